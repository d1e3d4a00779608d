"""GF(2) encoders for the synthetic QC codes and the seeded information bits.

Two independent encoders are provided so that each checks the other:

* ``encode_structured``: back-substitution through the dual-diagonal core.  With
  lambda_r the sum of row r's systematic circulants applied to the information blocks,
  the four core rows read
      row 0: lambda_0 + P^a p0 + p1 = 0        row 1: lambda_1 + p0 + p1 + p2 = 0
      row 2: lambda_2 + p2 + p3 = 0            row 3: lambda_3 + P^a p0 + p3 = 0
  and their sum gives p0 = lambda_0 + lambda_1 + lambda_2 + lambda_3, then p1, p2, p3
  follow row by row.
* ``encode_gaussian``: a generic solve of the 4Z x 4Z core system by Gauss-Jordan
  elimination over GF(2), which uses nothing of the dual-diagonal structure.

Extension parity blocks (rows r >= 4) are the GF(2) sum of the row's other circulants,
since each extension row holds an identity on its own parity column.

Circulant convention: (P^s x)[i] = x[(i + s) mod Z].
"""
from __future__ import annotations

import numpy as np

from .philox import philox4x32, seed_key

INFO_STREAM = 3


def info_bits(seed: int, batch: int, K: int, first_cw: int = 0) -> np.ndarray:
    """Seeded uniform information bits, uint8 [batch][K].

    Codeword b uses Philox counters (j, first_cw + b, 3, 0), j = 0, 1, ...; the 128 output
    bits of counter j are bits 128j .. 128j+127, word 0 first, least significant bit first.
    """
    k0, k1 = seed_key(seed)
    nblk = (K + 127) // 128
    j = np.arange(nblk, dtype=np.uint64)[None, :]
    cw = (np.arange(batch, dtype=np.uint64) + np.uint64(first_cw))[:, None]
    w = philox4x32(j, cw, INFO_STREAM, 0, k0, k1)
    words = np.stack(w, axis=-1).reshape(batch, nblk * 4)           # uint32
    by = words.view(np.uint8).reshape(batch, nblk * 16)                # little-endian bytes
    bits = np.unpackbits(by, axis=1, bitorder="little")[:, :K]
    return bits.astype(np.uint8)


def _circ(x: np.ndarray, s: int) -> np.ndarray:
    """P^s applied along the last axis: out[..., i] = x[..., (i + s) mod Z]."""
    return np.roll(x, -int(s), axis=-1)


def _lambda(base: np.ndarray, Z: int, K_b: int, ub: np.ndarray, r: int) -> np.ndarray:
    acc = np.zeros(ub.shape[:1] + (Z,), dtype=np.uint8)
    for c in range(K_b):
        v = int(base[r, c])
        if v >= 0:
            acc ^= _circ(ub[:, c, :], v % Z)
    return acc


def _extension(base: np.ndarray, Z: int, K_b: int, x: np.ndarray, n_rows: int) -> None:
    """Fill extension parity blocks of x ([B][cols][Z]) for rows 4..n_rows-1 in place."""
    for r in range(4, n_rows):
        acc = np.zeros(x.shape[:1] + (Z,), dtype=np.uint8)
        for c in range(K_b + 4):
            v = int(base[r, c])
            if v >= 0:
                acc ^= _circ(x[:, c, :], v % Z)
        if int(base[r, K_b + r]) != 0:
            raise ValueError("extension row must carry an identity on its parity column")
        x[:, K_b + r, :] = acc


def encode_structured(base: np.ndarray, K_b: int, Z: int, u: np.ndarray,
                      n_rows: int | None = None) -> np.ndarray:
    """Codewords uint8 [B][(K_b + n_rows) * Z] for information bits u [B][K_b * Z]."""
    M = base.shape[0]
    n_rows = M if n_rows is None else n_rows
    B = u.shape[0]
    x = np.zeros((B, K_b + n_rows, Z), dtype=np.uint8)
    x[:, :K_b, :] = u.reshape(B, K_b, Z)
    lam = [_lambda(base, Z, K_b, x, r) for r in range(4)]
    a = int(base[0, K_b]) % Z
    p0 = lam[0] ^ lam[1] ^ lam[2] ^ lam[3]
    p1 = lam[0] ^ _circ(p0, a)
    p2 = lam[1] ^ p0 ^ p1
    p3 = lam[2] ^ p2
    x[:, K_b + 0], x[:, K_b + 1], x[:, K_b + 2], x[:, K_b + 3] = p0, p1, p2, p3
    _extension(base, Z, K_b, x, n_rows)
    return x.reshape(B, -1)


def _gf2_inverse(A: np.ndarray) -> np.ndarray:
    """Inverse of a square uint8 GF(2) matrix by Gauss-Jordan elimination on packed rows."""
    n = A.shape[0]
    aug = np.concatenate([A.astype(np.uint8) & 1, np.eye(n, dtype=np.uint8)], axis=1)
    P = np.packbits(aug, axis=1)                      # rows as bytes
    for col in range(n):
        byte, bit = col >> 3, 7 - (col & 7)
        colbits = (P[:, byte] >> bit) & 1
        cand = np.nonzero(colbits[col:])[0]
        if cand.size == 0:
            raise ValueError("core parity matrix is singular over GF(2)")
        piv = col + int(cand[0])
        if piv != col:
            P[[col, piv]] = P[[piv, col]]
            colbits = (P[:, byte] >> bit) & 1
        rows = np.nonzero(colbits)[0]
        rows = rows[rows != col]
        if rows.size:
            P[rows] ^= P[col]
    full = np.unpackbits(P, axis=1)[:, : 2 * n]
    return full[:, n:]


def core_matrix(base: np.ndarray, K_b: int, Z: int) -> np.ndarray:
    """Dense 4Z x 4Z matrix of the core parity columns [K_b, K_b+4) in rows 0..3."""
    H = np.zeros((4 * Z, 4 * Z), dtype=np.uint8)
    i = np.arange(Z)
    for r in range(4):
        for k in range(4):
            v = int(base[r, K_b + k])
            if v >= 0:
                H[r * Z + i, k * Z + (i + v % Z) % Z] ^= 1
    return H


def encode_gaussian(base: np.ndarray, K_b: int, Z: int, u: np.ndarray,
                    n_rows: int | None = None, core_inverse: np.ndarray | None = None) -> np.ndarray:
    """Same codewords as encode_structured, by a generic GF(2) solve of the core system."""
    M = base.shape[0]
    n_rows = M if n_rows is None else n_rows
    B = u.shape[0]
    x = np.zeros((B, K_b + n_rows, Z), dtype=np.uint8)
    x[:, :K_b, :] = u.reshape(B, K_b, Z)
    rhs = np.concatenate([_lambda(base, Z, K_b, x, r) for r in range(4)], axis=1)  # [B][4Z]
    inv = _gf2_inverse(core_matrix(base, K_b, Z)) if core_inverse is None else core_inverse
    p = (rhs.astype(np.float32) @ inv.T.astype(np.float32)).astype(np.int64) & 1
    x[:, K_b:K_b + 4, :] = p.reshape(B, 4, Z).astype(np.uint8)
    _extension(base, Z, K_b, x, n_rows)
    return x.reshape(B, -1)
