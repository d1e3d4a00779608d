"""Seeded AWGN channel, demapper LLRs and the int8 quantiser.

The paper only names the demapper as the source of the channel LLR L_b (Sec. III).  The
channel used for the synthetic workloads:

* LLR = ln P(b=0)/P(b=1); bit 0 is sent as +A.
* BPSK: A = 1, one bit per real dimension, m = 1 bit per symbol.
* QPSK: Gray mapped, A = 1/sqrt(2) on each of I and Q, m = 2.  Each bit sees its own
  real dimension, so its LLR is that of BPSK with amplitude A.
* Es = 1, N0 = 1 / (R * m * Eb/N0), noise variance N0/2 per real dimension.
  LLR = 4 A y / N0.
* 16QAM / 64QAM: Gray-labelled PAM on each dimension with unit average symbol energy and
  max-log LLRs (min over the points with the bit at 1 minus the min over those at 0 of
  (y - x)^2, divided by N0).
* Gaussians come from Box-Muller on Philox uniforms: codeword b, real dimension 4j+k uses
  counter (j, b, 2, 0); words (0, 1) give dimensions 4j, 4j+1 and words (2, 3) give 4j+2,
  4j+3.  The same standard normals are reused at every Eb/N0 (common random numbers), so
  BLER curves over Eb/N0 are computed on identical noise shapes.
* int8 LLRs: q = clamp(round_half_even(scale * L), -127, 127) from the float32 LLR; -128
  is never produced, so |q| always fits in 7 bits.
"""
from __future__ import annotations

import math
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np

from .philox import philox4x32, seed_key

NOISE_STREAM = 2


def std_normals(seed: int, batch: int, n: int, first_cw: int = 0) -> np.ndarray:
    """Seeded standard normals, float64 [batch][n].

    Every value depends only on its own counter, so large requests are split over
    codeword ranges and generated on a thread pool (numpy releases the GIL inside its
    element-wise loops); the result is the same as one call over the whole range.
    """
    nblk = (n + 3) // 4
    workers = min(os.cpu_count() or 1, 16)
    if workers > 1 and batch >= 2 * workers and batch * nblk >= (1 << 20):
        out = np.empty((batch, n), dtype=np.float64)
        cuts = np.linspace(0, batch, workers + 1).astype(int)

        def part(i):
            lo, hi = int(cuts[i]), int(cuts[i + 1])
            out[lo:hi] = _std_normals(seed, hi - lo, n, first_cw + lo)

        with ThreadPoolExecutor(workers) as ex:
            list(ex.map(part, range(workers)))
        return out
    return _std_normals(seed, batch, n, first_cw)


def _std_normals(seed: int, batch: int, n: int, first_cw: int) -> np.ndarray:
    k0, k1 = seed_key(seed)
    nblk = (n + 3) // 4
    j = np.arange(nblk, dtype=np.uint64)[None, :]
    cw = (np.arange(batch, dtype=np.uint64) + np.uint64(first_cw))[:, None]
    w0, w1, w2, w3 = philox4x32(j, cw, NOISE_STREAM, 0, k0, k1)
    inv = 1.0 / 4294967296.0

    def unif(w):
        return (w.astype(np.float64) + 0.5) * inv          # in (0, 1), never 0

    out = np.empty((batch, nblk, 4), dtype=np.float64)
    for (ua, ub), k in (((w0, w1), 0), ((w2, w3), 2)):
        r = np.sqrt(-2.0 * np.log(unif(ua)))
        th = 2.0 * math.pi * unif(ub)
        out[:, :, k] = r * np.cos(th)
        out[:, :, k + 1] = r * np.sin(th)
    return out.reshape(batch, nblk * 4)[:, :n]


EBN0_STREAM = 4


def uniform_ebn0(seed: int, batch: int, lo: float, hi: float, first_cw: int = 0) -> np.ndarray:
    """Per-codeword Eb/N0 in dB, uniform in [lo, hi): codeword b uses word 0 of the Philox
    counter (b, 4, 0, 0)."""
    k0, k1 = seed_key(seed)
    cw = np.arange(batch, dtype=np.uint64) + np.uint64(first_cw)
    w = philox4x32(cw, EBN0_STREAM, 0, 0, k0, k1)[0]
    u = (w.astype(np.float64) + 0.5) / 4294967296.0
    return lo + (hi - lo) * u


def noise_n0(ebn0_db: float, rate: float, bits_per_symbol: int) -> float:
    ebn0 = 10.0 ** (ebn0_db / 10.0)
    return 1.0 / (rate * bits_per_symbol * ebn0)


def _pam_gray(m_half: int):
    """Gray-labelled PAM levels for m_half bits per dimension, unit-energy scaling later.

    Returns (levels [2^m], labels [2^m][m_half]) with levels -(L-1), ..., +(L-1) in steps of 2
    and the binary-reflected Gray label of each level index (bit 0 = most significant).
    """
    L = 1 << m_half
    idx = np.arange(L)
    gray = idx ^ (idx >> 1)
    levels = (2 * idx - (L - 1)).astype(np.float64)
    labels = ((gray[:, None] >> (m_half - 1 - np.arange(m_half))[None, :]) & 1).astype(np.uint8)
    return levels, labels


def pam_points(mh: int):
    """Unit-average-energy QAM per-dimension levels and their Gray labels.

    Square 2^(2 mh)-QAM is two Gray-labelled 2^mh-PAM axes; the scale makes the average
    energy of a 2-D symbol 1 (each axis carries 1/2).
    """
    levels, labels = _pam_gray(mh)
    L = len(levels)
    scale = math.sqrt(2.0 * (L * L - 1) / 3.0)
    return levels / scale, labels


def pam_map(groups: np.ndarray, mh: int) -> np.ndarray:
    """Map bit groups [..][mh] (first bit most significant in the label) to PAM levels."""
    pts, labels = pam_points(mh)
    L = len(pts)
    code = np.zeros(groups.shape[:-1], dtype=np.int64)
    for k in range(mh):
        code = (code << 1) | groups[..., k].astype(np.int64)
    lab_code = np.zeros(L, dtype=np.int64)
    for k in range(mh):
        lab_code = (lab_code << 1) | labels[:, k].astype(np.int64)
    inv = np.empty(L, dtype=np.int64)
    inv[lab_code] = np.arange(L)
    return pts[inv[code]]


def _pam_maxlog(y: np.ndarray, mh: int, n0) -> np.ndarray:
    pts, labels = pam_points(mh)
    d2 = (y[..., None] - pts) ** 2
    out = np.empty(y.shape + (mh,), dtype=np.float64)
    for k in range(mh):
        is1 = labels[:, k] == 1
        out[..., k] = (d2[..., is1].min(axis=-1) - d2[..., ~is1].min(axis=-1)) / n0
    return out


def pam_maxlog_llr(y: np.ndarray, mh: int, n0) -> np.ndarray:
    """Max-log bit LLRs [..][mh] of received per-dimension values y [B][..] (n0 a scalar or
    [B][1]).  Large inputs are split over rows on a thread pool (element-wise, so the result
    does not depend on the split)."""
    workers = min(os.cpu_count() or 1, 16)
    B = y.shape[0] if y.ndim else 1
    if workers < 2 or y.ndim < 2 or B < 2 * workers or y.size < (1 << 20):
        return _pam_maxlog(y, mh, n0)
    out = np.empty(y.shape + (mh,), dtype=np.float64)
    cuts = np.linspace(0, B, workers + 1).astype(int)
    n0a = np.asarray(n0, dtype=np.float64)

    def part(i):
        lo, hi = int(cuts[i]), int(cuts[i + 1])
        out[lo:hi] = _pam_maxlog(y[lo:hi], mh, n0a[lo:hi] if n0a.ndim else n0a)

    with ThreadPoolExecutor(workers) as ex:
        list(ex.map(part, range(workers)))
    return out


_BITS_PER_SYMBOL = {"BPSK": 1, "QPSK": 2, "16QAM": 4, "64QAM": 6}


def modulate_llr(bits: np.ndarray, ebn0_db, rate: float, modulation: str,
                 seed: int, first_cw: int = 0) -> np.ndarray:
    """Channel LLRs (float32 [B][n]) for transmitted bits [B][n] over AWGN.

    ebn0_db is one value for the whole batch or an array [B] with one value per codeword;
    a codeword's LLRs do not depend on which of the two forms carried its Eb/N0.
    """
    B, n = bits.shape
    m = _BITS_PER_SYMBOL.get(modulation)
    if m is None:
        raise ValueError(f"unknown modulation {modulation}")
    if np.ndim(ebn0_db) == 0:
        n0 = noise_n0(float(ebn0_db), rate, m)
        sigma = math.sqrt(n0 / 2.0)
    else:
        e = np.asarray(ebn0_db, dtype=np.float64).reshape(-1)
        if e.shape != (B,):
            raise ValueError("per-codeword Eb/N0 needs one value per codeword")
        n0s = [noise_n0(float(x), rate, m) for x in e]
        n0 = np.array(n0s)[:, None]
        sigma = np.array([math.sqrt(v / 2.0) for v in n0s])[:, None]
    if m <= 2:
        A = 1.0 if m == 1 else 1.0 / math.sqrt(2.0)
        y = A * (1.0 - 2.0 * bits.astype(np.float64)) + sigma * std_normals(seed, B, n, first_cw)
        return (4.0 * A * y / n0).astype(np.float32)
    mh = m // 2
    nsym_dims = (n + mh - 1) // mh                      # real dimensions used
    pad = nsym_dims * mh - n
    bp = np.concatenate([bits, np.zeros((B, pad), dtype=bits.dtype)], axis=1)
    x = pam_map(bp.reshape(B, nsym_dims, mh), mh)
    y = x + sigma * std_normals(seed, B, nsym_dims, first_cw)
    llr = pam_maxlog_llr(y, mh, n0)
    return llr.reshape(B, nsym_dims * mh)[:, :n].astype(np.float32)


def modulate_llr_sweep(bits: np.ndarray, ebn0s, rate: float, modulation: str, seed: int,
                       first_cw: int = 0):
    """Channel LLRs of the same transmitted bits at each Eb/N0 in `ebn0s` (a generator of
    float32 [B][n] arrays): the symbols and the standard normals are computed once, and each
    array equals modulate_llr(bits, e, rate, modulation, seed, first_cw)."""
    B, n = bits.shape
    m = _BITS_PER_SYMBOL.get(modulation)
    if m is None:
        raise ValueError(f"unknown modulation {modulation}")
    if m <= 2:
        A = 1.0 if m == 1 else 1.0 / math.sqrt(2.0)
        x = A * (1.0 - 2.0 * bits.astype(np.float64))
        z = std_normals(seed, B, n, first_cw)
        for e in ebn0s:
            n0 = noise_n0(float(e), rate, m)
            yield (4.0 * A * (x + math.sqrt(n0 / 2.0) * z) / n0).astype(np.float32)
        return
    mh = m // 2
    nsym_dims = (n + mh - 1) // mh
    pad = nsym_dims * mh - n
    bp = np.concatenate([bits, np.zeros((B, pad), dtype=bits.dtype)], axis=1)
    x = pam_map(bp.reshape(B, nsym_dims, mh), mh)
    z = std_normals(seed, B, nsym_dims, first_cw)
    for e in ebn0s:
        n0 = noise_n0(float(e), rate, m)
        llr = pam_maxlog_llr(x + math.sqrt(n0 / 2.0) * z, mh, n0)
        yield llr.reshape(B, nsym_dims * mh)[:, :n].astype(np.float32)


def quantize_int8(llr: np.ndarray, scale: float = 4.0) -> np.ndarray:
    """int8 LLRs: clamp(round_half_even(scale * L), -127, 127) from the float32 LLR."""
    x = np.rint(np.asarray(llr, dtype=np.float32) * np.float32(scale))
    return np.clip(x, -127, 127).astype(np.int8)


def to_fp16(llr: np.ndarray) -> np.ndarray:
    """float16 LLRs by round-to-nearest-even from the float32 LLR (numpy's conversion)."""
    return np.asarray(llr, dtype=np.float32).astype(np.float16)
