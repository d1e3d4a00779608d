"""Seeded synthetic quasi-cyclic base graphs shaped like the two 5G NR data-channel graphs.

The paper (Sec. II) describes the codes only structurally: a base graph H_BG of M_bg rows
and N_bg columns, the first K_b columns systematic, each non-zero entry lifted to a Z x Z
circulant, rate chosen by the number of rows used, and the first two information columns
punctured.  The 3GPP shift tables it relies on are not available, so the graphs here are
drawn from a seeded generator with the same shape:

* columns [0, K_b) systematic, [K_b, K_b+4) a dual-diagonal core parity part,
  [K_b+4, N_bg) degree-1 extension parity columns (one per extension row);
* core rows 0..3: column K_b carries shifts (a, 0, -, a) on rows (0, 1, 2, 3); columns
  K_b+1 (rows 0, 1), K_b+2 (rows 1, 2), K_b+3 (rows 2, 3) carry identities.  Summing the four
  core rows leaves only an identity on column K_b, so the core is invertible over GF(2);
* row 0 contains systematic column 0 and not column 1; rows 1..3 contain both.  With the
  layered schedule this lets noiseless LLRs recover both punctured columns in iteration 1;
* extension row r >= 4: an identity on column K_b+r, exactly one of columns {0, 1} (a
  seeded coin), and d_r - 2 further columns drawn from [2, K_b+4);
* every shift value V is drawn uniform in [0, 384); the circulant shift is V mod Z, so
  one base table serves every lifting size.

Circulant convention: check row i of block (r, c) with shift s connects variable
c*Z + ((i + s) mod Z).  -1 marks a zero block.

Draw order (Philox stream 1 of the seed): a; then for core rows 0..3 the systematic
column picks followed by their V values; then per extension row: d_r, the {0,1} coin,
the V of that column, the other column picks and their V values.  If any column below
K_b+4 ends with fewer than two edges the extension rows are drawn again from the same
stream (continuing it).
"""
from __future__ import annotations

from dataclasses import dataclass
from fractions import Fraction

import numpy as np

from .philox import PhiloxStream

V_RANGE = 384          # shift values are drawn in [0, 384) and reduced mod Z
GRAPH_STREAM = 1


@dataclass(frozen=True)
class GraphShape:
    name: str
    M: int              # base-graph rows
    N: int              # base-graph columns
    K_b: int            # systematic columns
    core_deg: int | None   # total degree of each core row (None: take every eligible column)
    ext_deg_lo: int
    ext_deg_hi: int     # inclusive


SHAPES = {
    # BG1-shaped: 46 x 68, 22 systematic columns, core rows of degree 19, extension rows 3..8
    "BG1": GraphShape("BG1", 46, 68, 22, 19, 3, 8),
    # BG2-shaped: 42 x 52, 10 systematic columns, core rows of degree 10, extension rows 3..10
    "BG2": GraphShape("BG2", 42, 52, 10, 10, 3, 10),
    # tiny code used for the brute-force ML comparison: 5 x 8, 3 systematic columns
    "TINY": GraphShape("TINY", 5, 8, 3, None, 3, 5),
}

# parity columns of each core row (offsets from K_b) and the fixed shift marker
# (None = identity, "a" = the drawn core shift)
_CORE_PARITY = {
    0: ((0, "a"), (1, None)),
    1: ((0, None), (1, None), (2, None)),
    2: ((2, None), (3, None)),
    3: ((0, "a"), (3, None)),
}


def _pick(stream: PhiloxStream, candidates: list[int], k: int) -> list[int]:
    """k distinct items from candidates by a partial Fisher-Yates shuffle."""
    pool = list(candidates)
    out = []
    for j in range(k):
        t = j + stream.uniform_int(len(pool) - j)
        pool[j], pool[t] = pool[t], pool[j]
        out.append(pool[j])
    return out


def generate_base_graph(kind: str, seed: int = 0) -> np.ndarray:
    """Return the int16 base table [M][N] (-1 = zero block, else V in [0, 384))."""
    sh = SHAPES[kind]
    M, N, Kb = sh.M, sh.N, sh.K_b
    st = PhiloxStream(seed, GRAPH_STREAM)
    H = np.full((M, N), -1, dtype=np.int16)
    a = st.uniform_int(V_RANGE)
    for r in range(4):
        for off, mark in _CORE_PARITY[r]:
            H[r, Kb + off] = a if mark == "a" else 0
        n_par = len(_CORE_PARITY[r])
        fixed = [0] if r == 0 else [0, 1]
        others = list(range(2, Kb))
        if sh.core_deg is None:
            chosen = fixed + others
        else:
            n_sys = sh.core_deg - n_par
            chosen = fixed + _pick(st, others, n_sys - len(fixed))
        for c in chosen:
            H[r, c] = st.uniform_int(V_RANGE)
    while True:
        Hx = H.copy()
        for r in range(4, M):
            d = sh.ext_deg_lo + st.uniform_int(sh.ext_deg_hi - sh.ext_deg_lo + 1)
            Hx[r, Kb + r] = 0
            c01 = st.uniform_int(2)
            Hx[r, c01] = st.uniform_int(V_RANGE)
            for c in _pick(st, list(range(2, Kb + 4)), d - 2):
                Hx[r, c] = st.uniform_int(V_RANGE)
        deg = (Hx[:, : Kb + 4] >= 0).sum(axis=0)
        if (deg >= 2).all():
            return Hx


# ----------------------------------------------------------------------------- rate

def rate_params(kind: str, Z: int, rate: Fraction | str | float) -> tuple[int, int]:
    """Rows used M' and transmitted bits N_tx for code rate R (Sec. II: rate by row count).

    N_tx = round(K / R) (half up); M' is the smallest row count with Z*(K_b + M' - 2) >= N_tx
    (never below the 4 core rows).  Bits of the last used column beyond N_tx are not sent.
    """
    sh = SHAPES[kind]
    R = Fraction(rate) if not isinstance(rate, Fraction) else rate
    K = sh.K_b * Z
    n_tx = int(Fraction(K) / R + Fraction(1, 2))
    m = 4
    while Z * (sh.K_b + m - 2) < n_tx:
        m += 1
    if m > sh.M:
        raise ValueError(f"rate {R} too low for {kind}")
    return m, n_tx


def expand_H(base: np.ndarray, Z: int, n_rows: int | None = None) -> np.ndarray:
    """Dense parity-check matrix (uint8) of the first n_rows base rows lifted by Z."""
    M, N = base.shape
    n_rows = M if n_rows is None else n_rows
    H = np.zeros((n_rows * Z, N * Z), dtype=np.uint8)
    i = np.arange(Z)
    for r in range(n_rows):
        for c in range(N):
            v = int(base[r, c])
            if v < 0:
                continue
            s = v % Z
            H[r * Z + i, c * Z + (i + s) % Z] ^= 1
    return H
