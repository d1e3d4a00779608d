"""Seeded synthetic decoding workloads: graph + info bits + codewords + channel LLRs.

Rate matching follows the paper's description (Sec. II): the first two information
columns are punctured and the rate is set by the number of base rows used.  Transmitted
bits are codeword positions [2Z, 2Z + N_tx); any bits of the last used column beyond N_tx
are not sent (their LLR is 0 at the decoder).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from fractions import Fraction

import numpy as np

from .channel import modulate_llr, quantize_int8, to_fp16
from .encode import encode_structured, info_bits
from .graphs import SHAPES, generate_base_graph, rate_params


@dataclass
class Workload:
    kind: str
    Z: int
    base: np.ndarray          # int16 [M][N]
    K_b: int
    n_rows: int               # M' rows used
    n_tx: int                 # transmitted bits per codeword
    punct_cols: int           # leading punctured columns (2 for the 5G-shaped codes)
    info: np.ndarray          # uint8 [B][K]
    codewords: np.ndarray     # uint8 [B][(K_b + n_rows) * Z]
    llr: np.ndarray           # float32 [B][n_tx]
    ebn0_db: float
    modulation: str
    meta: dict = field(default_factory=dict)

    @property
    def K(self) -> int:
        return self.K_b * self.Z

    @property
    def n_used(self) -> int:
        return (self.K_b + self.n_rows) * self.Z

    def llr_int8(self, scale: float = 4.0) -> np.ndarray:
        return quantize_int8(self.llr, scale)

    def llr_fp16(self) -> np.ndarray:
        return to_fp16(self.llr)


def make_workload(kind: str, Z: int, batch: int, ebn0_db, rate=None,
                  modulation: str = "QPSK", seed: int = 0, graph_seed: int | None = None,
                  punct_cols: int = 2, first_cw: int = 0, noiseless_llr: float | None = None,
                  base: np.ndarray | None = None) -> Workload:
    """Build a workload.  rate=None uses every base row (the lowest rate of the graph).

    noiseless_llr: if given, LLRs are +/- that value with no noise (the P2 pin).
    ebn0_db: one value, or an array with one value per codeword (the mean is kept in
    ``ebn0_db`` and the array in ``meta["ebn0_db"]``).
    """
    sh = SHAPES[kind]
    if base is None:
        base = generate_base_graph(kind, seed if graph_seed is None else graph_seed)
    if rate is None:
        n_rows = sh.M
        n_tx = (sh.K_b + n_rows - punct_cols) * Z
    else:
        n_rows, n_tx = rate_params(kind, Z, rate)
        if punct_cols != 2:
            raise ValueError("explicit rates assume the two punctured columns")
    K = sh.K_b * Z
    u = info_bits(seed, batch, K, first_cw)
    cw = encode_structured(base, sh.K_b, Z, u, n_rows)
    tx = cw[:, punct_cols * Z: punct_cols * Z + n_tx]
    R = float(Fraction(K, n_tx))
    if noiseless_llr is not None:
        llr = (noiseless_llr * (1.0 - 2.0 * tx.astype(np.float32))).astype(np.float32)
    else:
        llr = modulate_llr(tx, ebn0_db, R, modulation, seed, first_cw)
    meta = {"rate": R, "seed": seed}
    if np.ndim(ebn0_db) != 0:
        meta["ebn0_db"] = np.asarray(ebn0_db, dtype=np.float64)
    return Workload(kind, Z, base, sh.K_b, n_rows, n_tx, punct_cols, u, cw, llr,
                    float(np.mean(ebn0_db)), modulation, meta)
