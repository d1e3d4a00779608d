"""CPU oracle for layered min-sum LDPC decoding — TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg may use
this package.  The decoder itself is plain C (``ldpc_oracle.c``), built with gcc into
``liboracle.so`` next to this file; this module is argument marshalling only (ctypes, so
the GIL is released during each call and codeword ranges can run on several threads).

Every function follows the paper's method step by step (Sec. II code model, Sec. III
min-sum / layered schedule / stopping rule, Sec. IV per-row quantities); the C file's
header lists the readings taken where the paper is silent.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ldpc_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

LLR_INT8, LLR_FP16, LLR_FP32 = 0, 1, 2
NORMALISED, OFFSET, LEARNED, SUM_PRODUCT = 0, 1, 2, 3


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C99, -O2, no FP contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-std=c99", "-O2", "-ffp-contract=off", "-fno-fast-math",
                               "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB)
            P = ctypes.c_void_p
            i, f = ctypes.c_int, ctypes.c_float
            L.oracle_decode_layered.argtypes = [P, i, i, i, i, i, i, i, i, i, f, f, i, P, i, i,
                                                P, i, i, P, P, P, P]
            L.oracle_decode_layered.restype = i
            L.oracle_decode_flooding.argtypes = [P, i, i, i, i, i, i, i, i, f, f, i, i, P, i, i,
                                                 P, P, P]
            L.oracle_decode_flooding.restype = i
            L.oracle_check_node_f32.argtypes = [P, i, i, f, f, f, f, P]
            L.oracle_check_node_f32.restype = None
            L.oracle_check_node_i8.argtypes = [P, i, i, P]
            L.oracle_check_node_i8.restype = None
            L.oracle_syndrome_bits.argtypes = [P, i, i, i, i, i, P]
            L.oracle_syndrome_bits.restype = i
            L.oracle_edge_count.argtypes = [P, i, i, i, i, i]
            L.oracle_edge_count.restype = i
            L.oracle_learned_grad.argtypes = [P, i, i, i, i, i, i, i, P, i, P, P, i, i,
                                              ctypes.c_double, P, P, P, P, P]
            L.oracle_learned_grad.restype = i
            L.oracle_round_half.argtypes = [ctypes.c_double]
            L.oracle_round_half.restype = ctypes.c_float
            _lib = L
    return _lib


def _ptr(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


@dataclass
class DecodeResult:
    bits: np.ndarray          # uint8 [B][K] (0/1)
    iters: np.ndarray         # int32 [B]
    post: np.ndarray | None   # [B][N_used] posteriors (int8 / float16 / float32)
    c2v: np.ndarray | None    # [B][E*Z] check-to-variable messages, edge-major


def edge_count(base: np.ndarray, K_b: int, Z: int, n_rows: int) -> int:
    b = np.ascontiguousarray(base, dtype=np.int16)
    return lib().oracle_edge_count(_ptr(b), b.shape[0], b.shape[1], K_b, Z, n_rows)


def decode_layered(base, K_b, Z, n_rows, llr, *, llr_type=None, algo=NORMALISED, alpha=0.75,
                   offset=0.0, offset_q=1, learned=None, max_iter=8, early_stop=True,
                   punct=2, want_post=False, want_c2v=False, threads=1) -> DecodeResult:
    """Layered min-sum decode of llr [B][n_tx] (int8, float16 or float32)."""
    b = np.ascontiguousarray(base, dtype=np.int16)
    llr = np.ascontiguousarray(llr)
    if llr_type is None:
        llr_type = {np.dtype(np.int8): LLR_INT8, np.dtype(np.float16): LLR_FP16,
                    np.dtype(np.float32): LLR_FP32}[llr.dtype]
    B, n_tx = llr.shape
    K = K_b * Z
    N = (K_b + n_rows) * Z
    E = edge_count(b, K_b, Z, n_rows)
    bits = np.zeros((B, K), np.uint8)
    iters = np.zeros(B, np.int32)
    pdt = {LLR_INT8: np.int8, LLR_FP16: np.float16, LLR_FP32: np.float32}[llr_type]
    post = np.zeros((B, N), pdt) if want_post else None
    c2v = np.zeros((B, E * Z), pdt) if want_c2v else None
    lp = None
    if learned is not None:
        lp = np.ascontiguousarray(learned, dtype=np.float32)
    L = lib()

    def run(lo, hi):
        st = L.oracle_decode_layered(_ptr(b), b.shape[0], b.shape[1], K_b, Z, n_rows, punct,
                                     n_tx, llr_type, algo, alpha, offset, offset_q, _ptr(lp),
                                     max_iter, int(early_stop), _ptr(llr), lo, hi, _ptr(bits),
                                     _ptr(iters), _ptr(post), _ptr(c2v))
        if st != 0:
            raise ValueError(f"oracle_decode_layered failed with status {st}")

    _threaded(run, B, threads)
    return DecodeResult(bits, iters, post, c2v)


def decode_flooding(base, K_b, Z, n_rows, llr, *, algo=NORMALISED, alpha=0.75, offset=0.0,
                    max_iter=16, early_stop=True, punct=2, want_post=False,
                    threads=1) -> DecodeResult:
    """Flooding-schedule decode (fp32 min-sum, or exact sum-product with algo=SUM_PRODUCT)."""
    b = np.ascontiguousarray(base, dtype=np.int16)
    llr = np.ascontiguousarray(llr, dtype=np.float32)
    B, n_tx = llr.shape
    K = K_b * Z
    N = (K_b + n_rows) * Z
    bits = np.zeros((B, K), np.uint8)
    iters = np.zeros(B, np.int32)
    post = np.zeros((B, N), np.float32) if want_post else None
    L = lib()

    def run(lo, hi):
        st = L.oracle_decode_flooding(_ptr(b), b.shape[0], b.shape[1], K_b, Z, n_rows, punct,
                                      n_tx, algo, alpha, offset, max_iter, int(early_stop),
                                      _ptr(llr), lo, hi, _ptr(bits), _ptr(iters), _ptr(post))
        if st != 0:
            raise ValueError(f"oracle_decode_flooding failed with status {st}")

    _threaded(run, B, threads)
    return DecodeResult(bits, iters, post, None)


def _threaded(fn, B, threads):
    threads = max(1, min(int(threads), B)) if B else 1
    if threads == 1 or B == 0:
        fn(0, B)
        return
    edges = np.linspace(0, B, threads + 1).astype(int)
    ths = [threading.Thread(target=fn, args=(int(edges[k]), int(edges[k + 1])))
           for k in range(threads)]
    for t in ths:
        t.start()
    for t in ths:
        t.join()


def check_node_f32(v, mode=NORMALISED, alpha=0.75, offset=0.0, beta=1.0, gamma=0.0):
    v = np.ascontiguousarray(v, dtype=np.float32)
    out = np.zeros_like(v)
    lib().oracle_check_node_f32(_ptr(v), v.size, mode, alpha, offset, beta, gamma, _ptr(out))
    return out


def check_node_i8(v, offset_q=1):
    v = np.ascontiguousarray(v, dtype=np.int8)
    out = np.zeros_like(v)
    lib().oracle_check_node_i8(_ptr(v), v.size, offset_q, _ptr(out))
    return out


def syndrome_weight(base, K_b, Z, n_rows, bits) -> int:
    b = np.ascontiguousarray(base, dtype=np.int16)
    x = np.ascontiguousarray(bits, dtype=np.uint8)
    return int(lib().oracle_syndrome_bits(_ptr(b), b.shape[0], b.shape[1], K_b, Z, n_rows,
                                          _ptr(x)))


def learned_grad(base, K_b, Z, n_rows, llr, params, codewords, *, punct=2, want_post=False,
                 want_grad_llr=False, scale=None, iter_weights=None):
    """Loss (mean BCE of sigma(-L) against the codeword bits over batch x used bits) and its
    gradient with respect to the learned (beta, gamma) table [T][n_rows][2] (and optionally
    the channel LLRs), by reverse mode through the unrolled layered decoder.

    iter_weights ([T], optional): loss = sum_t w[t] * BCE(posteriors after iteration t);
    None is the final-posterior loss."""
    b = np.ascontiguousarray(base, dtype=np.int16)
    llr = np.ascontiguousarray(llr, dtype=np.float32)
    prm = np.ascontiguousarray(params, dtype=np.float32)
    T = prm.shape[0]
    B, n_tx = llr.shape
    N = (K_b + n_rows) * Z
    cw = np.ascontiguousarray(codewords[:, :N], dtype=np.uint8)
    if scale is None:
        scale = 1.0 / (B * N)
    gp = np.zeros(prm.shape, np.float64)
    gl = np.zeros((B, n_tx), np.float64) if want_grad_llr else None
    post = np.zeros((B, N), np.float32) if want_post else None
    loss = ctypes.c_double(0.0)
    iw = None
    if iter_weights is not None:
        iw = np.ascontiguousarray(iter_weights, dtype=np.float64)
        if iw.shape != (T,):
            raise ValueError("iter_weights needs one weight per iteration")
    st = lib().oracle_learned_grad(_ptr(b), b.shape[0], b.shape[1], K_b, Z, n_rows, punct, n_tx,
                                   _ptr(prm), T, _ptr(llr), _ptr(cw), 0, B, float(scale),
                                   _ptr(iw), _ptr(gp), _ptr(gl), _ptr(post), ctypes.byref(loss))
    if st != 0:
        raise ValueError(f"oracle_learned_grad failed with status {st}")
    return loss.value / (B * N), gp, gl, post


def round_half(x: float) -> float:
    return float(lib().oracle_round_half(float(x)))
