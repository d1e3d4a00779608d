"""GPU decoder vs the CPU oracle, through the C ABI, on the same seeded inputs.

int8: bit-exact in every posterior, every check-to-variable message, every hard bit and
every iteration count.  fp32: identical operations in the same order, so the same bar is
applied (the benchmark spec's tolerance of 1e-4 relative is asserted as well).  fp16: identical
hard bits and posteriors within 2^-7 of max|LLR| (IEEE binary16 arithmetic on both sides,
so exact agreement is expected and checked on the hard bits).
"""
import json
import os
from fractions import Fraction

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from synth import generate_base_graph, make_workload

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def ldpc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2009_05534_gb300 import build
    build.build()
    import paper_2009_05534_gb300 as pkg
    return pkg


def _gpu(ldpc, wl, llr, T, *, early_stop, n_rows=None, punct=2, debug=True, **kw):
    g = ldpc.Graph(wl.base, wl.K_b, wl.Z)
    t = torch.from_numpy(np.ascontiguousarray(llr)).cuda()
    out = ldpc.decode(g, t, T, early_stop=early_stop, n_rows=n_rows or 0, punct_cols=punct,
                      debug=debug, **kw)
    torch.cuda.synchronize()
    g.sync_status()
    res = [o.cpu().numpy() for o in out]
    g.close()
    return res


def _unpack(ldpc, packed, K):
    return ldpc.unpack_bits(packed, K)


# ------------------------------------------------------------------- int8 (headline path)
#
# threads_per_row (the paper's alpha): 1 = the high-throughput kernels (one thread per row
# pair), 2 and 4 = the low-latency kernel (alpha threads per row pair, shuffle reduce),
# 0 = the library's choice for the batch.

_REF = {}


def _ref_bg1(T):
    """Oracle decode of the 24-codeword BG1 Z=384 case (shared by every alpha)."""
    if T not in _REF:
        wl = make_workload("BG1", 384, 24, 1.25, seed=11)
        q = wl.llr_int8()
        _REF[T] = (wl, q, oracle.decode_layered(wl.base, wl.K_b, 384, wl.n_rows, q,
                                                algo=oracle.OFFSET, offset_q=1, max_iter=T,
                                                early_stop=False, want_post=True,
                                                want_c2v=True, threads=8))
    return _REF[T]


@pytest.mark.parametrize("tpr", [1, 2, 4])
@pytest.mark.parametrize("T", [1, 2, 5, 10])
def test_int8_bg1_z384_bit_exact(ldpc, T, tpr):
    wl, q, ref = _ref_bg1(T)
    bits, iters, post, c2v = _gpu(ldpc, wl, q, T, early_stop=False, threads_per_row=tpr)
    assert np.array_equal(post, ref.post)
    assert np.array_equal(c2v, ref.c2v)
    assert np.array_equal(_unpack(ldpc, bits, wl.K), ref.bits)
    assert (iters == T).all()


@pytest.mark.parametrize("tpr", [1, 4])
@pytest.mark.parametrize("ebn0", [0.5, 1.5, 2.5])
def test_int8_early_stop_iterations_exact(ldpc, ebn0, tpr):
    wl = make_workload("BG1", 384, 32, ebn0, seed=3)
    q = wl.llr_int8()
    ref = oracle.decode_layered(wl.base, wl.K_b, 384, wl.n_rows, q, algo=oracle.OFFSET,
                                offset_q=1, max_iter=10, early_stop=True, want_post=True,
                                threads=8)
    bits, iters, post, _ = _gpu(ldpc, wl, q, 10, early_stop=True, threads_per_row=tpr)
    assert np.array_equal(iters, ref.iters)
    assert np.array_equal(post, ref.post)
    assert np.array_equal(_unpack(ldpc, bits, wl.K), ref.bits)


@pytest.mark.parametrize("kind,Z,rate", [("BG1", 13, None), ("BG1", 40, "1/2"),
                                         ("BG2", 7, "2/3"), ("BG2", 96, "1/3"),
                                         ("BG1", 384, "8/9"), ("BG2", 2, None)])
@pytest.mark.parametrize("tpr", [1, 0])
def test_int8_ragged_shapes_and_rates(ldpc, kind, Z, rate, tpr):
    """Z not a multiple of the warp, odd Z, several row counts (rates); with the library's
    choice of alpha (the low-latency kernel for even Z at this batch)."""
    wl = make_workload(kind, Z, 9, 2.0, rate=None if rate is None else Fraction(rate), seed=4)
    q = wl.llr_int8()
    ref = oracle.decode_layered(wl.base, wl.K_b, Z, wl.n_rows, q, algo=oracle.OFFSET,
                                offset_q=1, max_iter=6, early_stop=True, want_post=True,
                                want_c2v=True)
    bits, iters, post, c2v = _gpu(ldpc, wl, q, 6, early_stop=True, n_rows=wl.n_rows,
                                  n_tx=wl.n_tx, threads_per_row=tpr)
    assert np.array_equal(iters, ref.iters)
    assert np.array_equal(post, ref.post)
    assert np.array_equal(c2v, ref.c2v)
    assert np.array_equal(_unpack(ldpc, bits, wl.K), ref.bits)


def test_int8_hand_examples(ldpc):
    for name, key in (("hand_layered_z2.json", "int8_offset1"),
                      ("hand_saturation_z1.json", "int8_offset1")):
        g = json.load(open(os.path.join(GOLDEN, name)))
        code, ex = g["code"], g[key]
        base = np.array(code["base"], np.int16)
        graph = ldpc.Graph(base, code["K_b"], code["Z"])
        llr = torch.tensor([ex["llr"]], dtype=torch.int8).cuda()
        for T in (1, 2):
            bits, iters, post, c2v = ldpc.decode(graph, llr, T, early_stop=False, punct_cols=0,
                                                 n_rows=code["n_rows"], debug=True)
            assert post.cpu().numpy()[0].tolist() == ex[f"T{T}"]["post"]
            assert c2v.cpu().numpy()[0].tolist() == ex[f"T{T}"]["c2v"]
        graph.close()


def test_int8_noiseless_one_iteration(ldpc):
    wl = make_workload("BG1", 384, 8, 0.0, noiseless_llr=8.0, seed=2)
    bits, iters, _, _ = _gpu(ldpc, wl, wl.llr_int8(), 10, early_stop=True)
    assert (iters == 1).all()
    assert np.array_equal(_unpack(ldpc, bits, wl.K), wl.info)


def test_empty_and_single_batch(ldpc):
    wl = make_workload("BG2", 16, 1, 3.0, seed=1)
    g = ldpc.Graph(wl.base, wl.K_b, 16)
    empty = torch.zeros((0, wl.n_tx), dtype=torch.int8, device="cuda")
    bits, iters = ldpc.decode(g, empty, 5)
    assert bits.shape[0] == 0 and iters.shape[0] == 0
    q = wl.llr_int8()
    ref = oracle.decode_layered(wl.base, wl.K_b, 16, wl.n_rows, q, algo=oracle.OFFSET,
                                max_iter=5)
    bits, iters = ldpc.decode(g, torch.from_numpy(q).cuda(), 5)
    torch.cuda.synchronize()
    assert np.array_equal(_unpack(ldpc, bits.cpu().numpy(), wl.K), ref.bits)
    assert iters.cpu().numpy().tolist() == ref.iters.tolist()
    g.close()


def test_invalid_calls_raise(ldpc):
    wl = make_workload("BG2", 16, 2, 3.0, seed=1)
    g = ldpc.Graph(wl.base, wl.K_b, 16)
    q = torch.from_numpy(wl.llr_int8()).cuda()
    with pytest.raises(ldpc.LdpcError):
        ldpc.decode(g, q, 0)                       # max_iter < 1
    with pytest.raises(ldpc.LdpcError):
        ldpc.decode(g, q, 5, n_rows=99)
    with pytest.raises(ldpc.LdpcError):
        ldpc.decode(g, q, 5, algo=ldpc.NORMALISED)   # int8 supports offset only
    with pytest.raises(ldpc.LdpcError):
        ldpc.decode(g, q, 5, n_tx=10 ** 6)
    with pytest.raises(ldpc.LdpcError):              # no 32-bit sum with n_tx may wrap
        ldpc.decode(g, q, 5, n_tx=2 ** 31 - 1)
    with pytest.raises(ldpc.LdpcError):
        ldpc.decode(g, q, 5, threads_per_row=3)      # alpha must be 0, 1, 2 or 4
    with pytest.raises(ldpc.LdpcError):                # low latency: int8 offset only
        ldpc.decode(g, q.float(), 5, threads_per_row=2)
    g.close()


# --------------------------------------------------------------- fp32 (BG2 Z=16, 8 iterations)

@pytest.mark.parametrize("ebn0", [0.0, 1.0, 2.0, 3.0])
def test_fp32_bg2_z16(ldpc, ebn0):
    wl = make_workload("BG2", 16, 200, ebn0, modulation="BPSK", seed=0)
    ref = oracle.decode_layered(wl.base, wl.K_b, 16, wl.n_rows, wl.llr, algo=oracle.NORMALISED,
                                alpha=0.75, max_iter=8, early_stop=True, want_post=True,
                                want_c2v=True, threads=4)
    bits, iters, post, c2v = _gpu(ldpc, wl, wl.llr, 8, early_stop=True,
                                  algo=ldpc.NORMALISED, alpha=0.75)
    assert np.array_equal(iters, ref.iters)
    assert np.array_equal(_unpack(ldpc, bits, wl.K), ref.bits)
    scale = np.maximum(np.abs(ref.post), 1e-30)
    assert (np.abs(post - ref.post) <= 1e-4 * scale).all()
    assert np.array_equal(post, ref.post)          # same operation order: exact
    assert np.array_equal(c2v, ref.c2v)


def test_fp32_hand_example(ldpc):
    g = json.load(open(os.path.join(GOLDEN, "hand_layered_z2.json")))
    code, ex = g["code"], g["fp32_normalised_0.75"]
    graph = ldpc.Graph(np.array(code["base"], np.int16), code["K_b"], code["Z"])
    llr = torch.tensor([ex["llr"]], dtype=torch.float32).cuda()
    _, _, post, c2v = ldpc.decode(graph, llr, 1, early_stop=False, punct_cols=0,
                                  n_rows=code["n_rows"], debug=True, algo=ldpc.NORMALISED)
    assert post.cpu().numpy()[0].tolist() == ex["T1"]["post"]
    assert c2v.cpu().numpy()[0].tolist() == ex["T1"]["c2v"]
    graph.close()


# ------------------------------------------------------------------------------- fp16

def test_fp16_bg1_z64(ldpc):
    wl = make_workload("BG1", 64, 48, 2.0, seed=8)
    h = wl.llr_fp16()
    ref = oracle.decode_layered(wl.base, wl.K_b, 64, wl.n_rows, h, algo=oracle.NORMALISED,
                                alpha=0.75, max_iter=8, early_stop=True, want_post=True,
                                threads=8)
    bits, iters, post, _ = _gpu(ldpc, wl, h, 8, early_stop=True, algo=ldpc.NORMALISED)
    gb = _unpack(ldpc, bits, wl.K)
    assert (gb == ref.bits).all(axis=1).mean() >= 0.9999
    assert np.array_equal(iters, ref.iters)
    tol = 2.0 ** -7 * float(np.abs(wl.llr).max())
    assert (np.abs(post.astype(np.float32) - ref.post.astype(np.float32)) <= tol).all()


def test_fp16_hand_example(ldpc):
    """The binary16 decoder on the hand-worked example whose every binary16 rounding
    (v = L - c, corrected magnitudes, posteriors, ties to even, binary16 parameters, the
    learned correction's two roundings) changes a value."""
    g = json.load(open(os.path.join(GOLDEN, "hand_layered_f16_z2.json")))
    code = g["code"]
    graph = ldpc.Graph(np.array(code["base"], np.int16), code["K_b"], code["Z"])
    llr = torch.tensor([g["llr"]], dtype=torch.float16).cuda()
    ex = g["normalised_0.75"]
    for T in (1, 2):
        bits, _, post, c2v = ldpc.decode(graph, llr, T, early_stop=False, punct_cols=0,
                                         n_rows=code["n_rows"], debug=True,
                                         algo=ldpc.NORMALISED, alpha=0.75)
        torch.cuda.synchronize()
        assert post.cpu().double().numpy()[0].tolist() == ex[f"T{T}"]["post"]
        assert c2v.cpu().double().numpy()[0].tolist() == ex[f"T{T}"]["c2v"]
    assert _unpack(ldpc, bits.cpu().numpy(), 4)[0].tolist() == ex["hard_bits_K"]
    lx = g["learned_T1"]
    tab = torch.tensor(lx["table"], dtype=torch.float32).cuda()
    _, _, post, c2v = ldpc.decode(graph, llr, 1, early_stop=False, punct_cols=0,
                                  n_rows=code["n_rows"], debug=True, algo=ldpc.LEARNED,
                                  learned=tab)
    torch.cuda.synchronize()
    graph.sync_status()
    assert post.cpu().double().numpy()[0].tolist() == lx["post"]
    assert c2v.cpu().double().numpy()[0].tolist() == lx["c2v"]
    ox = g["offset_0.3_T1"]
    _, _, post, c2v = ldpc.decode(graph, llr, 1, early_stop=False, punct_cols=0,
                                  n_rows=code["n_rows"], debug=True, algo=ldpc.OFFSET,
                                  offset=0.3)
    torch.cuda.synchronize()
    assert post.cpu().double().numpy()[0].tolist() == ox["post"]
    assert c2v.cpu().double().numpy()[0].tolist() == ox["c2v"]
    graph.close()


# ------------------------------------------------------- full size, the whole batch


@pytest.fixture(scope="module")
def headline():
    """The benchmark's workload: BG1 Z=384, 1024 codewords at 1.5 dB, int8."""
    wl = make_workload("BG1", 384, 1024, 1.5, seed=0)
    return wl, wl.llr_int8()


@pytest.mark.parametrize("early_stop", [False, True])
def test_int8_full_batch(ldpc, headline, early_stop):
    """Batch 1024, BG1 Z=384, T=10 in the benchmark's launch configuration (work counter,
    staging ahead, on-demand claims near the end of the batch, lane refill under the
    stopping rule): every codeword's hard bits and iteration count equal the oracle's."""
    wl, q = headline
    bits, iters = _gpu(ldpc, wl, q, 10, early_stop=early_stop, debug=False)
    ref = oracle.decode_layered(wl.base, wl.K_b, 384, wl.n_rows, q, algo=oracle.OFFSET,
                                max_iter=10, early_stop=early_stop, threads=16)
    assert np.array_equal(_unpack(ldpc, bits, wl.K), ref.bits)
    assert np.array_equal(iters, ref.iters)
    if early_stop:
        assert 1 <= ref.iters.min() and ref.iters.max() == 10 and ref.iters.mean() < 9


def test_int8_full_batch_posteriors(ldpc, headline):
    """The same batch with the stopping rule and the debug outputs: all 1024 codewords'
    final posteriors and check-to-variable messages equal the oracle's."""
    wl, q = headline
    bits, iters, post, c2v = _gpu(ldpc, wl, q, 10, early_stop=True, threads_per_row=1)
    ref = oracle.decode_layered(wl.base, wl.K_b, 384, wl.n_rows, q, algo=oracle.OFFSET,
                                max_iter=10, early_stop=True, want_post=True, want_c2v=True,
                                threads=16)
    assert np.array_equal(iters, ref.iters)
    assert np.array_equal(post, ref.post)
    assert np.array_equal(c2v, ref.c2v)
    assert np.array_equal(_unpack(ldpc, bits, wl.K), ref.bits)


@pytest.mark.parametrize("tpr", [1, 2, 4])
def test_int8_custom_table_degrees_11_to_18(ldpc, tpr):
    """A user base table with row degrees 11..18 (the predicated wide-row path; with alpha
    2 and 4, rows whose degree is not a multiple of alpha)."""
    rng = np.random.default_rng(7)
    M, K_b, Z = 6, 24, 32
    N = K_b + M
    base = np.full((M, N), -1, np.int16)
    for r in range(M):
        d = 11 + r + (r > 3)                  # 11, 12, 13, 14, 16, 17
        cols = rng.choice(K_b + r, size=d - 1, replace=False)
        base[r, cols] = rng.integers(0, 384, size=d - 1)
        base[r, K_b + r] = 0
    from synth import info_bits
    B = 12
    llr = rng.integers(-40, 41, size=(B, (N - 2) * Z)).astype(np.int8)
    ref = oracle.decode_layered(base, K_b, Z, M, llr, algo=oracle.OFFSET, offset_q=1,
                                max_iter=4, early_stop=False, want_post=True, want_c2v=True)
    g = ldpc.Graph(base, K_b, Z)
    bits, iters, post, c2v = ldpc.decode(g, torch.from_numpy(llr).cuda(), 4, early_stop=False,
                                         debug=True, threads_per_row=tpr)
    torch.cuda.synchronize()
    assert np.array_equal(post.cpu().numpy(), ref.post)
    assert np.array_equal(c2v.cpu().numpy(), ref.c2v)
    assert np.array_equal(ldpc.unpack_bits(bits.cpu().numpy(), K_b * Z), ref.bits)
    g.close()


@pytest.mark.parametrize("tpr", [1, 4])
def test_int8_dense_bg1_table_z384(ldpc, tpr):
    """A 46 x 68 table with more edges than fit the two-codeword Tensor-Memory message
    store (E > 340 at Z = 384): alpha 1 takes the shared-memory row-pair kernel; the
    one-codeword low-latency kernel holds it in Tensor Memory."""
    rng = np.random.default_rng(11)
    M, K_b, Z = 46, 22, 384
    N = K_b + M
    base = np.full((M, N), -1, np.int16)
    for r in range(M):
        d = int(rng.integers(8, 13))
        cols = rng.choice(K_b + 4, size=d - 1, replace=False)
        base[r, cols] = rng.integers(0, 384, size=d - 1)
        base[r, K_b + r] = 0
    assert (base >= 0).sum() > 340
    B = 6
    llr = rng.integers(-30, 31, size=(B, (N - 2) * Z)).astype(np.int8)
    ref = oracle.decode_layered(base, K_b, Z, M, llr, algo=oracle.OFFSET, offset_q=1,
                                max_iter=3, early_stop=False, want_post=True, want_c2v=True,
                                threads=6)
    g = ldpc.Graph(base, K_b, Z)
    bits, iters, post, c2v = ldpc.decode(g, torch.from_numpy(llr).cuda(), 3, early_stop=False,
                                         debug=True, threads_per_row=tpr)
    torch.cuda.synchronize()
    assert np.array_equal(post.cpu().numpy(), ref.post)
    assert np.array_equal(c2v.cpu().numpy(), ref.c2v)
    g.close()


# ------------------------------------- batch kernel: work counter, lane refill, streams

def test_batch_kernel_many_codewords_per_block_early_stop(ldpc):
    """Several codewords per block with varied iteration counts: lanes stop on their own,
    take the next codeword from the launch's work counter and start it at layer 0 while
    the other lane carries on; every codeword's bits and iteration count match the oracle,
    in three consecutive launches on one stream (the counter resets itself)."""
    n_sm = torch.cuda.get_device_properties(0).multi_processor_count
    B = 6 * n_sm + 11
    wl = make_workload("BG1", 40, B, 1.25, seed=23)
    q = wl.llr_int8()
    ref = oracle.decode_layered(wl.base, wl.K_b, 40, wl.n_rows, q, algo=oracle.OFFSET,
                                max_iter=10, early_stop=True, threads=8)
    assert len(np.unique(ref.iters)) >= 4               # the stopping rule is exercised
    g = ldpc.Graph(wl.base, wl.K_b, 40)
    t = torch.from_numpy(q).cuda()
    s = torch.cuda.Stream()
    nb = (wl.K + 7) // 8
    for rep in range(3):
        bits = torch.full((B, nb), 0xAB, dtype=torch.uint8, device="cuda")
        iters = torch.full((B,), -1, dtype=torch.int32, device="cuda")
        torch.cuda.synchronize()                        # the fills ran on another stream
        ldpc.decode(g, t, 10, early_stop=True, stream=s, bits=bits, iters=iters,
                    threads_per_row=1)
        torch.cuda.synchronize()
        assert np.array_equal(iters.cpu().numpy(), ref.iters), rep
        assert np.array_equal(_unpack(ldpc, bits.cpu().numpy(), wl.K), ref.bits), rep
    g.sync_status()
    g.close()


def test_batch_kernel_two_streams_share_a_graph(ldpc):
    """Decodes of one graph launched on two streams without a sync between them use
    separate work counters; both match the oracle."""
    n_sm = torch.cuda.get_device_properties(0).multi_processor_count
    B = 3 * n_sm
    wl = make_workload("BG2", 96, 2 * B, 1.0, seed=29)
    q = wl.llr_int8()
    ref = oracle.decode_layered(wl.base, wl.K_b, 96, wl.n_rows, q, algo=oracle.OFFSET,
                                max_iter=8, early_stop=True, threads=8)
    g = ldpc.Graph(wl.base, wl.K_b, 96)
    t = torch.from_numpy(q).cuda()
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    torch.cuda.synchronize()
    outs = []
    for k, s in enumerate(streams):
        outs.append(ldpc.decode(g, t[k * B:(k + 1) * B], 8, early_stop=True, stream=s,
                                threads_per_row=1))
    torch.cuda.synchronize()
    for k, (bits, iters) in enumerate(outs):
        sl = slice(k * B, (k + 1) * B)
        assert np.array_equal(iters.cpu().numpy(), ref.iters[sl]), k
        assert np.array_equal(_unpack(ldpc, bits.cpu().numpy(), wl.K), ref.bits[sl]), k
    g.close()


def test_batch_kernel_more_streams_than_counters(ldpc):
    """A graph has 64 work-counter pairs; decodes on further streams fall back to a fixed
    assignment of codewords to blocks and stay exact."""
    n_sm = torch.cuda.get_device_properties(0).multi_processor_count
    B = n_sm + 9                                   # beyond the low-latency range
    wl = make_workload("BG2", 32, B, 1.5, seed=31)
    q = wl.llr_int8()
    ref = oracle.decode_layered(wl.base, wl.K_b, 32, wl.n_rows, q, algo=oracle.OFFSET,
                                max_iter=6, early_stop=True, threads=8)
    g = ldpc.Graph(wl.base, wl.K_b, 32)
    t = torch.from_numpy(q).cuda()
    torch.cuda.synchronize()
    streams = [torch.cuda.Stream() for _ in range(70)]
    for k, s in enumerate(streams):
        bits, iters = ldpc.decode(g, t, 6, early_stop=True, stream=s, threads_per_row=1)
        s.synchronize()
        if k in (0, 63, 64, 69):
            assert np.array_equal(iters.cpu().numpy(), ref.iters), k
            assert np.array_equal(_unpack(ldpc, bits.cpu().numpy(), wl.K), ref.bits), k
    g.close()


# ------------------------------------------- cluster split (one codeword on two SMs)

@pytest.mark.parametrize("T", [1, 10])
def test_cluster_split_bit_exact(ldpc, T):
    """cluster_size 2: each codeword decoded by a pair of blocks that exchange posterior
    updates through distributed shared memory after every layer; every posterior, message,
    hard bit and iteration count equals the oracle's."""
    wl, q, ref = _ref_bg1(T)
    bits, iters, post, c2v = _gpu(ldpc, wl, q, T, early_stop=False, cluster_size=2)
    assert np.array_equal(post, ref.post)
    assert np.array_equal(c2v, ref.c2v)
    assert np.array_equal(_unpack(ldpc, bits, wl.K), ref.bits)
    assert (iters == T).all()


def test_cluster_split_early_stop_several_codewords(ldpc):
    """More codewords than clusters (each cluster decodes several in turn) with the stopping
    rule combined across the pair: iteration counts and bits match the oracle."""
    n_sm = torch.cuda.get_device_properties(0).multi_processor_count
    B = n_sm + 9
    wl = make_workload("BG1", 384, B, 1.5, seed=37)
    q = wl.llr_int8()
    ref = oracle.decode_layered(wl.base, wl.K_b, 384, wl.n_rows, q, algo=oracle.OFFSET,
                                max_iter=10, early_stop=True, threads=8)
    assert len(np.unique(ref.iters)) >= 3
    bits, iters = _gpu(ldpc, wl, q, 10, early_stop=True, debug=False, cluster_size=2)
    assert np.array_equal(iters, ref.iters)
    assert np.array_equal(_unpack(ldpc, bits, wl.K), ref.bits)


@pytest.mark.parametrize("kind,Z,rate", [("BG2", 4, None), ("BG1", 100, "2/3"),
                                         ("BG2", 256, "1/3")])
def test_cluster_split_other_shapes(ldpc, kind, Z, rate):
    """Small Z (one warp per block, spare threads) and other rates."""
    wl = make_workload(kind, Z, 5, 2.0, rate=None if rate is None else Fraction(rate), seed=Z)
    q = wl.llr_int8()
    ref = oracle.decode_layered(wl.base, wl.K_b, Z, wl.n_rows, q, algo=oracle.OFFSET,
                                max_iter=6, early_stop=True, want_post=True, want_c2v=True)
    bits, iters, post, c2v = _gpu(ldpc, wl, q, 6, early_stop=True, n_rows=wl.n_rows,
                                  n_tx=wl.n_tx, cluster_size=2)
    assert np.array_equal(iters, ref.iters)
    assert np.array_equal(post, ref.post)
    assert np.array_equal(c2v, ref.c2v)
    assert np.array_equal(_unpack(ldpc, bits, wl.K), ref.bits)


def test_cluster_split_row_maps_and_host_buffers(ldpc):
    """The cluster split through decode_rows (scattered pool rows in and out) and through the
    host-buffer entry point equals the oracle."""
    wl = make_workload("BG1", 96, 20, 1.75, seed=44)
    q = wl.llr_int8()
    g = ldpc.Graph(wl.base, wl.K_b, 96)
    perm = np.random.default_rng(4).permutation(20)
    in_rows = torch.tensor(perm[:12], dtype=torch.int32).cuda()
    out_rows = torch.tensor(perm[8:20], dtype=torch.int32).cuda()
    nb = (wl.K + 7) // 8
    bits = torch.zeros((20, nb), dtype=torch.uint8, device="cuda")
    iters = torch.full((20,), -1, dtype=torch.int32, device="cuda")
    ldpc.decode_rows(g, torch.from_numpy(q).cuda(), in_rows, out_rows, 6, bits=bits,
                     iters=iters, early_stop=True, cluster_size=2)
    torch.cuda.synchronize()
    ref = oracle.decode_layered(wl.base, wl.K_b, 96, wl.n_rows, q, algo=oracle.OFFSET,
                                max_iter=6, early_stop=True)
    assert np.array_equal(ldpc.unpack_bits(bits.cpu().numpy()[perm[8:20]], wl.K),
                          ref.bits[perm[:12]])
    assert np.array_equal(iters.cpu().numpy()[perm[8:20]], ref.iters[perm[:12]])
    hb, hi = ldpc.decode_host(g, torch.from_numpy(q), 6, early_stop=True, cluster_size=2)
    assert np.array_equal(ldpc.unpack_bits(hb.numpy(), wl.K), ref.bits)
    assert np.array_equal(hi.numpy(), ref.iters)
    g.close()


def test_cluster_split_rejections(ldpc):
    wl = make_workload("BG2", 16, 2, 3.0, seed=1)
    g = ldpc.Graph(wl.base, wl.K_b, 16)
    q = torch.from_numpy(wl.llr_int8()).cuda()
    with pytest.raises(ldpc.LdpcError):
        ldpc.decode(g, q, 5, cluster_size=3)               # 1 or 2
    with pytest.raises(ldpc.LdpcError):
        ldpc.decode(g, q.float(), 5, cluster_size=2)       # int8 only
    with pytest.raises(ldpc.LdpcError):
        ldpc.decode(g, q, 5, cluster_size=2, threads_per_row=4)
    g.close()
    wl = make_workload("BG2", 18, 2, 3.0, seed=1)          # Z not a multiple of 4
    g = ldpc.Graph(wl.base, wl.K_b, 18)
    with pytest.raises(ldpc.LdpcError):
        ldpc.decode(g, torch.from_numpy(wl.llr_int8()).cuda(), 5, cluster_size=2)
    g.close()


# ------------------------------------------------- low-latency strategy (alpha threads)

def test_low_latency_batch_beyond_sm_count(ldpc):
    """alpha = 2 asked for on a batch larger than the SM count: each block loops over several
    codewords, staging the next one's LLRs while it decodes; sampled codewords and every
    iteration count match the oracle."""
    n_sm = torch.cuda.get_device_properties(0).multi_processor_count
    B = 2 * n_sm + 7
    wl = make_workload("BG2", 128, B, 1.5, seed=21)
    q = wl.llr_int8()
    bits, iters = _gpu(ldpc, wl, q, 8, early_stop=True, debug=False, threads_per_row=2)
    rng = np.random.default_rng(1)
    idx = np.sort(rng.choice(B, 24, replace=False))
    idx[-1] = B - 1
    ref = oracle.decode_layered(wl.base, wl.K_b, 128, wl.n_rows, q[idx], algo=oracle.OFFSET,
                                max_iter=8, early_stop=True, threads=8)
    assert np.array_equal(_unpack(ldpc, bits, wl.K)[idx], ref.bits)
    assert np.array_equal(iters[idx], ref.iters)


def test_low_latency_row_maps(ldpc):
    """decode_rows through the alpha = 4 kernel: scattered pool rows in, scattered rows out."""
    wl = make_workload("BG1", 96, 20, 1.75, seed=8)
    q = wl.llr_int8()
    g = ldpc.Graph(wl.base, wl.K_b, 96)
    perm = np.random.default_rng(3).permutation(20)
    in_rows = torch.tensor(perm[:12], dtype=torch.int32).cuda()
    out_rows = torch.tensor(perm[8:20], dtype=torch.int32).cuda()
    nb = (wl.K + 7) // 8
    bits = torch.zeros((20, nb), dtype=torch.uint8, device="cuda")
    iters = torch.full((20,), -1, dtype=torch.int32, device="cuda")
    ldpc.decode_rows(g, torch.from_numpy(q).cuda(), in_rows, out_rows, 6, bits=bits,
                     iters=iters, early_stop=True, threads_per_row=4)
    torch.cuda.synchronize()
    ref = oracle.decode_layered(wl.base, wl.K_b, 96, wl.n_rows, q[perm[:12]],
                                algo=oracle.OFFSET, max_iter=6, early_stop=True)
    got = ldpc.unpack_bits(bits.cpu().numpy()[perm[8:20]], wl.K)
    assert np.array_equal(got, ref.bits)
    assert np.array_equal(iters.cpu().numpy()[perm[8:20]], ref.iters)
    g.close()


def test_every_alpha_decodes_a_lone_codeword_exactly(ldpc):
    """A lone codeword (the latency case), 10 iterations: the library's choice (0), the
    high-throughput kernel (1) and the low-latency kernel (2, 4) all give the oracle's
    posteriors and bits."""
    wl = make_workload("BG1", 384, 1, 1.5, seed=9)
    q = wl.llr_int8()
    ref = oracle.decode_layered(wl.base, wl.K_b, 384, wl.n_rows, q, algo=oracle.OFFSET,
                                max_iter=10, early_stop=False, want_post=True)
    for tpr in (0, 1, 2, 4):
        bits, iters, post, _ = _gpu(ldpc, wl, q, 10, early_stop=False, threads_per_row=tpr)
        assert np.array_equal(post, ref.post), tpr
        assert np.array_equal(_unpack(ldpc, bits, wl.K), ref.bits), tpr


# ------------------------------------------------------------------ host-buffer entry point

@pytest.mark.parametrize("B,pinned", [(700, True), (40, False), (1, True)])
def test_decode_host_equals_device_decode(ldpc, B, pinned):
    """ldpc_decode_host uploads in wave-sized chunks that overlap the decodes (700 = two full
    chunks and a ragged one); results equal the device-buffer decode, from pinned or pageable
    host memory."""
    wl = make_workload("BG1", 128, B, 1.75, seed=B)
    q = wl.llr_int8()
    g = ldpc.Graph(wl.base, wl.K_b, 128)
    host = torch.from_numpy(q)
    if pinned:
        host = host.pin_memory()
    hb, hi = ldpc.decode_host(g, host, 8, early_stop=True)
    db, di = ldpc.decode(g, torch.from_numpy(q).cuda(), 8, early_stop=True)
    torch.cuda.synchronize()
    assert np.array_equal(hb.numpy(), db.cpu().numpy())
    assert np.array_equal(hi.numpy(), di.cpu().numpy())
    ref = oracle.decode_layered(wl.base, wl.K_b, 128, wl.n_rows, q[:8], algo=oracle.OFFSET,
                                max_iter=8, early_stop=True, threads=8)
    assert np.array_equal(ldpc.unpack_bits(hb.numpy()[:8], wl.K), ref.bits)
    g.close()


# ------------------------------------------------------- bounded waits (failure handling)

def test_bounded_wait_times_out_and_context_survives(ldpc):
    """A barrier armed for a transfer that never comes: the bounded wait gives up and reports
    LDPC_ERR_TIMEOUT (no trap, no hang), and the next decode on the same context is exact."""
    st, cycles = ldpc.selftest_wait_timeout(1 << 14)
    assert st == 5                                   # LDPC_ERR_TIMEOUT
    assert cycles > 0
    wl = make_workload("BG1", 64, 4, 2.0, seed=5)
    q = wl.llr_int8()
    bits, iters = _gpu(ldpc, wl, q, 3, early_stop=False, debug=False)
    ref = oracle.decode_layered(wl.base, wl.K_b, 64, wl.n_rows, q, algo=oracle.OFFSET,
                                max_iter=3, early_stop=False)
    assert np.array_equal(_unpack(ldpc, bits, wl.K), ref.bits)
