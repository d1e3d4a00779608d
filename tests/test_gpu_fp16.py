"""binary16 decoder (messages in Tensor Memory) against the oracle's binary16 path.

Both sides perform the same IEEE binary16 operations in the same order with the correction
parameters rounded to binary16 once, so posteriors, messages, hard bits and iteration
counts must agree exactly (signed zeros compare equal).  Covers the three corrections,
early stop, the 16QAM/64QAM high-rate shape, the learned table at BG2 Z=128, ragged
batches and lifting sizes, the unstaged (n_tx not a multiple of 8) load, and the
one-codeword-per-block layout of large shapes (messages split between TMEM and shared
memory).  The kernels run here are the ones compiled for each row sequence and block
shape.
"""
from fractions import Fraction

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from synth import make_workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ldpc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2009_05534_gb300 import build
    build.build()
    import paper_2009_05534_gb300 as pkg
    # every decode here waits for the kernel compiled for its row sequence and block shape
    # (the generic kernel is checked against it in test_gpu_jit.py)
    prev = pkg.pair_jit(2) & 3
    yield pkg
    pkg.pair_jit(prev)


def _table(T, n_rows, seed):
    rng = np.random.default_rng(seed)
    t = np.zeros((T, n_rows, 2), np.float32)
    t[..., 0] = rng.uniform(0.4, 1.0, size=(T, n_rows))
    t[..., 1] = rng.uniform(0.0, 0.5, size=(T, n_rows))
    return t


def _run(ldpc, wl, T, mode, *, early_stop, n_tx=None, debug=True, seed=0):
    h = wl.llr_fp16()
    if n_tx is not None:
        h = np.ascontiguousarray(h[:, :n_tx])
    kw_o, kw_g = {}, {}
    if mode == "normalised":
        kw_o = dict(algo=oracle.NORMALISED, alpha=0.7)
        kw_g = dict(algo=ldpc.NORMALISED, alpha=0.7)
    elif mode == "normalised75":
        kw_o = dict(algo=oracle.NORMALISED, alpha=0.75)
        kw_g = dict(algo=ldpc.NORMALISED, alpha=0.75)
    elif mode == "offset":
        kw_o = dict(algo=oracle.OFFSET, offset=0.3)
        kw_g = dict(algo=ldpc.OFFSET, offset=0.3)
    else:
        tab = _table(T, wl.n_rows, seed)
        kw_o = dict(algo=oracle.LEARNED, learned=tab)
        kw_g = dict(algo=ldpc.LEARNED, learned=torch.from_numpy(tab).cuda())
    ntx = h.shape[1]
    ref = oracle.decode_layered(wl.base, wl.K_b, wl.Z, wl.n_rows, h, max_iter=T,
                                early_stop=early_stop, want_post=debug, want_c2v=debug,
                                threads=8, **kw_o)
    g = ldpc.Graph(wl.base, wl.K_b, wl.Z)
    out = ldpc.decode(g, torch.from_numpy(h).cuda(), T, early_stop=early_stop,
                      n_rows=wl.n_rows, n_tx=ntx, debug=debug, **kw_g)
    torch.cuda.synchronize()
    g.sync_status()
    res = [o.cpu().numpy() for o in out]
    g.close()
    return ref, res


def _check(ldpc, wl, ref, res, debug=True):
    bits, iters = res[0], res[1]
    assert np.array_equal(ldpc.unpack_bits(bits, wl.K), ref.bits)
    assert np.array_equal(iters, ref.iters)
    if debug:
        assert np.array_equal(res[2], ref.post)
        assert np.array_equal(res[3], ref.c2v)


@pytest.mark.parametrize("mode", ["normalised", "normalised75", "offset", "learned"])
@pytest.mark.parametrize("T", [1, 3, 8])
def test_bg1_z64_every_correction(ldpc, mode, T):
    wl = make_workload("BG1", 64, 10, 1.75, seed=40 + T)
    ref, res = _run(ldpc, wl, T, mode, early_stop=False, seed=T)
    _check(ldpc, wl, ref, res)


@pytest.mark.parametrize("mode", ["normalised75", "learned"])
def test_early_stop_iteration_counts(ldpc, mode):
    wl = make_workload("BG2", 64, 33, 3.0, seed=51)          # odd batch: an idle half
    ref, res = _run(ldpc, wl, 12, mode, early_stop=True, seed=5)
    assert (ref.iters < 12).any()
    _check(ldpc, wl, ref, res)


@pytest.mark.parametrize("mod", ["16QAM", "64QAM"])
def test_high_rate_qam_z384(ldpc, mod):
    """BG1-shaped Z=384 at rate 8/9 (5 rows) with max-log QAM LLRs, the high-load shape."""
    wl = make_workload("BG1", 384, 12, 4.5 if mod == "16QAM" else 7.0, rate=Fraction(8, 9),
                       modulation=mod, seed=61)
    ref, res = _run(ldpc, wl, 5, "normalised75", early_stop=False)
    _check(ldpc, wl, ref, res)


def test_learned_bg2_z128(ldpc):
    wl = make_workload("BG2", 128, 6, 2.0, seed=71, graph_seed=0)
    ref, res = _run(ldpc, wl, 10, "learned", early_stop=False, seed=7)
    _check(ldpc, wl, ref, res)


@pytest.mark.parametrize("Z", [2, 6, 30, 94, 382])
def test_ragged_lifting_sizes(ldpc, Z):
    """H = Z/2 not a multiple of 32 leaves spare threads in the last warp."""
    wl = make_workload("BG2", Z, 5, 2.5, seed=Z, rate=Fraction(1, 2) if Z > 100 else None)
    ref, res = _run(ldpc, wl, 4, "offset", early_stop=False)
    _check(ldpc, wl, ref, res)


def test_unstaged_load_and_shortened_tail(ldpc):
    """n_tx not a multiple of 8: the LLR rows are not 16-byte aligned, so they are read
    with plain loads; the bits beyond n_tx enter as zero LLRs."""
    wl = make_workload("BG1", 96, 7, 2.0, seed=81, rate=Fraction(2, 3))
    ref, res = _run(ldpc, wl, 4, "normalised75", early_stop=False, n_tx=wl.n_tx - 5)
    _check(ldpc, wl, ref, res)


@pytest.mark.parametrize("Z", [256, 320, 384])
def test_one_codeword_blocks(ldpc, Z):
    """BG1 at rate 1/3 needs more TMEM columns than two codewords' messages allow: one
    codeword per block, the first four warps' messages in TMEM and (Z = 320, 384) the
    remaining warps' messages in shared memory."""
    wl = make_workload("BG1", Z, 5, 1.5, seed=91)
    ref, res = _run(ldpc, wl, 3, "learned", early_stop=False, seed=9)
    _check(ldpc, wl, ref, res)


def test_large_batch_sampled(ldpc):
    """Batch 2048 at the high-rate shape (several codewords per block in turn); sampled
    codewords are decoded by the oracle one by one."""
    wl = make_workload("BG1", 384, 2048, 4.0, rate=Fraction(8, 9), modulation="16QAM", seed=3)
    h = wl.llr_fp16()
    g = ldpc.Graph(wl.base, wl.K_b, 384)
    bits, iters = ldpc.decode(g, torch.from_numpy(h).cuda(), 10, early_stop=True,
                              n_rows=wl.n_rows, algo=ldpc.NORMALISED, alpha=0.75)
    torch.cuda.synchronize()
    g.sync_status()
    gb = ldpc.unpack_bits(bits.cpu().numpy(), wl.K)
    it = iters.cpu().numpy()
    g.close()
    idx = np.sort(np.random.default_rng(1).choice(2048, 24, replace=False))
    ref = oracle.decode_layered(wl.base, wl.K_b, 384, wl.n_rows, h[idx], algo=oracle.NORMALISED,
                                alpha=0.75, max_iter=10, early_stop=True, threads=8)
    assert np.array_equal(gb[idx], ref.bits)
    assert np.array_equal(it[idx], ref.iters)


@pytest.mark.parametrize("kind,Z,mode", [("BG2", 128, "learned"), ("BG1", 64, "normalised75"),
                                         ("BG2", 94, "offset")])
def test_four_codeword_blocks_large_batch(ldpc, kind, Z, mode):
    """Batches larger than two codewords per SM at small Z run four codewords per block
    (BG2 Z=128: four warps' messages in TMEM, four in shared memory; BG1 Z=64: all in TMEM);
    sampled codewords match the oracle in every posterior and message."""
    B, T = 400, 6
    wl = make_workload(kind, Z, B, 2.0, seed=300 + Z, graph_seed=0)
    h = wl.llr_fp16()
    if mode == "learned":
        tab = _table(T, wl.n_rows, 12)
        kw_o, kw_g = (dict(algo=oracle.LEARNED, learned=tab),
                      dict(algo=ldpc.LEARNED, learned=torch.from_numpy(tab).cuda()))
    elif mode == "offset":
        kw_o, kw_g = dict(algo=oracle.OFFSET, offset=0.3), dict(algo=ldpc.OFFSET, offset=0.3)
    else:
        kw_o = dict(algo=oracle.NORMALISED, alpha=0.75)
        kw_g = dict(algo=ldpc.NORMALISED, alpha=0.75)
    g = ldpc.Graph(wl.base, wl.K_b, Z)
    bits, iters, post, c2v = ldpc.decode(g, torch.from_numpy(h).cuda(), T, early_stop=True,
                                         debug=True, **kw_g)
    torch.cuda.synchronize()
    g.sync_status()
    idx = np.sort(np.random.default_rng(Z).choice(B, 24, replace=False))
    ref = oracle.decode_layered(wl.base, wl.K_b, Z, wl.n_rows, h[idx], max_iter=T,
                                early_stop=True, want_post=True, want_c2v=True, threads=8,
                                **kw_o)
    assert np.array_equal(ldpc.unpack_bits(bits.cpu().numpy()[idx], wl.K), ref.bits)
    assert np.array_equal(iters.cpu().numpy()[idx], ref.iters)
    assert np.array_equal(post.cpu().numpy()[idx], ref.post)
    assert np.array_equal(c2v.cpu().numpy()[idx], ref.c2v)
    g.close()
