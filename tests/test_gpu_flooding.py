"""Flooding-schedule decoder (fp32 min-sum and sum-product) against the oracle's flooding
decoder on the same seeded inputs.

Min-sum: the same binary32 operations in the same order, posteriors summed in base-row
order on both sides, so every posterior, hard bit and iteration count must agree exactly.
Sum-product: binary64 tanh / atanh on both sides from different math libraries, so the
hard bits must agree on >= 99.99 % of codewords and the posteriors within 1e-4 of max|L|.
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
    return pkg


def _both(ldpc, wl, T, algo_o, algo_g, *, early_stop, **kw):
    ref = oracle.decode_flooding(wl.base, wl.K_b, wl.Z, wl.n_rows, wl.llr, algo=algo_o,
                                 max_iter=T, early_stop=early_stop, want_post=True, threads=8,
                                 **kw)
    g = ldpc.Graph(wl.base, wl.K_b, wl.Z)
    bits, iters, post = ldpc.decode_flooding(g, torch.from_numpy(wl.llr).cuda(), T,
                                             algo=algo_g, early_stop=early_stop,
                                             n_rows=wl.n_rows, want_post=True, **kw)
    torch.cuda.synchronize()
    g.sync_status()
    out = (ldpc.unpack_bits(bits.cpu().numpy(), wl.K), iters.cpu().numpy(), post.cpu().numpy())
    g.close()
    return ref, out


@pytest.mark.parametrize("T", [1, 4, 12])
@pytest.mark.parametrize("mode", ["normalised", "offset"])
def test_min_sum_bit_exact(ldpc, T, mode):
    wl = make_workload("BG1", 64, 8, 2.0, seed=200 + T)
    kw = dict(alpha=0.75) if mode == "normalised" else dict(offset=0.25)
    a_o = oracle.NORMALISED if mode == "normalised" else oracle.OFFSET
    a_g = ldpc.NORMALISED if mode == "normalised" else ldpc.OFFSET
    ref, (bits, iters, post) = _both(ldpc, wl, T, a_o, a_g, early_stop=False, **kw)
    assert np.array_equal(post, ref.post)
    assert np.array_equal(bits, ref.bits)
    assert np.array_equal(iters, ref.iters)


def test_min_sum_early_stop_and_rate(ldpc):
    wl = make_workload("BG2", 96, 21, 3.5, seed=211, rate=Fraction(1, 3))
    ref, (bits, iters, post) = _both(ldpc, wl, 20, oracle.NORMALISED, ldpc.NORMALISED,
                                     early_stop=True, alpha=0.75)
    assert (ref.iters < 20).any()
    assert np.array_equal(iters, ref.iters)
    assert np.array_equal(bits, ref.bits)
    assert np.array_equal(post, ref.post)


@pytest.mark.parametrize("kind,Z", [("BG2", 32), ("BG1", 384)])
def test_sum_product_close(ldpc, kind, Z):
    wl = make_workload(kind, Z, 6, 1.5 if kind == "BG1" else 2.5, seed=220 + Z)
    ref, (bits, iters, post) = _both(ldpc, wl, 6, oracle.SUM_PRODUCT, ldpc.SUM_PRODUCT,
                                     early_stop=False)
    assert (bits == ref.bits).all(axis=1).mean() >= 0.9999
    tol = 1e-4 * float(np.abs(ref.post).max())
    assert np.abs(post - ref.post).max() <= tol


def test_rejects_non_fp32_and_learned(ldpc):
    wl = make_workload("BG2", 16, 2, 2.0, seed=1)
    g = ldpc.Graph(wl.base, wl.K_b, 16)
    with pytest.raises(ValueError):
        ldpc.decode_flooding(g, torch.from_numpy(wl.llr_fp16()).cuda(), 4)
    tab = torch.zeros((4, wl.n_rows, 2), device="cuda")
    with pytest.raises(ldpc.LdpcError):
        ldpc.decode_flooding(g, torch.from_numpy(wl.llr).cuda(), 4, algo=ldpc.LEARNED,
                             learned=tab)
    # sum-product is a flooding-only rule
    with pytest.raises(ldpc.LdpcError):
        ldpc.decode(g, torch.from_numpy(wl.llr).cuda(), 4, algo=ldpc.SUM_PRODUCT)
    g.close()
