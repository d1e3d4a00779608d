"""Shapes the specialised kernels do not take: lifting sizes above 384 (up to the ABI's
1024) and binary16 at odd Z.  They run on the generic kernel (one thread per check row,
the codeword's posteriors and messages in shared memory, a block barrier per layer; Sec. III
layered schedule).  Every output against the oracle: bit-exact for int8, binary16 and fp32
(the same operations in the same order on both sides), with and without the stopping rule.
A shape whose codeword state does not fit in shared memory is rejected on the host before
any launch, and the graph stays usable."""
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


def _decode(ldpc, wl, llr, T, early_stop, **kw):
    g = ldpc.Graph(wl.base, wl.K_b, wl.Z)
    out = ldpc.decode(g, torch.from_numpy(np.ascontiguousarray(llr)).cuda(), T,
                      early_stop=early_stop, n_rows=wl.n_rows, n_tx=wl.n_tx, debug=True, **kw)
    torch.cuda.synchronize()
    g.sync_status()
    g.close()
    return [o.cpu().numpy() for o in out]


def _check(ldpc, wl, got, ref):
    assert np.array_equal(ldpc.unpack_bits(got[0], wl.K), ref.bits)
    assert np.array_equal(got[1], ref.iters)
    assert np.array_equal(got[2], ref.post)
    assert np.array_equal(got[3], ref.c2v)


# (kind, Z, rate, Eb/N0): Z = 1024 is the largest lifting size the ABI takes; 450 is even
# and above the specialised kernels' 384
INT8 = [("BG2", 1024, "2/3", 2.5), ("BG1", 1024, "8/9", 5.0), ("BG2", 450, "1/2", 2.0)]


@pytest.mark.parametrize("kind,Z,rate,ebn0", INT8)
@pytest.mark.parametrize("early_stop", [False, True])
def test_int8_beyond_384(ldpc, kind, Z, rate, ebn0, early_stop):
    wl = make_workload(kind, Z, 6, ebn0, rate=Fraction(rate), seed=Z + 7)
    q = wl.llr_int8()
    T = 6
    ref = oracle.decode_layered(wl.base, wl.K_b, Z, wl.n_rows, q, algo=oracle.OFFSET,
                                offset_q=1, max_iter=T, early_stop=early_stop,
                                want_post=True, want_c2v=True, threads=8)
    _check(ldpc, wl, _decode(ldpc, wl, q, T, early_stop), ref)


# binary16: odd Z (the specialised kernel needs row pairs) and Z above 384
F16 = [("BG2", 13, None, 2.0), ("BG2", 385, "1/2", 2.0), ("BG2", 512, "1/2", 2.0)]


@pytest.mark.parametrize("kind,Z,rate,ebn0", F16)
@pytest.mark.parametrize("early_stop", [False, True])
def test_binary16_odd_and_beyond_384(ldpc, kind, Z, rate, ebn0, early_stop):
    wl = make_workload(kind, Z, 5, ebn0, rate=None if rate is None else Fraction(rate),
                       seed=Z + 3)
    h = wl.llr_fp16()
    T = 5
    ref = oracle.decode_layered(wl.base, wl.K_b, Z, wl.n_rows, h, algo=oracle.NORMALISED,
                                alpha=0.75, max_iter=T, early_stop=early_stop,
                                want_post=True, want_c2v=True, threads=8)
    _check(ldpc, wl, _decode(ldpc, wl, h, T, early_stop, algo=ldpc.NORMALISED, alpha=0.75),
           ref)


def test_fp32_odd_z_beyond_384(ldpc):
    """Z = 449: odd and above 384, so the last warp of the block has idle threads."""
    wl = make_workload("BG2", 449, 5, 2.0, rate=Fraction(2, 3), modulation="BPSK", seed=449)
    T = 6
    ref = oracle.decode_layered(wl.base, wl.K_b, 449, wl.n_rows, wl.llr,
                                algo=oracle.NORMALISED, alpha=0.75, max_iter=T,
                                early_stop=True, want_post=True, want_c2v=True, threads=8)
    _check(ldpc, wl, _decode(ldpc, wl, wl.llr, T, True, algo=ldpc.NORMALISED, alpha=0.75),
           ref)


def test_state_beyond_shared_memory_is_rejected(ldpc):
    """BG1-shaped Z = 1024 at rate 1/3 holds 316 edges x 1024 message bytes, more than a
    block's shared memory: LDPC_ERR_UNSUPPORTED from the host, nothing launched; the same
    graph then decodes its rate-8/9 rows exactly."""
    wl = make_workload("BG1", 1024, 2, 2.0, seed=1031)
    hi = make_workload("BG1", 1024, 3, 5.0, rate=Fraction(8, 9), seed=1031)
    assert np.array_equal(wl.base, hi.base)
    g = ldpc.Graph(wl.base, wl.K_b, 1024)
    launches = ldpc.launch_count()
    with pytest.raises(ldpc.LdpcError):
        ldpc.decode(g, torch.from_numpy(wl.llr_int8()).cuda(), 5, n_rows=wl.n_rows,
                    n_tx=wl.n_tx)
    assert ldpc.launch_count() == launches
    qh = hi.llr_int8()
    out = ldpc.decode(g, torch.from_numpy(qh).cuda(), 4, early_stop=True, n_rows=hi.n_rows,
                      n_tx=hi.n_tx, debug=True)
    torch.cuda.synchronize()
    g.sync_status()
    g.close()
    ref = oracle.decode_layered(hi.base, hi.K_b, 1024, hi.n_rows, qh, algo=oracle.OFFSET,
                                offset_q=1, max_iter=4, early_stop=True, want_post=True,
                                want_c2v=True, threads=8)
    _check(ldpc, hi, [o.cpu().numpy() for o in out], ref)
