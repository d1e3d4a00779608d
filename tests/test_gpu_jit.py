"""The batch kernel compiled for a graph's row sequence (ldpc_pair_jit, blocking mode)
against the CPU oracle: bit-exact hard bits, iteration counts, final posteriors and
check-to-variable messages, at the headline size and on shapes whose rows start and end
mid-column (odd degrees, odd E), with and without the stopping rule.  The generic kernel
(compilation off) is run beside it on the same inputs."""
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
    prev = pkg.pair_jit(2) & 3
    yield pkg
    pkg.pair_jit(prev)


def _decode(ldpc, wl, q, T, *, early_stop, debug=True):
    g = ldpc.Graph(wl.base, wl.K_b, wl.Z)
    out = ldpc.decode(g, torch.from_numpy(np.ascontiguousarray(q)).cuda(), T,
                      early_stop=early_stop, n_rows=wl.n_rows, n_tx=wl.n_tx, debug=debug,
                      threads_per_row=1)
    torch.cuda.synchronize()
    g.sync_status()
    g.close()
    return [o.cpu().numpy() for o in out]


def _oracle(wl, q, T, early_stop, debug=True):
    return oracle.decode_layered(wl.base, wl.K_b, wl.Z, wl.n_rows, q,
                                 algo=oracle.OFFSET, offset_q=1, max_iter=T,
                                 early_stop=early_stop, want_post=debug, want_c2v=debug,
                                 threads=16)


@pytest.mark.parametrize("early_stop", [False, True])
def test_compiled_kernel_headline_batch(ldpc, early_stop):
    """BG1-shaped Z=384, 1024 codewords at 1.5 dB, T=10: the benchmark's launch."""
    wl = make_workload("BG1", 384, 1024, 1.5, seed=0)
    q = wl.llr_int8()
    bits, iters = _decode(ldpc, wl, q, 10, early_stop=early_stop, debug=False)
    assert ldpc.pair_jit(-1) & 4, "no kernel was compiled and loaded"
    assert not ldpc.pair_jit(-1) & 8, "a compilation failed"
    ref = _oracle(wl, q, 10, early_stop, debug=False)
    assert np.array_equal(ldpc.unpack_bits(bits, wl.K), ref.bits)
    assert np.array_equal(iters, ref.iters)


# odd and even Z, several rates (row counts), rows starting and ending mid-column
SHAPES = [("BG1", 384, None, 48, 1.25), ("BG2", 128, None, 96, 1.0),
          ("BG1", 13, None, 9, 2.0), ("BG1", 40, "1/2", 33, 2.5),
          ("BG2", 96, "1/3", 40, 2.0), ("BG1", 384, "8/9", 20, 5.5)]


@pytest.mark.parametrize("kind,Z,rate,B,ebn0", SHAPES)
@pytest.mark.parametrize("early_stop", [False, True])
def test_compiled_kernel_equals_oracle_and_generic(ldpc, kind, Z, rate, B, ebn0, early_stop):
    wl = make_workload(kind, Z, B, ebn0, rate=None if rate is None else Fraction(rate),
                       seed=Z + B)
    q = wl.llr_int8()
    T = 6
    got = _decode(ldpc, wl, q, T, early_stop=early_stop)
    ref = _oracle(wl, q, T, early_stop)
    assert np.array_equal(ldpc.unpack_bits(got[0], wl.K), ref.bits)
    assert np.array_equal(got[1], ref.iters)
    assert np.array_equal(got[2], ref.post)
    assert np.array_equal(got[3], ref.c2v)
    prev = ldpc.pair_jit(0) & 3
    try:
        gen = _decode(ldpc, wl, q, T, early_stop=early_stop)
    finally:
        ldpc.pair_jit(prev)
    for a, b in zip(got, gen):
        assert np.array_equal(a, b)


def test_background_mode_serves_and_then_switches(ldpc):
    """Mode 1: a new sequence decodes at once (generic kernel) while it compiles; once
    compiled, later decodes use the module; both give the oracle's results."""
    import time
    wl = make_workload("BG2", 160, 8, 2.0, seed=777)
    q = wl.llr_int8()
    ref = _oracle(wl, q, 4, True)
    ldpc.pair_jit(1)
    try:
        for k in range(40):
            got = _decode(ldpc, wl, q, 4, early_stop=True)
            assert np.array_equal(got[2], ref.post)
            assert np.array_equal(got[3], ref.c2v)
            time.sleep(0.25)
    finally:
        ldpc.pair_jit(2)


# binary16: the kernel compiled per row sequence and block shape against the generic one
F16_SHAPES = [("BG1", 384, None, 3, "normalised"), ("BG1", 384, "8/9", 40, "offset"),
              ("BG2", 128, None, 700, "learned"), ("BG1", 64, None, 20, "normalised")]


@pytest.mark.parametrize("kind,Z,rate,B,mode", F16_SHAPES)
def test_binary16_compiled_equals_generic(ldpc, kind, Z, rate, B, mode):
    """One, two and four codewords per block (messages all in TMEM, or partly in shared
    memory for the BG1-shaped Z=384 code at low rate); every output equal, bit for bit."""
    wl = make_workload(kind, Z, B, 2.5 if rate is None else 7.5,
                       rate=None if rate is None else Fraction(rate),
                       modulation="QPSK" if rate is None else "16QAM", seed=B)
    h = torch.from_numpy(wl.llr_fp16()).cuda()
    if mode == "normalised":
        kw = dict(algo=ldpc.NORMALISED, alpha=0.75)
    elif mode == "offset":
        kw = dict(algo=ldpc.OFFSET, offset=0.3)
    else:
        rng = np.random.default_rng(5)
        tab = np.zeros((6, wl.n_rows, 2), np.float32)
        tab[..., 0] = rng.uniform(0.4, 1.0, size=(6, wl.n_rows))
        tab[..., 1] = rng.uniform(0.0, 0.5, size=(6, wl.n_rows))
        kw = dict(algo=ldpc.LEARNED, learned=torch.from_numpy(tab).cuda())
    outs = []
    for m in (2, 0):
        prev = ldpc.pair_jit(m) & 3
        try:
            g = ldpc.Graph(wl.base, wl.K_b, wl.Z)
            o = ldpc.decode(g, h, 6, early_stop=True, n_rows=wl.n_rows, n_tx=wl.n_tx,
                            debug=True, **kw)
            torch.cuda.synchronize()
            g.sync_status()
            g.close()
            outs.append([x.cpu().numpy() for x in o])
        finally:
            ldpc.pair_jit(prev)
    for a, b in zip(*outs):
        assert np.array_equal(a.view(np.uint8), b.view(np.uint8))


def test_exit_during_background_compile_is_clean(ldpc):
    """A process that meets a new row sequence in the background mode and exits at once
    (the compilation still running) exits cleanly: the binding waits for it at exit."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    code = (
        "import sys, torch; sys.path.insert(0, %r)\n"
        "import paper_2009_05534_gb300 as ldpc\n"
        "from synth import make_workload\n"
        "ldpc.pair_jit(1)\n"
        "wl = make_workload('BG2', 96, 4, 2.0, seed=4242)\n"
        "g = ldpc.Graph(wl.base, wl.K_b, wl.Z)\n"
        "ldpc.decode(g, torch.from_numpy(wl.llr_int8()).cuda(), 5, threads_per_row=1)\n"
        "torch.cuda.synchronize()\n"
        "print('decoded', flush=True)\n" % root)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    assert "decoded" in r.stdout


@pytest.mark.parametrize("tpr", [2, 4])
@pytest.mark.parametrize("kind,Z,rate,B,ebn0", [("BG1", 384, None, 3, 1.25),
                                                ("BG2", 96, "1/3", 40, 2.0),
                                                ("BG1", 40, "1/2", 17, 2.5)])
def test_low_latency_compiled_equals_oracle_and_generic(ldpc, tpr, kind, Z, rate, B, ebn0):
    """The one-codeword low-latency kernel (alpha = 2, 4) compiled for the row sequence:
    every output against the oracle and the generic kernel, with the stopping rule."""
    wl = make_workload(kind, Z, B, ebn0, rate=None if rate is None else Fraction(rate),
                       seed=Z + B + tpr)
    q = wl.llr_int8()
    outs = []
    for m in (2, 0):
        prev = ldpc.pair_jit(m) & 3
        try:
            g = ldpc.Graph(wl.base, wl.K_b, wl.Z)
            o = ldpc.decode(g, torch.from_numpy(q).cuda(), 6, early_stop=True,
                            n_rows=wl.n_rows, n_tx=wl.n_tx, debug=True, threads_per_row=tpr)
            torch.cuda.synchronize()
            g.sync_status()
            g.close()
            outs.append([x.cpu().numpy() for x in o])
        finally:
            ldpc.pair_jit(prev)
    ref = _oracle(wl, q, 6, True)
    got = outs[0]
    assert np.array_equal(ldpc.unpack_bits(got[0], wl.K), ref.bits)
    assert np.array_equal(got[1], ref.iters)
    assert np.array_equal(got[2], ref.post)
    assert np.array_equal(got[3], ref.c2v)
    for a, b in zip(*outs):
        assert np.array_equal(a, b)
