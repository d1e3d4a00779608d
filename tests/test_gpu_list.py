"""Work-list decode (heterogeneous batches in one launch) against the oracle and against the
same codewords decoded alone."""
from fractions import Fraction

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from synth import make_workload

pytestmark = pytest.mark.gpu

ZS = (32, 64, 96, 128, 192, 256, 384)
RATES = {"BG1": ("1/3", "1/2", "2/3", "5/6", "8/9"), "BG2": ("1/5", "1/3", "1/2", "2/3", "5/6")}


@pytest.fixture(scope="module")
def ldpc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2009_05534_gb300 import build
    build.build()
    import paper_2009_05534_gb300 as pkg
    return pkg


def _mixed(ldpc, n, seed):
    rng = np.random.default_rng(seed)
    graphs, items, refs = {}, [], []
    for k in range(n):
        kind = "BG1" if rng.integers(2) else "BG2"
        Z = int(rng.choice(ZS))
        rate = Fraction(str(rng.choice(RATES[kind])))
        T = int(rng.choice([3, 6, 10]))
        wl = make_workload(kind, Z, 1, float(rng.uniform(0.5, 4.0)), rate=rate, seed=seed + k,
                           graph_seed=0)
        key = (kind, Z)
        if key not in graphs:
            graphs[key] = ldpc.Graph(wl.base, wl.K_b, Z)
        q = wl.llr_int8()
        llr = torch.from_numpy(q[0]).cuda()
        bits = torch.zeros(((wl.K + 7) // 8,), dtype=torch.uint8, device="cuda")
        it = torch.zeros((1,), dtype=torch.int32, device="cuda")
        items.append((graphs[key], llr, bits, it, wl.n_rows, wl.n_tx, T))
        refs.append((wl, q, T))
    return graphs, items, refs


@pytest.mark.parametrize("early_stop", [False, True])
def test_list_matches_oracle_and_alone(ldpc, early_stop):
    graphs, items, refs = _mixed(ldpc, 40, 100 + int(early_stop))
    ldpc.decode_list(items, early_stop=early_stop)
    torch.cuda.synchronize()
    for (g, llr, bits, it, n_rows, n_tx, T), (wl, q, _) in zip(items, refs):
        ref = oracle.decode_layered(wl.base, wl.K_b, wl.Z, wl.n_rows, q, algo=oracle.OFFSET,
                                    max_iter=T, early_stop=early_stop)
        got = ldpc.unpack_bits(bits.cpu().numpy()[None, :], wl.K)
        assert np.array_equal(got, ref.bits)
        assert int(it.item()) == int(ref.iters[0])
        # the same codeword decoded alone through the batch entry point
        b1, i1 = ldpc.decode(g, llr[None, :], T, n_rows=n_rows, n_tx=n_tx,
                             early_stop=early_stop)
        torch.cuda.synchronize()
        assert np.array_equal(b1.cpu().numpy()[0], bits.cpu().numpy())
        assert int(i1.item()) == int(it.item())
    for g in graphs.values():
        g.close()


def test_list_back_to_back_and_empty(ldpc):
    graphs, items, refs = _mixed(ldpc, 12, 7)
    ldpc.decode_list([])
    for _ in range(3):                    # reuse of the per-stream work table
        for (_, _, bits, it, *_r) in items:
            bits.zero_()
            it.zero_()
        ldpc.decode_list(items, early_stop=False)
    torch.cuda.synchronize()
    for (g, llr, bits, it, n_rows, n_tx, T), (wl, q, _) in zip(items, refs):
        ref = oracle.decode_layered(wl.base, wl.K_b, wl.Z, wl.n_rows, q, algo=oracle.OFFSET,
                                    max_iter=T, early_stop=False)
        assert np.array_equal(ldpc.unpack_bits(bits.cpu().numpy()[None, :], wl.K), ref.bits)
    for g in graphs.values():
        g.close()


def test_list_rejects_unsupported(ldpc):
    wl = make_workload("BG2", 13, 1, 2.0, seed=1)          # odd Z
    g = ldpc.Graph(wl.base, wl.K_b, 13)
    llr = torch.from_numpy(wl.llr_int8()[0]).cuda()
    bits = torch.zeros(((wl.K + 7) // 8,), dtype=torch.uint8, device="cuda")
    it = torch.zeros((1,), dtype=torch.int32, device="cuda")
    with pytest.raises(ldpc.LdpcError):
        ldpc.decode_list([(g, llr, bits, it, 0, 0, 5)])
    g.close()


@pytest.mark.parametrize("dtype", ["int8", "fp16", "fp32"])
def test_decode_rows_equals_gathered_batch(ldpc, dtype):
    """Row-mapped decode: codeword b reads pool row in_rows[b] and writes output row
    out_rows[b]; equal to decoding the gathered rows as a plain batch."""
    wl = make_workload("BG1", 128, 40, 2.0, seed=17, graph_seed=0)
    host = {"int8": wl.llr_int8(), "fp16": wl.llr_fp16(), "fp32": wl.llr}[dtype]
    kw = {} if dtype == "int8" else dict(algo=ldpc.NORMALISED, alpha=0.75)
    g = ldpc.Graph(wl.base, wl.K_b, 128)
    pool = torch.from_numpy(host).cuda()
    rng = np.random.default_rng(5)
    in_rows = rng.choice(40, 25, replace=False).astype(np.int32)
    out_rows = rng.permutation(64)[:25].astype(np.int32)
    nb = (wl.K + 7) // 8
    bits = torch.zeros((64, nb), dtype=torch.uint8, device="cuda")
    iters = torch.zeros((64,), dtype=torch.int32, device="cuda")
    ldpc.decode_rows(g, pool, torch.from_numpy(in_rows).cuda(), torch.from_numpy(out_rows).cuda(),
                     6, bits=bits, iters=iters, **kw)
    ref_b, ref_i = ldpc.decode(g, pool[torch.from_numpy(in_rows).long().cuda()], 6, **kw)
    torch.cuda.synchronize()
    assert np.array_equal(bits.cpu().numpy()[out_rows], ref_b.cpu().numpy())
    assert np.array_equal(iters.cpu().numpy()[out_rows], ref_i.cpu().numpy())
    untouched = np.setdiff1d(np.arange(64), out_rows)
    assert (bits.cpu().numpy()[untouched] == 0).all()
    with pytest.raises(ValueError):
        ldpc.decode_rows(g, pool, torch.tensor([40], dtype=torch.int32, device="cuda"),
                         torch.tensor([0], dtype=torch.int32, device="cuda"), 6, bits=bits,
                         iters=iters, **kw)
    g.close()
