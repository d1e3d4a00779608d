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


@pytest.mark.parametrize("tpr", [1, 2])
@pytest.mark.parametrize("early_stop", [False, True])
def test_list_matches_oracle_and_alone(ldpc, early_stop, tpr):
    """Each list kernel (tpr 1: one thread per row pair; 2: the low-latency one) against
    the oracle, and against the same codeword decoded alone."""
    graphs, items, refs = _mixed(ldpc, 40, 100 + int(early_stop))
    ldpc.decode_list(items, early_stop=early_stop, threads_per_row=tpr)
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


@pytest.mark.parametrize("tpr", [0, 1, 2])
def test_list_back_to_back_and_empty(ldpc, tpr):
    graphs, items, refs = _mixed(ldpc, 12, 7)
    ldpc.decode_list([], threads_per_row=tpr)
    for _ in range(3):                    # reuse of the per-stream work table
        for (_, _, bits, it, *_r) in items:
            bits.zero_()
            it.zero_()
        ldpc.decode_list(items, early_stop=False, threads_per_row=tpr)
    torch.cuda.synchronize()
    for (g, llr, bits, it, n_rows, n_tx, T), (wl, q, _) in zip(items, refs):
        ref = oracle.decode_layered(wl.base, wl.K_b, wl.Z, wl.n_rows, q, algo=oracle.OFFSET,
                                    max_iter=T, early_stop=False)
        assert np.array_equal(ldpc.unpack_bits(bits.cpu().numpy()[None, :], wl.K), ref.bits)
    for g in graphs.values():
        g.close()


def test_list_words_equals_record_array(ldpc):
    """The raw-word entry of the work list (the serving path's) decodes the same items as
    the record-array entry, and rejects arrays of the wrong shape or type."""
    graphs, items, refs = _mixed(ldpc, 24, 31)
    arr = np.zeros(len(items), dtype=ldpc.work_item_dtype)
    for k, (g, llr, bits, it, n_rows, n_tx, T) in enumerate(items):
        arr[k] = (g.handle.value, llr.data_ptr(), bits.data_ptr(), it.data_ptr(), n_rows,
                  n_tx, T)
    ldpc.decode_list_array(arr, early_stop=True)
    torch.cuda.synchronize()
    first = [(bits.cpu().numpy().copy(), int(it.item())) for (_, _, bits, it, *_r) in items]
    for (_, _, bits, it, *_r) in items:
        bits.zero_()
        it.zero_()
    words = arr.view(np.uint64).reshape(len(arr), ldpc.WORK_ITEM_WORDS)
    ldpc.decode_list_words(np.take(words, np.arange(len(arr)), axis=0), early_stop=True)
    torch.cuda.synchronize()
    for (b0, i0), (_, _, bits, it, *_r) in zip(first, items):
        assert np.array_equal(bits.cpu().numpy(), b0) and int(it.item()) == i0
    with pytest.raises(ValueError):
        ldpc.decode_list_words(words[:, :5].copy())
    with pytest.raises(ValueError):
        ldpc.decode_list_words(words.astype(np.int64))
    for g in graphs.values():
        g.close()


def test_list_small_lifting_sizes_and_many_items(ldpc):
    """Lifting sizes down to 2 (a single row pair: one busy warp, the rest of the block at
    the barriers only) and more items than SMs (blocks take several items in turn), low-
    latency list kernel against the one-thread kernel and the oracle."""
    rng = np.random.default_rng(77)
    graphs, items, refs = {}, [], []
    n_sm = torch.cuda.get_device_properties(0).multi_processor_count
    for k in range(n_sm + 40):
        Z = int(rng.choice([2, 4, 6, 10, 36, 384]))
        kind = "BG1" if rng.integers(2) else "BG2"
        wl = make_workload(kind, Z, 1, float(rng.uniform(0.0, 4.0)), seed=500 + k,
                           graph_seed=0)
        if (kind, Z) not in graphs:
            graphs[(kind, Z)] = ldpc.Graph(wl.base, wl.K_b, Z)
        q = wl.llr_int8()
        llr = torch.from_numpy(q[0]).cuda()
        bits = torch.zeros(((wl.K + 7) // 8,), dtype=torch.uint8, device="cuda")
        it = torch.zeros((1,), dtype=torch.int32, device="cuda")
        items.append((graphs[(kind, Z)], llr, bits, it, wl.n_rows, wl.n_tx, 6))
        refs.append((wl, q))
    outs = {}
    for tpr in (1, 2):
        for (_, _, bits, it, *_r) in items:
            bits.zero_()
            it.zero_()
        ldpc.decode_list(items, early_stop=True, threads_per_row=tpr)
        torch.cuda.synchronize()
        outs[tpr] = [(bits.cpu().numpy().copy(), int(it.item())) for (_, _, bits, it, *_r) in items]
    for k, ((wl, q), (b2, i2)) in enumerate(zip(refs, outs[2])):
        assert np.array_equal(b2, outs[1][k][0]) and i2 == outs[1][k][1]
        if k % 8 == 0:
            ref = oracle.decode_layered(wl.base, wl.K_b, wl.Z, wl.n_rows, q, algo=oracle.OFFSET,
                                        max_iter=6, early_stop=True)
            assert np.array_equal(ldpc.unpack_bits(b2[None, :], wl.K), ref.bits)
            assert i2 == int(ref.iters[0])
    for g in graphs.values():
        g.close()


def test_list_llr_rows_at_every_byte_alignment(ldpc):
    """Items whose LLR rows start at every offset modulo 16 inside one device buffer (the
    low-latency list kernel stages a row with 16-byte loads of its aligned middle and byte
    loads of both ragged ends): both list kernels against each other and the oracle."""
    rng = np.random.default_rng(41)
    graphs, wls, offs = {}, [], []
    pos = 0
    for k in range(32):
        kind = "BG1" if k % 2 else "BG2"
        Z = int(rng.choice([6, 32, 96, 384]))
        rate = Fraction(str(rng.choice(RATES[kind])))
        wl = make_workload(kind, Z, 1, float(rng.uniform(0.5, 3.0)), rate=rate, seed=900 + k,
                           graph_seed=0)
        if (kind, Z) not in graphs:
            graphs[(kind, Z)] = ldpc.Graph(wl.base, wl.K_b, Z)
        pos += (k % 16 - pos) % 16                   # row k starts at offset k mod 16
        offs.append(pos)
        wls.append(wl)
        pos += wl.n_tx
    host = np.zeros(pos + 16, np.int8)
    qs = []
    for wl, o in zip(wls, offs):
        q = wl.llr_int8()
        host[o:o + wl.n_tx] = q[0]
        qs.append(q)
    buf = torch.from_numpy(host).cuda()
    assert sorted({(buf.data_ptr() + o) % 16 for o in offs}) == list(range(16))
    outs = {}
    for tpr in (1, 2):
        items = []
        for wl, o in zip(wls, offs):
            bits = torch.zeros(((wl.K + 7) // 8,), dtype=torch.uint8, device="cuda")
            it = torch.zeros((1,), dtype=torch.int32, device="cuda")
            items.append((graphs[(wl.kind, wl.Z)], buf[o:o + wl.n_tx], bits, it, wl.n_rows,
                          wl.n_tx, 7))
        ldpc.decode_list(items, early_stop=True, threads_per_row=tpr)
        torch.cuda.synchronize()
        outs[tpr] = [(b.cpu().numpy(), int(i.item())) for (_, _, b, i, *_r) in items]
    for k, (wl, q) in enumerate(zip(wls, qs)):
        assert np.array_equal(outs[2][k][0], outs[1][k][0]) and outs[2][k][1] == outs[1][k][1]
        if k % 4 == 0:
            ref = oracle.decode_layered(wl.base, wl.K_b, wl.Z, wl.n_rows, q, algo=oracle.OFFSET,
                                        max_iter=7, early_stop=True)
            assert np.array_equal(ldpc.unpack_bits(outs[2][k][0][None, :], wl.K), ref.bits)
            assert outs[2][k][1] == int(ref.iters[0])
    for g in graphs.values():
        g.close()


def test_list_dense_graph_falls_back(ldpc):
    """A graph whose messages do not fit the low-latency kernel's Tensor Memory at two
    threads per row pair (52 rows of degree 19 at Z = 160: 520 slots, two warps per lane
    quarter) decodes through the one-thread kernel by default; asking for the low-latency
    kernel is refused, and so are 3 (invalid) and 4 threads per row pair (unsupported)."""
    rng = np.random.default_rng(3)
    M, K_b, Z = 52, 20, 160
    base = np.full((M, K_b + M), -1, np.int16)
    for r in range(M):
        cols = rng.choice(K_b + M, 19, replace=False)
        base[r, cols] = rng.integers(0, Z, 19)
    g = ldpc.Graph(base, K_b, Z)
    n_tx = (K_b + M - 2) * Z
    llr = torch.from_numpy(rng.integers(-20, 21, size=n_tx).astype(np.int8)).cuda()
    res = {}
    for tpr in (0, 1):
        bits = torch.zeros(((K_b * Z + 7) // 8,), dtype=torch.uint8, device="cuda")
        it = torch.zeros((1,), dtype=torch.int32, device="cuda")
        ldpc.decode_list([(g, llr, bits, it, M, n_tx, 5)], early_stop=False, threads_per_row=tpr)
        torch.cuda.synchronize()
        res[tpr] = (bits.cpu().numpy(), int(it.item()))
    assert np.array_equal(res[0][0], res[1][0]) and res[0][1] == res[1][1] == 5
    ref = oracle.decode_layered(base, K_b, Z, M, llr.cpu().numpy()[None, :], algo=oracle.OFFSET,
                                max_iter=5, early_stop=False)
    assert np.array_equal(ldpc.unpack_bits(res[0][0][None, :], K_b * Z), ref.bits)
    for tpr in (2, 3, 4):
        with pytest.raises(ldpc.LdpcError):
            ldpc.decode_list([(g, llr, bits, it, M, n_tx, 5)], threads_per_row=tpr)
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


@pytest.mark.parametrize("dtype", ["int8", "fp16"])
def test_decode_rows_host_maps_equals_gathered_batch(ldpc, dtype):
    """Row maps from host memory (the library stages and uploads them): several calls in a
    row on one stream, the last one larger than the first staging allocation, each equal
    to decoding its gathered rows as a plain batch; a negative row is rejected."""
    wl = make_workload("BG2", 64, 300, 1.5, seed=23, graph_seed=0)
    host = {"int8": wl.llr_int8(), "fp16": wl.llr_fp16()}[dtype]
    kw = {} if dtype == "int8" else dict(algo=ldpc.NORMALISED, alpha=0.75)
    g = ldpc.Graph(wl.base, wl.K_b, 64)
    pool = torch.from_numpy(host).cuda()
    nb = (wl.K + 7) // 8
    s = torch.cuda.Stream()
    rng = np.random.default_rng(9)
    outs = []
    for n in (17, 200, 290):
        in_rows = rng.choice(300, n, replace=False).astype(np.int32)
        out_rows = rng.permutation(320)[:n].astype(np.int32)
        bits = torch.zeros((320, nb), dtype=torch.uint8, device="cuda")
        iters = torch.zeros((320,), dtype=torch.int32, device="cuda")
        ldpc.decode_rows_host_maps(g, pool, in_rows, out_rows, 8, bits=bits, iters=iters,
                                   stream=s, **kw)
        outs.append((bits, iters, in_rows.copy(), out_rows))
        in_rows[:] = -7                   # the maps are read before the call returns
    torch.cuda.synchronize()
    for bits, iters, in_rows, out_rows in outs:
        ref_b, ref_i = ldpc.decode(g, pool[torch.from_numpy(in_rows).long().cuda()], 8, **kw)
        assert np.array_equal(bits.cpu().numpy()[out_rows], ref_b.cpu().numpy())
        assert np.array_equal(iters.cpu().numpy()[out_rows], ref_i.cpu().numpy())
        untouched = np.setdiff1d(np.arange(320), out_rows)
        assert (bits.cpu().numpy()[untouched] == 0).all()
    with pytest.raises(ldpc.LdpcError):
        ldpc.decode_rows_host_maps(g, pool, np.array([3, -1], np.int32),
                                   np.array([0, 1], np.int32), 8, bits=bits, iters=iters, **kw)
    g.close()


@pytest.mark.parametrize("early_stop", [False, True])
def test_compiled_list_kernel_matches_oracle(ldpc, early_stop):
    """The work-list kernel compiled for the BG1 row sequences (ldpc_list_jit_prepare): a
    mixed list whose BG1 items run compiled row sequences and whose BG2 items take the
    generic row loop in the same launch; every item against the oracle."""
    tabs = []
    for rate in RATES["BG1"]:
        wl = make_workload("BG1", 64, 1, 2.0, rate=Fraction(rate), seed=0, graph_seed=0)
        tabs.append((wl.base, wl.n_rows))
    ldpc.list_jit_prepare(tabs)
    try:
        graphs, items, refs = _mixed(ldpc, 48, 300 + int(early_stop))
        assert any(wl.kind == "BG1" for wl, _, _ in refs)
        assert any(wl.kind == "BG2" for wl, _, _ in refs)
        for rep in range(2):                         # the first call loads the module
            for _, _, bits, it, _, _, _ in items:
                bits.zero_()
                it.zero_()
            ldpc.decode_list(items, early_stop=early_stop, threads_per_row=2)
            torch.cuda.synchronize()
            for (g, llr, bits, it, n_rows, n_tx, T), (wl, q, _) in zip(items, refs):
                ref = oracle.decode_layered(wl.base, wl.K_b, wl.Z, wl.n_rows, q,
                                            algo=oracle.OFFSET, max_iter=T,
                                            early_stop=early_stop)
                got = ldpc.unpack_bits(bits.cpu().numpy()[None, :], wl.K)
                assert np.array_equal(got, ref.bits)
                assert int(it.item()) == int(ref.iters[0])
        for g in graphs.values():
            g.close()
    finally:
        ldpc.list_jit_prepare([])
