"""The allocation-free work-list decode (ldpc_decode_list_noalloc), for callers that cannot
allocate device memory (a host framework's fixed memory pool, a fixed memory map, or a path
where cudaMalloc would synchronise the device).  Its output must equal the regular
work-list decode's, on two calls in a row (the static work table is reused).  This file is
collected last so that a run stopping at the first failure has run every other test."""
from fractions import Fraction

import numpy as np
import pytest

torch = pytest.importorskip("torch")

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


def _items(ldpc, n, seed):
    rng = np.random.default_rng(seed)
    graphs, keep = {}, []
    table = np.zeros(n, dtype=ldpc.work_item_dtype)
    for k in range(n):
        kind = "BG1" if rng.integers(2) else "BG2"
        Z = int(rng.choice([32, 64, 96, 128, 192, 256, 384]))
        rate = Fraction(str(rng.choice(["1/3", "1/2", "2/3", "5/6"])))
        wl = make_workload(kind, Z, 1, float(rng.uniform(0.5, 4.0)), rate=rate, seed=seed + k,
                           graph_seed=0)
        if (kind, Z) not in graphs:
            graphs[(kind, Z)] = ldpc.Graph(wl.base, wl.K_b, Z)
        llr = torch.from_numpy(wl.llr_int8()[0]).cuda()
        keep.append(llr)
        table[k] = (graphs[(kind, Z)].handle.value, llr.data_ptr(), 0, 0, wl.n_rows, wl.n_tx,
                    int(rng.choice([4, 8, 10])))
    return graphs, keep, table


def _run(ldpc, table, noalloc, early_stop, tpr=0):
    n = len(table)
    nb = 1056
    bits = torch.zeros((n, nb), dtype=torch.uint8, device="cuda")
    iters = torch.zeros((n,), dtype=torch.int32, device="cuda")
    t = table.copy()
    t["hard_bits"] = bits.data_ptr() + np.arange(n) * nb
    t["iters"] = iters.data_ptr() + np.arange(n) * 4
    if noalloc:
        ldpc.decode_list_noalloc(t, early_stop=early_stop, threads_per_row=tpr)
    else:
        ldpc.decode_list_array(t, early_stop=early_stop, threads_per_row=tpr)
    torch.cuda.synchronize()
    return bits.cpu().numpy(), iters.cpu().numpy()


@pytest.mark.parametrize("tpr", [1, 2])
@pytest.mark.parametrize("early_stop", [True, False])
def test_noalloc_matches_list_decode_twice(ldpc, early_stop, tpr):
    """Both list kernels (one and two threads per row pair) through the allocation-free
    entry equal the regular entry's one-thread kernel."""
    graphs, keep, table = _items(ldpc, 48, 900 + int(early_stop))
    ref_bits, ref_iters = _run(ldpc, table, False, early_stop, tpr=1)
    for _ in range(2):                            # two calls in a row reuse the static table
        b, it = _run(ldpc, table, True, early_stop, tpr)
        assert np.array_equal(b, ref_bits)        # bit-exact, like every int8 path
        assert np.array_equal(it, ref_iters)
    for g in graphs.values():
        g.close()


def test_noalloc_rejects_oversize_list(ldpc):
    graphs, keep, table = _items(ldpc, 1, 5)
    big = np.repeat(table, 2049)
    with pytest.raises(ldpc.LdpcError):
        ldpc.decode_list_noalloc(big)
    for g in graphs.values():
        g.close()


def test_noalloc_allocates_nothing(ldpc):
    """The entry point's distinguishing claim: on a stream the library has never seen, the
    regular work-list decode allocates its per-stream workspace, the allocation-free one
    does not (the library counts every device and pinned-host allocation it makes)."""
    graphs, keep, table = _items(ldpc, 8, 77)
    n = len(table)
    bits = torch.zeros((n, 1056), dtype=torch.uint8, device="cuda")
    iters = torch.zeros((n,), dtype=torch.int32, device="cuda")
    t = table.copy()
    t["hard_bits"] = bits.data_ptr() + np.arange(n) * 1056
    t["iters"] = iters.data_ptr() + np.arange(n) * 4
    ldpc.decode_list_noalloc(t)                   # set-up on this device done before counting
    torch.cuda.synchronize()
    fresh = torch.cuda.Stream()
    before = ldpc.alloc_count()
    for _ in range(2):
        ldpc.decode_list_noalloc(t, stream=fresh)
    torch.cuda.synchronize()
    assert ldpc.alloc_count() == before
    ldpc.decode_list_array(t, stream=torch.cuda.Stream())   # a new stream's workspace
    torch.cuda.synchronize()
    assert ldpc.alloc_count() > before
    for g in graphs.values():
        g.close()
