"""Slot scheduler: FIFO admission by memory, continuous batching, latency bookkeeping
(CPU, fake backend), and on the GPU: each result is the same alone and in the mix."""
import numpy as np
import pytest

from paper_2009_05534_gb300.serve import SlotScheduler, latency_stats


class FakeBackend:
    """Each batch completes `delay` slots after its launch (device time = delay slots)."""

    def __init__(self, n_buffers, delay=2, slot_us=500.0):
        self.n, self.delay, self.now, self.slot_us = n_buffers, delay, 0, slot_us
        self.launched = []

    def capacity(self):
        return self.n

    def launch(self, slot, ids, outs):
        self.launched.append((slot, ids.tolist(), outs.tolist()))
        return slot + self.delay

    def done(self, handle):
        return self.now >= handle

    def wait(self, handle):
        self.now = max(self.now, handle)

    def finish(self, handle, ids, outs):
        return self.delay * self.slot_us


def test_fifo_admission_by_memory():
    be = FakeBackend(n_buffers=3, delay=2)
    sch = SlotScheduler(be, slot_us=500.0)
    sch.submit(7)
    for s in range(12):
        be.now = s
        sch.step()
    sch.drain()
    # slot 0 admits the first 3; buffers return when the batch completes (2 slots later)
    assert be.launched[0][:2] == (0, [0, 1, 2])
    order = [rid for _, ids, _ in be.launched for rid in ids]
    assert order == list(range(7))                     # first come, first served
    assert all(len(ids) <= 3 for _, ids, _ in be.launched)
    # a buffer is never handed out twice while in use
    live = {}
    for slot, ids, outs in be.launched:
        for o in outs:
            assert live.get(o, -10) + 2 <= slot
            live[o] = slot
    lat = sch.completed_latencies()
    assert lat.size == 7 and lat.min() == 1000.0 and lat.max() > 1000.0


def test_continuous_batching_overlaps_slots():
    be = FakeBackend(n_buffers=100, delay=3)
    sch = SlotScheduler(be, slot_us=500.0)
    for s in range(6):
        be.now = s
        sch.submit(4)
        sch.step()
    # new work was launched every slot while earlier batches were still in flight
    assert [slot for slot, _, _ in be.launched] == list(range(6))
    assert len(sch.in_flight) >= 2
    sch.drain()
    st = latency_stats(sch.completed_latencies())
    assert st["n"] == 24 and st["p99_us"] == 1500.0


class _RandomDelayBackend(FakeBackend):
    """Each batch completes a seeded random number of slots after its launch; slot_start
    calls are logged in order with the launches."""

    def __init__(self, n_buffers, seed):
        super().__init__(n_buffers)
        self.rng = np.random.default_rng(seed)
        self.log = []

    def slot_start(self):
        self.log.append("start")

    def launch(self, slot, ids, outs):
        self.log.append("launch")
        self.launched.append((slot, ids.tolist(), outs.tolist()))
        d = int(self.rng.integers(1, 5))
        return slot + d, d

    def done(self, handle):
        return self.now >= handle[0]

    def wait(self, handle):
        self.now = max(self.now, handle[0])

    def finish(self, handle, ids, outs):
        return handle[1] * self.slot_us


class _EagerScheduler(SlotScheduler):
    """Retires finished batches before every admission."""

    def step(self):
        self._retire()
        return super().step()


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_lazy_retirement_admits_as_eager(seed):
    """Retiring only when the arena is short (else after the launch) admits the same
    requests into the same buffers in the same slots as retiring first at every slot, and
    gives the same latencies; the backend hears of each slot boundary before its launch."""
    rng = np.random.default_rng(100 + seed)
    counts = rng.poisson(5, size=60)
    runs = []
    for cls in (SlotScheduler, _EagerScheduler):
        be = _RandomDelayBackend(n_buffers=12, seed=seed)
        sch = cls(be, slot_us=500.0)
        for s, n in enumerate(counts):
            be.now = s
            sch.submit(int(n))
            sch.step()
        sch.drain()
        runs.append((be, sch))
    (be_l, sch_l), (be_e, sch_e) = runs
    assert be_l.launched == be_e.launched
    assert np.array_equal(sch_l.completed_latencies(), sch_e.completed_latencies())
    assert sch_l.completed_latencies().size == counts.sum()
    # the arena ran short: some requests waited for buffers to come back
    n = sch_l.tail
    assert (sch_l.admit[:n] > sch_l.arrival[:n]).any()
    assert all(a == "start" for a, b in zip(be_l.log, be_l.log[1:]) if b == "launch")


@pytest.mark.gpu
def test_results_same_alone_and_in_mix():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from fractions import Fraction

    from paper_2009_05534_gb300 import build
    build.build()
    import paper_2009_05534_gb300 as ldpc
    from paper_2009_05534_gb300.serve import GpuBackend
    from synth import make_workload
    rng = np.random.default_rng(3)
    graphs, llrs, alone = {}, [], []
    n = 60
    table = np.zeros(n, dtype=ldpc.work_item_dtype)
    ks = np.zeros(n, np.int64)
    for i in range(n):
        kind = "BG1" if rng.integers(2) else "BG2"
        Z = int(rng.choice([32, 64, 96, 128, 192, 256, 384]))
        rate = Fraction(str(rng.choice(["1/3", "1/2", "2/3", "5/6"])))
        wl = make_workload(kind, Z, 1, float(rng.uniform(0.5, 4.0)), rate=rate, seed=500 + i,
                           graph_seed=0)
        if (kind, Z) not in graphs:
            graphs[(kind, Z)] = ldpc.Graph(wl.base, wl.K_b, Z)
        g = graphs[(kind, Z)]
        llr = torch.from_numpy(wl.llr_int8()[0]).cuda()
        llrs.append(llr)
        table[i] = (g.handle.value, llr.data_ptr(), 0, 0, wl.n_rows, wl.n_tx, 8)
        ks[i] = wl.K
        b, it = ldpc.decode(g, llr[None, :], 8, n_rows=wl.n_rows, n_tx=wl.n_tx)
        torch.cuda.synchronize()
        alone.append((b.cpu().numpy()[0], int(it.item())))
    kmax = max(g.K for g in graphs.values())
    be = GpuBackend(table, ks, n_buffers=16, kmax=kmax, n_streams=3, keep_results=True)
    sch = SlotScheduler(be, slot_us=500.0)
    for s in range(0, n, 7):                 # 7 arrivals per slot, only 16 buffers
        sch.submit(min(7, n - s))
        sch.step()
    sch.drain()
    assert len(be.results) == n
    for i, (b, it) in be.results.items():
        assert np.array_equal(b, alone[i][0]) and it == alone[i][1]
    assert (sch.completed_latencies() > 0).all()
    for g in graphs.values():
        g.close()


@pytest.mark.gpu
def test_learned_and_plain_served_together():
    """Learned requests (binary16, BG2-shaped Z=128, a (beta, gamma) table) share slots with
    plain int8 requests; each result equals the same codeword decoded alone."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from fractions import Fraction

    from paper_2009_05534_gb300 import build
    build.build()
    import paper_2009_05534_gb300 as ldpc
    from paper_2009_05534_gb300.serve import GpuBackend, LearnedClass
    from synth import make_workload
    rng = np.random.default_rng(4)
    T = 8
    wl_l = make_workload("BG2", 128, 24, 2.5, seed=900, graph_seed=0)
    g_l = ldpc.Graph(wl_l.base, wl_l.K_b, 128)
    pool = torch.from_numpy(wl_l.llr_fp16()).cuda()
    tab = np.zeros((T, wl_l.n_rows, 2), np.float32)
    tab[..., 0] = rng.uniform(0.4, 0.9, size=(T, wl_l.n_rows))
    tab[..., 1] = rng.uniform(0.0, 0.3, size=(T, wl_l.n_rows))
    tab_d = torch.from_numpy(tab).cuda()
    graphs, llrs = {}, []
    n = 48
    table = np.zeros(n, dtype=ldpc.work_item_dtype)
    ks = np.zeros(n, np.int64)
    pick = np.full(n, -1, np.int32)
    alone = []
    for i in range(n):
        if rng.integers(3) == 0:                               # learned request
            pick[i] = int(rng.integers(len(pool)))
            ks[i] = wl_l.K
            b, it = ldpc.decode(g_l, pool[pick[i]][None, :], T, algo=ldpc.LEARNED,
                                learned=tab_d)
            torch.cuda.synchronize()
            alone.append((b.cpu().numpy()[0], int(it.item())))
            continue
        Z = int(rng.choice([64, 128, 384]))
        wl = make_workload("BG1", Z, 1, 2.0, rate=Fraction(1, 2), seed=700 + i, graph_seed=0)
        if Z not in graphs:
            graphs[Z] = ldpc.Graph(wl.base, wl.K_b, Z)
        llr = torch.from_numpy(wl.llr_int8()[0]).cuda()
        llrs.append(llr)
        table[i] = (graphs[Z].handle.value, llr.data_ptr(), 0, 0, wl.n_rows, wl.n_tx, T)
        ks[i] = wl.K
        b, it = ldpc.decode(graphs[Z], llr[None, :], T, n_rows=wl.n_rows, n_tx=wl.n_tx)
        torch.cuda.synchronize()
        alone.append((b.cpu().numpy()[0], int(it.item())))
    assert (pick >= 0).sum() >= 8 and (pick < 0).sum() >= 8
    kmax = max([g.K for g in graphs.values()] + [g_l.K])
    be = GpuBackend(table, ks, n_buffers=12, kmax=kmax, n_streams=2, keep_results=True,
                    learned=LearnedClass(g_l, pool, tab_d, pick, T))
    sch = SlotScheduler(be, slot_us=500.0)
    for s in range(0, n, 5):
        sch.submit(min(5, n - s))
        sch.step()
    sch.drain()
    assert len(be.results) == n
    for i, (b, it) in be.results.items():
        assert np.array_equal(b, alone[i][0]) and it == alone[i][1], i
    for g in list(graphs.values()) + [g_l]:
        g.close()
