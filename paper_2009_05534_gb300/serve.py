"""Slot-driven continuous batching of LDPC transport blocks.

The paper sizes the decoder against the 5G slot (Sec. II: decoding should finish within one
slot of 250 us to 1 ms; Sec. V: the 500 us target at 10 iterations).  This module is the
serving loop around the decoder: transport blocks of mixed base graph, lifting size and
rate arrive continuously; at every slot boundary the server

1. admits waiting blocks first-come first-served while the output arena has room
   (admission by memory: a block that does not fit waits for a later slot),
2. decodes everything admitted in that slot with one work-list launch (`ldpc_decode_list`)
   on the next stream of a small round-robin pool, so new slots start while earlier ones
   are still running on the device; blocks for the learned decoder (one graph and
   (beta, gamma) table, binary16 LLRs) go to one row-mapped launch
   (`ldpc_decode_rows_host_maps`, which uploads the slot's row maps itself) on a stream of
   their own, and the slot completes when both have,
3. retires the slot batches whose completion event has fired (their output buffers return
   to the arena and their latencies are recorded); when the arena cannot take every
   waiting block this happens before admission instead.

Graphs live on the device for the server's lifetime.  Channel LLRs are read from device
memory (the demapper's output buffers); the decoder's messages and posteriors never leave
the SM.  Latency of a block = (slots it waited for admission) x slot length + device time
from the start of its admission slot to the completion of its slot batch (CUDA events; the
start event is recorded on an idle stream as the slot's first action, so it marks the slot
boundary even while the decode streams are busy and the host's retirement, admission and
launch work counts towards the latency).

Host cost per slot is kept independent of Python object churn: requests are integer ids
assigned in arrival order (so FIFO admission is a contiguous id range), their attributes
live in numpy arrays, and a slot's work items are gathered into one numpy record array that
is handed to the C ABI as-is.  `SlotScheduler` does not touch CUDA and is tested on the CPU
with a fake backend.
"""
from __future__ import annotations

import gc
import time
from dataclasses import dataclass

import numpy as np


@dataclass
class _Batch:
    slot: int
    ids: np.ndarray            # request ids of the batch
    outs: np.ndarray           # their output-buffer indices
    handle: object             # backend token


class SlotScheduler:
    """FIFO admission by output-buffer memory, one batch per slot, completion bookkeeping.

    backend must provide:
      capacity() -> int                               output buffers in the arena
      launch(slot, ids, outs) -> handle               asynchronous decode of requests `ids`
      done(handle) -> bool                            non-blocking completion test
      wait(handle) -> None                            blocking wait
      finish(handle, ids, outs) -> device_us          per-batch device latency, results kept
    and may provide slot_start() -> None, called first thing at every slot boundary.
    """

    def __init__(self, backend, slot_us: float = 500.0, max_requests: int = 1 << 22):
        self.backend = backend
        self.slot_us = float(slot_us)
        self.free = list(range(backend.capacity() - 1, -1, -1))   # stack of free buffers
        self.arrival = np.zeros(max_requests, np.int64)
        self.admit = np.full(max_requests, -1, np.int64)
        self.latency_us = np.full(max_requests, np.nan)
        self.head = 0                 # oldest waiting request id
        self.tail = 0                 # next request id
        self.in_flight: list[_Batch] = []
        self.slot = 0

    @property
    def n_waiting(self) -> int:
        return self.tail - self.head

    def submit(self, n: int) -> np.ndarray:
        """Register n arrivals in the current slot; returns their ids."""
        ids = np.arange(self.tail, self.tail + n)
        self.arrival[self.tail:self.tail + n] = self.slot
        self.tail += n
        return ids

    def _retire(self, block: bool = False):
        keep = []
        for b in self.in_flight:
            if block:
                self.backend.wait(b.handle)
            if block or self.backend.done(b.handle):
                dev_us = self.backend.finish(b.handle, b.ids, b.outs)
                self.latency_us[b.ids] = (b.slot - self.arrival[b.ids]) * self.slot_us + dev_us
                self.free.extend(b.outs.tolist())
            else:
                keep.append(b)
        self.in_flight = keep

    def step(self) -> np.ndarray:
        """One slot boundary: admit, launch, retire finished batches.  Returns admitted ids.

        A backend with a ``slot_start()`` method is told of the boundary first, so that its
        latency clock also covers the host work before the launch.  Finished batches are
        retired before admission only when the free buffers do not cover every waiting
        request (only then can retiring change what is admitted); otherwise after the
        launch, off the path to the device."""
        mark = getattr(self.backend, "slot_start", None)
        if mark is not None:
            mark()
        if self.n_waiting > len(self.free):
            self._retire()
        k = min(self.n_waiting, len(self.free))
        ids = np.arange(self.head, self.head + k)
        if k:
            outs = np.array(self.free[-k:][::-1], dtype=np.int64)
            del self.free[-k:]
            self.head += k
            self.admit[ids] = self.slot
            self.in_flight.append(_Batch(self.slot, ids, outs,
                                         self.backend.launch(self.slot, ids, outs)))
        self._retire()
        self.slot += 1
        return ids

    def drain(self, max_slots: int = 1 << 20):
        n = 0
        while self.n_waiting and n < max_slots:
            if not self.free:
                self._retire(block=True)
            self.step()
            n += 1
        self._retire(block=True)

    def completed_latencies(self) -> np.ndarray:
        lat = self.latency_us[:self.tail]
        return lat[~np.isnan(lat)]


def latency_stats(lat) -> dict:
    lat = np.asarray(lat, dtype=np.float64)
    if lat.size == 0:
        return {"n": 0}
    return {"n": int(lat.size), "p50_us": float(np.percentile(lat, 50)),
            "p99_us": float(np.percentile(lat, 99)), "max_us": float(lat.max())}


@dataclass
class LearnedClass:
    """Requests served by the learned decoder: one graph and (beta, gamma) table, their
    binary16 LLRs in a device pool; request id i uses pool row pick[i] (-1: plain request).
    """
    graph: object
    pool: object               # CUDA float16 [rows][n_tx]
    table: object              # CUDA float32 [T][n_rows][2]
    pick: np.ndarray           # int32 per request id
    max_iter: int
    n_rows: int = 0


class GpuBackend:
    """Device backend: output arena, round-robin streams, one work-list launch per slot.

    table: numpy record array (``work_item_dtype``), one row per request id, with graph,
    LLR pointer, n_rows, n_tx and max_iter filled in; the output pointers are set at
    admission from the arena.  ks: information bits per request id.  learned: optional
    LearnedClass; its requests of a slot are decoded by one row-mapped learned decode
    (`ldpc_decode_rows_host_maps`, row maps from host memory) on a stream of its own, into
    an arena of their own.  row_tables: optional (base table, n_rows) pairs of the served
    graphs and rates, for which the work-list kernel is compiled (`ldpc_list_jit_prepare`).

    Host work per slot is part of every block's latency (the slot's start event is recorded
    before it), so the per-slot path reuses what does not change: the decode options, the
    raw stream handles and a pool of timing events.
    """

    def __init__(self, table: np.ndarray, ks: np.ndarray, n_buffers: int, kmax: int,
                 n_streams: int = 4, early_stop: bool = True, keep_results: bool = False,
                 learned: LearnedClass | None = None, row_tables=None):
        import ctypes

        import torch

        import paper_2009_05534_gb300 as ldpc
        self.torch, self.ldpc = torch, ldpc
        if row_tables:
            # the work-list kernel compiled for the served graphs' row sequences (seconds
            # of host time, once; the first launch below loads it)
            ldpc.list_jit_prepare(row_tables)
        self.table = table
        # the table as raw words: row gathers and pointer patches on plain integers
        self.words = np.ascontiguousarray(table, dtype=ldpc.work_item_dtype).view(
            np.uint64).reshape(len(table), ldpc.WORK_ITEM_WORDS)
        self.w_bits = ldpc.WorkItem.hard_bits.offset // 8
        self.w_iters = ldpc.WorkItem.iters.offset // 8
        self.ks = ks
        self.early_stop = early_stop
        self.nb = (kmax + 7) // 8
        self.bits = torch.zeros((n_buffers, self.nb), dtype=torch.uint8, device="cuda")
        self.iters = torch.zeros((n_buffers,), dtype=torch.int32, device="cuda")
        # device address of every output buffer's hard bits and iteration count
        self.bits_addr = (self.bits.data_ptr()
                          + np.arange(n_buffers, dtype=np.uint64) * np.uint64(self.nb))
        self.iters_addr = self.iters.data_ptr() + np.arange(n_buffers, dtype=np.uint64) * 4
        self.n = n_buffers
        self.streams = [torch.cuda.Stream() for _ in range(n_streams)]
        self.sp = [ctypes.c_void_p(st.cuda_stream) for st in self.streams]
        self.opts = ldpc.make_opts(ldpc.LLR_INT8, early_stop=early_stop)
        self.clock = torch.cuda.Stream()          # idle stream: slot-boundary timestamps
        self.k = 0
        self.keep = keep_results
        self.results: dict = {}
        self.ev_pool: list = []
        self._start = None
        self.learned = learned
        if learned is not None:
            self.nb_l = (learned.graph.K + 7) // 8
            self.bits_l = torch.zeros((n_buffers, self.nb_l), dtype=torch.uint8, device="cuda")
            self.iters_l = torch.zeros((n_buffers,), dtype=torch.int32, device="cuda")
            # learned batches run on streams of their own, concurrently with the slot's
            # work-list launch
            self.lstreams = [torch.cuda.Stream() for _ in range(n_streams)]
            self.lsp = [ctypes.c_void_p(st.cuda_stream) for st in self.lstreams]
            self.opts_l = ldpc.make_opts(ldpc.LLR_FP16, algo=ldpc.LEARNED, learned=learned.table,
                                         n_rows=learned.n_rows, n_tx=learned.pool.shape[1],
                                         early_stop=early_stop)
        self._prime()

    def _prime(self):
        """The library allocates a stream's work table and row-map staging (device and
        pinned host memory, which can take milliseconds) on that stream's first launch;
        one throw-away launch per stream here, into output buffer 0, keeps that out of
        the slots."""
        z = np.zeros(1, np.int64)
        for j in range(len(self.streams)):
            if len(self.words):
                items = np.take(self.words, z, axis=0)
                items[:, self.w_bits] = np.take(self.bits_addr, z)
                items[:, self.w_iters] = np.take(self.iters_addr, z)
                self.ldpc.decode_list_words(items, stream=self.sp[j], opts=self.opts)
            lc = self.learned
            if lc is not None:
                self.ldpc.decode_rows_host_maps(lc.graph, lc.pool, z, z, lc.max_iter,
                                                bits=self.bits_l, iters=self.iters_l,
                                                stream=self.lsp[j], opts=self.opts_l)
        self.torch.cuda.synchronize()

    def capacity(self):
        return self.n

    def _event(self):
        return self.ev_pool.pop() if self.ev_pool else self.torch.cuda.Event(enable_timing=True)

    def slot_start(self):
        """Timestamp the slot boundary on the idle stream (the scheduler calls this first
        thing at every boundary; a slot that admits nothing keeps the event for the next)."""
        if self._start is None:
            self._start = self._event()
        self._start.record(self.clock)

    def launch(self, slot, ids, outs):
        if self._start is None:
            self.slot_start()
        start, self._start = self._start, None
        j = self.k % len(self.streams)
        self.k += 1
        lc = self.learned
        if lc is not None:
            sel = lc.pick[ids] >= 0
            ids_p, outs_p = ids[~sel], outs[~sel]
        else:
            ids_p, outs_p = ids, outs
        if len(ids_p):
            items = np.take(self.words, ids_p, axis=0)
            items[:, self.w_bits] = np.take(self.bits_addr, outs_p)
            items[:, self.w_iters] = np.take(self.iters_addr, outs_p)
            self.ldpc.decode_list_words(items, stream=self.sp[j], opts=self.opts)
        end = self._event()
        end.record(self.streams[j])
        end_l = None
        if lc is not None and sel.any():
            self.ldpc.decode_rows_host_maps(lc.graph, lc.pool, lc.pick[ids[sel]], outs[sel],
                                            lc.max_iter, bits=self.bits_l, iters=self.iters_l,
                                            stream=self.lsp[j], opts=self.opts_l)
            end_l = self._event()
            end_l.record(self.lstreams[j])
        return (start, end, end_l)

    def done(self, handle):
        return handle[1].query() and (handle[2] is None or handle[2].query())

    def wait(self, handle):
        handle[1].synchronize()
        if handle[2] is not None:
            handle[2].synchronize()

    def finish(self, handle, ids, outs):
        start, end, end_l = handle
        if self.keep:
            o = self.torch.from_numpy(outs).cuda()
            its = self.iters[o].cpu().numpy()
            bits = self.bits[o].cpu().numpy()
            if self.learned is not None:
                its_l = self.iters_l[o].cpu().numpy()
                bits_l = self.bits_l[o].cpu().numpy()
                is_l = self.learned.pick[ids] >= 0
            for k, (i, it, b) in enumerate(zip(ids.tolist(), its, bits)):
                if self.learned is not None and is_l[k]:
                    b, it = bits_l[k], its_l[k]
                self.results[i] = (b[: (int(self.ks[i]) + 7) // 8].copy(), int(it))
        t = start.elapsed_time(end)
        if end_l is not None:
            t = max(t, start.elapsed_time(end_l))
            self.ev_pool.append(end_l)
        self.ev_pool += (start, end)
        return t * 1e3


def run_paced(scheduler: SlotScheduler, counts, slot_us: float = 500.0) -> float:
    """counts[s] arrivals at slot s, slots paced in real time; returns the wall time.

    The interpreter's cyclic garbage collector is paused for the duration (a collection
    over the loop's many short-lived arrays can stall a slot by milliseconds) and run once
    afterwards."""
    was_enabled = gc.isenabled()
    gc.disable()
    try:
        t0 = time.perf_counter()
        for s, n in enumerate(counts):
            target = t0 + s * slot_us * 1e-6
            while time.perf_counter() < target:
                pass
            scheduler.submit(int(n))
            scheduler.step()
        scheduler.drain()
        return time.perf_counter() - t0
    finally:
        if was_enabled:
            gc.enable()
        gc.collect()
