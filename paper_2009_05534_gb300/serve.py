"""Slot-driven continuous batching of LDPC transport blocks.

The paper sizes the decoder against the 5G slot (Sec. II: decoding should finish within one
slot of 250 us to 1 ms; Sec. V: the 500 us target at 10 iterations).  This module is the
serving loop around the decoder: transport blocks of mixed base graph, lifting size and
rate arrive continuously; at every slot boundary the server

1. retires the slot batches whose completion event has fired (their output buffers return
   to the arena and their latencies are recorded),
2. admits waiting blocks first-come first-served while the output arena has room
   (admission by memory: a block that does not fit waits for a later slot),
3. decodes everything admitted in that slot with one work-list launch (`ldpc_decode_list`)
   on the next stream of a small round-robin pool, so new slots start while earlier ones
   are still running on the device; blocks for the learned decoder (one graph and
   (beta, gamma) table, binary16 LLRs) go to one row-mapped launch (`ldpc_decode_rows`) on
   a stream of their own, and the slot completes when both have.

Graphs live on the device for the server's lifetime.  Channel LLRs are read from device
memory (the demapper's output buffers); the decoder's messages and posteriors never leave
the SM.  Latency of a block = (slots it waited for admission) x slot length + device time
from the start of its admission slot to the completion of its slot batch (CUDA events; the
start event is recorded on an idle stream so it marks the slot boundary even while the
decode streams are busy).

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
        """One slot boundary: retire finished batches, admit, launch.  Returns admitted ids."""
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
    (`ldpc_decode_rows`) on the same stream, into an arena of their own.
    """

    def __init__(self, table: np.ndarray, ks: np.ndarray, n_buffers: int, kmax: int,
                 n_streams: int = 4, early_stop: bool = True, keep_results: bool = False,
                 learned: LearnedClass | None = None):
        import torch

        import paper_2009_05534_gb300 as ldpc
        self.torch, self.ldpc = torch, ldpc
        self.table = table
        self.ks = ks
        self.early_stop = early_stop
        self.nb = (kmax + 7) // 8
        self.bits = torch.zeros((n_buffers, self.nb), dtype=torch.uint8, device="cuda")
        self.iters = torch.zeros((n_buffers,), dtype=torch.int32, device="cuda")
        self.n = n_buffers
        self.streams = [torch.cuda.Stream() for _ in range(n_streams)]
        self.clock = torch.cuda.Stream()          # idle stream: slot-boundary timestamps
        self.k = 0
        self.keep = keep_results
        self.results: dict = {}
        self.learned = learned
        if learned is not None:
            self.nb_l = (learned.graph.K + 7) // 8
            self.bits_l = torch.zeros((n_buffers, self.nb_l), dtype=torch.uint8, device="cuda")
            self.iters_l = torch.zeros((n_buffers,), dtype=torch.int32, device="cuda")
            # learned batches run on streams of their own, concurrently with the slot's
            # work-list launch; their row maps go up from a pinned ring (a pageable copy
            # would stall the host until the stream drains)
            self.lstreams = [torch.cuda.Stream() for _ in range(n_streams)]
            self.ring = 64
            self.rows_pin = torch.zeros((self.ring, 2, n_buffers), dtype=torch.int32).pin_memory()
            self.rows_dev = torch.zeros((self.ring, 2, n_buffers), dtype=torch.int32,
                                        device="cuda")
            self.ring_ev = [None] * self.ring

    def capacity(self):
        return self.n

    def launch(self, slot, ids, outs):
        torch = self.torch
        s = self.streams[self.k % len(self.streams)]
        self.k += 1
        start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        start.record(self.clock)
        lc = self.learned
        if lc is not None:
            sel = lc.pick[ids] >= 0
            ids_p, outs_p = ids[~sel], outs[~sel]
        else:
            ids_p, outs_p = ids, outs
        if len(ids_p):
            items = self.table[ids_p].copy()
            items["hard_bits"] = self.bits.data_ptr() + outs_p * self.nb
            items["iters"] = self.iters.data_ptr() + outs_p * 4
            self.ldpc.decode_list_array(items, stream=s, early_stop=self.early_stop)
        end.record(s)
        end_l = None
        if lc is not None and sel.any():
            sl = self.lstreams[(self.k - 1) % len(self.lstreams)]
            r = (self.k - 1) % self.ring
            if self.ring_ev[r] is not None:
                self.ring_ev[r].synchronize()          # the copy that last used slot r
            n = int(sel.sum())
            pin = self.rows_pin[r].numpy()
            pin[0, :n] = lc.pick[ids[sel]]
            pin[1, :n] = outs[sel]
            dev = self.rows_dev[r]
            with torch.cuda.stream(sl):
                dev[:, :n].copy_(self.rows_pin[r][:, :n], non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(sl)
            self.ring_ev[r] = ev
            self.ldpc.decode_rows(lc.graph, lc.pool, dev[0, :n], dev[1, :n], lc.max_iter,
                                  bits=self.bits_l, iters=self.iters_l, stream=sl,
                                  algo=self.ldpc.LEARNED, learned=lc.table,
                                  n_rows=lc.n_rows, early_stop=self.early_stop,
                                  check_rows=False)
            end_l = torch.cuda.Event(enable_timing=True)
            end_l.record(sl)
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
