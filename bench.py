#!/usr/bin/env python
"""Throughput benchmark of the layered min-sum decoder.

Workload: seeded synthetic BG1-shaped graph (46 x 68, K_b = 22), Z = 384 (K = 8448),
rate 1/3 (N_tx = 25344), QPSK over AWGN at Eb/N0 = 1.5 dB, int8 LLRs (scale 4, saturate
+-127), offset min-sum with offset 1, 10 iterations, batch 1024 codewords per GPU.  The
headline runs a fixed 10 iterations (early stop off); a second measurement with early
stop on is reported beside it.  One step = one decode of the whole batch (every step of
the hot path: load, gather, v->c, check node, write-back, output).

Metric: decoded information Gbit/s = batch * K / time, timed with CUDA events on the
decode stream; inputs rotate over device copies totalling more than twice the L2 size, so
no step reads its LLRs from L2.  `--impl reference` times the CPU oracle instead.  The
clock record (nvidia-smi every 200 ms) spans the timed region and 1.5 s of the same decode
run untimed right after it, since the timed region is shorter than one sampling period.

Beside the headline the JSON line carries: the ALU roofline fraction and the profiled DRAM
traffic of the decode kernel; the early-stop figure; an end-to-end figure through the
host-buffer C-ABI call; a whole-rounds batch (8 codewords per SM) for context; and, on rank
0, the slot-serving leg (10 000 slots of mixed traffic, p50/p99 latency), the latency leg
(a lone codeword with each strategy, the cluster split, small batches), the BLER curve,
the flooding comparison, the rate-8/9 high-load leg (int8 and binary16) and the learned
tables against plain min-sum at equal BLER.  --no-<leg> flags skip them.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

KIND, Z, EBN0, BATCH, T_ITER, SEED = "BG1", 384, 1.5, 1024, 10, 0
WORKLOAD = "BG1-shaped 46x68 Z=384 K=8448 R=1/3 QPSK AWGN Eb/N0=1.5dB int8 offset-1 min-sum T=10"
L2_BYTES = 129 * 2 ** 20
METRIC = "decoded information throughput (BG1 Z=384, 10 it)"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--batch", type=int, default=BATCH)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--serve-slots", type=int, default=10000,
                    help="slots of the mixed-traffic serving measurement (0 = skip)")
    ap.add_argument("--no-high-load", dest="high_load", action="store_false",
                    help="skip the rate-8/9 QAM int8-vs-binary16 measurement")
    ap.add_argument("--no-learned", dest="learned", action="store_false",
                    help="skip the learned-vs-plain BLER and throughput measurement")
    ap.add_argument("--no-flooding", dest="flooding", action="store_false",
                    help="skip the flooding-schedule comparison")
    ap.add_argument("--no-latency", dest="latency", action="store_false",
                    help="skip the single-codeword latency measurement")
    ap.add_argument("--no-bler-curve", dest="bler_curve", action="store_false",
                    help="skip the BLER sweep over Eb/N0 of the headline workload")
    return ap.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def max_over_ranks(x: float) -> float:
    """The largest value of x over the ranks of the process group (x itself without one);
    the tensor lives where the backend needs it (CUDA for NCCL, host for gloo)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_gbps(world: int, steps: int, batch: int, K: int, seconds: float) -> float:
    """Whole-job information throughput: every rank decodes `batch` codewords per step."""
    return world * steps * batch * K / seconds / 1e9


def make_inputs(batch: int, rank: int, ebn0: float = EBN0):
    from synth import make_workload
    return make_workload(KIND, Z, batch, ebn0, modulation="QPSK", seed=SEED,
                         first_cw=rank * batch)


def headline_config(B: int, E: int, n_tx: int, in_bytes: int, world: int) -> dict:
    """The workload's `config` object, printed by both arms (GPU decoder and CPU oracle)."""
    n_copies = max(2, math.ceil(2.2 * L2_BYTES / in_bytes))
    return {"workload": WORKLOAD, "batch_per_gpu": B, "E": E, "n_tx": n_tx,
            "early_stop": False,
            "l2": f"inputs rotate over {n_copies} device copies "
                  f"({n_copies * in_bytes / 2**20:.0f} MiB > L2)",
            "parallelism": f"replicas x{world}"}


def cpu_model() -> str:
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu model")):
                return line.split(":", 1)[1].strip()
        import platform
        return platform.machine()
    except OSError:
        return "unknown"


def oracle_gbps(wl, q, seconds: float, threads: int):
    """Decode the sample repeatedly with the CPU oracle for about `seconds`."""
    import oracle
    n = min(len(q), max(threads * 2, 16))
    t0 = time.perf_counter()
    done = 0
    while True:
        oracle.decode_layered(wl.base, wl.K_b, Z, wl.n_rows, q[:n], algo=oracle.OFFSET,
                              offset_q=1, max_iter=T_ITER, early_stop=False, threads=threads)
        done += n
        el = time.perf_counter() - t0
        if el >= seconds:
            break
    return done * wl.K / el / 1e9, done, el


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms from just before the timed
    region to the end of the load window that follows it."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: str):
        self.index = index
        self.proc = None
        self.lines: list[str] = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", self.index, f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def wait_first(self, limit_s: float = 5.0):
        """Block until nvidia-smi has printed its first sample (its start-up must not fall
        inside the timed region), at most limit_s seconds."""
        t0 = time.perf_counter()
        while self.proc is not None and not self.lines and time.perf_counter() - t0 < limit_s:
            time.sleep(0.05)

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for nm, v in zip(names, f[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return None


def profiled_traffic(kernel_tag: str):
    """DRAM bytes per launch recorded from ncu in profiles/, if the kernel source still
    matches the hash recorded beside it (else None): sha256 of the kernel header and the
    runtime-compilation unit that builds it for the graph, concatenated."""
    import hashlib
    path = os.path.join(ROOT, "profiles", f"{kernel_tag}.md")
    csrc = os.path.join(ROOT, "paper_2009_05534_gb300", "csrc")
    try:
        text = open(path).read()
        blob = b"".join(open(os.path.join(csrc, f), "rb").read()
                        for f in ("pair_kernel.cuh", "pair_jit.cu"))
        h = hashlib.sha256(blob).hexdigest()[:16]
    except OSError:
        return None
    got, sha = None, None
    for line in text.splitlines():
        if line.startswith("traffic_bytes_per_launch:"):
            got = float(line.split(":", 1)[1].split()[0])
        if line.startswith("kernel_source_sha256_16:"):
            sha = line.split(":", 1)[1].strip()
    return got if (got is not None and sha == h) else None


# ------------------------------------------------------------------------- slot serving

SERVE_ZS = (32, 64, 96, 128, 192, 256, 384)
SERVE_RATES = ("1/3", "1/2", "2/3", "5/6", "8/9")
SERVE_MODS = (("QPSK", 3.0), ("16QAM", 7.0), ("64QAM", 11.0))


def serving_measure(n_slots: int, mean_tbs: float = 128.0, seed: int = 1, max_iter: int = 10,
                    learned_share: float = 0.125):
    """Mixed-traffic slot serving: Poisson(mean_tbs) transport blocks per 500 us slot
    (clipped to 64..512), each a uniformly drawn (BG1|BG2, Z, rate, modulation) codeword
    from a device-resident pool of synthetic int8 LLRs, plus (share `learned_share`, when
    the trained table is present) learned-decoder blocks (BG2-shaped Z=128, every row,
    binary16 QPSK LLRs); returns p50/p99 latency and throughput."""
    from fractions import Fraction

    import numpy as np
    import torch

    import paper_2009_05534_gb300 as ldpc
    from paper_2009_05534_gb300.serve import GpuBackend, SlotScheduler, latency_stats, run_paced
    from synth import make_workload
    rng = np.random.default_rng(seed)
    graphs, rows, ks, llrs, row_tables = {}, [], [], [], {}
    for kind in ("BG1", "BG2"):
        for Zs in SERVE_ZS:
            for rate in SERVE_RATES:
                for m, (mod, eb) in enumerate(SERVE_MODS):
                    wl = make_workload(kind, Zs, 2, eb, rate=Fraction(rate), modulation=mod,
                                       seed=seed * 1000 + len(rows), graph_seed=0)
                    if (kind, Zs) not in graphs:
                        graphs[(kind, Zs)] = ldpc.Graph(wl.base, wl.K_b, Zs)
                    row_tables[(kind, rate)] = (wl.base, wl.n_rows)
                    q = torch.from_numpy(wl.llr_int8()).cuda()
                    for b in range(2):
                        llrs.append(q[b])
                        rows.append((graphs[(kind, Zs)].handle.value, q[b].data_ptr(), 0, 0,
                                     wl.n_rows, wl.n_tx, max_iter))
                        ks.append(wl.K)
    pool = np.array(rows, dtype=ldpc.work_item_dtype)
    ks = np.array(ks, np.int64)
    counts = np.clip(rng.poisson(mean_tbs, size=n_slots), 64, 512)
    total = int(counts.sum())
    pick = rng.integers(0, len(pool), size=total)
    table, kreq = pool[pick], ks[pick]
    kmax = max(g.K for g in graphs.values())
    learned, n_learned = None, 0
    path = os.path.join(ROOT, "paper_2009_05534_gb300", "tables", LEARNED_TABLE)
    if learned_share > 0 and os.path.exists(path):
        from paper_2009_05534_gb300.serve import LearnedClass
        from paper_2009_05534_gb300.train_learned import load_table
        tab, meta = load_table(path)
        wl = make_workload("BG2", 128, 256, 3.0, modulation="QPSK", seed=seed * 1000 + 999,
                           graph_seed=0)
        g_l = graphs[("BG2", 128)]
        lpool = torch.from_numpy(wl.llr_fp16()).cuda()
        is_l = rng.random(total) < learned_share
        lpick = np.where(is_l, rng.integers(0, len(lpool), size=total), -1).astype(np.int32)
        kreq = np.where(is_l, wl.K, kreq)
        n_learned = int(is_l.sum())
        learned = LearnedClass(g_l, lpool, torch.from_numpy(tab).cuda(), lpick,
                               int(meta["T"]), 0)
        ldpc.decode(g_l, lpool[:8], learned.max_iter, algo=ldpc.LEARNED, learned=learned.table)
    be = GpuBackend(table, kreq, n_buffers=4096, kmax=kmax, n_streams=4, early_stop=True,
                    learned=learned, row_tables=list(row_tables.values()))
    sch = SlotScheduler(be, slot_us=500.0, max_requests=total + 1)
    # warm-up: a few slots outside the measurement
    warm = SlotScheduler(GpuBackend(np.tile(pool, 4), np.tile(ks, 4), n_buffers=1024,
                                    kmax=kmax), slot_us=500.0, max_requests=4 * len(pool) + 1)
    run_paced(warm, [len(pool)] * 4)
    torch.cuda.synchronize()
    wall = run_paced(sch, counts.tolist(), 500.0)
    st = latency_stats(sch.completed_latencies())
    for g in graphs.values():
        g.close()
    del llrs
    return {"slots": n_slots, "slot_us": 500.0, "tbs": total, "mean_tbs_per_slot":
            float(counts.mean()), "p50_us": st.get("p50_us"), "p99_us": st.get("p99_us"),
            "max_us": st.get("max_us"), "gbps": float(kreq.sum()) / wall / 1e9,
            "max_iter": max_iter, "early_stop": True, "learned_tbs": n_learned,
            "list_kernel": "compiled for the served row sequences (ldpc_list_jit_prepare)",
            "traffic": "BG1|BG2 x Z{32..384} x R{1/3..8/9} x QPSK/16QAM/64QAM int8"
                       + (f"; {learned_share:.3f} of blocks learned (BG2 Z=128 R=1/5 "
                          "binary16, 10 iterations)" if learned is not None else "")}


# ----------------------------------------------------------- BLER over the Eb/N0 sweep

def bler_curve_measure(graph, batch: int = 1024, ebn0s=None):
    """The headline workload's Eb/N0 sweep (0.5 .. 2.5 dB in 0.25 dB steps, batch 1024,
    int8 offset min-sum, cap 10 iterations with the stopping rule): BLER and mean
    iterations per point, decoded on the GPU."""
    import numpy as np
    import torch

    import paper_2009_05534_gb300 as ldpc
    if ebn0s is None:
        ebn0s = [0.5 + 0.25 * k for k in range(9)]
    out = {"workload": "BG1-shaped Z=384 R=1/3 QPSK int8 offset-1, cap 10, stopping rule, "
                       f"{batch} codewords per point; LLR scale 4 (the headline quantiser) "
                       "and scale 2 (same kernel, coarser input quantisation)"}
    for scale in (4.0, 2.0):
        pts = []
        for eb in ebn0s:
            wl = make_inputs(batch, 0, eb)
            bits, iters = ldpc.decode(graph, torch.from_numpy(wl.llr_int8(scale)).cuda(),
                                      T_ITER, early_stop=True)
            got = ldpc.unpack_bits(bits.cpu().numpy(), wl.K)
            pts.append({"ebn0_db": eb, "bler": float((got != wl.info).any(1).mean()),
                        "ber": float((got != wl.info).mean()),
                        "mean_iterations": float(iters.float().mean())})
        out[f"scale_{scale:g}"] = pts
    return out


# ------------------------------------------------------------------- single-codeword latency

def full_rounds_measure(wl, graph, n_sm: int, alu_peak: float, reps: int = 10):
    """Context for the headline: the batch kernel holds two codewords per SM, so a batch of
    1024 on 152 SMs leaves its fourth round a third full.  The same workload at a batch of
    four full rounds (8 codewords per SM), 10 iterations: throughput and ALU roofline
    fraction without that tail."""
    import torch

    import paper_2009_05534_gb300 as ldpc
    from synth import make_workload
    B = 8 * n_sm
    w = make_workload("BG1", 384, B, EBN0, seed=5, graph_seed=0)
    q = w.llr_int8()
    n_copies = max(2, math.ceil(2.2 * L2_BYTES / q.nbytes))
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        bufs = [torch.from_numpy(q).cuda() for _ in range(n_copies)]
    torch.cuda.synchronize()

    def run(k):
        ldpc.decode(graph, bufs[k % n_copies], T_ITER, early_stop=False, stream=stream)

    for k in range(3):
        run(k)
    sec = _timed(run, reps, stream)
    del bufs
    E = int((w.base[:w.n_rows] >= 0).sum())
    achieved = T_ITER * E * 384 * B / sec
    return {"batch": B, "gbps": B * w.K / sec / 1e9, "ms_per_launch": sec * 1e3,
            "roofline_frac": achieved / alu_peak}


def latency_measure(wl, graph, reps: int = 50):
    """Latency of one codeword alone (batch 1, the headline workload, 10 iterations, early
    stop off): CUDA events around each launch on an otherwise idle stream; median and max.
    int8 with the paper's two strategies (Sec. IV): alpha = 1 thread per row pair (the
    high-throughput kernel) and alpha = 2, 4 cooperating threads per row pair (the
    low-latency kernel, the library's choice for a batch that does not fill the SMs), and
    the binary16 decoder, and the cluster split (one codeword on two SMs).  Then small
    batches (up to two codewords per SM) with alpha 1, 2 and 4 and the cluster split, which
    sets where the library switches strategy."""
    import torch

    import paper_2009_05534_gb300 as ldpc
    stream = torch.cuda.Stream()
    q = torch.from_numpy(wl.llr_int8()[:1]).cuda()

    def lat(dt, n, **kw):
        ts = []
        for k in range(n + 3):
            s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s.record(stream)
            ldpc.decode(graph, dt, T_ITER, early_stop=False, stream=stream, **kw)
            e.record(stream)
            torch.cuda.synchronize()
            if k >= 3:
                ts.append(s.elapsed_time(e) * 1e3)
        return {"median_us": statistics.median(ts), "max_us": max(ts),
                "per_iteration_us": statistics.median(ts) / T_ITER}

    out = {"int8": lat(q, reps, algo=ldpc.OFFSET)}
    out["int8_by_alpha"] = {str(a): lat(q, reps, algo=ldpc.OFFSET, threads_per_row=a)
                            for a in (1, 2, 4)}
    # the cluster split: two blocks on two SMs per codeword (alpha 2 in each)
    out["int8_cluster2"] = lat(q, reps, algo=ldpc.OFFSET, cluster_size=2)
    out["fp16"] = lat(torch.from_numpy(wl.llr_fp16()[:1]).cuda(), reps, algo=ldpc.NORMALISED,
                      alpha=0.75)
    n_sm = torch.cuda.get_device_properties(0).multi_processor_count
    small = {}
    full = wl.llr_int8()
    for b in sorted({1, n_sm // 4, n_sm // 2, n_sm, 2 * n_sm}):
        if b > full.shape[0]:
            continue
        qb = torch.from_numpy(full[:b]).cuda()
        small[str(b)] = {str(a): lat(qb, 10, algo=ldpc.OFFSET, threads_per_row=a)["median_us"]
                         for a in (1, 2, 4)}
        small[str(b)]["cluster2"] = lat(qb, 10, algo=ldpc.OFFSET, cluster_size=2)["median_us"]
    out["batch_us_by_alpha"] = small
    return {"workload": "one BG1-shaped Z=384 R=1/3 codeword, 10 iterations", **out}


# ------------------------------------------------------------------- high load (R = 8/9)

# Eb/N0 grids per modulation that carry every decoder and cap through BLER 1e-1 .. 1e-3 on
# the BG1-shaped graph at rate 8/9 (set from an oracle sweep of 256 codewords per point)
HIGH_LOAD = (("16QAM", [6.875 + 0.125 * k for k in range(15)]),
             ("64QAM", [10.875 + 0.125 * k for k in range(15)]))


def _timed(fn, reps: int, stream):
    import torch
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s.record(stream)
    for k in range(reps):
        fn(k)
    e.record(stream)
    torch.cuda.synchronize()
    return s.elapsed_time(e) / 1e3 / reps


def _crossings(ebn0s, blers, levels=(1e-1, 1e-2, 1e-3)):
    """Eb/N0 where a BLER curve first falls to each level (log-linear between points, a
    zero counting as below every level), None where it never does."""
    out = {}
    for lv in levels:
        at = None
        for k in range(len(ebn0s) - 1):
            b0, b1 = blers[k], blers[k + 1]
            if b0 > lv >= b1:
                if b1 <= 0.0:
                    at = ebn0s[k + 1]
                else:
                    t = math.log(b0 / lv) / math.log(b0 / b1)
                    at = ebn0s[k] + t * (ebn0s[k + 1] - ebn0s[k])
                break
        if at is None and blers and blers[0] <= lv:
            at = ebn0s[0]
        out[f"{lv:g}"] = at
    return out


def high_load_measure(batch: int = 8192, caps=(5, 10, 20), reps: int = 3, seed: int = 2,
                      alu_peak: float | None = None):
    """BG1-shaped Z=384 at rate 8/9 (5 rows, N_tx = 9504), 16QAM / 64QAM max-log LLRs,
    batch 8192, iteration caps 5/10/20 with early stop: int8 (offset 1, LLR scale 4, the
    headline quantiser), int8 at LLR scale 2 and binary16 (normalised 0.75) message storage
    side by side, over an Eb/N0 grid per modulation (the same codewords and noise at every
    point).  Per point: Gbit/s, BLER, mean iterations; per decoder and cap: the Eb/N0 where
    BLER reaches 1e-1, 1e-2 and 1e-3; and the ALU roofline fraction of the int8 and
    binary16 decodes (executed edge updates over the int8x4 or fp16x2 issue peak).  Inputs
    rotate over device copies larger than L2."""
    from fractions import Fraction

    import numpy as np
    import torch

    import paper_2009_05534_gb300 as ldpc
    from synth import make_workload
    from synth.channel import modulate_llr_sweep, quantize_int8, to_fp16
    stream = torch.cuda.Stream()
    points, summary = [], []
    decoders = (("int8", 4.0, dict(algo=ldpc.OFFSET)), ("int8_scale2", 2.0, dict(algo=ldpc.OFFSET)),
                ("fp16", None, dict(algo=ldpc.NORMALISED, alpha=0.75)))
    for mod, grid in HIGH_LOAD:
        wl = make_workload("BG1", 384, batch, grid[0], rate=Fraction(8, 9), modulation=mod,
                           seed=seed, graph_seed=0)
        E = int((wl.base[:wl.n_rows] >= 0).sum())
        g = ldpc.Graph(wl.base, wl.K_b, 384)
        info = torch.from_numpy(wl.info).cuda()
        tx = wl.codewords[:, wl.punct_cols * 384: wl.punct_cols * 384 + wl.n_tx]
        curve = {(name, T): [] for name, _, _ in decoders for T in caps}
        for eb, llr in zip(grid, modulate_llr_sweep(tx, grid, wl.meta["rate"], mod, seed)):
            for name, scale, kw in decoders:
                host = quantize_int8(llr, scale) if scale else to_fp16(llr)
                n_copies = max(2, math.ceil(2.2 * L2_BYTES / host.nbytes))
                with torch.cuda.stream(stream):
                    b0 = torch.from_numpy(host).cuda()
                    bufs = [b0] + [b0.clone() for _ in range(n_copies - 1)]
                torch.cuda.synchronize()
                for T in caps:
                    bits = iters = None

                    def run(k):
                        nonlocal bits, iters
                        bits, iters = ldpc.decode(g, bufs[k % n_copies], T, n_rows=wl.n_rows,
                                                  n_tx=wl.n_tx, early_stop=True, stream=stream,
                                                  **kw)

                    for k in range(2):
                        run(k)
                    sec = _timed(run, reps, stream)
                    got = torch.from_numpy(ldpc.unpack_bits(bits.cpu().numpy(), wl.K)).cuda()
                    bler = float((got != info).any(1).float().mean())
                    mit = float(iters.float().mean())
                    pt = {"modulation": mod, "ebn0_db": eb, "max_iter": T, "dtype": name,
                          "gbps": batch * wl.K / sec / 1e9, "bler": bler,
                          "mean_iterations": mit}
                    if alu_peak:
                        # executed edge updates / s over the issue peak of the lane format
                        peak = alu_peak if name.startswith("int8") else alu_peak / 2
                        pt["roofline_frac"] = mit * E * 384 * batch / sec / peak
                    points.append(pt)
                    curve[(name, T)].append(bler)
                del bufs
        for (name, T), bl in curve.items():
            summary.append({"modulation": mod, "dtype": name, "max_iter": T,
                            "ebn0_db_at_bler": _crossings(grid, bl)})
        g.close()
    return {"workload": "BG1-shaped Z=384 K=8448 R=8/9 (5 rows, N_tx=9504), batch "
                        f"{batch}, early stop, inputs rotate over copies > L2; int8 = LLR "
                        "scale 4 (the headline quantiser), int8_scale2 = LLR scale 2; "
                        "roofline_frac: executed edge updates over the int8x4 (int8) or "
                        "fp16x2 (binary16) issue peak",
            "points": points, "bler_crossings": summary}


# ------------------------------------------------------------ flooding baseline (Sec. V)

def flooding_measure(wl, graph, q_dev, batch: int = 512, reps: int = 3):
    """The paper's comparison schedule on the headline codewords: flooding min-sum
    (normalised 0.75, fp32) and sum-product with a cap of 2T = 20 iterations against the
    layered int8 decoder with a cap of T = 10, all stopping at a valid codeword: Gbit/s,
    BLER and mean iterations of each on the same codewords."""
    import torch

    import paper_2009_05534_gb300 as ldpc
    stream = torch.cuda.Stream()
    llr = torch.from_numpy(wl.llr[:batch]).cuda()
    info = wl.info[:batch]
    out = {"batch": batch}
    ws = torch.empty((int(ldpc.lib().ldpc_flooding_workspace_floats(graph.handle, batch, 0)),),
                     dtype=torch.float32, device="cuda")
    for name, algo, T in (("flooding_min_sum", ldpc.NORMALISED, 2 * T_ITER),
                          ("flooding_sum_product", ldpc.SUM_PRODUCT, 2 * T_ITER)):
        res = {}

        def run(k):
            res["o"] = ldpc.decode_flooding(graph, llr, T, algo=algo, alpha=0.75,
                                            early_stop=True, stream=stream, workspace=ws)

        run(0)
        sec = _timed(run, reps, stream)
        bits = ldpc.unpack_bits(res["o"][0].cpu().numpy(), wl.K)
        out[name] = {"max_iter": T, "gbps": batch * wl.K / sec / 1e9,
                     "bler": float((bits != info).any(1).mean()),
                     "mean_iterations": float(res["o"][1].float().mean())}

    def run_l(k):
        res["l"] = ldpc.decode(graph, q_dev[:batch], T_ITER, early_stop=True, stream=stream)

    run_l(0)
    sec = _timed(run_l, reps, stream)
    bits = ldpc.unpack_bits(res["l"][0].cpu().numpy(), wl.K)
    out["layered_int8"] = {"max_iter": T_ITER, "gbps": batch * wl.K / sec / 1e9,
                           "bler": float((bits != info).any(1).mean()),
                           "mean_iterations": float(res["l"][1].float().mean())}
    return out


# -------------------------------------------------------- learned vs plain (BG2, Z = 128)

LEARNED_TABLE = "learned_bg2_z128_t10.json"
# (table file, base graph, Z, Eb/N0 grid of the comparison, fresh codewords per point,
# throughput batch) of each trained table: the grids bracket both decoders' BLER 1e-2
LEARNED_CASES = (
    (LEARNED_TABLE, "BG2", 128,
     (1.5, 1.75, 2.0, 2.25, 2.5, 2.75, 3.0, 3.5, 3.75, 4.0, 4.25), 8192, 8192),
    ("learned_bg1_z384_t10.json", "BG1", 384,
     (0.75, 0.875, 1.0, 1.125, 1.25, 1.375, 1.5), 4096, 2048),
)


def learned_measure(table_file: str = LEARNED_TABLE, kind: str = "BG2", Z: int = 128,
                    grid=LEARNED_CASES[0][3], n_cw: int = 8192, batch: int = 8192,
                    reps: int = 5):
    """A trained (beta, gamma) table against plain normalised min-sum (alpha 0.75) on the
    same fresh codewords: BLER per Eb/N0 at T = 10 (binary16 LLRs and messages), the Eb/N0
    of BLER 1e-2 for each, decode throughput of both at T = 10 and, with early stop, at the
    plain decoder's BLER-1e-2 point, and each decoder with early stop at its own BLER-1e-2
    point (Gbit/s at equal BLER)."""
    import torch

    import paper_2009_05534_gb300 as ldpc
    from paper_2009_05534_gb300.train_learned import (TABLE_DIR, bler_sweep, ebn0_at,
                                                      load_table)
    from synth import make_workload
    path = os.path.join(TABLE_DIR, table_file)
    if not os.path.exists(path):
        return None
    table, meta = load_table(path)
    T = int(meta["T"])
    wl0 = make_workload(kind, Z, 1, 1.0, seed=0, graph_seed=0)
    g = ldpc.Graph(wl0.base, wl0.K_b, Z)
    tab = torch.from_numpy(table).cuda()
    curves = bler_sweep(g, kind, Z, T, {"plain": None, "learned": tab}, list(grid), n_cw,
                        4096, seed=77_000)
    at = {k: ebn0_at(list(grid), v, 1e-2) for k, v in curves.items()}
    eb_op = at["plain"] if at["plain"] is not None else grid[-1]
    stream = torch.cuda.Stream()
    kws = {"plain": dict(algo=ldpc.NORMALISED, alpha=0.75),
           "learned": dict(algo=ldpc.LEARNED, learned=tab)}

    def throughput(eb, names, early_stops, seed):
        """Gbit/s and mean iterations of each decoder on `batch` fresh codewords at eb."""
        wl = make_workload(kind, Z, batch, float(eb), seed=seed, graph_seed=0)
        host = wl.llr_fp16()
        n_copies = max(2, math.ceil(2.2 * L2_BYTES / host.nbytes))
        with torch.cuda.stream(stream):
            b0 = torch.from_numpy(host).cuda()
            bufs = [b0] + [b0.clone() for _ in range(n_copies - 1)]
        torch.cuda.synchronize()
        res = {}
        for es in early_stops:
            for name in names:
                out = {}

                def run(k):
                    out["o"] = ldpc.decode(g, bufs[k % n_copies], T, early_stop=es,
                                           stream=stream, **kws[name])

                for k in range(2):
                    run(k)
                sec = _timed(run, reps, stream)
                got = ldpc.unpack_bits(out["o"][0].cpu().numpy(), wl.K)
                res[f"{name}{'_early_stop' if es else ''}"] = {
                    "gbps": batch * wl.K / sec / 1e9,
                    "mean_iterations": float(out["o"][1].float().mean()),
                    "bler": float((got != wl.info).any(1).mean())}
        return res

    # both decoders at the plain decoder's BLER-1e-2 point, fixed T and with early stop
    thr = throughput(eb_op, ("plain", "learned"), (False, True), 78_000)
    # equal BLER: each decoder with early stop at its own BLER-1e-2 Eb/N0
    equal = {}
    for name in ("plain", "learned"):
        if at[name] is not None:
            r = throughput(at[name], (name,), (True,), 79_000)[f"{name}_early_stop"]
            equal[name] = {"ebn0_db": at[name], **r}
    return {"workload": meta.get("code"), "T": T, "llr": "binary16", "eval_codewords": n_cw,
            "ebn0_db": list(grid), "bler_plain": curves["plain"],
            "bler_learned": curves["learned"], "ebn0_at_bler_1e-2": at,
            "gain_db": (at["plain"] - at["learned"]) if None not in at.values() else None,
            "throughput_ebn0_db": eb_op, "throughput_batch": batch, "throughput": thr,
            "equal_bler_1e-2_early_stop": equal,
            "training": {k: meta["training"].get(k) for k in
                         ("codewords", "epochs", "steps", "lr", "ebn0_db", "loss", "gradient")}}


# ----------------------------------------------------------------------------- reference

def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    threads = os.cpu_count() or 1
    n = args.batch                 # the GPU arm's batch: every step decodes all of it
    wl = make_inputs(n, 0)
    q = wl.llr_int8()
    import oracle
    E = oracle.edge_count(wl.base, wl.K_b, Z, wl.n_rows)
    for _ in range(args.warmup):
        oracle.decode_layered(wl.base, wl.K_b, Z, wl.n_rows, q, algo=oracle.OFFSET,
                              max_iter=T_ITER, early_stop=False, threads=threads)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.decode_layered(wl.base, wl.K_b, Z, wl.n_rows, q, algo=oracle.OFFSET,
                              max_iter=T_ITER, early_stop=False, threads=threads)
        times.append(time.perf_counter() - t0)
    tot = sum(times)
    val = n * wl.K * args.steps / tot / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": val,
        "unit": "Gbit/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * tot / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int8", "data": "synthetic",
        "config": headline_config(n, E, wl.n_tx, q.nbytes, world),
        "cpu_baseline": {"value": val, "unit": "Gbit/s", "cores": threads, "kind": "oracle",
                         "sample": f"the whole {n}-codeword batch per step on {threads} "
                                   f"threads ({cpu_model()}), LLRs in host memory"},
        "e2e": {"value": val, "unit": "Gbit/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------------- ours

def run_ours(args):
    import numpy as np
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import paper_2009_05534_gb300 as ldpc
    # every leg compiles the batch kernel for its row sequence at first use and waits
    # (inside its warm-up), so that no timed region runs the generic kernel meanwhile
    ldpc.pair_jit(2)
    B = args.batch
    wl = make_inputs(B, rank)
    q = wl.llr_int8()
    ldpc.pair_jit_prepare(wl.base, wl.n_rows)
    graph = ldpc.Graph(wl.base, wl.K_b, Z)
    E = graph.edges()
    stream = torch.cuda.Stream()
    in_bytes = q.nbytes
    n_copies = max(2, math.ceil(2.2 * L2_BYTES / in_bytes))
    with torch.cuda.stream(stream):
        host = torch.from_numpy(q)
        bufs = [host.cuda(non_blocking=False) for _ in range(n_copies)]
        nbytes = (wl.K + 7) // 8
        bits = torch.empty((B, nbytes), dtype=torch.uint8, device="cuda")
        iters = torch.empty((B,), dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()

    def step(k, early_stop=False, buf=None):
        ldpc.decode(graph, bufs[k % n_copies] if buf is None else buf, T_ITER, bits=bits,
                    iters=iters, stream=stream, early_stop=early_stop)

    for k in range(args.warmup):
        step(k)
    torch.cuda.synchronize()
    graph.sync_status(stream)
    # correctness spot check against the LLRs' own decode stays in the test-suite

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    idx = vis.split(",")[local] if vis else str(local)
    sampler = ClockSampler(idx)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    barrier()
    torch.cuda.synchronize()
    sampler.start()
    sampler.wait_first()
    time.sleep(0.2)
    l0 = ldpc.launch_count()
    t_wall0 = time.perf_counter()
    for k in range(args.steps):
        ev[k][0].record(stream)
        step(k)
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall0
    launches = ldpc.launch_count() - l0
    # the timed region lasts milliseconds, less than the sampler's 200 ms period: the same
    # decode keeps running, untimed, for 1.5 s after it, so the clock record is taken under
    # that load (every LLR copy holds the same codewords, so the outputs do not change)
    soak_end, k = time.perf_counter() + 1.5, args.steps
    while time.perf_counter() < soak_end:
        for _ in range(64):
            step(k)
            k += 1
        torch.cuda.synchronize()
    barrier()
    clocks = sampler.stop()
    if clocks is not None:
        clocks["window"] = "timed region, then 1.5 s of the same decode right after it"
    graph.sync_status(stream)
    # what the timed decode returned (every copy holds the same LLRs): BLER of the fixed
    # 10-iteration decode, read after the timed region
    got = ldpc.unpack_bits(bits.cpu().numpy(), wl.K)
    headline_bler = {"fixed_iterations": {
        "max_iter": T_ITER, "bler": float((got != wl.info).any(1).mean()),
        "ber": float((got != wl.info).mean()), "mean_iterations": float(T_ITER)}}
    per = [a.elapsed_time(b) / 1e3 for a, b in ev]         # seconds per step (= per launch)
    elapsed = max_over_ranks(ev[0][0].elapsed_time(ev[-1][1]) / 1e3)
    value = job_gbps(world, args.steps, B, wl.K, elapsed)
    kern = sum(per) / len(per)

    # early stop on (same data, 10-iteration cap): mean iterations and throughput
    es_ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
    es_ev[0].record(stream)
    for k in range(args.steps):
        step(k, early_stop=True)
    es_ev[1].record(stream)
    torch.cuda.synchronize()
    es_time = es_ev[0].elapsed_time(es_ev[1]) / 1e3
    mean_it = float(iters.float().mean().item())
    es_gbps = args.steps * B * wl.K / es_time / 1e9
    got = ldpc.unpack_bits(bits.cpu().numpy(), wl.K)
    headline_bler["early_stop"] = {"max_iter": T_ITER,
                                   "bler": float((got != wl.info).any(1).mean()),
                                   "ber": float((got != wl.info).mean()),
                                   "mean_iterations": mean_it}
    headline_bler["note"] = ("Eb/N0 1.5 dB, LLR scale 4: at a fixed 10 iterations the 8-bit "
                             "posteriors saturate and most codewords decode wrongly (a "
                             "throughput measurement only); with the stopping rule the "
                             "decoder stops at the valid codeword")

    # end to end through the host-buffer C-ABI call (pinned memory, copies timed)
    pin = torch.from_numpy(q).pin_memory()
    hbits = torch.empty((B, nbytes), dtype=torch.uint8).pin_memory()
    hit = torch.empty((B,), dtype=torch.int32).pin_memory()
    for _ in range(2):
        ldpc.decode_host(graph, pin, T_ITER, bits=hbits, iters=hit, stream=stream,
                         early_stop=False)
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        ldpc.decode_host(graph, pin, T_ITER, bits=hbits, iters=hit, stream=stream,
                         early_stop=False)
    e2e_t = max_over_ranks(time.perf_counter() - t0)
    e2e = job_gbps(world, args.steps, B, wl.K, e2e_t)

    peaks = measured_peaks()
    props = torch.cuda.get_device_properties(local)
    n_sm = props.multi_processor_count
    f_max = (peaks or {}).get("sm_max_mhz") or 2070.0
    edge_updates = T_ITER * E * Z * B
    alu_peak = n_sm * f_max * 1e6 * 512.0 / 12.0            # edge updates / s (int8x4 issue)
    achieved = edge_updates / kern
    hbm_peak = (peaks or {}).get("hbm_gbs")
    alg_bytes = B * (wl.n_tx + nbytes + 4)
    traffic = profiled_traffic("layered_int8_bg1_z384")

    # the single-GPU side measurements run on rank 0 only (replicas would repeat them)
    aux = rank == 0
    full_rounds = full_rounds_measure(wl, graph, n_sm, alu_peak) if aux else None
    serving = serving_measure(args.serve_slots) if aux and args.serve_slots > 0 else None
    latency = latency_measure(wl, graph) if aux and args.latency else None
    bler_curve = bler_curve_measure(graph) if aux and args.bler_curve else None
    flooding = flooding_measure(wl, graph, bufs[0]) if aux and args.flooding else None
    high_load = high_load_measure(alu_peak=alu_peak) if aux and args.high_load else None
    learned = learned_bg1 = None
    if aux and args.learned:
        learned = learned_measure()
        learned_bg1 = learned_measure(*LEARNED_CASES[1][:3], grid=LEARNED_CASES[1][3],
                                      n_cw=LEARNED_CASES[1][4], batch=LEARNED_CASES[1][5])

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        threads = os.cpu_count() or 1
        g, done, el = oracle_gbps(wl, q, 12.0, threads)
        g1, done1, el1 = oracle_gbps(wl, q, 4.0, 1)
        cpu = {"value": g, "unit": "Gbit/s", "cores": threads, "kind": "oracle",
               "sample": f"first {min(len(q), max(threads * 2, 16))} codewords of the batch, "
                         f"decoded repeatedly ({done} codewords in {el:.1f} s, {cpu_model()})",
               "single_thread": {"value": g1, "unit": "Gbit/s",
                                 "sample": f"{done1} codewords in {el1:.1f} s on 1 thread"}}
    if rank == 0:
        line = {
            "metric": METRIC,
            "value": value, "unit": "Gbit/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * elapsed / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "int8", "data": "synthetic",
            "config": headline_config(B, E, wl.n_tx, in_bytes, world),
            "roofline": {"bound": "alu", "achieved": achieved / 1e9, "peak": alu_peak / 1e9,
                         "unit": "Gedge/s", "frac": achieved / alu_peak,
                         "traffic": traffic,
                         "peak_basis": f"{n_sm} SMs x {f_max:.0f} MHz x 512/12 edge updates "
                                       "per SM per clock (int8x4 issue, 12 lane-ops/edge)",
                         "algorithmic_bytes": alg_bytes,
                         "hbm_frac": (alg_bytes / kern / 1e9 / hbm_peak) if hbm_peak else None,
                         "kernel_ms": 1e3 * kern},
            "early_stop": {"value": es_gbps, "unit": "Gbit/s", "mean_iterations": mean_it,
                           "ebn0_db": EBN0},
            "headline_bler": headline_bler,
            "e2e": {"value": e2e, "unit": "Gbit/s", "h2d_bytes_per_step": in_bytes,
                    "d2h_bytes_per_step": B * (nbytes + 4)},
            "full_rounds": full_rounds,
            "serving": serving,
            "latency": latency,
            "bler_curve": bler_curve,
            "flooding": flooding,
            "high_load": high_load,
            "learned": learned,
            "learned_bg1": learned_bg1,
            "gpu_launches": launches,
            "clocks": clocks,
            "wall_s": t_wall,
        }
        if cpu:
            line["cpu_baseline"] = cpu
        print(json.dumps(line), flush=True)
    graph.close()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
