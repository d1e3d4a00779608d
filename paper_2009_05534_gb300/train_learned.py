"""Train a learned min-sum table and compare it with plain normalised min-sum.

The learned check rule scales and offsets the min-sum magnitude per (iteration, base row):
m' = beta[t][r] * max(m - gamma[t][r], 0) (the per-row, per-iteration extension of the
single correction factor of Sec. III).  This module holds the recipe around the kernels:

* a training set of seeded synthetic codewords (random information bits, the structured
  encoder, QPSK over AWGN at an Eb/N0 drawn per codeword), generated once and kept on the
  device as binary16 LLRs and codeword bits;
* Adam on the binary cross-entropy of the posteriors after every iteration (mean over
  iterations; the final-posterior loss alone is an option), over several seeded shuffles
  (epochs) of that set, with checkpoint / resume;
* a BLER sweep over Eb/N0 on fresh codewords, decoding the same LLRs with the plain and the
  learned table through the regular decode entry point, and the Eb/N0 at which each curve
  crosses a target BLER (log-linear interpolation between grid points);
* the trained table with its recipe and results as a small JSON file.

Command line (GPU):
    python -m paper_2009_05534_gb300.train_learned --out table.json [--codewords N ...]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import time

import numpy as np

from . import LEARNED, NORMALISED, Graph, decode, unpack_bits
from . import learned as _learned

TABLE_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tables")


def training_set(kind: str, Z: int, n_cw: int, batch: int, ebn0_lo: float, ebn0_hi: float,
                 seed: int, rate=None, log=None):
    """(llr float16 CUDA [n_cw][n_tx], codewords uint8 CUDA [n_cw][N], n_rows, base)."""
    import torch
    from concurrent.futures import ThreadPoolExecutor
    from synth import make_workload, uniform_ebn0

    def gen(k):
        lo = k * batch
        b = min(batch, n_cw - lo)
        e = uniform_ebn0(seed, b, ebn0_lo, ebn0_hi, first_cw=lo)
        return make_workload(kind, Z, b, e, rate=rate, seed=seed, graph_seed=0, first_cw=lo)

    n_b = (n_cw + batch - 1) // batch
    llr = cw = None
    with ThreadPoolExecutor(1) as ex:
        nxt = ex.submit(gen, 0)
        for k in range(n_b):
            wl = nxt.result()
            if k + 1 < n_b:
                nxt = ex.submit(gen, k + 1)
            if llr is None:
                llr = torch.empty((n_cw, wl.n_tx), dtype=torch.float16, device="cuda")
                cw = torch.empty((n_cw, wl.codewords.shape[1]), dtype=torch.uint8,
                                 device="cuda")
                n_rows, base = wl.n_rows, wl.base
            lo = k * batch
            llr[lo:lo + len(wl.llr)] = torch.from_numpy(wl.llr_fp16()).cuda()
            cw[lo:lo + len(wl.llr)] = torch.from_numpy(wl.codewords).cuda()
            if log and (k % 32 == 0 or k + 1 == n_b):
                log(f"generated {lo + len(wl.llr)} / {n_cw} codewords")
    return llr, cw, n_rows, base


def train_table(graph: Graph, n_rows: int, T: int, llr, cw, *, batch: int, epochs: int,
                lr: float, seed: int, checkpoint=None, log_every: int = 0,
                every_iteration: bool = True, detach: bool = False):
    """Adam over `epochs` seeded shuffles of the device-resident training set; the loss is
    the mean over iterations of the BCE after each iteration (or the final BCE only)."""
    import torch
    n = llr.shape[0]
    per_epoch = n // batch
    g = torch.Generator().manual_seed(seed)
    perms = [torch.randperm(n, generator=g).cuda() for _ in range(epochs)]

    def batch_fn(k):
        e, j = divmod(k, per_epoch)
        idx = perms[e][j * batch:(j + 1) * batch]
        return llr.index_select(0, idx).float(), cw.index_select(0, idx)

    w = np.full(T, 1.0 / T) if every_iteration else None
    return _learned.train(graph, n_rows, T, batch_fn, n_steps=per_epoch * epochs, lr=lr,
                          checkpoint=checkpoint, checkpoint_every=64, log_every=log_every,
                          iter_weights=w, detach=detach)


def bler_sweep(graph: Graph, kind: str, Z: int, T: int, tables: dict, ebn0s, n_cw: int,
               batch: int, seed: int, rate=None, early_stop: bool = False, log=None):
    """BLER per Eb/N0 for each decoder on the same fresh codewords.

    tables maps a name to None (plain normalised min-sum, alpha 0.75) or to a learned
    (beta, gamma) table; every decoder runs T iterations on binary16 LLRs.
    """
    import torch
    from synth import make_workload
    out = {name: [] for name in tables}
    for eb in ebn0s:
        err = {name: 0 for name in tables}
        done = 0
        while done < n_cw:
            b = min(batch, n_cw - done)
            wl = make_workload(kind, Z, b, float(eb), rate=rate, seed=seed, graph_seed=0,
                               first_cw=done)
            l16 = torch.from_numpy(wl.llr_fp16()).cuda()
            for name, tab in tables.items():
                kw = (dict(algo=NORMALISED, alpha=0.75) if tab is None
                      else dict(algo=LEARNED, learned=tab))
                bits, _ = decode(graph, l16, T, n_rows=wl.n_rows, n_tx=wl.n_tx,
                                 early_stop=early_stop, **kw)
                got = unpack_bits(bits.cpu().numpy(), wl.K)
                err[name] += int((got != wl.info).any(1).sum())
            done += b
        for name in tables:
            out[name].append(err[name] / n_cw)
        if log:
            log(f"Eb/N0 {eb:.2f} dB: " + ", ".join(f"{k} {out[k][-1]:.5f}" for k in tables))
    return out


def ebn0_at(ebn0s, bler, target: float):
    """Eb/N0 where a BLER curve first falls to `target` (log-linear between grid points);
    None if it never does on the grid."""
    for i in range(len(ebn0s)):
        if bler[i] <= target:
            if i == 0:
                return float(ebn0s[0])
            b0, b1 = bler[i - 1], bler[i]
            if b1 <= 0.0:
                return float(ebn0s[i])
            f = (math.log(b0) - math.log(target)) / (math.log(b0) - math.log(b1))
            return float(ebn0s[i - 1] + f * (ebn0s[i] - ebn0s[i - 1]))
    return None


def save_table(path, table, meta: dict):
    t = np.asarray(table.cpu() if hasattr(table, "cpu") else table, dtype=np.float32)
    doc = dict(meta)
    doc["shape"] = list(t.shape)
    doc["table"] = [[[float(x) for x in row] for row in it] for it in t]
    with open(path, "w") as f:
        json.dump(doc, f, indent=1)


def load_table(path):
    """(table float32 [T][n_rows][2], metadata dict)."""
    with open(path) as f:
        doc = json.load(f)
    return np.asarray(doc.pop("table"), dtype=np.float32), doc


def main(argv=None):
    import torch
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--kind", default="BG2")
    ap.add_argument("--Z", type=int, default=128)
    ap.add_argument("--T", type=int, default=10)
    ap.add_argument("--codewords", type=int, default=1 << 20)
    ap.add_argument("--batch", type=int, default=4096)
    ap.add_argument("--epochs", type=int, default=4)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--ebn0-lo", type=float, default=0.5)
    ap.add_argument("--ebn0-hi", type=float, default=2.5)
    ap.add_argument("--seed", type=int, default=1000)
    ap.add_argument("--eval-codewords", type=int, default=1 << 16)
    ap.add_argument("--eval-grid", default="1.5:4.5:0.25")
    ap.add_argument("--loss", choices=("every", "final"), default="every",
                    help="BCE after every iteration (mean) or of the final posteriors only")
    ap.add_argument("--grad", choices=("local", "full"), default="local",
                    help="with --loss every: each iteration's parameters follow their own "
                         "term (local) or the whole unrolled chain (full)")
    ap.add_argument("--checkpoint", default=None)
    ap.add_argument("--eval-only", action="store_true",
                    help="re-evaluate the table already in --out (no training): BLER sweep of "
                         "--eval-codewords fresh codewords per point over --eval-grid, "
                         "written into the file's eval record")
    ap.add_argument("--out", required=True)
    a = ap.parse_args(argv)

    def log(msg):
        print(f"[{time.strftime('%H:%M:%S')}] {msg}", flush=True)

    if a.eval_only:
        return evaluate_only(a, log)

    t0 = time.time()
    llr, cw, n_rows, base = training_set(a.kind, a.Z, a.codewords, a.batch, a.ebn0_lo,
                                         a.ebn0_hi, a.seed, log=log)
    t_gen = time.time() - t0
    from synth import SHAPES
    graph = Graph(base, SHAPES[a.kind].K_b, a.Z)
    t1 = time.time()
    table, hist = train_table(graph, n_rows, a.T, llr, cw, batch=a.batch, epochs=a.epochs,
                              lr=a.lr, seed=a.seed, checkpoint=a.checkpoint, log_every=32,
                              every_iteration=a.loss == "every",
                              detach=a.loss == "every" and a.grad == "local")
    torch.cuda.synchronize()
    t_train = time.time() - t1
    del llr, cw
    lo, hi, st = (float(x) for x in a.eval_grid.split(":"))
    grid = [round(lo + k * st, 4) for k in range(int(round((hi - lo) / st)) + 1)]
    curves = bler_sweep(graph, a.kind, a.Z, a.T, {"plain": None, "learned": table}, grid,
                        a.eval_codewords, a.batch, a.seed + 1, log=log)
    res = {name: ebn0_at(grid, curves[name], 1e-2) for name in curves}
    log(f"Eb/N0 at BLER 1e-2: {res}")
    meta = {
        "code": f"{a.kind}-shaped synthetic graph (generator seed 0), Z={a.Z}, every base row "
                f"(rate {SHAPES[a.kind].K_b}/{SHAPES[a.kind].K_b + n_rows - 2})",
        "T": a.T, "n_rows": n_rows,
        "training": {"codewords": a.codewords, "batch": a.batch, "epochs": a.epochs,
                     "steps": len(hist), "optimizer": "Adam", "lr": a.lr,
                     "loss": ("mean over iterations of the BCE after each iteration"
                              if a.loss == "every" else "BCE of the final posteriors"),
                     "gradient": ("per-iteration partial derivatives (adjoints reset at "
                                  "iteration boundaries)"
                                  if a.loss == "every" and a.grad == "local"
                                  else "full reverse mode through the unrolled iterations"),
                     "ebn0_db": [a.ebn0_lo, a.ebn0_hi], "modulation": "QPSK",
                     "seed": a.seed, "llr_storage": "binary16",
                     "loss_first": float(hist[0]), "loss_last": float(hist[-1]),
                     "loss_every_32": [float(x) for x in hist[::32]],
                     "generate_s": round(t_gen, 1), "train_s": round(t_train, 1)},
        "eval": {"codewords_per_point": a.eval_codewords, "seed": a.seed + 1,
                 "llr": "binary16", "early_stop": False, "ebn0_db": grid,
                 "bler_plain": curves["plain"], "bler_learned": curves["learned"],
                 "ebn0_at_bler_1e-2": res},
    }
    save_table(a.out, table, meta)
    log(f"wrote {a.out}")
    graph.close()


def evaluate_only(a, log):
    """BLER sweep of a trained table against plain min-sum on fresh codewords; the table
    file's eval record is replaced by the new one."""
    import torch
    from synth import SHAPES, make_workload
    table, meta = load_table(a.out)
    T = int(meta["T"])
    wl0 = make_workload(a.kind, a.Z, 1, 1.0, seed=0, graph_seed=0)
    graph = Graph(wl0.base, SHAPES[a.kind].K_b, a.Z)
    lo, hi, st = (float(x) for x in a.eval_grid.split(":"))
    grid = [round(lo + k * st, 4) for k in range(int(round((hi - lo) / st)) + 1)]
    seed = int(meta.get("eval", {}).get("seed", a.seed + 1)) + 100_000
    t0 = time.time()
    curves = bler_sweep(graph, a.kind, a.Z, T, {"plain": None,
                                                "learned": torch.from_numpy(table).cuda()},
                        grid, a.eval_codewords, a.batch, seed, log=log)
    res = {name: ebn0_at(grid, curves[name], 1e-2) for name in curves}
    log(f"Eb/N0 at BLER 1e-2: {res}")
    meta["eval"] = {"codewords_per_point": a.eval_codewords,
                    "codewords_total": a.eval_codewords * len(grid), "seed": seed,
                    "llr": "binary16", "early_stop": False, "ebn0_db": grid,
                    "bler_plain": curves["plain"], "bler_learned": curves["learned"],
                    "ebn0_at_bler_1e-2": res, "eval_s": round(time.time() - t0, 1)}
    save_table(a.out, table, meta)
    log(f"wrote {a.out}")
    graph.close()


if __name__ == "__main__":
    main()
