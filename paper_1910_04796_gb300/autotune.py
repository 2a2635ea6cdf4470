"""Autotuner of the FP64 stack kernels.

The paper's LIBCUSMM (Sec. II) tunes its kernels per block shape (m, n, k)
over read/write strategy, threads per block, elements per thread and tiling.
This library's FP64 stack kernels expose a smaller space (team of 1, 2 or 4
warps per C block; 128- or 256-thread CTAs; see dbcsr_opts.kernel), chosen
per C-block shape (m, n). For each shape the tuner builds a synthetic
block-sparse product of that shape (inner sizes from the workload's set),
times every variant through the C ABI with the library's own CUDA-event
kernel timer, keeps the fastest and writes the table as JSON:

    {"device": ..., "entries": [[m, n, variant, tflops_best, {variant: tflops}], ...]}

``load_table`` hands a table to the library (dbcsr_set_tuning).

Usage (on the GPU): python -m paper_1910_04796_gb300.autotune --sizes 5 13 23 26 32 --out table.json
"""
from __future__ import annotations

import argparse
import json
import os
import statistics

import numpy as np

from . import dbcsr, synth

HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_TABLE = os.path.join(HERE, "tuning", "gb300_fp64.json")


def _case(m, n, ksizes, seed, nb=48, p=0.5):
    rng = np.random.default_rng(seed)
    ks = rng.choice(np.asarray(ksizes, np.int32), nb).astype(np.int32)
    A = synth.make_matrix(rng, np.full(nb, m, np.int32), ks, synth.bernoulli_mask(rng, nb, nb, p))
    B = synth.make_matrix(rng, ks, np.full(nb, n, np.int32), synth.bernoulli_mask(rng, nb, nb, p))
    return A, B


def tune_shape(m, n, ksizes, reps=3, seed=0):
    """TFLOP/s of every variant on a synthetic (m, n, k in ksizes) product; returns (best, all)."""
    A, B = _case(m, n, ksizes, seed)
    Ag, Bg = dbcsr.Matrix.from_blocks(A), dbcsr.Matrix.from_blocks(B)
    Cg = dbcsr.Matrix.create(A.row_sizes, B.col_sizes, np.zeros(0, np.int32), np.zeros(0, np.int32))
    res = {}
    for v in range(4):
        times = []
        for _ in range(reps + 1):
            dbcsr.multiply("N", "N", 1.0, Ag, Bg, 0.0, Cg, path="stacks", kernel=v + 1, timing=True)
            st = dbcsr.stats()
            times.append(st["ms_kernel"])
        ms = statistics.median(times[1:])
        res[v] = st["useful_flops"] / (ms / 1e3) / 1e12
    for M in (Ag, Bg, Cg):
        M.release()
    best = max(res, key=res.get)
    return best, res


def tune(msizes, nsizes, ksizes, reps=3):
    entries = []
    for m in msizes:
        for n in nsizes:
            best, res = tune_shape(int(m), int(n), ksizes, reps)
            entries.append([int(m), int(n), int(best), res[best], {str(k): v for k, v in res.items()}])
    return entries


def load_table(path=DEFAULT_TABLE) -> bool:
    """Hand a tuned table to the library; False if the file does not exist."""
    if not os.path.exists(path):
        return False
    with open(path) as f:
        t = json.load(f)
    dbcsr.set_tuning([(e[0], e[1], e[2]) for e in t["entries"]])
    return True


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--sizes", type=int, nargs="+", default=[5, 13, 22, 23, 26, 32])
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--out", default=DEFAULT_TABLE)
    args = ap.parse_args()
    import torch
    dbcsr.init()
    entries = tune(args.sizes, args.sizes, args.sizes, args.reps)
    os.makedirs(os.path.dirname(os.path.abspath(args.out)), exist_ok=True)
    with open(args.out, "w") as f:
        json.dump({"device": torch.cuda.get_device_name(), "kernel": "FP64 stack kernels",
                   "entries": entries}, f, indent=1)
    for e in entries:
        print(e[0], e[1], "best variant", e[2], f"{e[3]:.3f} TFLOP/s", e[4])


if __name__ == "__main__":
    main()
