"""Autotuner of the FP64 stack kernels.

The paper's LIBCUSMM (Sec. II) tunes its kernels per block shape (m, n, k)
over read/write strategy, threads per block, elements per thread and tiling.
This library's FP64 stack kernels expose a smaller space (team of 1, 2 or 4
warps per C block, see dbcsr_opts.kernel; variant 1 runs as variant 0),
chosen per C-block shape (m, n). For each shape the tuner builds a synthetic
block-sparse product of that shape (inner sizes from the workload's set),
times every variant through the C ABI with the library's own CUDA-event
kernel timer, keeps the fastest and writes the table as JSON:

    {"device": ..., "entries": [[m, n, variant, tflops_best, {variant: tflops}], ...]}

``load_table`` hands a table to the library (dbcsr_set_tuning).

Usage (on the GPU): python -m paper_1910_04796_gb300.autotune --sizes 5 13 23 26 32 --out table.json

With --model the tuner times only a random fraction of the (m, n, k) shapes,
fits the regression-tree performance model of ``perfmodel`` to them and
predicts the variant of every (m, n) and of every (m, n, k) up to --max-edge
(the paper's approach to a kernel space too large to time exhaustively; the
library applies the (m, n, k) choice by the inner size of a C block's first
product). The model file holds the (m, n) entries, the (m, n, k) table as a
string of variant digits ("variants_mnk") and the training records, so a
refit needs no GPU (--records). With --evaluate it also times the held-out
shapes and reports how close each table's choices come to the measured
optimum, and how the library does applying both tables (kernel 0) beside a
forced run of the variant the (m, n, k) table chose.
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
# every (m, n) up to 32 predicted by the regression-tree model from a 20 % sample
MODEL_TABLE = os.path.join(HERE, "tuning", "gb300_fp64_model.json")


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


def applied_tflops(m, n, k, variant, reps=3, seed=0):
    """TFLOP/s of the library's own choice (kernel 0: the tuning tables) and of
    the forced ``variant``, timed alternately on the same (m, n, k) case."""
    A, B = _case(m, n, [k], seed)
    Ag, Bg = dbcsr.Matrix.from_blocks(A), dbcsr.Matrix.from_blocks(B)
    Cg = dbcsr.Matrix.create(A.row_sizes, B.col_sizes, np.zeros(0, np.int32), np.zeros(0, np.int32))
    times = {0: [], variant + 1: []}
    for _ in range(reps + 1):
        for kern in times:
            dbcsr.multiply("N", "N", 1.0, Ag, Bg, 0.0, Cg, path="stacks", kernel=kern, timing=True)
            st = dbcsr.stats()
            times[kern].append(st["ms_kernel"])
    for M in (Ag, Bg, Cg):
        M.release()
    return tuple(st["useful_flops"] / (statistics.median(times[kern][1:]) / 1e3) / 1e12 for kern in times)


def measure(shapes, reps=3, seed=0):
    """Records (m, n, k, variant, TFLOP/s) of every variant on each (m, n, k) shape."""
    out = []
    for i, (m, n, k) in enumerate(shapes):
        _, res = tune_shape(int(m), int(n), [int(k)], reps, seed + i)
        out += [(int(m), int(n), int(k), v, float(t)) for v, t in res.items()]
    return out


def encode_mnk(entries_mnk, max_edge):
    """The (m, n, k) table as one string of variant digits, index
    ((m-1)*E + (n-1))*E + (k-1) for E = max_edge."""
    d = np.zeros((max_edge, max_edge, max_edge), np.int8)
    for m, n, k, v in entries_mnk:
        d[m - 1, n - 1, k - 1] = v
    return "".join(map(str, d.ravel().tolist()))


def decode_mnk(code, max_edge):
    d = np.frombuffer(code.encode(), np.uint8).astype(np.int32) - ord("0")
    d = d.reshape(max_edge, max_edge, max_edge)
    return [(m + 1, n + 1, k + 1, int(d[m, n, k])) for m in range(max_edge) for n in range(max_edge)
            for k in range(max_edge)]


def model_tune(sizes, train_frac, reps, max_edge, evaluate, seed=0, recs=None):
    """Fit the performance model on a random subset of shapes.

    Returns (per-(m, n) entries, per-(m, n, k) entries, report, training
    records); ``recs`` (records of an earlier run) skips the timing of the
    training shapes.
    """
    import itertools
    from . import perfmodel
    shapes = list(itertools.product(sizes, sizes, sizes))
    rng = np.random.default_rng(seed)
    rng.shuffle(shapes)
    ntrain = max(1, int(round(train_frac * len(shapes))))
    train, held = shapes[:ntrain], shapes[ntrain:]
    if recs is None:
        recs = measure(train, reps, seed)
    model = perfmodel.PerfModel(perfmodel.RandomForest(seed=seed)).fit(recs)
    edges = range(1, max_edge + 1)
    entries = [[m, n, v, t, {}] for (m, n, v, t) in model.table(edges, edges, sizes)]
    entries_mnk = [[m, n, k, v] for (m, n, k, v, t) in model.table_mnk(edges, edges, edges)]
    report = {"shapes": len(shapes), "timed_for_training": len(train), "train_frac": train_frac,
              "sizes": list(map(int, sizes))}
    if evaluate and held:
        hrec = measure(held, reps, seed + 10_000)
        measured = {}
        for (m, n, k, v, t) in hrec:
            measured.setdefault((m, n, k), {})[v] = t
        chosen = {s: model.best_variant(*s) for s in measured}
        report["held_out_model"] = perfmodel.choice_quality(measured, chosen)
        report["held_out_default_variant0"] = perfmodel.choice_quality(measured, {s: 0 for s in measured})
        # the tables the library uses: per (m, n), and per (m, n, k) where set
        tab = {(e[0], e[1]): e[2] for e in entries}
        report["held_out_mn_table"] = perfmodel.choice_quality(measured, {s: tab[(s[0], s[1])] for s in measured})
        tab3 = {(e[0], e[1], e[2]): e[3] for e in entries_mnk}
        report["held_out_mnk_table"] = perfmodel.choice_quality(measured, {s: tab3[s] for s in measured})
        # the library applying both tables (kernel 0), timed on the held-out
        # cases beside a forced run of the variant the (m, n, k) table chose
        dbcsr.set_tuning([(e[0], e[1], e[2]) for e in entries])
        dbcsr.set_tuning_mnk(entries_mnk)
        try:
            best_r, chosen_r = [], []
            for i, sh in enumerate(held):
                sh = tuple(int(x) for x in sh)
                ta, tf = applied_tflops(*sh, tab3[sh], reps=reps, seed=seed + 10_000 + i)
                best_r.append(ta / max(measured[sh].values()))
                chosen_r.append(ta / tf)
        finally:
            dbcsr.set_tuning_mnk([])
            dbcsr.set_tuning([])
        best_r, chosen_r = np.asarray(best_r), np.asarray(chosen_r)
        report["held_out_library_applied"] = {
            "shapes": len(best_r), "mean_of_best": float(best_r.mean()), "min_of_best": float(best_r.min()),
            "within_5pct": float(np.mean(best_r >= 0.95)),
            "mean_of_forced_choice": float(chosen_r.mean()), "min_of_forced_choice": float(chosen_r.min())}
    return entries, entries_mnk, report, recs


def tune(msizes, nsizes, ksizes, reps=3):
    entries = []
    for m in msizes:
        for n in nsizes:
            best, res = tune_shape(int(m), int(n), ksizes, reps)
            entries.append([int(m), int(n), int(best), res[best], {str(k): v for k, v in res.items()}])
    return entries


def load_table(path=DEFAULT_TABLE, model_path=MODEL_TABLE) -> bool:
    """Hand the tuning tables to the library: the model's predictions for every
    (m, n), overridden by the shapes that were timed (dbcsr_set_tuning), and
    the model's per-(m, n, k) predictions where the model file has them
    (dbcsr_set_tuning_mnk); False if neither file exists."""
    entries, mnk = {}, []
    for p in (model_path, path):
        if p and os.path.exists(p):
            with open(p) as f:
                d = json.load(f)
            for e in d["entries"]:
                entries[(int(e[0]), int(e[1]))] = int(e[2])
            if p == model_path and "variants_mnk" in d:
                mnk = decode_mnk(d["variants_mnk"]["variants"], int(d["variants_mnk"]["max_edge"]))
    if not entries and not mnk:
        return False
    dbcsr.set_tuning([(m, n, v) for (m, n), v in sorted(entries.items())])
    dbcsr.set_tuning_mnk(mnk)
    return True


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--sizes", type=int, nargs="+", default=[5, 13, 22, 23, 26, 32])
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--out", default=DEFAULT_TABLE)
    ap.add_argument("--model", action="store_true", help="time a subset, predict the rest (regression trees)")
    ap.add_argument("--train-frac", type=float, default=0.2)
    ap.add_argument("--max-edge", type=int, default=32, help="table covers m, n = 1 .. max-edge")
    ap.add_argument("--evaluate", action="store_true", help="also time the held-out shapes and score the model")
    ap.add_argument("--report", default=None, help="JSON file for the model's evaluation")
    ap.add_argument("--records", default=None,
                    help="reuse the training records of this model file instead of timing the training shapes")
    args = ap.parse_args()
    import torch
    dbcsr.init()
    if args.model:
        recs = None
        if args.records:
            with open(args.records) as f:
                recs = [tuple(r) for r in json.load(f)["records"]]
        entries, entries_mnk, report, recs = model_tune(args.sizes, args.train_frac, args.reps, args.max_edge,
                                                        args.evaluate, recs=recs)
        with open(args.out, "w") as f:
            json.dump({"device": torch.cuda.get_device_name(), "kernel": "FP64 stack kernels",
                       "model": "random forest of regression trees", "report": report, "entries": entries,
                       "variants_mnk": {"max_edge": args.max_edge,
                                        "index": "((m-1)*max_edge + (n-1))*max_edge + (k-1)",
                                        "variants": encode_mnk(entries_mnk, args.max_edge)},
                       "records": [list(r) for r in recs]}, f, indent=1)
        if args.report:
            with open(args.report, "w") as f:
                json.dump(report, f, indent=1)
        print(json.dumps(report, indent=1))
        return
    entries = tune(args.sizes, args.sizes, args.sizes, args.reps)
    os.makedirs(os.path.dirname(os.path.abspath(args.out)), exist_ok=True)
    with open(args.out, "w") as f:
        json.dump({"device": torch.cuda.get_device_name(), "kernel": "FP64 stack kernels",
                   "entries": entries}, f, indent=1)
    for e in entries:
        print(e[0], e[1], "best variant", e[2], f"{e[3]:.3f} TFLOP/s", e[4])


if __name__ == "__main__":
    main()
