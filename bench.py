#!/usr/bin/env python3
"""Benchmark of the GB300 local block-sparse multiply C = alpha*op(A)*op(B) + beta*C.

Metric: useful FP64 TFLOP/s -- sum over the block products the multiply needs
of 2*m*n*k, divided by the time of one whole dbcsr_multiply (stack
generation or densification, the product kernels, undensification), inputs
resident in HBM. Densified zeros and emulation slice work are not counted.

Default workload: the dense limit, N = 11'264 as a 512 x 512 grid of 22 x 22
blocks at 100% occupancy, entries U[-1,1], C = A*B + C (beta = 1). It is the
paper's "square matrix" experiment with its block size 22 (Sec. IV), scaled
to one GPU. Every input is larger than L2 (1 GB each, L2 is 129 MB), so no
flush is needed between steps.

One JSON line on stdout (rank 0). ``--impl reference`` times the CPU oracle
(the plain FP64 block-triple loop) on a bounded sample of the same workload.
Multi-GPU: replicas only (the single-GPU product does not shard here); each
rank runs its own replica, value = all ranks' useful flops / max time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}
# nominal dense rates (TFLOP/s) used to scale the measured bf16 peak to other dtypes
NOMINAL = {"bf16": 2250.0, "tf32": 1100.0, "fp64": 1.25}


def peaks():
    try:
        with open(PEAKS_FILE) as f:
            p = json.load(f)
        return p, "measured"
    except Exception:
        return dict(FALLBACK), "fallback"


TRAFFIC_TABLE = os.path.join(ROOT, "profiles", "dram_traffic.md")


def traffic_rows(precision, path):
    """{workload: DRAM bytes (read + write) per launch of the dominant kernel}
    from the ncu captures recorded in profiles/dram_traffic.md, for rows whose
    kernel source file is unchanged since (its SHA-256 is recorded with the
    number)."""
    import hashlib
    try:
        lines = open(TRAFFIC_TABLE).read().splitlines()
    except OSError:
        return {}
    out = {}
    for ln in lines:
        cells = [c.strip() for c in ln.strip().strip("|").split("|")]
        if len(cells) != 7 or cells[1] != precision or cells[2] != path:
            continue
        try:
            with open(os.path.join(ROOT, cells[4]), "rb") as f:
                if hashlib.sha256(f.read()).hexdigest() != cells[5]:
                    continue
            out[cells[0]] = float(cells[6])
        except (OSError, ValueError):
            continue
    return out


def dram_traffic(workload_name, precision, path):
    """DRAM bytes per launch of the dominant kernel on this workload, or None
    (no capture of it, or the kernel changed since)."""
    return traffic_rows(precision, path).get(workload_name)


def workload(name, scale, occ=0.1):
    from paper_1910_04796_gb300 import synth
    if name == "dense-limit":
        nblk = max(2, int(round(512 * scale)))
        return synth.workload_dense_limit(seed=1, nblk=nblk, bs=22)
    if name == "small-sparse":
        return synth.workload_small_sparse(0)
    if name == "uneven":
        nblk = max(10, int(round(4000 * scale)))
        return synth.workload_uneven(seed=3, nblk=nblk, width=max(1, int(400 * scale)))
    if name == "precision-dense":
        n = max(64, int(round(16384 * scale / 32)) * 32)
        return synth.workload_precision_dense(seed=4, n=n)
    if name == "precision-sparse":
        nblk = max(8, int(round(1024 * scale)))
        return synth.workload_precision_sparse(seed=5, nblk=nblk)
    if name == "hybrid":
        nblk = max(16, int(round(256 * scale)))
        return synth.workload_hybrid(seed=6, nblk=nblk, panel=max(1, nblk // 16))
    if name == "occupancy":
        nblk = max(8, int(round(256 * scale)))
        w = synth.workload_precision_sparse(seed=7, nblk=nblk, occ=occ)
        w.name = f"occupancy-{occ:g}-{nblk}x{nblk}-bs32"
        return w
    if name.startswith("tall-skinny"):
        v = name.split("-")[-1]
        mn = max(64, int(round(4096 * scale / 32)) * 32)
        kk = max(64, int(round(131072 * scale / 32)) * 32)
        return synth.workload_tall_skinny(seed=2, variant=v, mn=mn, kk=kk)
    raise SystemExit(f"unknown workload {name}")


class Clocks:
    """nvidia-smi sampling of SM clocks, board power and throttle reasons.

    Each sample carries nvidia-smi's own timestamp; ``window(t0, t1)`` (host
    time.time() values) restricts the summary to the samples taken inside the
    timed region. Sampling starts before the warm-up, so that the region is
    covered from its first step."""
    Q = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []
        self.t0 = self.t1 = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def window(self, t0, t1):
        self.t0, self.t1 = t0, t1

    @staticmethod
    def _when(stamp):
        import datetime
        try:
            return datetime.datetime.strptime(stamp, "%Y/%m/%d %H:%M:%S.%f").timestamp()
        except ValueError:
            return None

    def summary(self):
        sm, mx, pw, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 8:
                continue
            if self.t0 is not None:
                w = self._when(f[0])
                if w is None or w < self.t0 or w > self.t1:
                    continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            try:
                pw.append(float(f[3]))
            except ValueError:
                pass
            for n, v in zip(names, f[4:8]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm), "power_w": statistics.median(pw) if pw else None}


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        if args.impl == "reference":     # the oracle runs on the host cores: no GPU
            dist.init_process_group("gloo")
        else:
            torch.cuda.set_device(local)
            dist.init_process_group("nccl")
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    """Largest value over the ranks (timings: the job ends with its slowest rank)."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_value(useful_flops_per_step, world, steps, seconds):
    """Whole-job TFLOP/s: every rank ran `steps` steps of the same workload (replicas)."""
    return useful_flops_per_step * world * steps / seconds / 1e12


def cpu_oracle_sample(w, rows, threads=0):
    """Time the CPU oracle on the given C block rows of the workload."""
    from oracle import oracle as O
    t0 = time.perf_counter()
    O.multiply(w.transa, w.transb, w.alpha, w.A, w.B, w.beta, w.C, rows=rows, nthreads=threads)
    dt = time.perf_counter() - t0
    # useful flops of the sampled rows: sum over products in those rows of 2*m*n*k
    A, B = w.A, w.B
    ta, tb = w.transa in "TC", w.transb in "TC"
    a_r = A.blk_col if ta else A.blk_row
    a_k = A.blk_row if ta else A.blk_col
    a_m = (A.col_sizes if ta else A.row_sizes)
    kk = (A.row_sizes if ta else A.col_sizes)
    b_k = B.blk_col if tb else B.blk_row
    b_j = B.blk_row if tb else B.blk_col
    b_n = (B.row_sizes if tb else B.col_sizes)
    nk = len(kk)
    bn_sum = np.zeros(nk)
    np.add.at(bn_sum, b_k, b_n[b_j].astype(np.float64))
    sel = np.isin(a_r, np.asarray(rows))
    fl = float((2.0 * a_m[a_r[sel]] * kk[a_k[sel]] * bn_sum[a_k[sel]]).sum())
    return fl, dt


def run_reference(args, world, rank):
    """Reference arm: the CPU oracle as it stands, on a bounded sample of the workload."""
    if rank != 0:
        return 0
    from oracle import oracle as O
    w = workload(args.workload, args.scale, args.occ)
    nrows = len(w.A.col_sizes if w.transa in "TC" else w.A.row_sizes)
    threads = O.threads()
    rows = list(range(0, nrows, max(1, nrows // max(1, args.ref_rows))))[:args.ref_rows]
    vals = []
    for _ in range(args.warmup):   # warm-up steps of one C block row each
        cpu_oracle_sample(w, rows[:1], threads)
    flops_tot, t_tot = 0.0, 0.0
    for _ in range(args.steps):
        fl, dt = cpu_oracle_sample(w, rows, threads)
        flops_tot += fl
        t_tot += dt
        vals.append(fl / dt / 1e12)
    value = flops_tot / t_tot / 1e12
    sample = f"{len(rows)} of {nrows} C block rows per step (oracle, OpenMP over C block rows)"
    line = {
        "impl": "reference", "metric": "useful FP64 TFLOP/s, block-sparse C+=A*B", "value": value,
        "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000.0 * t_tot / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w.name, "sample": sample, "warmup_sample": "one C block row per warm-up step"},
        "cpu_baseline": {"value": value, "unit": "TFLOP/s", "cores": threads, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def time_steps(fn, steps, warmup, world, region=False):
    """Seconds of `steps` calls of fn on the device (CUDA events), and of wall
    time; with region=True also the host time.time() bounds of the timed steps."""
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    h0 = time.time()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    h1 = time.time()
    barrier(world)
    wall = time.perf_counter() - t0
    if region:
        return e0.elapsed_time(e1) / 1000.0, wall, (h0, h1)
    return e0.elapsed_time(e1) / 1000.0, wall


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="dense-limit")
    ap.add_argument("--scale", type=float, default=1.0)
    ap.add_argument("--precision", default="auto", choices=["auto", "fp64", "ozaki", "tf32", "fp32"])
    ap.add_argument("--path", default="auto", choices=["auto", "stacks", "dense", "hybrid"])
    ap.add_argument("--slices", type=int, default=0)
    ap.add_argument("--occ", type=float, default=0.1, help="block occupancy of the 'occupancy' workload")
    ap.add_argument("--hybrid-panel", type=int, default=-1,
                    help="block rows per panel on the hybrid path (-1: the workload's panel height, else automatic)")
    ap.add_argument("--hybrid-fill", type=int, default=0, help="densify panels at least this %% occupied (0: 50)")
    ap.add_argument("--kernel", type=int, default=0,
                    help="stack kernel choice passed to dbcsr_multiply (0 = automatic)")
    ap.add_argument("--ref-rows", type=int, default=48, help="C block rows per oracle sample")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--e2e-serial", action="store_true",
                    help="end to end: wait for each upload before the next call (the copies do not overlap)")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-legs", action="store_true", help="skip the plain-FP64 comparison legs")
    args = ap.parse_args()
    world, rank, local = dist_setup(args)
    if args.impl == "reference":
        return run_reference(args, world, rank)

    import torch
    from paper_1910_04796_gb300 import dbcsr

    torch.cuda.set_device(local)
    dbcsr.init()
    pk, pk_kind = peaks()
    from paper_1910_04796_gb300 import autotune
    tuned = autotune.load_table()   # per-shape FP64 stack-kernel choice, if tuned on this GPU type
    w = workload(args.workload, args.scale, args.occ)
    precision = args.precision
    if precision == "auto":
        precision = "ozaki" if dbcsr.has_precision("ozaki") else "fp64"
    rs = w.A.col_sizes if w.transa in "TC" else w.A.row_sizes
    cs = w.B.row_sizes if w.transb in "TC" else w.B.col_sizes

    # resident inputs (device data, created once)
    A = dbcsr.Matrix.from_blocks(w.A)
    B = dbcsr.Matrix.from_blocks(w.B)
    C0 = w.C
    if C0 is not None:
        Cm = dbcsr.Matrix.from_blocks(C0)
    else:
        Cm = dbcsr.Matrix.create(rs, cs, np.zeros(0, np.int32), np.zeros(0, np.int32))

    hpanel = args.hybrid_panel if args.hybrid_panel >= 0 else int(w.extra.get("panel", 0))

    def step(prec=precision, path=args.path, timing=False):
        dbcsr.multiply(w.transa, w.transb, w.alpha, A, B, w.beta, Cm, path=path, precision=prec,
                       ozaki_slices=args.slices, kernel=args.kernel, timing=timing, hybrid_panel=hpanel,
                       hybrid_fill_pct=args.hybrid_fill)

    step()
    st = dbcsr.stats()
    useful = st["useful_flops"]
    with Clocks(local) as clk:
        time.sleep(0.5)   # the sampler's first lines come after its start-up
        secs, wall, region = time_steps(step, args.steps, max(args.warmup, 3) - 1, world, region=True)
        clk.window(*region)
    launches = dbcsr.stats()["kernel_launches"] * args.steps
    secs = max_over_ranks(secs, world)
    value = aggregate_value(useful, world, args.steps, secs)
    # live timing of the dominant kernel (CUDA events on the library stream)
    mains, totals = [], []
    for _ in range(max(1, min(3, args.steps))):
        step(timing=True)
        s2 = dbcsr.stats()
        # the hybrid path runs several product kernels: time the whole product phase
        mains.append(s2["ms_main"] if s2["path"] == dbcsr.PATH_HYBRID else s2["ms_kernel"])
        totals.append(s2["ms_total"])
    main_ms = statistics.median(mains)
    s2 = dbcsr.stats()
    path_taken = {dbcsr.PATH_DENSE: "dense", dbcsr.PATH_STACKS: "stacks", dbcsr.PATH_HYBRID: "hybrid"}[s2["path"]]
    if precision == "fp64" and path_taken == "stacks":
        # DFMA on the CUDA cores' FP64 pipe: SMs x 2 FMAs per clock (the nominal
        # 1.25 TFLOP/s at 2 070 MHz over 152 SMs) x 2 flops x the SM clock seen under load
        bound, unit = "alu", "TFLOP/s"
        sms = torch.cuda.get_device_properties(local).multi_processor_count
        mhz = clk.summary().get("sm_mhz") or clk.summary().get("sm_max_mhz") or 2070.0
        peak = sms * 2 * 2 * mhz * 1e6 / 1e12
        peak_note = f"FP64 FMA = {sms} SMs x 2 per clock x 2 x {mhz:.0f} MHz"
        achieved = s2["main_flops"] / (main_ms / 1e3) / 1e12
    elif precision == "fp64":
        # FP64 tensor-core MMA (dense) or a mix (hybrid): the measured bf16 rate x the nominal ratio
        bound, unit = "tensor", "TFLOP/s"
        peak = pk["bf16_tflops"] * NOMINAL["fp64"] / NOMINAL["bf16"]
        peak_note = f"FP64 = {pk_kind} bf16 burst x nominal FP64/bf16 (1.25/2250)"
        achieved = s2["main_flops"] / (main_ms / 1e3) / 1e12
    elif precision == "ozaki":
        bound, unit = "tensor", "TFLOP/s"
        peak = pk["bf16_tflops_sustained"] if main_ms > 1000 else pk["bf16_tflops"]
        peak_note = f"bf16 {'sustained' if main_ms > 1000 else 'burst'} ({pk_kind})"
        achieved = s2["main_flops"] / (main_ms / 1e3) / 1e12
    elif precision == "fp32":
        # plain FP32 FMA on the CUDA cores: SMs x 128 lanes x 2 flops x the SM clock seen under load
        bound, unit = "alu", "TFLOP/s"
        sms = torch.cuda.get_device_properties(local).multi_processor_count
        mhz = clk.summary().get("sm_mhz") or clk.summary().get("sm_max_mhz") or 2070.0
        peak = sms * 128 * 2 * mhz * 1e6 / 1e12
        peak_note = f"FP32 FMA = {sms} SMs x 128 lanes x 2 x {mhz:.0f} MHz"
        achieved = s2["main_flops"] / (main_ms / 1e3) / 1e12
    else:
        bound, unit = "tensor", "TFLOP/s"
        peak = pk["bf16_tflops"] * NOMINAL["tf32"] / NOMINAL["bf16"]
        peak_note = f"TF32 = {pk_kind} bf16 burst x nominal TF32/bf16 (1100/2250)"
        achieved = s2["main_flops"] / (main_ms / 1e3) / 1e12
    roofline = {"bound": bound, "achieved": achieved, "peak": peak, "unit": unit, "frac": achieved / peak,
                "traffic": dram_traffic(w.name, precision, path_taken),
                # captures of smaller cases of the same kernel (their own workloads;
                # traffic does not grow in proportion to the work, so none is scaled)
                "traffic_small_cases": {k: v for k, v in traffic_rows(precision, path_taken).items()
                                        if k != w.name} or None,
                "kernel_ms": main_ms,
                "algorithmic_flops": s2["main_flops"], "peak_source": peak_note}

    # end to end through the C ABI with host buffers (H2D of inputs and D2H of C inside);
    # measured before the comparison legs, which leave large allocations and a hot GPU behind
    e2e = None
    if not args.no_e2e:
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()
        hA, hB = pin(w.A.data), pin(w.B.data)
        hC = pin(C0.data) if C0 is not None else None
        # the result is read into pinned host memory too (allocated once, like the inputs)
        hOut = pin(np.zeros(max(1, int(Cm.info()[3])), np.float64))
        out = None

        phases = []   # host time per step of the creates, the multiply and the read-back

        def e2e_step():
            nonlocal out
            t0 = time.perf_counter()
            # --e2e-serial: every upload finished before the next call (no overlap)
            wait = dbcsr.sync if args.e2e_serial else (lambda: None)
            Ah = dbcsr.Matrix.create(w.A.row_sizes, w.A.col_sizes, w.A.blk_row, w.A.blk_col, hA)
            wait()
            Bh = dbcsr.Matrix.create(w.B.row_sizes, w.B.col_sizes, w.B.blk_row, w.B.blk_col, hB)
            wait()
            if C0 is not None:
                Ch = dbcsr.Matrix.create(C0.row_sizes, C0.col_sizes, C0.blk_row, C0.blk_col, hC)
            else:
                Ch = dbcsr.Matrix.create(rs, cs, np.zeros(0, np.int32), np.zeros(0, np.int32))
            wait()
            t1 = time.perf_counter()
            dbcsr.multiply(w.transa, w.transb, w.alpha, Ah, Bh, w.beta, Ch, path=args.path, precision=precision,
                           ozaki_slices=args.slices, kernel=args.kernel, hybrid_panel=hpanel,
                           hybrid_fill_pct=args.hybrid_fill)
            t2 = time.perf_counter()
            out = Ch.data(hOut)
            t3 = time.perf_counter()
            for m in (Ah, Bh, Ch):
                m.release()
            phases.append((t1 - t0, t2 - t1, t3 - t2, time.perf_counter() - t0))

        e2e_steps = max(1, args.steps)
        s_e2e, _ = time_steps(e2e_step, e2e_steps, 2, world)
        s_e2e = max_over_ranks(s_e2e, world)
        timed = phases[-e2e_steps:]
        h2d = (hA.nbytes + hB.nbytes + (hC.nbytes if hC is not None else 0)
               + 4 * 2 * (w.A.nblks + w.B.nblks + (C0.nblks if C0 is not None else 0)))
        e2e = {"value": useful * world * e2e_steps / s_e2e / 1e12, "unit": "TFLOP/s",
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(out.nbytes if out is not None else 0),
               # median host time of each call group per step: the creates return while
               # page-locked values still copy, so their copies overlap the multiply
               "phases_ms": {k: 1e3 * statistics.median(p[q] for p in timed)
                             for q, k in enumerate(("creates", "multiply", "read_back"))},
               # host time of whole steps: a few slow steps (shared host links) pull the mean down
               "step_ms": {"median": 1e3 * statistics.median(p[3] for p in timed),
                           "max": 1e3 * max(p[3] for p in timed)}}

    # comparison legs on the same GPU and inputs: the plain FP64 paths, the
    # emulated and TF32 paths with their error against the GPU FP64 result
    legs, accuracy = {}, {}
    if not args.no_legs and rank == 0:
        dense_ok = w.A.nblks == len(w.A.row_sizes) * len(w.A.col_sizes)
        combos = [("fp64_stacks", "fp64", "stacks"), ("ozaki_stacks", "ozaki", "stacks")]
        if dense_ok:
            combos = [("fp64_dense", "fp64", "dense"), ("ozaki_dense", "ozaki", "dense"),
                      ("tf32_dense", "tf32", "dense")] + combos
        ref_c = None
        for name, prec, path in combos:
            try:
                Cl = dbcsr.Matrix.from_blocks(C0) if C0 is not None else dbcsr.Matrix.create(
                    rs, cs, np.zeros(0, np.int32), np.zeros(0, np.int32))
                dbcsr.multiply(w.transa, w.transb, w.alpha, A, B, w.beta, Cl, path=path, precision=prec,
                               timing=True)
                legs[name] = useful / (dbcsr.stats()["ms_total"] / 1e3) / 1e12
                out = Cl.data_device()
                if prec == "fp64" and ref_c is None:
                    ref_c = out
                elif ref_c is not None and out.numel() == ref_c.numel():
                    nA = float(torch.linalg.vector_norm(A.data_device()))
                    nB = float(torch.linalg.vector_norm(B.data_device()))
                    accuracy[name + "_vs_fp64"] = float(torch.linalg.vector_norm(out - ref_c)) / (nA * nB)
                Cl.release()
            except Exception as e:  # report, do not hide
                legs[name] = f"error: {e}"
        if args.workload == "small-sparse":
            # the kept plan + CUDA graph replay of the same multiply (latency-bound case)
            Cl = dbcsr.Matrix.create(rs, cs, np.zeros(0, np.int32), np.zeros(0, np.int32))
            dbcsr.multiply("N", "N", 1.0, A, B, 0.0, Cl, path="stacks", reuse_plan=True)
            s_rep, _ = time_steps(lambda: dbcsr.multiply("N", "N", 1.0, A, B, 0.0, Cl, path="stacks",
                                                         reuse_plan=True), 50, 3, 1)
            legs["fp64_stacks_graph_replay"] = useful * 50 / s_rep / 1e12
            legs["graph_replay_us_per_multiply"] = s_rep / 50 * 1e6
            Cl.release()

    cpu = None
    if not args.no_cpu and rank == 0 and world == 1:
        from oracle import oracle as O
        nrows = len(rs)
        nsel = min(args.ref_rows, nrows)
        rows = list(range(0, nrows, max(1, nrows // nsel)))[:nsel]
        fl, dt = cpu_oracle_sample(w, rows, O.threads())
        cpu = {"value": fl / dt / 1e12, "unit": "TFLOP/s", "cores": O.threads(), "kind": "oracle",
               "sample": f"{len(rows)} of {nrows} C block rows ({dt:.1f} s)"}
        # the same oracle on one thread, on an eighth of that sample
        rows1 = rows[::8] or rows[:1]
        fl1, dt1 = cpu_oracle_sample(w, rows1, 1)
        cpu["single_thread"] = {"value": fl1 / dt1 / 1e12, "unit": "TFLOP/s", "cores": 1,
                                "sample": f"{len(rows1)} of {nrows} C block rows ({dt1:.1f} s)"}

    if rank == 0:
        line = {
            "metric": "useful FP64 TFLOP/s, block-sparse C+=A*B", "value": value, "unit": "TFLOP/s",
            "n_gpus": world, "steps": args.steps, "warmup": max(args.warmup, 3),
            "ms_per_step": 1000.0 * secs / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64" if precision == "fp64" else
            ("f64 (emulated: int8-valued slices on bf16 tensor cores)" if precision == "ozaki" else
             "f32" if precision == "fp32" else "tf32"),
            "data": "synthetic",
            "config": {"workload": w.name, "path": path_taken, "precision": precision,
                       "useful_flops_per_step": useful, "n_products": st["n_products"],
                       "l2": "inputs larger than L2 (no flush)" if useful > 1e9 else "inputs in L2",
                       **({"dense_panels": s2["dense_panels"]} if path_taken == "hybrid" else {}),
                       "parallelism": f"replicas x{world}"},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches),
            "clocks": clk.summary(), "legs_tflops": legs, "accuracy_normwise": accuracy,
            "tuned_table": tuned, "wall_s": wall,
        }
        print(json.dumps(line), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
