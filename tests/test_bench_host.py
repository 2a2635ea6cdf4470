"""Host logic of bench.py that needs no GPU (CPU only).

* roofline.traffic: the DRAM bytes recorded from an ncu capture are reported
  only while the kernel's source file still has the SHA-256 recorded with them,
  so a number taken on older code is never reported for newer code;
* the clock summary taken from nvidia-smi samples (median SM clock, maximum,
  throttle reasons seen);
* the roofline denominators: MEASURED_PEAKS.json, else the stated fallback;
* the reference arm (the oracle on the host cores) works and prints on rank 0
  only, with the warm-up steps it reports;
* on two gloo ranks: the set-up, the maximum of the ranks' timings that every
  rank sees, and the reference arm's single line from rank 0.
"""
import hashlib
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _table(tmp_path, src_rel, sha, value, workload="w-small", precision="ozaki", path="dense"):
    t = tmp_path / "traffic.md"
    t.write_text(
        "| workload | precision | path | kernel | source | sha256 | dram bytes per launch |\n"
        "|---|---|---|---|---|---|---|\n"
        f"| {workload} | {precision} | {path} | k_x | {src_rel} | {sha} | {value} |\n")
    return str(t)


def test_traffic_reported_only_for_the_recorded_source(tmp_path, monkeypatch):
    src = tmp_path / "kernel.cu"
    src.write_bytes(b"__global__ void k_x() {}\n")
    sha = hashlib.sha256(src.read_bytes()).hexdigest()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "TRAFFIC_TABLE", _table(tmp_path, "kernel.cu", sha, 123456789))
    assert bench.dram_traffic("w-small", "ozaki", "dense") == 123456789.0
    # another workload, precision or path has no number
    assert bench.dram_traffic("w-other", "ozaki", "dense") is None
    assert bench.dram_traffic("w-small", "fp64", "dense") is None
    assert bench.dram_traffic("w-small", "ozaki", "stacks") is None
    # the kernel changed after the capture: the number is withheld
    src.write_bytes(b"__global__ void k_x() { /* changed */ }\n")
    assert bench.dram_traffic("w-small", "ozaki", "dense") is None


def test_small_case_rows_listed_apart(tmp_path, monkeypatch):
    # captures of smaller cases of the same kernel are listed by workload; none
    # stands in for another workload's number
    src = tmp_path / "kernel.cu"
    src.write_bytes(b"k")
    sha = hashlib.sha256(b"k").hexdigest()
    t = tmp_path / "traffic.md"
    t.write_text("| workload | precision | path | kernel | source | sha256 | dram bytes per launch |\n"
                 "|---|---|---|---|---|---|---|\n"
                 f"| w-a | ozaki | dense | k_x | kernel.cu | {sha} | 10 |\n"
                 f"| w-b | ozaki | dense | k_x | kernel.cu | {sha} | 20 |\n"
                 f"| w-c | fp64 | dense | k_x | kernel.cu | {sha} | 30 |\n"
                 f"| w-d | ozaki | dense | k_x | kernel.cu | {'0' * 64} | 40 |\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "TRAFFIC_TABLE", str(t))
    assert bench.traffic_rows("ozaki", "dense") == {"w-a": 10.0, "w-b": 20.0}
    assert bench.dram_traffic("w-full", "ozaki", "dense") is None


def test_traffic_missing_or_malformed_gives_none(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "TRAFFIC_TABLE", str(tmp_path / "absent.md"))
    assert bench.dram_traffic("w-small", "ozaki", "dense") is None
    src = tmp_path / "kernel.cu"
    src.write_bytes(b"x")
    sha = hashlib.sha256(b"x").hexdigest()
    monkeypatch.setattr(bench, "TRAFFIC_TABLE", _table(tmp_path, "kernel.cu", sha, "n/a"))
    assert bench.dram_traffic("w-small", "ozaki", "dense") is None
    monkeypatch.setattr(bench, "TRAFFIC_TABLE", _table(tmp_path, "gone.cu", sha, 5))
    assert bench.dram_traffic("w-small", "ozaki", "dense") is None


def test_committed_traffic_rows_name_existing_sources():
    rows = [ln for ln in open(bench.TRAFFIC_TABLE).read().splitlines() if ln.count("|") == 8]
    data = [[c.strip() for c in r.strip().strip("|").split("|")] for r in rows[2:]]
    assert data, "no traffic rows"
    for cells in data:
        assert os.path.exists(os.path.join(ROOT, cells[4])), cells[4]
        assert len(cells[5]) == 64 and int(cells[5], 16) >= 0
        assert float(cells[6]) > 0


def test_clock_summary():
    c = bench.Clocks()
    c.lines = [
        "2026/12/04 10:00:00.100, 1965, 2070, 1180.2, Not Active, Not Active, Not Active, Active",
        "2026/12/04 10:00:00.200, 1890, 2070, 1201.0, Not Active, Not Active, Not Active, Active",
        "2026/12/04 10:00:00.300, 2010, 2070, 1150.7, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
        "2026/12/04 10:00:00.400, [N/A], 2070, 1, Not Active, Not Active, Not Active, Not Active",
    ]
    s = c.summary()
    assert s == {"sm_mhz": 1965.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3,
                 "power_w": 1180.2}
    c.lines.append("2026/12/04 10:00:00.500, 1200, 2070, 900.0, Active, Not Active, Active, Not Active")
    assert c.summary()["reasons"] == ["hw_slowdown", "sw_power_cap", "sw_thermal_slowdown"]
    # only the samples inside the timed region count
    t = bench.Clocks._when("2026/12/04 10:00:00.150")
    c.window(t, t + 0.2)
    s = c.summary()
    assert s["samples"] == 2 and s["sm_mhz"] == 1950.0 and s["reasons"] == ["sw_power_cap"]
    c.window(t + 10, t + 11)
    assert c.summary()["reasons"] == ["unsampled"]
    empty = bench.Clocks()
    assert empty.summary() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}


def test_peaks_measured_else_fallback(tmp_path, monkeypatch):
    p, src = bench.peaks()
    if os.path.exists(bench.PEAKS_FILE):
        assert src == "measured" and p["hbm_gbs"] > 0 and p["bf16_tflops"] > 0
    monkeypatch.setattr(bench, "PEAKS_FILE", str(tmp_path / "absent.json"))
    p, src = bench.peaks()
    assert src == "fallback"
    assert (p["hbm_gbs"], p["bf16_tflops"], p["bf16_tflops_sustained"]) == (6800.0, 1900.0, 1700.0)


def test_aggregate_value_counts_every_replica():
    # two replicas, 5 steps of 2e12 useful flops each, in 4 s: 5 TFLOP/s for the job
    assert bench.aggregate_value(2.0e12, 2, 5, 4.0) == 5.0


def test_reference_arm_runs_on_rank_zero_only(capsys):
    import argparse
    args = argparse.Namespace(workload="small-sparse", scale=1.0, occ=0.1, steps=1, warmup=3, ref_rows=4)
    assert bench.run_reference(args, 2, 1) == 0          # rank 1: no work, no line
    assert capsys.readouterr().out == ""
    assert bench.run_reference(args, 2, 0) == 0          # rank 0 prints the one line
    import json
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["warmup"] == 3
    assert line["cpu_baseline"]["kind"] == "oracle" and line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]


def _rank_worker(rank, world, port, out_dir):
    import argparse
    import contextlib
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    args = argparse.Namespace(impl="reference", workload="small-sparse", scale=1.0, occ=0.1, steps=1,
                              warmup=3, ref_rows=2)
    w, r, _ = bench.dist_setup(args)
    # each rank's timing differs; every rank must see the slowest one
    slowest = bench.max_over_ranks(1.5 + r, w)
    bench.barrier(w)
    with open(os.path.join(out_dir, f"out{rank}.txt"), "w") as f, contextlib.redirect_stdout(f):
        rc = bench.run_reference(args, w, r)
    with open(os.path.join(out_dir, f"max{rank}.txt"), "w") as f:
        f.write(f"{w} {r} {slowest} {rc}")


def test_two_gloo_ranks_reduce_max_and_print_once(tmp_path):
    import multiprocessing as mp
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_rank_worker, args=(r, 2, port, str(tmp_path))) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(2):
        w, rr, slowest, rc = (tmp_path / f"max{r}.txt").read_text().split()
        assert (int(w), int(rr), float(slowest), int(rc)) == (2, r, 2.5, 0)
    import json
    assert (tmp_path / "out1.txt").read_text() == ""          # rank 1: no work, no line
    lines = (tmp_path / "out0.txt").read_text().strip().splitlines()
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
