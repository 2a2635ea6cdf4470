"""CPU tests of the distributed exchange (Sec. II: Cannon for general shapes,
an O(1)-communication scheme for tall-skinny shapes) on gloo ranks.

The local product on the CPU ranks is the oracle's (tests may call it); the
exchange, the skew and shift schedule and the partial-sum reduction are the
library's. Pinned against the oracle's single-process product of the same
matrices: same result pattern, normwise difference within 1e-13 (the
distributed sum adds the inner panels in a different order).
"""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from oracle import oracle as O
from paper_1910_04796_gb300 import cannon, synth


def _oracle_mm(Ap, Bp, Cacc):
    r = O.multiply("N", "N", 1.0, Ap, Bp, 1.0 if Cacc is not None else 0.0, Cacc)
    return synth.BlockSparse(np.asarray(r.row_sizes, np.int32), np.asarray(r.col_sizes, np.int32),
                             np.asarray(r.blk_row, np.int32), np.asarray(r.blk_col, np.int32), np.asarray(r.data))


def _mats(seed, nbr=11, nbk=13, nbc=9, p=0.35):
    rng = np.random.default_rng(seed)
    return synth.random_small(rng, nbr, nbk, nbc, p=p, sizes=(2, 3, 5, 7))[:2]


def test_split_and_schedule():
    assert cannon.split_ranges(10, 3) == [(0, 4), (4, 7), (7, 10)]
    assert cannon.split_ranges(2, 3) == [(0, 1), (1, 2), (2, 2)]
    for q in (1, 2, 3, 4):
        for i in range(q):
            for j in range(q):
                s = cannon.cannon_schedule(q, i, j)
                assert sorted(s) == list(range(q))          # every inner panel exactly once
                # after each shift the left neighbour holds what this rank held
                for t in range(q - 1):
                    assert cannon.cannon_schedule(q, i, (j - 1) % q)[t + 1] == s[t]
                    assert cannon.cannon_schedule(q, (i - 1) % q, j)[t + 1] == s[t]
    with pytest.raises(ValueError):
        cannon.grid_side(3)


def test_panels_reassemble():
    A, _ = _mats(1)
    parts = []
    for r in cannon.split_ranges(len(A.row_sizes), 3):
        for c in cannon.split_ranges(len(A.col_sizes), 2):
            parts.append((cannon.sub_panel(A, r, c), r[0], c[0]))
    M = cannon.place(parts, A.row_sizes, A.col_sizes)
    assert np.array_equal(O.densify(M), O.densify(A))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, kind, seed, out_dir):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    A, B = _mats(seed)
    if kind == "cannon":
        C, (r0, c0) = cannon.cannon_multiply(A, B, rank, world, local_mm=_oracle_mm)
        np.savez(os.path.join(out_dir, f"c{rank}.npz"), rs=C.row_sizes, cs=C.col_sizes, br=C.blk_row,
                 bc=C.blk_col, data=C.data, r0=r0, c0=c0)
    else:
        C = cannon.tallskinny_multiply(A, B, rank, world, local_mm=_oracle_mm)
        if rank == 0:
            np.savez(os.path.join(out_dir, "c0.npz"), rs=C.row_sizes, cs=C.col_sizes, br=C.blk_row,
                     bc=C.blk_col, data=C.data, r0=0, c0=0)
    dist.barrier()
    dist.destroy_process_group()


def _run(kind, world, seed, tmp_path):
    ctx = mp.get_context("spawn")
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, kind, seed, str(tmp_path))) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    A, B = _mats(seed)
    parts = []
    for f in sorted(os.listdir(tmp_path)):
        z = np.load(os.path.join(tmp_path, f))
        parts.append((synth.BlockSparse(z["rs"], z["cs"], z["br"], z["bc"], z["data"]), int(z["r0"]), int(z["c0"])))
    got = cannon.place(parts, A.row_sizes, B.col_sizes)
    ref = O.multiply("N", "N", 1.0, A, B, 0.0)
    assert np.array_equal(got.blk_row, ref.blk_row) and np.array_equal(got.blk_col, ref.blk_col)
    err = O.normwise_error(O.densify(got), O.densify(ref), O.densify(A), O.densify(B))
    assert err <= 1e-13


@pytest.mark.parametrize("world", [1, 4])
def test_cannon_matches_single_process(world, tmp_path):
    _run("cannon", world, 11, tmp_path)


@pytest.mark.parametrize("world", [2, 3])
def test_tallskinny_matches_single_process(world, tmp_path):
    _run("tallskinny", world, 12, tmp_path)
