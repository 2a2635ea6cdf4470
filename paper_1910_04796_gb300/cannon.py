"""Distributed data-layout exchange of the paper's multiplication (Sec. II).

Above the local product the paper distributes the matrices over MPI ranks
and moves panels with one of two schemes: Cannon's algorithm for general
shapes (each rank communicates O(1/sqrt(P)) of the data) and, for tall and
skinny products with one large dimension, a scheme whose communication per
rank is O(1). Point-to-point messages are asynchronous, and the local product
starts once a step's panels have arrived.

Here the ranks are ``torch.distributed`` processes (gloo on CPU for tests,
NCCL or gloo across GPUs) and the local product is a callback:
``local_mm(A_panel, B_panel, C_acc) -> C_acc + A_panel @ B_panel`` on
``synth.BlockSparse`` panels. ``gpu_local_mm`` runs it through this library's
C ABI on the rank's GPU; it is the default and fails loudly without a GPU.

Cannon on a q x q grid (P = q^2), block rows of A and C split into q
contiguous ranges R_0..R_{q-1}, the inner block dimension into K_0..K_{q-1},
block columns of B and C into C_0..C_{q-1}. Rank (i, j) owns C(R_i, C_j).
After the initial skew it holds A(R_i, K_s) and B(K_s, C_j) with
s = (i + j) mod q; each of the q steps multiplies the held panels into C,
then passes A to the left neighbour (i, j-1) and B to the upper neighbour
(i-1, j), so that at step t it holds s = (i + j + t) mod q.

Tall-skinny (the inner dimension large): rank r owns A(:, K_r) and B(K_r, :)
over P ranges of the inner dimension, multiplies them locally, and the P
partial C matrices are summed on rank 0 in rank order (every rank sends one
C-sized message, independent of P).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import synth


# ------------------------------------------------------------ panels and grid
def split_ranges(n: int, parts: int) -> list[tuple[int, int]]:
    """n blocks into `parts` contiguous ranges whose sizes differ by at most one."""
    base, extra = divmod(n, parts)
    out, lo = [], 0
    for p in range(parts):
        hi = lo + base + (1 if p < extra else 0)
        out.append((lo, hi))
        lo = hi
    return out


def grid_side(world: int) -> int:
    q = int(round(world ** 0.5))
    if q * q != world:
        raise ValueError(f"Cannon needs a square number of ranks, got {world}")
    return q


def cannon_schedule(q: int, i: int, j: int) -> list[int]:
    """Inner panel index that rank (i, j) multiplies at each of the q steps."""
    return [(i + j + t) % q for t in range(q)]


def sub_panel(M: synth.BlockSparse, rows: tuple[int, int], cols: tuple[int, int]) -> synth.BlockSparse:
    """Blocks of M in block rows [rows) x block columns [cols), re-indexed from 0."""
    rs = np.asarray(M.row_sizes)
    cs = np.asarray(M.col_sizes)
    br = np.asarray(M.blk_row)
    bc = np.asarray(M.blk_col)
    sizes = rs[br].astype(np.int64) * cs[bc]
    off = np.concatenate([[0], np.cumsum(sizes)])
    keep = np.nonzero((br >= rows[0]) & (br < rows[1]) & (bc >= cols[0]) & (bc < cols[1]))[0]
    data = np.concatenate([M.data[off[b]:off[b + 1]] for b in keep]) if len(keep) else np.zeros(0)
    return synth.BlockSparse(rs[rows[0]:rows[1]].copy(), cs[cols[0]:cols[1]].copy(),
                             (br[keep] - rows[0]).astype(np.int32), (bc[keep] - cols[0]).astype(np.int32),
                             np.ascontiguousarray(data, dtype=np.float64))


def place(parts: list[tuple[synth.BlockSparse, int, int]], row_sizes, col_sizes) -> synth.BlockSparse:
    """Assemble panels (panel, first block row, first block column) into one matrix, CSR order."""
    rs = np.asarray(row_sizes, np.int32)
    cs = np.asarray(col_sizes, np.int32)
    entries = []
    for P, r0, c0 in parts:
        prs, pcs = np.asarray(P.row_sizes), np.asarray(P.col_sizes)
        pos = 0
        for i, j in zip(np.asarray(P.blk_row), np.asarray(P.blk_col)):
            n = int(prs[i]) * int(pcs[j])
            entries.append((int(i) + r0, int(j) + c0, P.data[pos:pos + n]))
            pos += n
    entries.sort(key=lambda e: (e[0], e[1]))
    br = np.array([e[0] for e in entries], np.int32)
    bc = np.array([e[1] for e in entries], np.int32)
    data = np.concatenate([e[2] for e in entries]) if entries else np.zeros(0)
    return synth.BlockSparse(rs, cs, br, bc, data)


# ------------------------------------------------------------- messages
_HDR = 5   # nbr, nbc, nblks, ndata, unused


def _pack(M: synth.BlockSparse):
    import torch
    hdr = torch.tensor([len(M.row_sizes), len(M.col_sizes), len(M.blk_row), len(M.data), 0], dtype=torch.int64)
    ints = torch.from_numpy(np.concatenate([np.asarray(M.row_sizes, np.int64), np.asarray(M.col_sizes, np.int64),
                                            np.asarray(M.blk_row, np.int64), np.asarray(M.blk_col, np.int64)]))
    data = torch.from_numpy(np.ascontiguousarray(M.data, dtype=np.float64))
    return hdr, ints, data


def _unpack(hdr, ints, data) -> synth.BlockSparse:
    nbr, nbc, nb = int(hdr[0]), int(hdr[1]), int(hdr[2])
    v = ints.numpy()
    return synth.BlockSparse(v[:nbr].astype(np.int32), v[nbr:nbr + nbc].astype(np.int32),
                             v[nbr + nbc:nbr + nbc + nb].astype(np.int32),
                             v[nbr + nbc + nb:nbr + nbc + 2 * nb].astype(np.int32), data.numpy().copy())


def exchange(send_to: int, recv_from: int, M: synth.BlockSparse) -> synth.BlockSparse:
    """Send M to one rank and receive a panel from another, asynchronously (isend / irecv)."""
    import torch
    import torch.distributed as dist
    hdr, ints, data = _pack(M)
    rh = torch.zeros(_HDR, dtype=torch.int64)
    reqs = [dist.isend(hdr, send_to), dist.irecv(rh, recv_from)]
    for r in reqs:
        r.wait()
    ri = torch.zeros(int(rh[0] + rh[1] + 2 * rh[2]), dtype=torch.int64)
    rd = torch.zeros(int(rh[3]), dtype=torch.float64)
    reqs = [dist.isend(ints, send_to), dist.isend(data, send_to), dist.irecv(ri, recv_from),
            dist.irecv(rd, recv_from)]
    for r in reqs:
        r.wait()
    return _unpack(rh, ri, rd)


# ------------------------------------------------------------ local product
def gpu_local_mm(Ap: synth.BlockSparse, Bp: synth.BlockSparse, Cacc: synth.BlockSparse | None,
                 precision: str = "fp64") -> synth.BlockSparse:
    """C_acc + A_panel @ B_panel through this library on the rank's GPU."""
    from . import dbcsr
    A = dbcsr.Matrix.from_blocks(Ap)
    B = dbcsr.Matrix.from_blocks(Bp)
    if Cacc is not None:
        Cm = dbcsr.Matrix.from_blocks(Cacc)
    else:
        Cm = dbcsr.Matrix.create(Ap.row_sizes, Bp.col_sizes, np.zeros(0, np.int32), np.zeros(0, np.int32))
    dbcsr.multiply("N", "N", 1.0, A, B, 1.0 if Cacc is not None else 0.0, Cm, precision=precision)
    rows, cols, _ = Cm.index()   # blocks in CSR order, data() concatenated in that order
    data = Cm.data()
    out = synth.BlockSparse(np.asarray(Ap.row_sizes, np.int32), np.asarray(Bp.col_sizes, np.int32),
                            np.asarray(rows, np.int32), np.asarray(cols, np.int32), np.asarray(data))
    for M in (A, B, Cm):
        M.release()
    return out


@dataclass
class Layout:
    """Block ranges of the q x q grid."""
    rows: list[tuple[int, int]]
    inner: list[tuple[int, int]]
    cols: list[tuple[int, int]]


def cannon_layout(A: synth.BlockSparse, B: synth.BlockSparse, q: int) -> Layout:
    return Layout(split_ranges(len(A.row_sizes), q), split_ranges(len(A.col_sizes), q),
                  split_ranges(len(B.col_sizes), q))


def cannon_multiply(A: synth.BlockSparse, B: synth.BlockSparse, rank: int, world: int, local_mm=None):
    """This rank's C panel (C(R_i, C_j), local block indices) of C = A @ B by Cannon's algorithm.

    Every rank passes the same global A and B (the test builds them from one
    seed); it keeps only its initial panels, so the result depends only on the
    exchanged data."""
    local_mm = local_mm or gpu_local_mm
    q = grid_side(world)
    i, j = divmod(rank, q)
    L = cannon_layout(A, B, q)
    s0 = (i + j) % q
    # after the skew: A(R_i, K_s0), B(K_s0, C_j)
    Ap = sub_panel(A, L.rows[i], L.inner[s0])
    Bp = sub_panel(B, L.inner[s0], L.cols[j])
    C = None
    left, right = i * q + (j - 1) % q, i * q + (j + 1) % q
    up, down = ((i - 1) % q) * q + j, ((i + 1) % q) * q + j
    for t in range(q):
        C = local_mm(Ap, Bp, C)
        if t + 1 < q:
            Ap = exchange(left, right, Ap)
            Bp = exchange(up, down, Bp)
    if C is None:
        C = synth.BlockSparse(np.asarray(A.row_sizes[L.rows[i][0]:L.rows[i][1]], np.int32),
                              np.asarray(B.col_sizes[L.cols[j][0]:L.cols[j][1]], np.int32),
                              np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros(0))
    return C, (L.rows[i][0], L.cols[j][0])


def tallskinny_multiply(A: synth.BlockSparse, B: synth.BlockSparse, rank: int, world: int, local_mm=None):
    """C = A @ B with the inner dimension split over the ranks; the sum of the
    partial products is returned on rank 0 (None elsewhere)."""
    import torch
    import torch.distributed as dist
    local_mm = local_mm or gpu_local_mm
    ks = split_ranges(len(A.col_sizes), world)[rank]
    Cr = local_mm(sub_panel(A, (0, len(A.row_sizes)), ks), sub_panel(B, ks, (0, len(B.col_sizes))), None)
    if rank != 0:
        hdr, ints, data = _pack(Cr)
        for t in (hdr, ints, data):
            dist.send(t, 0)
        return None
    parts = [Cr]
    for src in range(1, world):
        rh = torch.zeros(_HDR, dtype=torch.int64)
        dist.recv(rh, src)
        ri = torch.zeros(int(rh[0] + rh[1] + 2 * rh[2]), dtype=torch.int64)
        rd = torch.zeros(int(rh[3]), dtype=torch.float64)
        dist.recv(ri, src)
        dist.recv(rd, src)
        parts.append(_unpack(rh, ri, rd))
    return sum_blocks(parts)


def sum_blocks(parts: list[synth.BlockSparse]) -> synth.BlockSparse:
    """Blockwise sum of matrices with the same block sizes, in list order."""
    rs, cs = np.asarray(parts[0].row_sizes), np.asarray(parts[0].col_sizes)
    acc: dict[tuple[int, int], np.ndarray] = {}
    for P in parts:
        pos = 0
        for i, j in zip(np.asarray(P.blk_row), np.asarray(P.blk_col)):
            n = int(rs[i]) * int(cs[j])
            blk = P.data[pos:pos + n]
            key = (int(i), int(j))
            acc[key] = acc[key] + blk if key in acc else blk.copy()
            pos += n
    keys = sorted(acc)
    return synth.BlockSparse(rs.astype(np.int32), cs.astype(np.int32), np.array([k[0] for k in keys], np.int32),
                             np.array([k[1] for k in keys], np.int32),
                             np.concatenate([acc[k] for k in keys]) if keys else np.zeros(0))
