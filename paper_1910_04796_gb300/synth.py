"""Seeded synthetic inputs shaped like the paper's workloads.

This module only draws random numbers and lays them out as block index +
concatenated column-major block data; it holds none of the product's
arithmetic, so both the GPU library's tests and the CPU oracle's tests can take
their inputs from here. All draws use ``numpy.random.default_rng(seed)``.

The paper's own workloads (Sec. IV) are synthetic square (M=N=K=63'360) and
tall-and-skinny (M=N=1'408, K=1'982'464) matrices with uniform block sizes 22
or 64; the workloads below keep those block sizes and shapes, scaled to one GPU.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class BlockSparse:
    """A block-sparse matrix as plain arrays.

    row_sizes/col_sizes: int32 block sizes; blk_row/blk_col: int32 coordinates
    of the stored blocks (row-major order here, any order is accepted by the
    library); data: float64, the blocks concatenated in that order, each
    column-major (rows fastest).
    """
    row_sizes: np.ndarray
    col_sizes: np.ndarray
    blk_row: np.ndarray
    blk_col: np.ndarray
    data: np.ndarray

    @property
    def shape(self):
        return int(self.row_sizes.sum()), int(self.col_sizes.sum())

    @property
    def nblks(self):
        return int(len(self.blk_row))


@dataclass
class Workload:
    name: str
    A: BlockSparse
    B: BlockSparse
    C: BlockSparse | None
    alpha: float = 1.0
    beta: float = 0.0
    transa: str = "N"
    transb: str = "N"
    extra: dict = field(default_factory=dict)


def _nelem(row_sizes, col_sizes, br, bc):
    return int((row_sizes[br].astype(np.int64) * col_sizes[bc].astype(np.int64)).sum())


def make_matrix(rng, row_sizes, col_sizes, keep_mask=None, blocks=None, dist="uniform",
                int_range=8, scale_exp=None):
    """Block-sparse matrix with the given sizes and kept blocks.

    keep_mask: bool [nbr, nbc] (or ``blocks`` = (br, bc) arrays). dist:
    'uniform' U[-1,1], 'normal' N(0,1), 'int' integers in [-int_range,
    int_range], 'wide' U[-1,1]*10**U(-scale_exp, scale_exp).
    """
    row_sizes = np.asarray(row_sizes, np.int32)
    col_sizes = np.asarray(col_sizes, np.int32)
    if blocks is None:
        br, bc = np.nonzero(keep_mask)
    else:
        br, bc = blocks
    br = np.asarray(br, np.int32)
    bc = np.asarray(bc, np.int32)
    n = _nelem(row_sizes, col_sizes, br, bc)
    if dist == "uniform":
        data = rng.uniform(-1.0, 1.0, n)
    elif dist == "normal":
        data = rng.standard_normal(n)
    elif dist == "int":
        data = rng.integers(-int_range, int_range + 1, n).astype(np.float64)
    elif dist == "wide":
        e = scale_exp if scale_exp is not None else 4.0
        data = rng.uniform(-1.0, 1.0, n) * 10.0 ** rng.uniform(-e, e, n)
    else:
        raise ValueError(dist)
    return BlockSparse(row_sizes, col_sizes, br, bc, data)


def bernoulli_mask(rng, nbr, nbc, p):
    return rng.random((nbr, nbc)) < p


def banded_mask(rng, nbr, nbc, mean_occ, width):
    """Block (i,j) kept with probability c*exp(-|i-j|/width), c set so the mean is mean_occ."""
    i = np.arange(nbr)[:, None]
    j = np.arange(nbc)[None, :]
    w = np.exp(-np.abs(i - j) / float(width))
    c = mean_occ / w.mean()
    return rng.random((nbr, nbc)) < np.minimum(1.0, c * w)


def banded_blocks(rng, nbr, nbc, mean_occ, width, chunk=256):
    """Same as banded_mask, drawn row-chunk by row-chunk (large grids)."""
    j = np.arange(nbc)[None, :]
    # normalisation constant from the exact mean of the band weights
    d = np.abs(np.arange(nbr)[:, None] - np.arange(nbc)[None, :]) if nbr * nbc <= 4_000_000 else None
    if d is not None:
        wmean = np.exp(-d / float(width)).mean()
    else:
        acc = 0.0
        for r0 in range(0, nbr, chunk):
            i = np.arange(r0, min(nbr, r0 + chunk))[:, None]
            acc += np.exp(-np.abs(i - j) / float(width)).sum()
        wmean = acc / (nbr * nbc)
    c = mean_occ / wmean
    brs, bcs = [], []
    for r0 in range(0, nbr, chunk):
        i = np.arange(r0, min(nbr, r0 + chunk))[:, None]
        p = np.minimum(1.0, c * np.exp(-np.abs(i - j) / float(width)))
        keep = rng.random(p.shape) < p
        r, cc = np.nonzero(keep)
        brs.append(r + r0)
        bcs.append(cc)
    return np.concatenate(brs).astype(np.int32), np.concatenate(bcs).astype(np.int32)


def uneven_sizes(rng, n, choices=(5, 13, 23, 26, 32), weights=(0.2, 0.3, 0.2, 0.2, 0.1)):
    return rng.choice(np.asarray(choices, np.int32), size=n, p=np.asarray(weights)).astype(np.int32)


def dense_matrix(rng, nbr, nbc, bs_r, bs_c, dist="uniform", scale_exp=None):
    """100%-occupancy block matrix with uniform block sizes (the dense limit)."""
    rs = np.full(nbr, bs_r, np.int32)
    cs = np.full(nbc, bs_c, np.int32)
    br = np.repeat(np.arange(nbr, dtype=np.int32), nbc)
    bc = np.tile(np.arange(nbc, dtype=np.int32), nbr)
    return make_matrix(rng, rs, cs, blocks=(br, bc), dist=dist, scale_exp=scale_exp)


# --------------------------------------------------------------------------
# The five workloads (block-sparse small case; dense limit; tall-skinny dense;
# uneven-block banded; precision study). ``scale`` < 1 shrinks a workload's
# block grid for quick tests while keeping its block sizes and occupancy.
# --------------------------------------------------------------------------
def workload_small_sparse(seed=0):
    """20x20 block grid, block size 13, A and B at 10% Bernoulli occupancy, U[-1,1], beta=0."""
    rng = np.random.default_rng(seed)
    rs = np.full(20, 13, np.int32)
    A = make_matrix(rng, rs, rs, bernoulli_mask(rng, 20, 20, 0.1))
    B = make_matrix(rng, rs, rs, bernoulli_mask(rng, 20, 20, 0.1))
    return Workload("sparse-20x20-bs13-10pct", A, B, None, 1.0, 0.0)


def workload_dense_limit(seed=1, nblk=512, bs=22):
    """N = nblk*bs dense (512x512 grid of 22x22 blocks = 11'264), C random, beta = 1."""
    rng = np.random.default_rng(seed)
    A = dense_matrix(rng, nblk, nblk, bs, bs)
    B = dense_matrix(rng, nblk, nblk, bs, bs)
    Cm = dense_matrix(rng, nblk, nblk, bs, bs)
    return Workload(f"dense-N{nblk * bs}-bs{bs}-beta1", A, B, Cm, 1.0, 1.0)


def workload_tall_skinny(seed=2, variant="a", transb="N", mn=4096, kk=131072, bs=32):
    """(a) M=N=mn, K=kk; (b) M=kk, N=K=mn. Block size bs, N(0,1), alpha=1, beta=0.

    For transb='T' the stored B is the transpose, so op(B) has the same shape.
    """
    rng = np.random.default_rng(seed)
    if variant == "a":
        M, N, K = mn, mn, kk
    else:
        M, N, K = kk, mn, mn
    A = dense_matrix(rng, M // bs, K // bs, bs, bs, dist="normal")
    if transb == "N":
        B = dense_matrix(rng, K // bs, N // bs, bs, bs, dist="normal")
    else:
        B = dense_matrix(rng, N // bs, K // bs, bs, bs, dist="normal")
    return Workload(f"tallskinny-{variant}-M{M}-N{N}-K{K}-bs{bs}-{transb}", A, B, None, 1.0, 0.0,
                    "N", transb)


def workload_uneven(seed=3, nblk=4000, occ=0.01, width=400):
    """nblk^2 grid, sizes i.i.d. {5,13,23,26,32} w (.2,.3,.2,.2,.1), banded 1%, U[-1,1], beta=0."""
    rng = np.random.default_rng(seed)
    sizes = uneven_sizes(rng, nblk)
    ba = banded_blocks(rng, nblk, nblk, occ, width)
    bb = banded_blocks(rng, nblk, nblk, occ, width)
    A = make_matrix(rng, sizes, sizes, blocks=ba)
    B = make_matrix(rng, sizes, sizes, blocks=bb)
    return Workload(f"uneven-{nblk}x{nblk}-banded{occ}", A, B, None, 1.0, 0.0)


def workload_precision_dense(seed=4, n=16384, bs=32):
    """Dense N x N, entries U[-1,1]*10^U(-4,4) (wide dynamic range), beta=0."""
    rng = np.random.default_rng(seed)
    A = dense_matrix(rng, n // bs, n // bs, bs, bs, dist="wide", scale_exp=4.0)
    B = dense_matrix(rng, n // bs, n // bs, bs, bs, dist="wide", scale_exp=4.0)
    return Workload(f"precision-dense-N{n}-wide", A, B, None, 1.0, 0.0)


def workload_precision_sparse(seed=5, nblk=1024, bs=32, occ=0.1):
    """nblk^2 grid of 32x32 blocks at 10% Bernoulli occupancy, U[-1,1], beta=0."""
    rng = np.random.default_rng(seed)
    rs = np.full(nblk, bs, np.int32)
    A = make_matrix(rng, rs, rs, bernoulli_mask(rng, nblk, nblk, occ))
    B = make_matrix(rng, rs, rs, bernoulli_mask(rng, nblk, nblk, occ))
    return Workload(f"precision-sparse-{nblk}x{nblk}-bs{bs}", A, B, None, 1.0, 0.0)


def panel_mask(rng, nbr, nbc, panel, dense_every=2, sparse_occ=0.05):
    """Block rows in panels of `panel` rows: every `dense_every`-th panel fully
    occupied, the others Bernoulli(sparse_occ) -- a sparse matrix with dense
    sub-panels (input of the hybrid path)."""
    mask = rng.random((nbr, nbc)) < sparse_occ
    for r0 in range(0, nbr, panel * dense_every):
        mask[r0:r0 + panel, :] = True
    return mask


def workload_hybrid(seed=6, nblk=256, bs=32, panel=16, dense_every=2, sparse_occ=0.05, b_occ=1.0):
    """nblk^2 grid of bs x bs blocks; A alternates dense and sparse panels of
    `panel` block rows, B at b_occ occupancy (dense by default), U[-1,1], beta=0."""
    rng = np.random.default_rng(seed)
    rs = np.full(nblk, bs, np.int32)
    A = make_matrix(rng, rs, rs, panel_mask(rng, nblk, nblk, panel, dense_every, sparse_occ))
    B = make_matrix(rng, rs, rs, bernoulli_mask(rng, nblk, nblk, b_occ))
    return Workload(f"hybrid-{nblk}x{nblk}-bs{bs}-panel{panel}", A, B, None, 1.0, 0.0,
                    extra={"panel": panel, "sparse_occ": sparse_occ, "b_occ": b_occ})


def random_small(rng, nbr, nbk, nbc, p=0.5, sizes=(1, 2, 3, 4, 5), dist="uniform",
                 with_c=False, c_p=0.3):
    """Tiny random block-sparse A (nbr x nbk), B (nbk x nbc) and optional C."""
    rsz = rng.choice(np.asarray(sizes, np.int32), nbr).astype(np.int32)
    ksz = rng.choice(np.asarray(sizes, np.int32), nbk).astype(np.int32)
    csz = rng.choice(np.asarray(sizes, np.int32), nbc).astype(np.int32)
    A = make_matrix(rng, rsz, ksz, bernoulli_mask(rng, nbr, nbk, p), dist=dist)
    B = make_matrix(rng, ksz, csz, bernoulli_mask(rng, nbk, nbc, p), dist=dist)
    Cm = make_matrix(rng, rsz, csz, bernoulli_mask(rng, nbr, nbc, c_p), dist=dist) if with_c else None
    return A, B, Cm


def transpose_blocks(M: BlockSparse) -> BlockSparse:
    """Stored transpose: block (i,j) becomes block (j,i) holding the transposed data.

    Used to build inputs whose op(.) = 'T' view equals a given matrix; it is a
    relayout of random inputs, not a step of the product.
    """
    rs = np.asarray(M.row_sizes)
    cs = np.asarray(M.col_sizes)
    parts = []
    pos = 0
    for i, j in zip(M.blk_row, M.blk_col):
        m, n = int(rs[i]), int(cs[j])
        blk = M.data[pos:pos + m * n].reshape((m, n), order="F")
        parts.append(blk.T.reshape(-1, order="F"))
        pos += m * n
    data = np.concatenate(parts) if parts else np.zeros(0)
    return BlockSparse(cs.copy(), rs.copy(), np.asarray(M.blk_col).copy(),
                       np.asarray(M.blk_row).copy(), data)
