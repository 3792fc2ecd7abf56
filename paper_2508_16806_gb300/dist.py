"""Host-side plan of one LP partitioned across ranks (one GPU per rank).

The products of Algorithm 1 split by blocks of rows: rank r owns a contiguous
block of the rows of K (its part of y, q, the sense flags and of K x) and a
contiguous block of the columns (its part of x, c, l, u and of K^T y).  It keeps
the rows of K it owns (all their columns) and the rows of K^T it owns (all their
rows of K), so that each product needs the whole vector it multiplies:

  per step attempt   all-gather x'   (each rank contributes its columns)
                     all-gather y'   (each rank contributes its rows)
                     all-reduce 3 sums (||dx||^2, ||dy||^2, dy^T K dx: the
                     Algorithm 5 decision, taken identically on every rank)
  per KKT check      all-reduce the row- and column-side sums of the check
                     (Section 2.3.2 / 2.4.2 terms; maxima by a max-reduce)

Blocks are balanced by nonzeros.  The collectives move equal-sized pieces, so
each rank's piece of a gathered vector is padded to the largest block and the
gathered vector lives in a padded layout: entry j of block b sits at
b * width + (j - lo_b).  Column (and row) indices of the local matrices are
rewritten once, on the host, into that layout, so the SpMV kernels gather from
the padded vector directly.  The partition is a pure function of the LP and
the world size: every rank computes the same plan without communication.

This module is the host logic only; it moves no data and runs no arithmetic
of the method.
"""
from __future__ import annotations

import dataclasses

import numpy as np


def balanced_blocks(ptr: np.ndarray, parts: int) -> np.ndarray:
    """Boundaries b[0..parts] of `parts` contiguous blocks of the rows of a CSR
    structure with row pointers `ptr`, each holding about nnz / parts nonzeros:
    b[r] is the first row whose nonzero start reaches r * nnz / parts (and at
    least b[r - 1]).  Empty blocks are allowed when there are fewer rows than
    parts."""
    ptr = np.asarray(ptr, dtype=np.int64)
    rows = ptr.shape[0] - 1
    nnz = int(ptr[-1])
    b = np.zeros(parts + 1, dtype=np.int64)
    for r in range(1, parts):
        target = (nnz * r) // parts
        b[r] = max(int(np.searchsorted(ptr[:-1], target, side="left")), int(b[r - 1]))
        b[r] = min(b[r], rows)
    b[parts] = rows
    return b


def transpose_structure(m: int, n: int, row_ptr, col_idx):
    """CSR of K^T: (t_ptr[n + 1], t_row[nnz], t_perm[nnz]) with rows of K in
    ascending order inside each column; t_perm maps an entry of K^T to the
    nonzero of K it is."""
    row_ptr = np.asarray(row_ptr, dtype=np.int64)
    col_idx = np.asarray(col_idx, dtype=np.int64)
    rows = np.repeat(np.arange(m, dtype=np.int64), np.diff(row_ptr))
    order = np.lexsort((rows, col_idx))
    t_ptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(t_ptr, col_idx + 1, 1)
    t_ptr = np.cumsum(t_ptr)
    return t_ptr, rows[order], order


@dataclasses.dataclass
class RankPart:
    """What rank `rank` holds.  Indices in k_col / t_row point into the padded
    gathered vectors (width col_width / row_width per block)."""
    rank: int
    world: int
    rows: tuple            # [lo, hi) rows of K (entries of y, q, sense)
    cols: tuple            # [lo, hi) columns of K (entries of x, c, l, u)
    row_width: int         # padded piece of y per rank
    col_width: int         # padded piece of x per rank
    k_ptr: np.ndarray      # CSR of K[rows, :]  (local row pointers)
    k_col: np.ndarray      # padded column positions
    k_nz: np.ndarray       # nonzero index in the original K of each entry
    t_ptr: np.ndarray      # CSR of K^T[cols, :] (local)
    t_row: np.ndarray      # padded row positions
    t_nz: np.ndarray       # nonzero index in the original K of each entry


def padded_index(idx: np.ndarray, bounds: np.ndarray, width: int) -> np.ndarray:
    """Position of global index idx in the padded layout of blocks `bounds`."""
    blk = np.searchsorted(bounds, idx, side="right") - 1
    return blk * width + (idx - bounds[blk])


def partition(m: int, n: int, row_ptr, col_idx, world: int):
    """The plan of every rank (list of RankPart) and the row / column block
    boundaries."""
    row_ptr = np.asarray(row_ptr, dtype=np.int64)
    col_idx = np.asarray(col_idx, dtype=np.int64)
    rb = balanced_blocks(row_ptr, world)
    t_ptr, t_row, t_perm = transpose_structure(m, n, row_ptr, col_idx)
    cb = balanced_blocks(t_ptr, world)
    rw = int(max(1, np.max(np.diff(rb))))
    cw = int(max(1, np.max(np.diff(cb))))
    parts = []
    for r in range(world):
        r0, r1 = int(rb[r]), int(rb[r + 1])
        c0, c1 = int(cb[r]), int(cb[r + 1])
        a, b = int(row_ptr[r0]), int(row_ptr[r1])
        k_ptr = row_ptr[r0:r1 + 1] - a
        k_col = padded_index(col_idx[a:b], cb, cw)
        ta, tb = int(t_ptr[c0]), int(t_ptr[c1])
        tp = t_ptr[c0:c1 + 1] - ta
        tr = padded_index(t_row[ta:tb], rb, rw)
        parts.append(RankPart(r, world, (r0, r1), (c0, c1), rw, cw, k_ptr, k_col,
                              np.arange(a, b, dtype=np.int64), tp, tr, t_perm[ta:tb]))
    return parts, rb, cb


def pad_piece(v: np.ndarray, width: int) -> np.ndarray:
    """A rank's piece of a vector, zero-padded to the common width."""
    out = np.zeros(width, dtype=v.dtype)
    out[: v.shape[0]] = v
    return out


def unpad(gathered: np.ndarray, bounds: np.ndarray, width: int) -> np.ndarray:
    """The global vector from its padded gathered layout."""
    return np.concatenate([gathered[r * width: r * width + int(bounds[r + 1] - bounds[r])]
                           for r in range(len(bounds) - 1)])


def step_bytes_per_rank(m: int, n: int, world: int, value_bytes: int = 4) -> dict:
    """Bytes one rank sends and receives per step attempt in the two
    all-gathers (padded pieces; ring algorithm: each rank receives the other
    world - 1 pieces) and per check in the all-reduce of the check sums."""
    rw = -(-m // world)
    cw = -(-n // world)
    gather = (world - 1) * (rw + cw) * value_bytes
    return {"allgather_recv": gather, "decision_allreduce": 3 * 8, "check_allreduce": 29 * 8}


def partition_by_nnz(nnz, world: int) -> list:
    """Independent LPs shared among `world` ranks by their nonzeros: largest
    first, each to the rank with the fewest nonzeros so far (ties: the lower
    rank).  Returns each rank's LP indices in ascending order.  A pure function
    of the sizes, so every rank computes the same shares without communication."""
    nnz = np.asarray(nnz, dtype=np.int64)
    order = sorted(range(nnz.shape[0]), key=lambda k: (-int(nnz[k]), k))
    load = [0] * world
    share = [[] for _ in range(world)]
    for k in order:
        r = min(range(world), key=lambda i: (load[i], i))
        share[r].append(k)
        load[r] += int(nnz[k])
    return [sorted(s) for s in share]
