"""Seeded synthetic LP generators.

These build the input problems that both the CUDA solver and the FP64 CPU oracle
consume.  The module holds no solver arithmetic: it only draws random data and
assembles a CSR constraint matrix, right-hand side, cost vector and bounds.

Problem form (Section 2.2 of the paper):

    min c^T x   s.t.  K x  (>= | =)  q   row-wise,   l <= x <= u

where ``sense[i] == 1`` marks an inequality row (K_i x >= q_i, a row of G with
right-hand side h) and ``sense[i] == 0`` an equality row (a row of A with
right-hand side b).  Bounds may be +-inf.

Planted optimum ("feasible and bounded by construction"): a primal point x0 in
the box, a dual point y0 (non-negative on inequality rows) and reduced costs
lambda0 that agree with x0's bound activity are drawn first; then
q = K x0 (minus a slack only on inequality rows whose y0 is zero) and
c = K^T y0 + lambda0.  The pair (x0, y0) satisfies the KKT conditions of
Section 2.3.2 exactly, so c^T x0 is the optimal objective.
"""
from __future__ import annotations

import dataclasses
import numpy as np


@dataclasses.dataclass
class LP:
    m: int
    n: int
    row_ptr: np.ndarray   # int64, m+1
    col_idx: np.ndarray   # int32, nnz (ascending within each row)
    vals: np.ndarray      # float64, nnz
    sense: np.ndarray     # uint8, m   (1: row >= q_i, 0: row == q_i)
    c: np.ndarray         # float64, n
    q: np.ndarray         # float64, m
    l: np.ndarray         # float64, n  (-inf allowed)
    u: np.ndarray         # float64, n  (+inf allowed)
    x_star: np.ndarray | None = None   # planted primal optimum (if any)
    y_star: np.ndarray | None = None   # planted dual optimum (if any)
    name: str = ""

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    @property
    def f_star(self):
        if self.x_star is None:
            return None
        return float(self.c @ self.x_star)

    def row_of_nnz(self) -> np.ndarray:
        return np.repeat(np.arange(self.m, dtype=np.int64), np.diff(self.row_ptr))

    def dense(self) -> np.ndarray:
        """Dense copy of K (small problems only)."""
        K = np.zeros((self.m, self.n))
        K[self.row_of_nnz(), self.col_idx] = self.vals
        return K

    def matvec(self, x: np.ndarray) -> np.ndarray:
        """K x, used only to assemble planted right-hand sides."""
        prod = self.vals * x[self.col_idx]
        return np.bincount(self.row_of_nnz(), weights=prod, minlength=self.m)

    def rmatvec(self, y: np.ndarray) -> np.ndarray:
        """K^T y, used only to assemble planted costs."""
        prod = self.vals * y[self.row_of_nnz()]
        return np.bincount(self.col_idx, weights=prod, minlength=self.n)


# --------------------------------------------------------------------------
# sparsity patterns
# --------------------------------------------------------------------------

def _csr_from_rows_cols(m: int, n: int, rows: np.ndarray, cols: np.ndarray,
                        rng: np.random.Generator, resample: bool = True):
    """Sort (row, col) pairs, re-drawing duplicate columns inside a row, and
    return row_ptr, col_idx (ascending columns within each row) and the
    per-row counts.  ``rows`` must already be grouped (non-decreasing)."""
    rows = rows.astype(np.int64)
    cols = cols.astype(np.int64)
    for _ in range(64):
        key = rows * n + cols
        order = np.argsort(key, kind="stable")
        key = key[order]
        rows = rows[order]
        cols = cols[order]
        dup = np.zeros(key.shape[0], dtype=bool)
        dup[1:] = key[1:] == key[:-1]
        nd = int(dup.sum())
        if nd == 0 or not resample:
            break
        cols[dup] = rng.integers(0, n, nd)
    key = rows * n + cols
    order = np.argsort(key, kind="stable")
    rows = rows[order]
    cols = cols[order]
    keep = np.ones(rows.shape[0], dtype=bool)
    keep[1:] = (rows[1:] != rows[:-1]) | (cols[1:] != cols[:-1])
    rows = rows[keep]
    cols = cols[keep]
    counts = np.bincount(rows, minlength=m).astype(np.int64)
    row_ptr = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    return row_ptr, cols.astype(np.int32)


def bernoulli_pattern(m: int, n: int, density: float, rng: np.random.Generator):
    """Each entry of the m x n matrix is kept independently with probability
    ``density`` (2% uniform-random sparsity of the small test problem)."""
    mask = rng.random((m, n)) < density
    rows, cols = np.nonzero(mask)
    counts = np.bincount(rows, minlength=m).astype(np.int64)
    row_ptr = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    return row_ptr, cols.astype(np.int32)


def lengths_pattern(m: int, n: int, lengths: np.ndarray, rng: np.random.Generator):
    """Row i gets ``lengths[i]`` distinct uniformly random columns."""
    lengths = np.minimum(lengths.astype(np.int64), n)
    rows = np.repeat(np.arange(m, dtype=np.int64), lengths)
    cols = rng.integers(0, n, rows.shape[0])
    return _csr_from_rows_cols(m, n, rows, cols, rng)


def power_law_lengths(m: int, lo: int, hi: int, alpha: float,
                      rng: np.random.Generator) -> np.ndarray:
    """Discrete power law P(L) ~ L^-alpha on lo..hi (inverse-CDF sampling)."""
    support = np.arange(lo, hi + 1, dtype=np.float64)
    pmf = support ** (-alpha)
    cdf = np.cumsum(pmf)
    cdf /= cdf[-1]
    idx = np.searchsorted(cdf, rng.random(m), side="right")
    idx = np.minimum(idx, support.shape[0] - 1)
    return (lo + idx).astype(np.int64)


# --------------------------------------------------------------------------
# planted optimum
# --------------------------------------------------------------------------

def plant(m: int, n: int, row_ptr, col_idx, vals, sense, rng: np.random.Generator,
          frac_lower: float = 0.3, frac_upper: float = 0.2, name: str = "",
          literal_slack: bool = False) -> LP:
    """Assemble a feasible, bounded LP whose optimum (x0, y0) is known.

    x0 ~ U[0,1] in boxes l = 0, u ~ U[1,5]; 30% of coordinates moved to their
    lower bound and 20% to their upper bound; y0 ~ N(0,1), clamped >= 0 on
    inequality rows; q = K x0 except on inequality rows with y0 == 0, which get
    a U[0,1] slack; lambda0 ~ U[0,1] at lower-active, -U[0,1] at upper-active
    coordinates, 0 elsewhere; c = K^T y0 + lambda0.

    ``literal_slack=True`` gives every inequality row a slack (the literal text
    of the workload description).  That LP is still feasible and bounded, but
    (x0, y0) is then not optimal, so x_star/y_star are not recorded.
    """
    l = np.zeros(n)
    u = rng.uniform(1.0, 5.0, n)
    x0 = rng.uniform(0.0, 1.0, n)
    which = rng.random(n)
    at_l = which < frac_lower
    at_u = (which >= frac_lower) & (which < frac_lower + frac_upper)
    x0[at_l] = l[at_l]
    x0[at_u] = u[at_u]
    y0 = rng.standard_normal(m)
    ineq = sense.astype(bool)
    y0[ineq] = np.maximum(y0[ineq], 0.0)
    lp = LP(m, n, row_ptr, col_idx, vals, sense, np.zeros(n), np.zeros(m), l, u, name=name)
    Kx = lp.matvec(x0)
    slack = rng.uniform(0.0, 1.0, m)
    if literal_slack:
        has_slack = ineq
    else:
        has_slack = ineq & (y0 == 0.0)
    q = Kx - np.where(has_slack, slack, 0.0)
    lam = np.zeros(n)
    lam[at_l] = rng.uniform(0.0, 1.0, int(at_l.sum()))
    lam[at_u] = -rng.uniform(0.0, 1.0, int(at_u.sum()))
    c = lp.rmatvec(y0) + lam
    lp.c = c
    lp.q = q
    if not literal_slack:
        lp.x_star = x0
        lp.y_star = y0
    return lp


def _sense_half(m: int) -> np.ndarray:
    """First half of the rows are inequalities, the rest equalities."""
    s = np.zeros(m, dtype=np.uint8)
    s[: m - m // 2] = 1
    return s


def random_planted(m: int, n: int, lengths: np.ndarray | None = None,
                   density: float | None = None, seed: int = 0, name: str = "",
                   sense: np.ndarray | None = None) -> LP:
    """Planted LP on either a Bernoulli pattern (``density``) or given row
    lengths; values ~ N(0,1); half inequality, half equality rows."""
    rng = np.random.default_rng(seed)
    if density is not None:
        row_ptr, col_idx = bernoulli_pattern(m, n, density, rng)
    else:
        row_ptr, col_idx = lengths_pattern(m, n, lengths, rng)
    vals = rng.standard_normal(int(row_ptr[-1]))
    if sense is None:
        sense = _sense_half(m)
    return plant(m, n, row_ptr, col_idx, vals, sense, rng, name=name)


# --------------------------------------------------------------------------
# the five workloads
# --------------------------------------------------------------------------

def small_dense_lp(seed: int = 20250816) -> LP:
    """200 x 400 LP (100 >= rows, 100 = rows), 2% Bernoulli sparsity,
    entries ~ N(0,1), planted optimum."""
    return random_planted(200, 400, density=0.02, seed=seed, name="lp200x400")


def power_law_lp(m: int = 1_000_000, n: int = 2_000_000, lo: int = 4, hi: int = 5000,
                 alpha: float = 2.1, seed: int = 20250817) -> LP:
    """Large random LP with power-law row lengths (alpha = 2.1 on lo..hi),
    values ~ N(0,1), half >= / half = rows, planted optimum.  With lo = 4 the
    mean row length is about 20 (nnz ~ 20M at m = 1M)."""
    rng = np.random.default_rng(seed)
    lengths = power_law_lengths(m, lo, hi, alpha, rng)
    row_ptr, col_idx = lengths_pattern(m, n, lengths, rng)
    vals = rng.standard_normal(int(row_ptr[-1]))
    return plant(m, n, row_ptr, col_idx, vals, _sense_half(m), rng,
                 name=f"powerlaw{m}x{n}")


def dispatch_lp(n_gen: int = 5000, n_base: int = 15000, n_cont: int = 40,
                lo: int = 10, hi: int = 200, seed: int = 20250818) -> LP:
    """Economic-dispatch-shaped block LP.

    Generators x_j in [Pmin_j, Pmax_j] (Pmin ~ U[0,50], Pmax = Pmin + U[10,200]),
    costs ~ U[10,100]; one balance row sum(x) = D with D = sum(x0) for a
    dispatch x0 drawn inside the box; ``n_base`` flow rows with a log-uniform
    number (lo..hi) of N(0, 0.3) shift factors, written as -a.x >= -F with
    F = a.x0 + U[0,1] |a.x0| + 0.1; ``n_cont`` contingency blocks repeat the
    base patterns with every coefficient scaled by U[0.9, 1.1] and limits
    recomputed from x0.  The optimum is not planted (costs are given)."""
    rng = np.random.default_rng(seed)
    pmin = rng.uniform(0.0, 50.0, n_gen)
    pmax = pmin + rng.uniform(10.0, 200.0, n_gen)
    cost = rng.uniform(10.0, 100.0, n_gen)
    x0 = rng.uniform(pmin, pmax)
    lengths = np.exp(rng.uniform(np.log(lo), np.log(hi), n_base)).astype(np.int64)
    lengths = np.clip(lengths, lo, hi)
    b_rp, b_ci = lengths_pattern(n_base, n_gen, lengths, rng)
    b_nnz = int(b_rp[-1])
    b_val = rng.normal(0.0, 0.3, b_nnz)
    blocks_vals = [b_val]
    for _ in range(n_cont):
        blocks_vals.append(b_val * rng.uniform(0.9, 1.1, b_nnz))
    nblk = n_cont + 1
    m = 1 + nblk * n_base
    # row 0: balance, dense over all generators
    rp = np.zeros(m + 1, dtype=np.int64)
    rp[1] = n_gen
    blk_len = np.diff(b_rp)
    tiled = np.tile(blk_len, nblk)
    np.cumsum(tiled, out=rp[2:])
    rp[2:] += n_gen
    ci = np.concatenate([np.arange(n_gen, dtype=np.int32)] + [b_ci] * nblk)
    flow_vals = np.concatenate(blocks_vals)
    vals = np.concatenate([np.ones(n_gen), -flow_vals])
    # limits: a.x0 per flow row
    row_of = np.repeat(np.arange(nblk * n_base, dtype=np.int64), tiled)
    ax0 = np.bincount(row_of, weights=flow_vals * x0[np.tile(b_ci, nblk)],
                      minlength=nblk * n_base)
    F = ax0 + rng.uniform(0.0, 1.0, nblk * n_base) * np.abs(ax0) + 0.1
    q = np.concatenate([[x0.sum()], -F])
    sense = np.ones(m, dtype=np.uint8)
    sense[0] = 0
    return LP(m, n_gen, rp, ci, vals, sense, cost, q, pmin, pmax,
              name=f"dispatch{m}x{n_gen}")


def _batch_draws(k: int, m_lo: int, m_hi: int, k_lo: int, k_hi: int, seed: int):
    rng = np.random.default_rng(seed + k)
    m = int(np.exp(rng.uniform(np.log(m_lo), np.log(m_hi))))
    lengths = rng.integers(k_lo, k_hi + 1, m)
    return rng, m, lengths


def batch_lp(k: int, m_lo: int = 500, m_hi: int = 50_000, k_lo: int = 5, k_hi: int = 20,
             seed: int = 20250819) -> LP:
    """LP k of the batch workload: m ~ log-uniform[m_lo, m_hi], n = 2m, row
    lengths ~ U{k_lo..k_hi}, planted optimum; seed ``seed + k``."""
    rng, m, lengths = _batch_draws(k, m_lo, m_hi, k_lo, k_hi, seed)
    n = 2 * m
    row_ptr, col_idx = lengths_pattern(m, n, lengths, rng)
    vals = rng.standard_normal(int(row_ptr[-1]))
    return plant(m, n, row_ptr, col_idx, vals, _sense_half(m), rng, name=f"batch{k}_{m}x{n}")


def batch_nnz(count: int = 512, m_lo: int = 500, m_hi: int = 50_000, k_lo: int = 5,
              k_hi: int = 20, seed: int = 20250819) -> np.ndarray:
    """Nonzeros of LPs 0..count-1 of the batch workload before duplicate
    columns are re-drawn (an upper bound within a few per mille), from their
    first draws only: no LP is built."""
    out = np.empty(count, dtype=np.int64)
    for k in range(count):
        _, m, lengths = _batch_draws(k, m_lo, m_hi, k_lo, k_hi, seed)
        out[k] = int(np.minimum(lengths, 2 * m).sum())
    return out


def batch_lps(count: int = 512, m_lo: int = 500, m_hi: int = 50_000,
              k_lo: int = 5, k_hi: int = 20, seed: int = 20250819,
              indices=None) -> list[LP]:
    """``count`` independent planted LPs (``batch_lp``), or the LPs ``indices``
    of that list."""
    ks = range(count) if indices is None else indices
    return [batch_lp(int(k), m_lo, m_hi, k_lo, k_hi, seed) for k in ks]


def adjoint_lp(m: int = 100_000, n: int = 200_000, per_row: int = 20,
               seed: int = 20250820):
    """Planted LP with ``per_row`` nonzeros in every row, plus a target
    x_target ~ U[0,1] for the loss ||x_K - x_target||^2."""
    rng = np.random.default_rng(seed)
    lengths = np.full(m, per_row, dtype=np.int64)
    row_ptr, col_idx = lengths_pattern(m, n, lengths, rng)
    vals = rng.standard_normal(int(row_ptr[-1]))
    lp = plant(m, n, row_ptr, col_idx, vals, _sense_half(m), rng, name=f"adj{m}x{n}")
    x_target = rng.uniform(0.0, 1.0, n)
    return lp, x_target


def shuffle_sense(lp: LP, seed: int) -> LP:
    """Same LP with inequality / equality rows interleaved at random
    (a row permutation), for tests of the sense mask."""
    rng = np.random.default_rng(seed)
    perm = rng.permutation(lp.m)
    lens = np.diff(lp.row_ptr)[perm]
    rp = np.zeros(lp.m + 1, dtype=np.int64)
    np.cumsum(lens, out=rp[1:])
    ci = np.concatenate([lp.col_idx[lp.row_ptr[i]:lp.row_ptr[i + 1]] for i in perm]) \
        if lp.m else lp.col_idx
    vv = np.concatenate([lp.vals[lp.row_ptr[i]:lp.row_ptr[i + 1]] for i in perm]) \
        if lp.m else lp.vals
    out = LP(lp.m, lp.n, rp, ci.astype(np.int32), vv, lp.sense[perm].copy(),
             lp.c.copy(), lp.q[perm].copy(), lp.l.copy(), lp.u.copy(), name=lp.name + "_shuf")
    out.x_star = lp.x_star
    out.y_star = None if lp.y_star is None else lp.y_star[perm]
    return out


def from_dense(K, sense, c, q, l, u, name: str = "dense") -> LP:
    """CSR LP from a dense matrix (zeros dropped); small hand-made problems."""
    K = np.asarray(K, dtype=np.float64)
    m, n = K.shape
    rows, cols = np.nonzero(K)
    counts = np.bincount(rows, minlength=m).astype(np.int64)
    row_ptr = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])

    def vec(v):
        return np.array([float(t) for t in v], dtype=np.float64)

    return LP(m, n, row_ptr, cols.astype(np.int32), K[rows, cols].copy(),
              np.asarray(sense, dtype=np.uint8), vec(c), vec(q), vec(l), vec(u), name=name)


def ragged_lp(seed: int = 7, m: int = 10000, n: int = 6000) -> LP:
    """Planted LP whose row lengths hit every SpMV code path: empty rows,
    1 / 31 / 32 / 33 nonzeros, rows around the shared-memory staging sizes
    (2047..2049, 4095..4097, 4500, 5000), three dense columns (long rows of
    K^T, about m/2 entries each) and an empty column 0."""
    rng = np.random.default_rng(seed)
    special = [0, 0, 1, 31, 32, 33, 1023, 1024, 1025, 2047, 2048, 2049, 4095, 4096, 4097,
               4500, 5000]
    lengths = rng.integers(1, 12, m)
    pos = rng.choice(m, len(special), replace=False)
    lengths[pos] = special
    rows = np.repeat(np.arange(m, dtype=np.int64), lengths)
    cols = rng.integers(1, n, rows.shape[0])
    row_ptr, col_idx = _csr_from_rows_cols(m, n, rows, cols, rng)
    # three dense columns: append (i, j) for j in {5, 6, 7} on a quarter of the rows
    keep_r = np.repeat(np.arange(m, dtype=np.int64), np.diff(row_ptr))
    chunks = [np.flatnonzero(rng.random(m) < 0.5) for _ in range(3)]
    extra_r = np.concatenate(chunks)
    extra_c = np.concatenate([np.full(len(ch), j) for ch, j in zip(chunks, (5, 6, 7))])
    rows = np.concatenate([keep_r, extra_r])
    cols = np.concatenate([col_idx.astype(np.int64), extra_c])
    key = rows * n + cols
    key = np.unique(key)
    rows, cols = key // n, key % n
    keep = (cols != 0) & (rows != pos[0])      # empty column 0 and an empty row
    rows, cols = rows[keep], cols[keep]
    counts = np.bincount(rows, minlength=m).astype(np.int64)
    row_ptr = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    vals = rng.standard_normal(int(row_ptr[-1]))
    sense = (rng.random(m) < 0.5).astype(np.uint8)
    return plant(m, n, row_ptr, cols.astype(np.int32), vals, sense, rng, name="ragged")


# --------------------------------------------------------------------------
# infeasible and unbounded variants (for the detection tests)
# --------------------------------------------------------------------------

def _append_rows(lp: LP, rows_cols, rows_vals, senses, qs, name: str) -> LP:
    """lp with extra rows appended (each given by its columns and values)."""
    rp = [lp.row_ptr]
    ci = [lp.col_idx]
    va = [lp.vals]
    end = int(lp.row_ptr[-1])
    for cols, vals in zip(rows_cols, rows_vals):
        order = np.argsort(cols)
        ci.append(np.asarray(cols, dtype=np.int32)[order])
        va.append(np.asarray(vals, dtype=np.float64)[order])
        end += len(cols)
        rp.append(np.array([end], dtype=np.int64))
    return LP(lp.m + len(qs), lp.n, np.concatenate(rp), np.concatenate(ci), np.concatenate(va),
              np.concatenate([lp.sense, np.asarray(senses, dtype=np.uint8)]), lp.c.copy(),
              np.concatenate([lp.q, np.asarray(qs, dtype=np.float64)]), lp.l.copy(), lp.u.copy(),
              name=name)


def contradictory_rows_lp(lp: LP, seed: int = 1, gap: float = 1.0, width: int = 8) -> LP:
    """Primal-infeasible variant: two >= rows a^T x >= b and -a^T x >= gap - b
    on ``width`` random columns (so a^T x >= b and a^T x <= b - gap)."""
    rng = np.random.default_rng(seed)
    cols = rng.choice(lp.n, width, replace=False)
    a = rng.standard_normal(width)
    b = float(rng.uniform(-1.0, 1.0))
    return _append_rows(lp, [cols, cols], [a, -a], [1, 1], [b, gap - b],
                        name=lp.name + "+contradiction")


def unbounded_column_lp(lp: LP, seed: int = 2, width: int = 6) -> LP:
    """Dual-infeasible variant: one more column x_new >= 0 with cost -1 whose
    entries are positive and sit only in >= rows, so x_new can grow forever."""
    rng = np.random.default_rng(seed)
    ge = np.flatnonzero(lp.sense)
    rows = np.sort(rng.choice(ge, min(width, len(ge)), replace=False))
    n = lp.n
    counts = np.diff(lp.row_ptr)
    add = np.zeros(lp.m, dtype=np.int64)
    add[rows] = 1
    row_ptr = np.zeros(lp.m + 1, dtype=np.int64)
    np.cumsum(counts + add, out=row_ptr[1:])
    col_idx = np.empty(int(row_ptr[-1]), dtype=np.int32)
    vals = np.empty(int(row_ptr[-1]))
    newv = rng.uniform(0.5, 2.0, len(rows))
    k = 0
    for i in range(lp.m):
        a, b = int(lp.row_ptr[i]), int(lp.row_ptr[i + 1])
        s = int(row_ptr[i])
        col_idx[s:s + b - a] = lp.col_idx[a:b]
        vals[s:s + b - a] = lp.vals[a:b]
        if add[i]:
            col_idx[s + b - a] = n
            vals[s + b - a] = newv[k]
            k += 1
    return LP(lp.m, n + 1, row_ptr, col_idx, vals, lp.sense.copy(),
              np.concatenate([lp.c, [-1.0]]), lp.q.copy(), np.concatenate([lp.l, [0.0]]),
              np.concatenate([lp.u, [np.inf]]), name=lp.name + "+unbounded")
