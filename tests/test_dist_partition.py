"""Host logic of the single-LP row partition across ranks (paper_2508_16806_gb300.dist).

- The plan: row and column blocks balanced by nonzeros, every nonzero held once
  in the K part and once in the K^T part, padded positions that round-trip.
- The exchange, on CPU with the gloo backend at world size 2: each rank runs
  fixed-step PDHG steps (Algorithm 1, theta = 1) on its blocks with the two
  all-gathers of x' and y' and the all-reduce of the Algorithm 5 sums, and the
  result equals the FP64 oracle's unpartitioned steps; the check sums reduced
  across ranks equal the oracle's termination quantities.
The per-rank arithmetic here is a plain numpy stand-in for the GPU kernels;
no rank waits on another except through the collectives.
"""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2508_16806_gb300 import dist as D
from paper_2508_16806_gb300 import synth


def _lps():
    return {"small": synth.small_dense_lp(), "ragged": synth.ragged_lp(),
            "powerlaw": synth.power_law_lp(3000, 6000, 4, 500, seed=5)}


@pytest.mark.parametrize("world", [1, 2, 3, 8])
@pytest.mark.parametrize("name", ["small", "ragged", "powerlaw"])
def test_plan_covers_every_nonzero_once(name, world):
    lp = _lps()[name]
    parts, rb, cb = D.partition(lp.m, lp.n, lp.row_ptr, lp.col_idx, world)
    assert rb[0] == 0 and rb[-1] == lp.m and np.all(np.diff(rb) >= 0)
    assert cb[0] == 0 and cb[-1] == lp.n and np.all(np.diff(cb) >= 0)
    k_all = np.sort(np.concatenate([p.k_nz for p in parts]))
    t_all = np.sort(np.concatenate([p.t_nz for p in parts]))
    np.testing.assert_array_equal(k_all, np.arange(lp.nnz))
    np.testing.assert_array_equal(t_all, np.arange(lp.nnz))
    # balance: no block exceeds its share by more than the longest row
    row_len = np.diff(lp.row_ptr)
    per = [lp.row_ptr[rb[r + 1]] - lp.row_ptr[rb[r]] for r in range(world)]
    assert max(per) <= lp.nnz / world + row_len.max() + 1
    # padded positions round-trip
    v = np.arange(lp.n, dtype=float)
    pieces = [D.pad_piece(v[cb[r]:cb[r + 1]], parts[0].col_width) for r in range(world)]
    np.testing.assert_array_equal(D.unpad(np.concatenate(pieces), cb, parts[0].col_width), v)
    full = np.concatenate(pieces)
    for p in parts:
        np.testing.assert_array_equal(full[p.k_col], lp.col_idx[p.k_nz])


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _local_matvec(ptr, pos, nz, vals, vfull):
    out = np.zeros(len(ptr) - 1)
    for i in range(len(ptr) - 1):
        a, b = ptr[i], ptr[i + 1]
        out[i] = vals[nz[a:b]] @ vfull[pos[a:b]]
    return out


def _worker(rank, world, port, name, steps, tau, sigma, q):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    lp = _lps()[name]
    parts, rb, cb = D.partition(lp.m, lp.n, lp.row_ptr, lp.col_idx, world)
    p = parts[rank]
    (r0, r1), (c0, c1) = p.rows, p.cols

    def gather(piece, width):
        out = torch.zeros(world * width, dtype=torch.float64)
        dist.all_gather_into_tensor(out, torch.from_numpy(D.pad_piece(piece, width)))
        return out.numpy()

    # start x = proj_X(0), y = 0 (the oracle's start)
    x_loc = np.clip(np.zeros(c1 - c0), lp.l[c0:c1], lp.u[c0:c1])
    y_loc = np.zeros(r1 - r0)
    xf = gather(x_loc, p.col_width)
    yf = gather(y_loc, p.row_width)
    kx_loc = _local_matvec(p.k_ptr, p.k_col, p.k_nz, lp.vals, xf)
    for _ in range(steps):
        kty_loc = _local_matvec(p.t_ptr, p.t_row, p.t_nz, lp.vals, yf)
        xn = np.clip(x_loc - tau * (lp.c[c0:c1] - kty_loc), lp.l[c0:c1], lp.u[c0:c1])
        xnf = gather(xn, p.col_width)
        kxn = _local_matvec(p.k_ptr, p.k_col, p.k_nz, lp.vals, xnf)
        yn = y_loc + sigma * (lp.q[r0:r1] - (2 * kxn - kx_loc))
        ge = lp.sense[r0:r1] == 1
        yn[ge] = np.maximum(yn[ge], 0.0)
        ynf = gather(yn, p.row_width)
        # Algorithm 5 terms, summed over the ranks
        dx, dy = xn - x_loc, yn - y_loc
        s = torch.tensor([dx @ dx, dy @ dy, dy @ (kxn - kx_loc)], dtype=torch.float64)
        dist.all_reduce(s)
        x_loc, y_loc, kx_loc, xf, yf = xn, yn, kxn, xnf, ynf
    # check sums of the termination quantities on the final point (unscaled)
    kty_loc = _local_matvec(p.t_ptr, p.t_row, p.t_nz, lp.vals, yf)
    r = lp.q[r0:r1] - kx_loc
    r[lp.sense[r0:r1] == 1] = np.maximum(r[lp.sense[r0:r1] == 1], 0.0)
    v = lp.c[c0:c1] - kty_loc
    lf, uf = np.isfinite(lp.l[c0:c1]), np.isfinite(lp.u[c0:c1])
    lam = np.where(lf & uf, v, np.where(lf, np.maximum(v, 0), np.where(uf, np.minimum(v, 0), 0)))
    d = v - lam
    lt = np.where(lam > 0, lp.l[c0:c1] * lam, 0.0) + np.where(lam < 0, lp.u[c0:c1] * lam, 0.0)
    chk = torch.tensor([r @ r, lp.q[r0:r1] @ y_loc, d @ d, lp.c[c0:c1] @ x_loc, lt.sum()],
                       dtype=torch.float64)
    dist.all_reduce(chk)
    if rank == 0:
        q.put((D.unpad(xf, cb, p.col_width), D.unpad(yf, rb, p.row_width), s.numpy(),
               chk.numpy()))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("name", ["small", "ragged"])
def test_two_ranks_gloo_match_oracle_steps(oracle_mod, name):
    lp = _lps()[name]
    steps, tau, sigma = 12, 0.3, 0.4
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, name, steps, tau, sigma, q))
             for r in range(2)]
    for pr in procs:
        pr.start()
    x, y, s, chk = q.get(timeout=300)
    for pr in procs:
        pr.join(timeout=120)
        assert pr.exitcode == 0
    xo, yo = oracle_mod.start_point(lp)
    for _ in range(steps):
        xp, yp = xo, yo
        xo, yo = oracle_mod.pdhg_step(lp, xo, yo, tau, sigma)
    # summation orders differ (column blocks against the oracle's scatter over
    # rows): 2-norm relative agreement, as for the GPU iterates
    assert np.linalg.norm(x - xo) <= 1e-10 * np.linalg.norm(xo)
    assert np.linalg.norm(y - yo) <= 1e-10 * np.linalg.norm(yo)
    dx, dy = xo - xp, yo - yp
    kdx = oracle_mod.spmv(lp, dx)
    np.testing.assert_allclose(s, [dx @ dx, dy @ dy, dy @ kdx], rtol=1e-10, atol=1e-14)
    k = oracle_mod.kkt(lp, xo, yo)
    assert np.sqrt(chk[0]) == pytest.approx(k["pres"], rel=1e-10)
    assert np.sqrt(chk[2]) == pytest.approx(k["dres"], rel=1e-10)
    assert chk[3] == pytest.approx(k["pobj"], rel=1e-10, abs=1e-12)
    assert chk[1] + chk[4] == pytest.approx(k["dobj"], rel=1e-10, abs=1e-12)


def test_exchange_volume():
    b = D.step_bytes_per_rank(1_000_000, 2_000_000, 8)
    # seven padded pieces of 125,000 + 250,000 FP32 values per attempt
    assert b["allgather_recv"] == 7 * (125_000 + 250_000) * 4


@pytest.mark.parametrize("world", [1, 2, 3, 8])
def test_batch_shares_by_nnz(world):
    """One list of independent LPs shared among ranks by nonzeros (the batch
    workload's multi-rank form): every LP exactly once, each rank's load within
    one LP of the mean, the same shares on every call."""
    nnz = synth.batch_nnz(64 * world)
    shares = D.partition_by_nnz(nnz, world)
    assert sorted(k for s in shares for k in s) == list(range(64 * world))
    loads = [int(nnz[s].sum()) if s else 0 for s in shares]
    assert max(loads) - min(loads) <= int(nnz.max())
    assert shares == D.partition_by_nnz(nnz, world)
    assert all(s == sorted(s) for s in shares)


def test_batch_lp_by_index_matches_list():
    lps = synth.batch_lps(count=6)
    some = synth.batch_lps(indices=[5, 2])
    for a, b in zip(some, [lps[5], lps[2]]):
        np.testing.assert_array_equal(a.col_idx, b.col_idx)
        np.testing.assert_array_equal(a.vals, b.vals)
    nnz = synth.batch_nnz(6)
    for lp, est in zip(lps, nnz):
        assert lp.nnz <= est <= lp.nnz * 1.01
