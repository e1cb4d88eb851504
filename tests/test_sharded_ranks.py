"""The bin-sharded multi-GPU path's host logic (paper_2012_04534_gb300/
sharded.py) on two gloo ranks on the CPU.  Each rank's shard is served by
the FP64 oracle restricted to the rows of its run of the bin union (the run
comes from the library's host-only sfs_shard_run); the solver's control
flow, collectives and update order are the product's.  Sharded A, A^H, the
gradient, the power-iteration L and 60 FISTA iterations agree with the
single-process oracle to rounding, and both ranks end with the same x."""
import math
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

PARAMS = dict(Nx=6, Ny=5, dx=0.5e-3, dy=0.5e-3, Nz=8, z0=10e-3, dz=0.15e-3, c=5900.0, fs=40e6,
              Nt=128, fc=5e6, frac_bw=0.7, theta=0.0)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


class OracleShard:
    """The oracle's A restricted to the rows of one run of the bin union, with
    the vector operations the solver asks of a shard, in FP64 on the CPU."""

    def __init__(self, go, idx, nshards, shard):
        import oracle as O
        from paper_2012_04534_gb300 import sfs
        self.O = O
        self.full = O.LateralFFTOperator(go, idx)
        bins = np.unique(idx)
        first, count = sfs.shard_run(bins.size, nshards, shard)
        self.mask = np.isin(idx, bins[first:first + count])
        self.S, self.M = idx.shape
        self.V = go.V
        self.shape_x, self.shape_y = (go.Nz, go.Ny, go.Nx), idx.shape

    def zeros(self, shape):
        return torch.zeros(shape, dtype=torch.complex128)

    def apply_A_into(self, x, y):
        v = self.full.apply_A(x.numpy())
        yn = y.numpy()
        yn[self.mask] = v[self.mask]

    def apply_AH(self, y):
        return torch.from_numpy(self.full.apply_AH(np.where(self.mask, y.numpy(), 0)).copy())

    def normal_residual(self, x, y, out):
        r = np.where(self.mask, self.full.apply_A(x.numpy()) - y.numpy(), 0)
        out.numpy()[...] = self.full.apply_AH(r)
        return out

    def prox_momentum(self, x, gamma, grad, lam, L, beta):
        xn, gn, g = x.numpy(), gamma.numpy(), grad.numpy()
        xp = xn.copy()
        xn[...] = self.O.soft_threshold(gn - g / L, lam / L)
        gn[...] = xn + beta * (xn - xp)

    def sumsq(self, v):
        return float(np.vdot(v.numpy(), v.numpy()).real)

    def max_abs(self, v):
        return float(np.abs(v.numpy()).max())

    def scale(self, v, a):
        v.numpy()[...] *= a

    def randn(self, v, seed):
        rng = np.random.default_rng(seed)
        v.numpy()[...] = rng.standard_normal(v.shape) + 1j * rng.standard_normal(v.shape)

    def add(self, a, b):
        a.numpy()[...] += b.numpy()


def problem():
    import oracle as O
    import synth
    go = O.Geometry(**PARAMS)
    idx = O.select_indices(go, O.SEL_RANDOM, 7, True, 3)
    ref = O.LateralFFTOperator(go, idx)
    x_true = synth.scene((go.Nz, go.Ny, go.Nx), 4, "uniform", seed=5)
    y0 = ref.apply_A(x_true)
    sig = synth.noise_scale(float(np.vdot(y0, y0).real), y0.size, 20.0)
    y = y0 + sig * synth.unit_noise(y0.shape, seed=6)
    return go, idx, ref, x_true, y


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    from paper_2012_04534_gb300 import sharded
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        go, idx, ref, x_true, y = problem()

        def allreduce(t):
            dist.all_reduce(torch.view_as_real(t), op=dist.ReduceOp.SUM)

        solver = sharded.ShardedSolver([OracleShard(go, idx, world, rank)], allreduce)
        yt = torch.from_numpy(y)
        xt = torch.from_numpy(x_true)
        res = {"A": solver.apply_A(xt).numpy().copy(), "AH": solver.apply_AH(yt).numpy().copy(),
               "grad": solver.gradient(xt, yt).numpy().copy()}
        res["L"], res["L_ok"] = solver.lipschitz(max_iter=2000, rtol=1e-12, seed=7, safety=0.0)
        lam = 0.05 * float(np.abs(ref.apply_AH(y)).max())
        L = res["L"] * 1.001
        res["x"] = solver.fista(yt, lam, L, 60).numpy().copy()
        res["x_mu"] = solver.fista(yt, -0.05, L, 60).numpy().copy()
        out[rank] = res
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_the_bins():
    import oracle as O
    from tests._common import ensure_built
    ensure_built()
    world, port = 2, _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        res = [out[r] for r in range(world)]
    go, idx, ref, x_true, y = problem()

    def rel(a, b):
        return np.linalg.norm(a - b) / np.linalg.norm(b)

    for r in res:
        assert rel(r["A"], ref.apply_A(x_true)) <= 1e-13
        assert rel(r["AH"], ref.apply_AH(y)) <= 1e-13
        assert rel(r["grad"], ref.apply_AH(ref.apply_A(x_true) - y)) <= 1e-12
    A = O.dense_A(go, idx)
    smax2 = np.linalg.svd(A, compute_uv=False)[0] ** 2
    assert res[0]["L_ok"] and abs(res[0]["L"] - smax2) <= 1e-9 * smax2
    L = res[0]["L"] * 1.001
    lam = 0.05 * float(np.abs(ref.apply_AH(y)).max())
    x_ref = O.fista(ref.apply_A, ref.apply_AH, y, lam, L, 60)
    assert np.abs(x_ref).max() > 0
    for r in res:
        assert rel(r["x"], x_ref) <= 1e-11
        assert rel(r["x_mu"], x_ref) <= 1e-11
    # every rank holds the same replica of the iterate
    assert np.array_equal(res[0]["x"], res[1]["x"])


def test_shard_runs_partition_the_union():
    """sfs_shard_run (host only): the runs are contiguous, cover 0..U-1
    once, and differ in length by at most one."""
    from paper_2012_04534_gb300 import sfs
    from tests._common import ensure_built
    ensure_built()
    for U in (1, 7, 81, 163):
        for n in range(1, min(U, 9) + 1):
            runs = [sfs.shard_run(U, n, j) for j in range(n)]
            assert runs[0][0] == 0
            assert all(a[0] + a[1] == b[0] for a, b in zip(runs, runs[1:]))
            assert runs[-1][0] + runs[-1][1] == U
            lens = [c for _, c in runs]
            assert max(lens) - min(lens) <= 1 and min(lens) >= 1
    with pytest.raises(sfs.SfsError):
        sfs.shard_run(3, 2, 2)
