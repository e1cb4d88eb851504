"""The bin-sharded split (sfs_operator_shard, sfs_normal_residual,
sfs_prox_momentum, paper_2012_04534_gb300/sharded.py) on one GPU: one
process holds every shard and adds their partials where separate GPUs would
all-reduce.  Against the unsharded operator and the FP64 oracle: the rows of
each shard, A^H and the gradient as sums of partials, the power-iteration
L, and FISTA (1e-4 of the oracle)."""
import numpy as np
import pytest

import oracle as O
import synth
from tests._common import crandn, ensure_built, geom_params, oracle_geometry, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sfs():
    ensure_built()
    import torch
    from paper_2012_04534_gb300 import sfs as mod
    torch.cuda.init()
    return mod


def to_dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.complex64)).cuda()


def to_host(t):
    import torch
    torch.cuda.synchronize()
    return t.cpu().numpy().astype(np.complex128)


@pytest.mark.parametrize("case", [
    (dict(Nx=10, Ny=10, Nz=16, dz=0.15e-3, Nt=256), 12, 2, "fp32"),
    (dict(Nx=12, Ny=9, Nz=21, dz=0.15e-3, Nt=256), 10, 3, "fp32"),
    (dict(Nx=40, Ny=36, Nz=10, dz=0.15e-3, Nt=256), 10, 4, "fp32"),   # 128 x 128 planes
    (dict(Nx=10, Ny=10, Nz=16, dz=0.15e-3, Nt=256), 12, 2, "bf16"),
])
def test_sharded_operator_and_fista(sfs, case):
    from paper_2012_04534_gb300 import sharded
    over, M, n, mode = case
    params = geom_params(**over)
    g = sfs.Geometry(**params)
    go = oracle_geometry(params)
    idx = O.select_indices(go, O.SEL_RANDOM, M, True, 21)
    prec = sfs.PRECISION_NAMES[mode]
    full = sfs.Operator.from_indices(g, idx, precision=prec)
    shards = [sharded.GpuShard.build(g, idx, n, j, precision=prec) for j in range(n)]
    bins = np.unique(idx)
    for j, sh in enumerate(shards):
        info = sh.op.info
        first, count = sfs.shard_run(bins.size, n, j)
        assert (info["nshards"], info["shard"], info["shard_first"], info["U"], info["U_all"]) == \
            (n, j, first, count, bins.size)
    solver = sharded.ShardedSolver(shards)
    ref = O.LateralFFTOperator(go, idx)
    rng = np.random.default_rng(22)
    x = crandn(rng, g.Nz, g.Ny, g.Nx)
    y = crandn(rng, g.S, M)
    xd, yd = to_dev(x), to_dev(y)
    tol = 1e-5 if mode == "fp32" else 2.0 ** -8
    # each shard writes exactly the rows of its bins
    y_full = to_host(full.apply_A(xd))
    for j, sh in enumerate(shards):
        yj = sh.zeros(sh.shape_y)
        sh.apply_A_into(xd, yj)
        yj = to_host(yj)
        first, count = sfs.shard_run(bins.size, n, j)
        mask = np.isin(idx, bins[first:first + count])
        assert np.all(yj[~mask] == 0)
        assert rel_err(yj[mask], y_full[mask]) <= 1e-6
    assert rel_err(to_host(solver.apply_A(xd)), ref.apply_A(x)) <= tol
    assert rel_err(to_host(solver.apply_AH(yd)), ref.apply_AH(y)) <= tol
    assert rel_err(to_host(solver.gradient(xd, yd)), ref.apply_AH(ref.apply_A(x) - y)) <= tol
    # the unsharded operator's gradient through the same entry point
    assert rel_err(to_host(full.normal_residual(xd, yd)), ref.apply_AH(ref.apply_A(x) - y)) <= tol
    if mode != "fp32":
        return
    L_ref, _ = O.power_iteration(ref.apply_A, ref.apply_AH, full.shape_x, 1, max_iter=3000, rtol=1e-12)
    # FP32 vectors: the estimate's relative change settles near 1e-7, so stop at 1e-6
    L_sh, ok = solver.lipschitz(max_iter=3000, rtol=1e-6, seed=3, safety=0.0)
    assert ok and abs(L_sh - L_ref) <= 1e-4 * L_ref
    L = L_ref * 1.001
    x_true = synth.scene(full.shape_x, 4, "uniform", seed=23)
    y0 = ref.apply_A(x_true)
    sig = synth.noise_scale(float(np.vdot(y0, y0).real), y0.size, 20.0)
    ys = (y0 + sig * synth.unit_noise(y0.shape, seed=24)).astype(np.complex64).astype(complex)
    lam = O.lambda_from_mu(ref.apply_AH, ys, 0.05)
    x_ref = O.fista(ref.apply_A, ref.apply_AH, ys, lam, L, 100)
    x_sh = to_host(solver.fista(to_dev(ys), lam, L, 100))
    assert np.abs(x_ref).max() > 0
    assert rel_err(x_sh, x_ref) <= 1e-4
    assert rel_err(x_sh, to_host(full.fista(to_dev(ys), lam, L, 100))) <= 1e-5
    # mu rule: lambda from the all-reduced A^H y
    assert rel_err(to_host(solver.fista(to_dev(ys), -0.05, L, 100)), x_ref) <= 1e-4


def test_shard_arguments(sfs):
    params = geom_params(Nx=6, Ny=5, Nz=4, dz=0.15e-3, Nt=128)
    g = sfs.Geometry(**params)
    go = oracle_geometry(params)
    idx = O.select_indices(go, O.SEL_RANDOM, 3, False, 1)      # one shared set: U = 3
    with pytest.raises(sfs.SfsError):
        sfs.Operator.shard(g, idx, 4, 0)                       # more shards than bins
    with pytest.raises(sfs.SfsError):
        sfs.Operator.shard(g, idx, 2, 2)
    ops = [sfs.Operator.shard(g, idx, 3, j) for j in range(3)]
    assert [o.info["U"] for o in ops] == [1, 1, 1]
    import torch
    x = torch.zeros(ops[0].shape_x, dtype=torch.complex64, device="cuda")
    with pytest.raises(sfs.SfsError):
        sfs.prox_momentum(x, x.clone(), x.clone(), -1.0, 1.0, 0.0)   # lambda < 0
