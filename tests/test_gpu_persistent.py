"""sfs_fista_persistent: the FISTA loops of several groups of scenes (different
scan grids, lateral FFT sizes 32 / 64 / 128, depths, bin counts, BF16 and
FP16 tables, 1 / 2 / 4 scenes per table tile) in one persistent kernel.

Its contractions are the grouped solve's code on the same units and its
plane steps the one-CTA plane engine, so per scene it must agree with
sfs_fista_grouped to the rounding of the plane engine variant (the grouped
solve runs 128 x 128 planes as 4-CTA clusters when a launch holds few
planes): 1e-4 after 40 iterations of a 16-bit operator.  A one-group solve
with lambda from the FP64 oracle is also compared with the oracle's FISTA
within the 16-bit FISTA bar of the precision tests (4e-3 after 60
iterations).
"""
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


# (geometry, M, scenes, precision, scenes per table tile)
GROUPS = [
    (dict(Nx=12, Ny=10, Nz=20, Nt=128), 8, 3, "bf16", 4),    # 32 x 32 planes
    (dict(Nx=20, Ny=18, Nz=33, Nt=256), 10, 5, "fp16", 2),   # 64 x 64 planes, FP16 scales
    (dict(Nx=40, Ny=36, Nz=10, Nt=256), 10, 2, "bf16", 1),   # 128 x 128 quadrant planes
    (dict(Nx=16, Ny=16, Nz=64, Nt=256), 12, 4, "bf16", 4),
]


def build_groups(sfs, groups, seed):
    ops, ys, Ls = [], [], []
    rng = np.random.default_rng(seed)
    for k, (geo, M, B, mode, nb) in enumerate(groups):
        params = geom_params(dz=0.15e-3, **geo)
        go = oracle_geometry(params)
        idx = O.select_indices(go, O.SEL_RANDOM, M, True, seed + k)
        g = sfs.Geometry(**params)
        op = sfs.Operator.from_indices(g, idx, precision=sfs.PRECISION_NAMES[mode])
        op._geom = g
        op.set_batch_tile(B, nb)
        ops.append(op)
        Ls.append(op.lipschitz(max_iter=200, rtol=1e-6, seed=1, safety=1e-2)[0])
        scenes = []
        for b in range(B):
            x_true = synth.scene(op.shape_x, 3, "uniform", seed=seed + 10 * k + b)
            xd = to_dev(x_true[None])
            y0 = to_host(op.apply_A_batched(xd))[0]
            sig = synth.noise_scale(float(np.vdot(y0, y0).real), y0.size, 20.0)
            scenes.append(y0 + sig * crandn(rng, *y0.shape) / np.sqrt(2.0))
        ys.append(to_dev(np.stack(scenes)))
    return ops, ys, Ls


def test_persistent_equals_grouped(sfs):
    ops, ys, Ls = build_groups(sfs, GROUPS, 900)
    xg = [to_host(x) for x in sfs.fista_grouped(ops, ys, Ls, -0.05, 40)]
    xp = [to_host(x) for x in sfs.fista_persistent(ops, ys, Ls, -0.05, 40)]
    for g in range(len(ops)):
        assert np.abs(xg[g]).max() > 0
        for b in range(xg[g].shape[0]):
            assert rel_err(xp[g][b], xg[g][b]) <= 1e-4, (g, b)
    # the second call replays the cached graph: the same result bit for bit
    xp2 = [to_host(x) for x in sfs.fista_persistent(ops, ys, Ls, -0.05, 40)]
    for g in range(len(ops)):
        assert np.array_equal(xp2[g], xp[g])
    st = sfs.persistent_step_times()
    assert len(st) == 8 and all(v > 0 for v in st)
    assert all(st[4 + i] <= st[i] * 1.05 + 1e-3 for i in range(3))  # busy within the step
    # every group with one scene per table tile: the same results
    xp1 = [to_host(x) for x in sfs.fista_persistent(ops, ys, Ls, -0.05, 40, nb_policy=1)]
    for g in range(len(ops)):
        for b in range(xg[g].shape[0]):
            assert rel_err(xp1[g][b], xg[g][b]) <= 1e-4, (g, b)
    # the tile tuner times the four policies and picks the fastest
    c, ms = sfs.autotune_persistent(ops, ys, Ls, -0.05, probe_iters=4, reps=2)
    assert c in (0, 1, 2, 4) and all(v > 0 for v in ms) and ms[(0, 1, 2, 4).index(c)] == min(ms)
    for op in ops:
        assert op.check_status() == 0


def test_largest_group_count(sfs):
    """SFS_MAX_GROUPS groups (operators of a few small geometries and depths,
    one or two scenes each) in one grouped and one persistent solve: every
    scene agrees between the two and with its operator's own batched solve."""
    G = sfs.SFS_MAX_GROUPS
    ops, ys, Ls = [], [], []
    rng = np.random.default_rng(55)
    for k in range(G):
        Nx, Ny = (6, 6) if k % 3 == 0 else (10, 8) if k % 3 == 1 else (20, 18)
        params = geom_params(Nx=Nx, Ny=Ny, Nz=8 + 4 * (k % 4), dz=0.15e-3, Nt=128)
        go = oracle_geometry(params)
        M = 4 + k % 5
        idx = O.select_indices(go, O.SEL_RANDOM, M, True, 500 + k)
        g = sfs.Geometry(**params)
        op = sfs.Operator.from_indices(g, idx, precision=sfs.SFS_PREC_BF16)
        op._geom = g
        ops.append(op)
        Ls.append(op.lipschitz(max_iter=100, rtol=1e-5, seed=1, safety=1e-2)[0])
        ys.append(to_dev(crandn(rng, 1 + k % 2, op.S, M)))
    xg = [to_host(x) for x in sfs.fista_grouped(ops, ys, Ls, -0.05, 12)]
    xp = [to_host(x) for x in sfs.fista_persistent(ops, ys, Ls, -0.05, 12)]
    for k in (0, 1, 2, 31, G - 1):
        xb = to_host(ops[k].fista_batched(ys[k], -0.05, Ls[k], 12))
        assert np.abs(xb).max() > 0
        assert rel_err(xg[k], xb) <= 1e-5, k
    for k in range(G):
        assert rel_err(xp[k], xg[k]) <= 1e-4, k
    for op in ops:
        assert op.check_status() == 0


def test_persistent_one_group_matches_oracle(sfs):
    geo, M = dict(Nx=24, Ny=20, Nz=12, Nt=256), 10
    params = geom_params(dz=0.15e-3, **geo)
    go = oracle_geometry(params)
    idx = O.select_indices(go, O.SEL_RANDOM, M, True, 77)
    g = sfs.Geometry(**params)
    op = sfs.Operator.from_indices(g, idx, precision=sfs.SFS_PREC_BF16)
    ref = O.LateralFFTOperator(go, idx)
    x_true = synth.scene(op.shape_x, 4, "uniform", seed=78)
    y0 = ref.apply_A(x_true)
    sig = synth.noise_scale(float(np.vdot(y0, y0).real), y0.size, 20.0)
    y = (y0 + sig * synth.unit_noise(y0.shape, seed=79)).astype(np.complex64).astype(complex)
    L, _ = O.power_iteration(ref.apply_A, ref.apply_AH, op.shape_x, 1, max_iter=400, rtol=1e-10)
    L *= 1.001
    lam = O.lambda_from_mu(ref.apply_AH, y, 0.05)
    x_ref = O.fista(ref.apply_A, ref.apply_AH, y, lam, L, 60)
    (xp,) = sfs.fista_persistent([op], [to_dev(y[None])], [L], lam, 60)
    assert np.abs(x_ref).max() > 0
    assert rel_err(to_host(xp)[0], x_ref) <= 4e-3


@pytest.mark.parametrize("kind", ["fp32", "bf16x2", "line"])
def test_persistent_rejects_other_operators(sfs, kind):
    """FP32, two-part 16-bit and line-scan operators, and a tile policy other
    than 0, 1, 2 or 4, are refused."""
    if kind == "line":
        params = geom_params(Nx=16, Ny=1, Nz=8, dz=0.15e-3, Nt=128)
        prec = sfs.SFS_PREC_BF16
    else:
        params = geom_params(Nx=8, Ny=8, Nz=8, dz=0.15e-3, Nt=128)
        prec = sfs.PRECISION_NAMES[kind]
    go = oracle_geometry(params)
    g = sfs.Geometry(**params)
    op = sfs.Operator.from_indices(g, O.select_indices(go, O.SEL_RANDOM, 4, True, 5), precision=prec)
    y = to_dev(np.zeros((1, op.S, op.M)))
    with pytest.raises(sfs.SfsError):
        sfs.fista_persistent([op], [y], [1.0], -0.05, 5)
    if kind == "line":
        g2 = sfs.Geometry(**geom_params(Nx=8, Ny=8, Nz=8, dz=0.15e-3, Nt=128))
        op2 = sfs.Operator.from_indices(g2, O.select_indices(oracle_geometry(geom_params(
            Nx=8, Ny=8, Nz=8, dz=0.15e-3, Nt=128)), O.SEL_RANDOM, 4, True, 5), precision=sfs.SFS_PREC_BF16)
        with pytest.raises(sfs.SfsError):
            sfs.fista_persistent([op2], [to_dev(np.zeros((1, op2.S, op2.M)))], [1.0], -0.05, 5, nb_policy=3)
