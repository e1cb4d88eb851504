"""Batched scenes sharing one operator (sfs_apply_A_batched,
sfs_apply_AH_batched, sfs_fista_batched) against the single-scene calls and
the FP64 oracle.

A batched call runs the same arithmetic on every scene as the single-scene
call: per-scene results agree with it to FP32 rounding (<= 1e-6 relative),
and with the oracle at the precision's own tolerance (FP32 1e-5, BF16 2^-8,
BF16X2 4 * 2^-16, FP16 2^-11, FP16X2 1e-5; see test_gpu_precision.py for
their derivation).
"""
import numpy as np
import pytest

import oracle as O
import synth
from tests._common import crandn, ensure_built, geom_params, oracle_geometry, rel_err

pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-5, "bf16": 2.0 ** -8, "bf16x2": 4 * 2.0 ** -16, "fp16": 2.0 ** -11, "fp16x2": 1e-5}


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


# (Nx, Ny, Nz, Nt, M, batch): area and line scans, ragged depths and bin
# unions, batches that are not multiples of the 16-bit kernels' group of 4
CASES = [
    (12, 10, 20, 128, 12, 3),
    (16, 16, 33, 256, 10, 5),
    (32, 1, 64, 256, 32, 4),
    (8, 8, 70, 512, 40, 2),
    (5, 3, 1, 128, 1, 7),
]


@pytest.mark.parametrize("mode", list(TOL))
@pytest.mark.parametrize("case", CASES)
def test_batched_apply_equals_single_and_oracle(sfs, mode, case):
    Nx, Ny, Nz, Nt, M, B = case
    params = geom_params(Nx=Nx, Ny=Ny, Nz=Nz, dz=0.15e-3, Nt=Nt)
    go = oracle_geometry(params)
    idx = O.select_indices(go, O.SEL_RANDOM, M, True, 17)
    g = sfs.Geometry(**params)
    op = sfs.Operator.from_indices(g, idx, precision=sfs.PRECISION_NAMES[mode])
    A = O.dense_A(go, idx)
    rng = np.random.default_rng(23)
    x = crandn(rng, B, Nz, Ny, Nx)
    y = crandn(rng, B, g.S, M)
    yb = to_host(op.apply_A_batched(to_dev(x)))
    xb = to_host(op.apply_AH_batched(to_dev(y)))
    for b in range(B):
        ys = to_host(op.apply_A(to_dev(x[b])))
        xs = to_host(op.apply_AH(to_dev(y[b])))
        assert rel_err(yb[b], ys) <= 1e-6
        assert rel_err(xb[b], xs) <= 1e-6
        assert rel_err(yb[b], A @ x[b].ravel()) <= TOL[mode]
        assert rel_err(xb[b], A.conj().T @ y[b].ravel()) <= TOL[mode]


@pytest.mark.parametrize("mode", list(TOL))
def test_batched_fista_equals_single_scene_solves(sfs, mode):
    """Six scenes of the 32 x 32 x 128 workload geometry (U = 81) with their
    own scatterers and noise, lambda by the mu rule per scene: the batched
    solve returns every scene's single-scene iterate."""
    w = synth.WORKLOADS["vol32"]
    params = synth.geometry_params("vol32")
    go = oracle_geometry(params)
    idx = O.select_indices(go, O.SEL_RANDOM, w["M"], True, 1001)
    g = sfs.Geometry(**params)
    op = sfs.Operator.from_indices(g, idx, precision=sfs.PRECISION_NAMES[mode])
    B = 6
    ys = []
    for b in range(B):
        xt = synth.scene(op.shape_x, w["n_scatter"], w["amp"], seed=50 + b)
        y0 = to_host(op.apply_A(to_dev(xt)))
        sig = synth.noise_scale(float(np.vdot(y0, y0).real), y0.size, w["snr_db"])
        ys.append(y0 + sig * synth.unit_noise(y0.shape, seed=70 + b))
    y = np.stack(ys)
    L, _ = op.lipschitz(max_iter=300, rtol=1e-6, seed=2, safety=1e-3)
    xb = to_host(op.fista_batched(to_dev(y), -w["mu"], L, 40))
    for b in range(B):
        xs = to_host(op.fista(to_dev(y[b]), -w["mu"], L, 40))
        assert np.abs(xs).max() > 0
        assert rel_err(xb[b], xs) <= 1e-5


def test_batched_fp32_fista_matches_oracle(sfs):
    """Three scenes of a 10 x 10 x 16 geometry, 100 iterations, identical L and
    lambda on both sides: each batched iterate within 1e-4 of the FP64 FISTA."""
    params = geom_params(Nx=10, Ny=10, Nz=16, dz=0.15e-3, Nt=256)
    go = oracle_geometry(params)
    idx = O.select_indices(go, O.SEL_RANDOM, 12, True, 5)
    g = sfs.Geometry(**params)
    op = sfs.Operator.from_indices(g, idx)
    ref = O.LateralFFTOperator(go, idx)
    L, _ = O.power_iteration(ref.apply_A, ref.apply_AH, op.shape_x, 1, max_iter=400, rtol=1e-10)
    L *= 1.001
    ys, refs = [], []
    for b in range(3):
        xt = synth.scene(op.shape_x, 4, "uniform", seed=90 + b)
        y0 = ref.apply_A(xt)
        sig = synth.noise_scale(float(np.vdot(y0, y0).real), y0.size, 20.0)
        yb = (y0 + sig * synth.unit_noise(y0.shape, seed=95 + b)).astype(np.complex64).astype(complex)
        ys.append(yb)
    lam = O.lambda_from_mu(ref.apply_AH, ys[0], 0.05)   # one lambda for every scene
    for yb in ys:
        refs.append(O.fista(ref.apply_A, ref.apply_AH, yb, lam, L, 100))
    xb = to_host(op.fista_batched(to_dev(np.stack(ys)), lam, L, 100))
    for b in range(3):
        assert rel_err(xb[b], refs[b]) <= 1e-4
    # warm start: every scene from its own x_0 (the oracle's 30th iterate),
    # 30 more iterations with the momentum restarted at t = 1
    x0 = [O.fista(ref.apply_A, ref.apply_AH, yb, lam, L, 30) for yb in ys]
    xw = to_host(op.fista_batched(to_dev(np.stack(ys)), lam, L, 30, x=to_dev(np.stack(x0)),
                                  warm_start=True))
    for b in range(3):
        rw = O.fista(ref.apply_A, ref.apply_AH, ys[b], lam, L, 30, x0=x0[b])
        assert rel_err(xw[b], rw) <= 1e-4


@pytest.mark.parametrize("mode", ["fp32", "bf16"])
def test_largest_batch(sfs, mode):
    """SFS_MAX_BATCH scenes in one batched call (the 16-bit kernels' last
    table tile full, 64 tiles of 4): sampled scenes (first, ragged middle,
    last) equal their single-scene A, A^H and FISTA."""
    B = sfs.SFS_MAX_BATCH
    params = geom_params(Nx=8, Ny=6, Nz=12, dz=0.15e-3, Nt=128)
    go = oracle_geometry(params)
    idx = O.select_indices(go, O.SEL_RANDOM, 6, True, 31)
    g = sfs.Geometry(**params)
    op = sfs.Operator.from_indices(g, idx, precision=sfs.PRECISION_NAMES[mode])
    rng = np.random.default_rng(32)
    x = crandn(rng, B, g.Nz, g.Ny, g.Nx)
    y = crandn(rng, B, g.S, 6)
    yb = to_host(op.apply_A_batched(to_dev(x)))
    xb = to_host(op.apply_AH_batched(to_dev(y)))
    L, _ = op.lipschitz(max_iter=200, rtol=1e-6, seed=1, safety=1e-3)
    fb = to_host(op.fista_batched(to_dev(y), -0.05, L, 15))
    for b in (0, 1, 77, 130, B - 2, B - 1):
        assert rel_err(yb[b], to_host(op.apply_A(to_dev(x[b])))) <= 1e-6
        assert rel_err(xb[b], to_host(op.apply_AH(to_dev(y[b])))) <= 1e-6
        fs = to_host(op.fista(to_dev(y[b]), -0.05, L, 15))
        assert np.abs(fs).max() > 0
        assert rel_err(fb[b], fs) <= 1e-5


def test_batched_invalid_arguments(sfs):
    import ctypes
    import torch
    g = sfs.Geometry(**geom_params(Nx=4, Ny=4, Nz=4, dz=0.15e-3, Nt=64))
    op = sfs.Operator.select(g, O.SEL_RANDOM, 3, True, 0)
    x = torch.zeros((2,) + op.shape_x, dtype=torch.complex64, device="cuda")
    y = torch.zeros((2,) + op.shape_y, dtype=torch.complex64, device="cuda")
    L = sfs.lib()
    for B in (0, -1, sfs.SFS_MAX_BATCH + 1):
        assert L.sfs_apply_A_batched(op.handle, B, ctypes.c_void_p(x.data_ptr()),
                                     ctypes.c_void_p(y.data_ptr()), None) == sfs.SFS_ERR_INVALID_ARG
    assert L.sfs_fista_batched(op.handle, 2, ctypes.c_void_p(y.data_ptr()), 0.1, -1.0, 5,
                               ctypes.c_void_p(x.data_ptr()), 0, None) == sfs.SFS_ERR_INVALID_ARG
    # only SFS_FISTA_WARM_START is a batched flag
    assert L.sfs_fista_batched(op.handle, 2, ctypes.c_void_p(y.data_ptr()), 0.1, 1.0, 5,
                               ctypes.c_void_p(x.data_ptr()), sfs.SFS_FISTA_RESUME,
                               None) == sfs.SFS_ERR_INVALID_ARG
    with pytest.raises(ValueError):
        op.apply_A_batched(x[:, :, :, :2].contiguous())


def test_grouped_solve_equals_per_operator_batched_solves(sfs):
    """Three geometries (a line scan and two area scans, FP32 and BF16
    contractions) solved by one sfs_fista_grouped call: every scene equals the
    operator's own batched solve; a second call replays the cached graph."""
    import torch
    specs = [(dict(Nx=24, Ny=1, Nz=40, Nt=256), 12, 2, "fp32"),
             (dict(Nx=10, Ny=8, Nz=20, Nt=128), 10, 3, "bf16"),
             (dict(Nx=12, Ny=12, Nz=33, Nt=256), 16, 1, "fp32")]
    ops, ys, Ls = [], [], []
    rng = np.random.default_rng(41)
    for k, (geo, M, B, mode) in enumerate(specs):
        params = geom_params(dz=0.15e-3, **geo)
        go = oracle_geometry(params)
        idx = O.select_indices(go, O.SEL_RANDOM, M, True, 60 + k)
        g = sfs.Geometry(**params)
        op = sfs.Operator.from_indices(g, idx, precision=sfs.PRECISION_NAMES[mode])
        op._geom = g
        L, _ = op.lipschitz(max_iter=200, rtol=1e-6, seed=1, safety=1e-3)
        ops.append(op)
        Ls.append(L)
        ys.append(to_dev(crandn(rng, B, op.S, M)))
    xs = sfs.fista_grouped(ops, ys, Ls, -0.05, 25)
    for op, y, L, x in zip(ops, ys, Ls, xs):
        ref = to_host(op.fista_batched(y, -0.05, L, 25))
        assert rel_err(to_host(x), ref) <= 1e-6
    xs2 = sfs.fista_grouped(ops, ys, Ls, -0.05, 25)
    for a, b in zip(xs, xs2):
        assert torch.equal(a, b)
    with pytest.raises(sfs.SfsError):
        sfs.fista_grouped([ops[0], ops[0]], [ys[0], ys[0]], [Ls[0], Ls[0]], -0.05, 5)


def test_grouped_priority_orders_give_identical_results(sfs):
    """The three priority orders of the grouped graph (cheapest first,
    largest first, none) schedule the same kernels: every scene's result is
    the same bit for bit, and each order captures its own graph."""
    import torch
    specs = [(dict(Nx=24, Ny=1, Nz=40, Nt=256), 12, 2, "fp32"),
             (dict(Nx=10, Ny=8, Nz=20, Nt=128), 10, 3, "bf16"),
             (dict(Nx=20, Ny=18, Nz=33, Nt=256), 16, 2, "bf16")]
    ops, ys, Ls = [], [], []
    rng = np.random.default_rng(43)
    for k, (geo, M, B, mode) in enumerate(specs):
        params = geom_params(dz=0.15e-3, **geo)
        go = oracle_geometry(params)
        idx = O.select_indices(go, O.SEL_RANDOM, M, True, 80 + k)
        g = sfs.Geometry(**params)
        op = sfs.Operator.from_indices(g, idx, precision=sfs.PRECISION_NAMES[mode])
        op._geom = g
        ops.append(op)
        Ls.append(op.lipschitz(max_iter=200, rtol=1e-6, seed=1, safety=1e-3)[0])
        ys.append(to_dev(crandn(rng, B, op.S, M)))
    outs = []
    try:
        for order in (sfs.SFS_GROUPED_CHEAPEST_FIRST, sfs.SFS_GROUPED_LARGEST_FIRST,
                      sfs.SFS_GROUPED_NO_PRIORITY):
            sfs.set_grouped_order(order)
            outs.append([x.clone() for x in sfs.fista_grouped(ops, ys, Ls, -0.05, 20)])
            assert len(sfs.grouped_times(len(ops))) == len(ops)
    finally:
        sfs.set_grouped_order(sfs.SFS_GROUPED_CHEAPEST_FIRST)
    assert any(float(x.abs().max()) > 0 for x in outs[0])
    for o in outs[1:]:
        for a, b in zip(o, outs[0]):
            assert torch.equal(a, b)


@pytest.mark.parametrize("mode", ["bf16", "fp16"])
def test_batch_tile_choice_keeps_results_and_autotune_picks_one(sfs, mode):
    """Five scenes with one table tile serving 1, 2 or 4 of them: each
    scene's products and sums are the same, so A, A^H and FISTA agree bit for
    bit; sfs_autotune_batch picks one of the tiles it timed."""
    params = geom_params(Nx=12, Ny=10, Nz=40, dz=0.15e-3, Nt=256)
    go = oracle_geometry(params)
    idx = O.select_indices(go, O.SEL_RANDOM, 10, True, 71)
    g = sfs.Geometry(**params)
    op = sfs.Operator.from_indices(g, idx, precision=sfs.PRECISION_NAMES[mode])
    B = 5
    rng = np.random.default_rng(72)
    x = to_dev(crandn(rng, B, g.Nz, g.Ny, g.Nx))
    y = to_dev(crandn(rng, B, g.S, 10))
    outs = []
    for nb in (1, 2, 4):
        op.set_batch_tile(B, nb)
        outs.append((to_host(op.apply_A_batched(x)), to_host(op.apply_AH_batched(y)),
                     to_host(op.fista_batched(y, -0.05, 1.0e9, 20))))
    for o in outs[1:]:
        for a, b in zip(o, outs[0]):
            assert np.array_equal(a, b)
    nb, ms = op.autotune(B, reps=3)
    assert nb in (1, 2, 4)
    assert all(np.isfinite(ms)) and ms[[1, 2, 4].index(nb)] == min(ms)
    assert np.array_equal(to_host(op.fista_batched(y, -0.05, 1.0e9, 20)), outs[0][2])
    op32 = sfs.Operator.from_indices(g, idx)
    assert op32.autotune(B)[0] == 0


def test_grouped_completion_times(sfs):
    """sfs_grouped_times after a grouped solve: one time per group, each
    positive and within the whole call's event-timed span; the small group
    finishes no later than the solve."""
    import torch
    specs = [(dict(Nx=8, Ny=1, Nz=16, Nt=128), 6, 2), (dict(Nx=16, Ny=16, Nz=40, Nt=256), 16, 3)]
    ops, ys, Ls = [], [], []
    rng = np.random.default_rng(81)
    for k, (geo, M, B) in enumerate(specs):
        params = geom_params(dz=0.15e-3, **geo)
        go = oracle_geometry(params)
        idx = O.select_indices(go, O.SEL_RANDOM, M, True, 80 + k)
        g = sfs.Geometry(**params)
        op = sfs.Operator.from_indices(g, idx)
        op._geom = g
        ops.append(op)
        Ls.append(op.lipschitz(max_iter=100, rtol=1e-5, seed=1, safety=1e-2)[0])
        ys.append(to_dev(crandn(rng, B, op.S, M)))
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sfs.fista_grouped(ops, ys, Ls, -0.05, 30)   # capture
    torch.cuda.synchronize()
    a.record()
    sfs.fista_grouped(ops, ys, Ls, -0.05, 30)
    b.record()
    torch.cuda.synchronize()
    total = a.elapsed_time(b)
    t = sfs.grouped_times(2)
    assert len(t) == 2 and all(0 < v <= total * 1.01 + 0.05 for v in t)
    with pytest.raises(sfs.SfsError):
        sfs.grouped_times(3)


@pytest.mark.parametrize("mode", ["fp32", "fp16"])
def test_quadrant_planes_as_clusters_and_one_cta_agree(sfs, mode):
    """128 x 128 planes run as one cluster of four CTAs per plane while the
    launch holds few planes (2 n <= 3 SMs), one CTA per plane otherwise.  A
    batch large enough for the one-CTA kernels and single-scene solves (the
    cluster kernels) must give the same FISTA iterates to FP32 rounding
    (FP32: also the oracle's); FP16 also exercises the per-plane maxima gathered across the
    cluster."""
    import torch
    params = geom_params(Nx=40, Ny=36, Nz=10, dz=0.15e-3, Nt=256)
    go = oracle_geometry(params)
    g = sfs.Geometry(**params)
    idx = O.select_indices(go, O.SEL_RANDOM, 10, True, 61)
    op = sfs.Operator.from_indices(g, idx, precision=sfs.PRECISION_NAMES[mode])
    assert op.info["Px"] == 128
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    U = op.info["U"]
    B = (3 * sms) // (2 * min(U, g.Nz)) + 1          # past the cluster rule for both plane kernels
    assert 2 * B * g.Nz > 3 * sms and 2 * B * U > 3 * sms
    ref = O.LateralFFTOperator(go, idx)
    ys = []
    for b in range(B):
        x_true = synth.scene(op.shape_x, 3, "uniform", seed=300 + b)
        y0 = ref.apply_A(x_true) if b < 2 else None
        if y0 is None:
            ys.append(crandn(np.random.default_rng(400 + b), g.S, op.M) * 0.1)
            continue
        sig = synth.noise_scale(float(np.vdot(y0, y0).real), y0.size, 20.0)
        ys.append((y0 + sig * synth.unit_noise(y0.shape, seed=500 + b)).astype(np.complex64).astype(complex))
    Y = np.stack(ys)
    L, _ = op.lipschitz(max_iter=300, rtol=1e-6, seed=2, safety=1e-3)
    xb = to_host(op.fista_batched(to_dev(Y), -0.05, L, 60))
    for b in (0, 1, B - 1):
        xs = to_host(op.fista(to_dev(Y[b]), -0.05, L, 60))
        # the one-CTA engine applies the quadrant twiddles as two factors, the
        # cluster CTAs as one: FP32 roundings apart, carried through 60 steps
        assert rel_err(xb[b], xs) <= 1e-5
    if mode == "fp32":
        lam = O.lambda_from_mu(ref.apply_AH, Y[0], 0.05)
        x_ref = O.fista(ref.apply_A, ref.apply_AH, Y[0], lam, L, 60)
        assert np.abs(x_ref).max() > 0
        assert rel_err(xb[0], x_ref) <= 1e-4
