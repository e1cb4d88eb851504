"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Tolerances (complex64 path vs FP64 oracle):
  * A x and A^H y: relative 2-norm error <= 1e-5
  * FISTA iterate after 200 iterations with identical L and lambda: <= 1e-4
  * integer selection: bit-exact
"""
import math

import numpy as np
import pytest

import oracle as O
import synth
from tests._common import crandn, ensure_built, geom_params, oracle_geometry, rel_err

pytestmark = pytest.mark.gpu

TOL_OP = 1e-5
TOL_FISTA = 1e-4


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


def make_pair(sfs, params, strategy=O.SEL_RANDOM, M=8, per_position=True, seed=7):
    g = sfs.Geometry(**params)
    op = sfs.Operator.select(g, strategy, M, per_position, seed)
    go = oracle_geometry(params)
    idx = O.select_indices(go, strategy, M, per_position, seed)
    assert np.array_equal(op.idx, idx)
    return g, op, go, idx


# (Nx, Ny, Nz, Nt, M): line scans and area scans spanning several kappa tiles,
# a ragged depth count (not a multiple of 16) and a ragged bin union
SMALL_CASES = [
    (32, 1, 64, 256, 32),     # the 2-D line-scan workload geometry
    (12, 10, 20, 128, 12),    # 3-D, P = 32: 16 tiles of 64 wavenumbers
    (7, 1, 5, 64, 3),
    (1, 1, 9, 64, 4),         # a single A-scan
    (16, 16, 33, 256, 10),
    (5, 3, 1, 128, 1),        # one depth, one bin
]


@pytest.mark.parametrize("case", SMALL_CASES)
def test_apply_A_and_AH_match_dense_oracle(sfs, case):
    Nx, Ny, Nz, Nt, M = case
    params = geom_params(Nx=Nx, Ny=Ny, Nz=Nz, dz=0.15e-3, Nt=Nt)
    g, op, go, idx = make_pair(sfs, params, M=M)
    A = O.dense_A(go, idx)
    rng = np.random.default_rng(11)
    x = crandn(rng, Nz, Ny, Nx)
    y = crandn(rng, g.S, M)
    ya = to_host(op.apply_A(to_dev(x)))
    xa = to_host(op.apply_AH(to_dev(y)))
    ref_y = (A @ x.ravel()).reshape(g.S, M)
    ref_x = (A.conj().T @ y.ravel()).reshape(Nz, Ny, Nx)
    assert rel_err(ya, ref_y) <= TOL_OP
    assert rel_err(xa, ref_x) <= TOL_OP
    # element-wise: no entry off by more than 1e-4 of the largest entry
    assert np.abs(ya - ref_y).max() <= 1e-4 * np.abs(ref_y).max()
    assert np.abs(xa - ref_x).max() <= 1e-4 * np.abs(ref_x).max()


@pytest.mark.parametrize("strategy", [O.SEL_RANDOM, O.SEL_CONTIGUOUS, O.SEL_EQUISPACED,
                                      O.SEL_MAXIMAL, O.SEL_ENERGY])
@pytest.mark.parametrize("per_position", [True, False])
def test_strategies_select_and_apply(sfs, strategy, per_position):
    params = geom_params(Nx=9, Ny=6, Nz=11, dz=0.15e-3, Nt=256)
    g, op, go, idx = make_pair(sfs, params, strategy=strategy, M=10,
                               per_position=per_position, seed=99)
    # mask agrees with the index sets
    for s in range(g.S):
        bits = [k for k in range(g.Nt // 2 + 1) if (op.mask[s, k // 32] >> (k % 32)) & 1]
        assert bits == idx[s].tolist()
    assert op.info["U"] == len(np.unique(idx))
    A = O.dense_A(go, idx)
    rng = np.random.default_rng(3)
    x = crandn(rng, g.Nz, g.Ny, g.Nx)
    assert rel_err(to_host(op.apply_A(to_dev(x))), A @ x.ravel()) <= TOL_OP


@pytest.mark.parametrize("name", ["line2d", "vol32"])
def test_host_time_gate_pulse_rate_and_band_equal_the_oracle(sfs, name):
    """The library's readings of the geometry (t0 on the sample grid, the
    pulse rate alpha, the candidate band and its rung) are the oracle's."""
    w = synth.WORKLOADS[name]
    params = synth.geometry_params(name)
    go = oracle_geometry(params)
    op = sfs.Operator.select(sfs.Geometry(**params), O.SEL_CONTIGUOUS, w["M"], False, 0)
    info = op.info
    assert round(info["t0"] * go.fs) == round(go.t0 * go.fs)
    assert abs(info["t0"] * go.fs - round(info["t0"] * go.fs)) <= 1e-6
    assert info["alpha"] == pytest.approx(go.alpha, rel=1e-13)
    k_lo, k_hi, b = O.candidate_band(go, w["M"])
    assert (info["k_lo"], info["k_hi"]) == (k_lo, k_hi) and info["band_db"] == b


def test_directivity_geometry(sfs):
    params = geom_params(Nx=10, Ny=8, Nz=12, dz=0.2e-3, Nt=256, theta=math.radians(30))
    g, op, go, idx = make_pair(sfs, params, M=9)
    A = O.dense_A(go, idx)
    rng = np.random.default_rng(5)
    x = crandn(rng, g.Nz, g.Ny, g.Nx)
    y = crandn(rng, g.S, 9)
    assert rel_err(to_host(op.apply_A(to_dev(x))), A @ x.ravel()) <= TOL_OP
    assert rel_err(to_host(op.apply_AH(to_dev(y))), A.conj().T @ y.ravel()) <= TOL_OP


def test_operator_from_given_indices_and_user_t0(sfs):
    params = geom_params(Nx=6, Ny=6, Nz=8, dz=0.15e-3, Nt=128, t0=3.0e-6)
    go = oracle_geometry(params)
    rng = np.random.default_rng(8)
    idx = np.sort(np.stack([rng.choice(np.arange(3, 60), 5, replace=False)
                            for _ in range(36)]), axis=1).astype(np.int32)
    g = sfs.Geometry(**params)
    op = sfs.Operator.from_indices(g, idx)
    A = O.dense_A(go, idx)
    x = crandn(rng, 8, 6, 6)
    assert rel_err(to_host(op.apply_A(to_dev(x))), A @ x.ravel()) <= TOL_OP


def test_adjoint_identity_on_gpu(sfs):
    params = synth.geometry_params("vol32")
    g = sfs.Geometry(**params)
    op = sfs.Operator.select(g, O.SEL_RANDOM, 64, True, 5)
    rng = np.random.default_rng(1)
    x = crandn(rng, *op.shape_x)
    y = crandn(rng, *op.shape_y)
    Ax = to_host(op.apply_A(to_dev(x))).astype(np.complex128)
    AHy = to_host(op.apply_AH(to_dev(y))).astype(np.complex128)
    lhs = np.vdot(y, Ax)
    rhs = np.vdot(AHy, x)
    # If each operator is within TOL_OP of the exact one (relative, in norm),
    # Cauchy-Schwarz bounds the mismatch by TOL_OP (|y| |Ax| + |A^H y| |x|); a
    # wrong conjugate, sign or index breaks the identity by O(1) of that scale.
    scale = (np.linalg.norm(y) * np.linalg.norm(Ax) + np.linalg.norm(AHy) * np.linalg.norm(x))
    assert abs(lhs - rhs) <= TOL_OP * scale


def test_vol32_full_size_against_structured_and_dense_rows(sfs):
    """The 32 x 32 x 128 workload at full size: whole outputs against the FP64
    lateral-FFT oracle, and 400 sampled rows of A against the dense definition."""
    w = synth.WORKLOADS["vol32"]
    params = synth.geometry_params("vol32")
    g, op, go, idx = make_pair(sfs, params, M=w["M"], seed=1001)
    assert op.info["U"] == 81
    rng = np.random.default_rng(2)
    x = synth.scene((g.Nz, g.Ny, g.Nx), 40, "uniform", seed=4) + 0.01 * crandn(rng, g.Nz, g.Ny, g.Nx)
    y = crandn(rng, g.S, w["M"])
    ya = to_host(op.apply_A(to_dev(x)))
    xa = to_host(op.apply_AH(to_dev(y)))
    ref = O.LateralFFTOperator(go, idx)
    assert rel_err(ya, ref.apply_A(x)) <= TOL_OP
    assert rel_err(xa, ref.apply_AH(y)) <= TOL_OP
    rows = rng.choice(g.S * w["M"], 400, replace=False)
    dense = O.A_rows(go, idx, rows) @ x.ravel()
    assert rel_err(ya.ravel()[rows], dense) <= TOL_OP


def test_max_abs_AH_and_lipschitz(sfs):
    params = geom_params(Nx=8, Ny=8, Nz=16, dz=0.15e-3, Nt=128)
    g, op, go, idx = make_pair(sfs, params, M=6)
    A = O.dense_A(go, idx)
    rng = np.random.default_rng(4)
    y = crandn(rng, g.S, 6)
    ref = np.abs(A.conj().T @ y.ravel()).max()
    assert op.max_abs_AH(to_dev(y)) == pytest.approx(ref, rel=1e-5)
    smax2 = np.linalg.svd(A, compute_uv=False)[0] ** 2
    L, converged = op.lipschitz(max_iter=3000, rtol=1e-7, seed=3, safety=0.0)
    assert converged
    assert L == pytest.approx(smax2, rel=1e-4)
    L2, _ = op.lipschitz(max_iter=3000, rtol=1e-7, seed=3, safety=1e-3)
    assert L2 == pytest.approx(L * 1.001, rel=1e-9)


def _fista_case(sfs, params, M, n_scatter, iters, mu=0.05, snr_db=20.0, seed=1):
    g, op, go, idx = make_pair(sfs, params, M=M, seed=seed + 100)
    ref = O.LateralFFTOperator(go, idx)
    x_true = synth.scene((g.Nz, g.Ny, g.Nx), n_scatter, "uniform", seed=seed)
    y0 = ref.apply_A(x_true)
    sig = synth.noise_scale(float(np.vdot(y0, y0).real), y0.size, snr_db)
    y = (y0 + sig * synth.unit_noise(y0.shape, seed=seed + 7)).astype(np.complex64)
    y = y.astype(np.complex128)
    L, _ = O.power_iteration(ref.apply_A, ref.apply_AH, x_true.shape, seed, max_iter=400,
                             rtol=1e-10)
    L *= 1.001
    lam = O.lambda_from_mu(ref.apply_AH, y, mu)
    x_ref = O.fista(ref.apply_A, ref.apply_AH, y, lam, L, iters)
    x_gpu = to_host(op.fista(to_dev(y), lam, L, iters))
    return x_gpu, x_ref, op, ref, y, lam, L


@pytest.mark.parametrize("case", [
    ("line2d", dict(), 32, 3, 200),
    ("small3d", dict(Nx=12, Ny=12, Nz=24, dz=0.15e-3, Nt=256), 16, 5, 200),
    # 128 x 128 lateral FFT planes (2 * 40 - 1 > 64), a non-square scan
    ("p128", dict(Nx=40, Ny=36, Nz=10, dz=0.15e-3, Nt=256), 10, 4, 200),
])
def test_fista_200_iterations_matches_oracle(sfs, case):
    name, over, M, ns, iters = case
    params = synth.geometry_params("line2d") if name == "line2d" else geom_params(**over)
    x_gpu, x_ref, *_ = _fista_case(sfs, params, M, ns, iters)
    assert np.abs(x_ref).max() > 0
    assert rel_err(x_gpu, x_ref) <= TOL_FISTA


def test_fista_mu_rule_warm_start_and_monitor(sfs):
    params = geom_params(Nx=10, Ny=10, Nz=16, dz=0.15e-3, Nt=256)
    x_gpu, x_ref, op, ref, y, lam, L = _fista_case(sfs, params, 12, 4, 60)
    # lambda < 0: mu rule evaluated on the device gives the same iterate
    x_mu = to_host(op.fista(to_dev(y), -0.05, L, 60))
    assert rel_err(x_mu, x_ref) <= TOL_FISTA
    # warm start: 30 + 30 restarted iterations equal the oracle restarted alike
    x30 = op.fista(to_dev(y), lam, L, 30)
    x_w = to_host(op.fista(to_dev(y), lam, L, 30, x=x30, warm_start=True))
    r30 = O.fista(ref.apply_A, ref.apply_AH, y, lam, L, 30)
    r_w = O.fista(ref.apply_A, ref.apply_AH, y, lam, L, 30, x0=r30)
    assert rel_err(x_w, r_w) <= TOL_FISTA
    # objective monitor: 1/2||A gamma_k - y||^2 + lam ||x_k||_1
    _, hist = op.fista(to_dev(y), lam, L, 10, obj_hist=True)
    beta, _ = O.fista_momentum(10)
    gam = np.zeros(op.shape_x, complex)
    xp = gam.copy()
    for k in range(10):
        r = ref.apply_A(gam) - y
        xk = O.soft_threshold(gam - ref.apply_AH(r) / L, lam / L)
        mon = 0.5 * np.vdot(r, r).real + lam * np.abs(xk).sum()
        assert hist[k] == pytest.approx(mon, rel=1e-4)
        gam = xk + beta[k] * (xk - xp)
        xp = xk
    # zero iterations return zero; lambda above ||A^H y||_inf gives zero
    assert np.all(to_host(op.fista(to_dev(y), lam, L, 0)) == 0)
    big = float(np.abs(ref.apply_AH(y)).max()) * 1.01
    assert np.all(to_host(op.fista(to_dev(y), big, L, 20)) == 0)


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_fista_recovers_isolated_scatterers_noiseless_on_gpu(sfs, prec):
    """Noiseless data of isolated scatterers (at least 4 voxels apart) and a
    small mu: the 4 largest magnitudes of the GPU iterate sit exactly on the
    true positions (the recovery the oracle is pinned by, here through the
    C ABI, Algorithm 1 with the mu rule evaluated on the device)."""
    params = geom_params(Nx=10, Ny=10, Nz=16, dz=0.15e-3, Nt=256)
    go = oracle_geometry(params)
    idx = O.select_indices(go, O.SEL_RANDOM, 16, True, 77)
    g = sfs.Geometry(**params)
    op = sfs.Operator.from_indices(g, idx, precision=sfs.PRECISION_NAMES[prec])
    x_true = synth.scene(op.shape_x, 4, "unit", seed=13, min_sep=4)
    y = O.LateralFFTOperator(go, idx).apply_A(x_true)
    L, _ = op.lipschitz(max_iter=2000, rtol=1e-9, seed=1, safety=1e-3)
    x = to_host(op.fista(to_dev(y), -0.02, L, 400))
    top = np.argsort(np.abs(x).ravel())[-4:]
    assert set(top.tolist()) == set(np.nonzero(x_true.ravel())[0].tolist())


def test_fista_on_zero_data_stays_zero(sfs):
    """y = 0: the mu rule gives lambda = 0 and the gradient is zero at
    x = 0, so every iterate is exactly zero (no division by lambda or by a
    norm of the data anywhere on the path)."""
    params = geom_params(Nx=12, Ny=10, Nz=20, dz=0.15e-3, Nt=128)
    g = sfs.Geometry(**params)
    op = sfs.Operator.select(g, O.SEL_RANDOM, 8, True, 3)
    y = np.zeros(op.shape_y, complex)
    for lam in (-0.05, 0.0, 0.1):
        x = to_host(op.fista(to_dev(y), lam, 1.0, 25))
        assert np.all(x == 0), lam
    assert op.max_abs_AH(to_dev(y)) == 0.0


@pytest.mark.parametrize("case", [
    ("fp32", dict(Nx=10, Ny=10, Nz=16, dz=0.15e-3, Nt=256), 12),
    ("fp16", dict(Nx=10, Ny=10, Nz=16, dz=0.15e-3, Nt=256), 12),
    ("fp32", dict(Nx=40, Ny=36, Nz=10, dz=0.15e-3, Nt=256), 10),   # 128 x 128 planes
])
def test_fista_resumed_from_state_is_bit_exact(sfs, case):
    """Algorithm 1's state (gamma_{k+1}, x_k, t_{k+1}) through the ABI: 30
    iterations, then 30 resumed from the state buffer, equal 60 iterations in
    one call bit for bit, and the FP64 oracle's 60 within the FISTA bar; a
    restart from x_30 (momentum back at t = 1) differs."""
    import torch
    mode, over, M = case
    params = geom_params(**over)
    g = sfs.Geometry(**params)
    go = oracle_geometry(params)
    idx = O.select_indices(go, O.SEL_RANDOM, M, True, 9)
    op = sfs.Operator.from_indices(g, idx, precision=sfs.PRECISION_NAMES[mode])
    ref = O.LateralFFTOperator(go, idx)
    x_true = synth.scene(op.shape_x, 4, "uniform", seed=10)
    y0 = ref.apply_A(x_true)
    sig = synth.noise_scale(float(np.vdot(y0, y0).real), y0.size, 20.0)
    y = (y0 + sig * synth.unit_noise(y0.shape, seed=11)).astype(np.complex64).astype(complex)
    L, _ = O.power_iteration(ref.apply_A, ref.apply_AH, op.shape_x, 1, max_iter=400, rtol=1e-10)
    L *= 1.001
    lam = O.lambda_from_mu(ref.apply_AH, y, 0.05)
    yd = to_dev(y)
    x60 = to_host(op.fista(yd, lam, L, 60))
    state = op.new_fista_state()
    x30 = op.fista(yd, lam, L, 30, state=state)
    torch.cuda.synchronize()
    st = state.cpu().numpy()
    assert np.array_equal(st[op.V:2 * op.V].reshape(op.shape_x), x30.cpu().numpy())
    t31, k = st[2 * op.V:].view(np.float64)[0], st[2 * op.V:].view(np.int64)[1]
    _, t_ref = O.fista_momentum(30)
    assert k == 30 and t31 == pytest.approx(t_ref, rel=1e-15)
    x_res = to_host(op.fista(yd, lam, L, 30, state=state, resume=True))
    assert np.array_equal(x_res, x60)
    assert state.cpu().numpy()[2 * op.V:].view(np.int64)[1] == 60
    x_ref = O.fista(ref.apply_A, ref.apply_AH, y, lam, L, 60)
    assert rel_err(x_res, x_ref) <= (TOL_FISTA if mode == "fp32" else 4e-3)
    x_warm = to_host(op.fista(yd, lam, L, 30, x=x30.clone(), warm_start=True))
    assert rel_err(x_warm, x60) > 1e-6
    # RESUME needs a state buffer and excludes WARM_START
    with pytest.raises(sfs.SfsError):
        op.fista(yd, lam, L, 5, resume=True)
    with pytest.raises(sfs.SfsError):
        op.fista(yd, lam, L, 5, state=state, resume=True, warm_start=True)


def test_deterministic_and_stream_ordered(sfs):
    import torch
    params = geom_params(Nx=16, Ny=16, Nz=32, dz=0.15e-3, Nt=256)
    g = sfs.Geometry(**params)
    op = sfs.Operator.select(g, O.SEL_RANDOM, 16, True, 3)
    rng = np.random.default_rng(0)
    x = to_dev(crandn(rng, *op.shape_x))
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        y1 = op.apply_A(x)
        y2 = op.apply_A(x)
    s.synchronize()
    assert torch.equal(y1, y2)


def test_invalid_arguments_on_gpu(sfs):
    import torch
    params = geom_params(Nx=4, Ny=4, Nz=4, dz=0.15e-3, Nt=64)
    g = sfs.Geometry(**params)
    op = sfs.Operator.select(g, O.SEL_RANDOM, 3, True, 0)
    x = torch.zeros(op.shape_x, dtype=torch.complex64, device="cuda")
    with pytest.raises(ValueError):
        op.apply_A(x[:, :, :2].contiguous())
    with pytest.raises(sfs.SfsError):
        op.fista(torch.zeros(op.shape_y, dtype=torch.complex64, device="cuda"), 0.1, -1.0, 5)
    # misaligned device pointer
    buf = torch.zeros(op.V + 1, dtype=torch.complex64, device="cuda")
    y = torch.zeros(op.shape_y, dtype=torch.complex64, device="cuda")
    L = sfs.lib()
    import ctypes
    rc = L.sfs_apply_A(op.handle, ctypes.c_void_p(buf.data_ptr() + 8), ctypes.c_void_p(y.data_ptr()), None)
    assert rc == sfs.SFS_ERR_INVALID_ARG
    bad = np.array([[5, 5, 6]] * 16, dtype=np.int32)
    with pytest.raises(sfs.SfsError):
        sfs.Operator.from_indices(g, bad)


@pytest.mark.parametrize("theta_deg", [0.0, 25.0])
def test_frobenius_norm_and_sigma_estimate(sfs, theta_deg):
    """||A||_F^2 of Sec. IV-C from the closed-form magnitudes equals the dense
    oracle's (1e-12), and the estimate ||A||_F / N^(1/4) lies between the
    bounds ||A||_F / sqrt(N) <= sigma_max <= ||A||_F."""
    params = geom_params(Nx=7, Ny=5, Nz=9, dz=0.2e-3, Nt=128, theta=math.radians(theta_deg))
    g, op, go, idx = make_pair(sfs, params, M=6, seed=31)
    A = O.dense_A(go, idx)
    fro2, sigma_hat = op.frobenius()
    assert fro2 == pytest.approx(float(np.linalg.norm(A) ** 2), rel=1e-12)
    smax = float(np.linalg.svd(A, compute_uv=False)[0])
    N = min(A.shape)
    assert math.sqrt(fro2) / math.sqrt(N) <= smax * (1 + 1e-12) <= math.sqrt(fro2) * (1 + 1e-12)
    assert sigma_hat == pytest.approx(math.sqrt(fro2) / N ** 0.25, rel=1e-12)


# tolerances of the modes against the FP64 oracle (derived in
# test_gpu_precision.py): relative 2-norm, and element-wise against the
# largest entry
P128_TOL = {"fp32": (TOL_OP, 10 * TOL_OP), "bf16": (2.0 ** -8, 8 * 2.0 ** -8),
            "fp16": (2.0 ** -11, 8 * 2.0 ** -11)}


@pytest.mark.parametrize("mode", list(P128_TOL))
def test_128_point_planes_match_oracle(sfs, mode):
    """A 48 x 40 scan pads its planes to 128 x 128 (the 1024-thread plane
    kernels): single and batched (3 scenes in one 16-bit group) A and A^H
    against the FP64 lateral-FFT oracle."""
    params = geom_params(Nx=48, Ny=40, Nz=14, dz=0.15e-3, Nt=256)
    go = oracle_geometry(params)
    idx = O.select_indices(go, O.SEL_RANDOM, 12, True, 31)
    g = sfs.Geometry(**params)
    op = sfs.Operator.from_indices(g, idx, precision=sfs.PRECISION_NAMES[mode])
    assert op.info["Px"] == 128 and op.info["Py"] == 128
    ref = O.LateralFFTOperator(go, idx)
    rng = np.random.default_rng(32)
    x = crandn(rng, 3, g.Nz, g.Ny, g.Nx)
    y = crandn(rng, 3, g.S, 12)
    tol, tol_el = P128_TOL[mode]
    yb = to_host(op.apply_A_batched(to_dev(x)))
    xb = to_host(op.apply_AH_batched(to_dev(y)))
    for b in range(3):
        ry, rx = ref.apply_A(x[b]), ref.apply_AH(y[b])
        assert rel_err(yb[b], ry) <= tol
        assert rel_err(xb[b], rx) <= tol
        assert np.abs(yb[b] - ry).max() <= tol_el * np.abs(ry).max()
        assert np.abs(xb[b] - rx).max() <= tol_el * np.abs(rx).max()
    assert rel_err(to_host(op.apply_A(to_dev(x[0]))), yb[0]) <= 1e-6
    assert rel_err(to_host(op.apply_AH(to_dev(y[0]))), xb[0]) <= 1e-6


@pytest.mark.parametrize("mode", list(P128_TOL))
def test_vol64_full_size_sampled_outputs(sfs, mode):
    """The 64 x 64 x 256 workload (Nt = 1024, M = 128, 128 x 128 planes) at
    full size: 24 sampled entries of A x against rows of the dense
    definition (Eq. (4)), 16 sampled voxels of A^H y against its columns,
    within the mode's norm-wise bar."""
    w = synth.WORKLOADS["vol64"]
    params = synth.geometry_params("vol64")
    go = oracle_geometry(params)
    idx = O.select_indices(go, O.SEL_RANDOM, w["M"], True, 1002)
    g = sfs.Geometry(**params)
    op = sfs.Operator.from_indices(g, idx, precision=sfs.PRECISION_NAMES[mode])
    rng = np.random.default_rng(33)
    x = synth.scene((g.Nz, g.Ny, g.Nx), None, "uniform", seed=5, p_bernoulli=1e-4)
    x = x + 0.01 * crandn(rng, g.Nz, g.Ny, g.Nx)
    y = crandn(rng, g.S, w["M"])
    ya = to_host(op.apply_A(to_dev(x))).ravel()
    xa = to_host(op.apply_AH(to_dev(y))).ravel()
    tol, tol_el = P128_TOL[mode]
    rows = rng.choice(g.S * w["M"], 24, replace=False)
    ref_y = np.concatenate([O.A_rows(go, idx, rows[i:i + 6]) @ x.ravel() for i in range(0, 24, 6)])
    vox = rng.choice(g.V, 16, replace=False)
    ref_x = O.A_cols(go, idx, vox).conj().T @ y.ravel()
    # norm-wise on the sampled entries against the dense definition (the
    # element-wise bound, normalised by the oracle's largest entry, is in
    # test_gpu_fullsize.py with the whole applies)
    assert rel_err(ya[rows], ref_y) <= tol
    assert rel_err(xa[vox], ref_x) <= tol


@pytest.mark.parametrize("mode", ["fp32", "fp16"])
def test_128_point_batched_fista(sfs, mode):
    """FISTA on 128 x 128 planes (one 4-CTA cluster per plane in the
    residual and update kernels), three scenes in one batched call: each
    equals its single-scene solve, and the FP64 FISTA within 1e-4 (FP32) or
    4e-3 (FP16 contractions, u = 2^-11 per apply)."""
    params = geom_params(Nx=40, Ny=36, Nz=10, dz=0.15e-3, Nt=256)
    go = oracle_geometry(params)
    idx = O.select_indices(go, O.SEL_RANDOM, 10, True, 41)
    g = sfs.Geometry(**params)
    op = sfs.Operator.from_indices(g, idx, precision=sfs.PRECISION_NAMES[mode])
    ref = O.LateralFFTOperator(go, idx)
    L, _ = O.power_iteration(ref.apply_A, ref.apply_AH, op.shape_x, 1, max_iter=400, rtol=1e-10)
    L *= 1.001
    ys = []
    for b in range(3):
        xt = synth.scene(op.shape_x, 4, "uniform", seed=42 + b)
        y0 = ref.apply_A(xt)
        sig = synth.noise_scale(float(np.vdot(y0, y0).real), y0.size, 20.0)
        ys.append((y0 + sig * synth.unit_noise(y0.shape, seed=45 + b)).astype(np.complex64).astype(complex))
    lam = O.lambda_from_mu(ref.apply_AH, ys[0], 0.05)
    xb = to_host(op.fista_batched(to_dev(np.stack(ys)), lam, L, 60))
    for b in range(3):
        xs = to_host(op.fista(to_dev(ys[b]), lam, L, 60))
        x_ref = O.fista(ref.apply_A, ref.apply_AH, ys[b], lam, L, 60)
        assert rel_err(xb[b], xs) <= 1e-6
        assert rel_err(xb[b], x_ref) <= (1e-4 if mode == "fp32" else 4e-3)
