"""GPU parity of the reduced- and split-precision depth contractions.

Each precision mode (include/sfs.h, sfs_precision) is compared with the FP64
oracle at a tolerance derived from the arithmetic of its stored table:

  * TF32X3: table and spectra split into TF32 hi + lo, three products; FP32-
    level, so the FP32 bars hold: A, A^H <= 1e-5, FISTA(200) <= 1e-4.
  * BF16: every real table component is the BF16 rounding of the FP32 value,
    relative error <= u = 2^-8; the spectra are split into BF16 hi + lo
    (<= 2^-16) and products accumulate in FP32.  An output is a sum of such
    products with independent rounding errors, so its relative 2-norm error
    stays below u: the bar is u (2-norm) and 8u of the largest entry
    (element-wise).
  * BF16X2: table stored as BF16 hi + lo (remainder rounded again), relative
    error <= 2^-16 per component, spectra alike; the bar is 4 * 2^-16 in norm.
  * FP16: as BF16 with u = 2^-11 (11 significant bits).  Both operands are
    scaled by powers of two into FP16's range, which is exact, so the bars
    are u and 8u whatever the scale of the input; FP16X2 (table hi + lo,
    about 2^-22) is held to the FP32 bars.
"""
import numpy as np
import pytest

import oracle as O
import synth
from tests._common import crandn, ensure_built, geom_params, oracle_geometry, rel_err

pytestmark = pytest.mark.gpu

U_BF16 = 2.0 ** -8
U_FP16 = 2.0 ** -11
TOL = {
    "tf32x3": (1e-5, 1e-4),
    "bf16": (U_BF16, 8 * U_BF16),
    "bf16x2": (4 * 2.0 ** -16, 4e-4),
    "fp16": (U_FP16, 8 * U_FP16),
    "fp16x2": (1e-5, 1e-4),
}
MODES = list(TOL)


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


def make_pair(sfs, params, mode, M=8, seed=7, strategy=O.SEL_RANDOM, per_position=True):
    go = oracle_geometry(params)
    idx = O.select_indices(go, strategy, M, per_position, seed)
    g = sfs.Geometry(**params)
    op = sfs.Operator.from_indices(g, idx, precision=sfs.PRECISION_NAMES[mode])
    assert op.info["precision"] == sfs.PRECISION_NAMES[mode]
    return g, op, go, idx


# line scans and area scans; ragged depth counts (not multiples of 32), bin
# unions beyond one tile of 64 and of 128, a single A-scan, one depth
CASES = [
    (32, 1, 64, 256, 32),
    (12, 10, 20, 128, 12),
    (7, 1, 5, 64, 3),
    (1, 1, 9, 64, 4),
    (16, 16, 33, 256, 10),
    (5, 3, 1, 128, 1),
    (8, 8, 70, 512, 40),     # U > 128 bins: two bin tiles forward, three chunks adjoint
]


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("case", CASES)
def test_precision_apply_matches_dense_oracle(sfs, mode, case):
    Nx, Ny, Nz, Nt, M = case
    params = geom_params(Nx=Nx, Ny=Ny, Nz=Nz, dz=0.15e-3, Nt=Nt)
    g, op, go, idx = make_pair(sfs, params, mode, M=M)
    A = O.dense_A(go, idx)
    rng = np.random.default_rng(11)
    x = crandn(rng, Nz, Ny, Nx)
    y = crandn(rng, g.S, M)
    ya = to_host(op.apply_A(to_dev(x)))
    xa = to_host(op.apply_AH(to_dev(y)))
    ref_y = (A @ x.ravel()).reshape(g.S, M)
    ref_x = (A.conj().T @ y.ravel()).reshape(Nz, Ny, Nx)
    tol, tol_el = TOL[mode]
    assert rel_err(ya, ref_y) <= tol
    assert rel_err(xa, ref_x) <= tol
    assert np.abs(ya - ref_y).max() <= tol_el * np.abs(ref_y).max()
    assert np.abs(xa - ref_x).max() <= tol_el * np.abs(ref_x).max()


@pytest.mark.parametrize("mode", MODES)
def test_precision_vol32_full_size(sfs, mode):
    """The 32 x 32 x 128 workload (U = 81) in each mode: whole outputs against
    the FP64 lateral-FFT oracle and 300 sampled rows of A against the dense
    definition; the adjoint identity within the mode's tolerance."""
    w = synth.WORKLOADS["vol32"]
    params = synth.geometry_params("vol32")
    g, op, go, idx = make_pair(sfs, params, mode, M=w["M"], seed=1001)
    assert op.info["U"] == 81
    rng = np.random.default_rng(2)
    x = synth.scene((g.Nz, g.Ny, g.Nx), 40, "uniform", seed=4) + 0.01 * crandn(rng, g.Nz, g.Ny, g.Nx)
    y = crandn(rng, g.S, w["M"])
    ya = to_host(op.apply_A(to_dev(x)))
    xa = to_host(op.apply_AH(to_dev(y)))
    ref = O.LateralFFTOperator(go, idx)
    tol, _ = TOL[mode]
    assert rel_err(ya, ref.apply_A(x)) <= tol
    assert rel_err(xa, ref.apply_AH(y)) <= tol
    rows = rng.choice(g.S * w["M"], 300, replace=False)
    assert rel_err(ya.ravel()[rows], O.A_rows(go, idx, rows) @ x.ravel()) <= tol
    # adjoint identity: a wrong conjugate, sign or index breaks it by O(1)
    lhs = np.vdot(y, ya)
    rhs = np.vdot(xa, x)
    scale = np.linalg.norm(y) * np.linalg.norm(ya) + np.linalg.norm(xa) * np.linalg.norm(x)
    assert abs(lhs - rhs) <= tol * scale


@pytest.mark.parametrize("case", [
    ("line2d", dict(), 32, 3, 200),
    ("small3d", dict(Nx=12, Ny=12, Nz=24, dz=0.15e-3, Nt=256), 16, 5, 200),
])
def test_tf32x3_fista_200_iterations_matches_oracle(sfs, case):
    name, over, M, ns, iters = case
    params = synth.geometry_params("line2d") if name == "line2d" else geom_params(**over)
    g, op, go, idx = make_pair(sfs, params, "tf32x3", M=M, seed=101)
    ref = O.LateralFFTOperator(go, idx)
    x_true = synth.scene((g.Nz, g.Ny, g.Nx), ns, "uniform", seed=1)
    y0 = ref.apply_A(x_true)
    sig = synth.noise_scale(float(np.vdot(y0, y0).real), y0.size, 20.0)
    y = (y0 + sig * synth.unit_noise(y0.shape, seed=8)).astype(np.complex64).astype(complex)
    L, _ = O.power_iteration(ref.apply_A, ref.apply_AH, x_true.shape, 1, max_iter=400, rtol=1e-10)
    L *= 1.001
    lam = O.lambda_from_mu(ref.apply_AH, y, 0.05)
    x_ref = O.fista(ref.apply_A, ref.apply_AH, y, lam, L, iters)
    x_gpu = to_host(op.fista(to_dev(y), lam, L, iters))
    assert rel_err(x_gpu, x_ref) <= 1e-4


@pytest.mark.parametrize("mode", ["bf16", "bf16x2", "fp16", "fp16x2"])
def test_reduced_precision_fista_reaches_fp32_nmse(sfs, mode):
    """FISTA with a reduced-precision operator on a noisy 16 x 16 x 40 scene:
    after the same 150 iterations its NMSE against the true scene is within
    0.1 dB of the FP32 operator's (the table's rounding, 2^-8 relative, sits
    far below the 20 dB noise), and its largest magnitudes sit on the same
    voxels.  (The l1 penalty shrinks amplitudes, so the NMSE itself stays a
    few dB below 0.)"""
    params = geom_params(Nx=16, Ny=16, Nz=40, dz=0.15e-3, Nt=256)
    go = oracle_geometry(params)
    idx = O.select_indices(go, O.SEL_RANDOM, 16, True, 21)
    g = sfs.Geometry(**params)
    op32 = sfs.Operator.from_indices(g, idx)
    oph = sfs.Operator.from_indices(g, idx, precision=sfs.PRECISION_NAMES[mode])
    ref = O.LateralFFTOperator(go, idx)
    x_true = synth.scene((g.Nz, g.Ny, g.Nx), 6, "uniform", seed=9)
    y0 = ref.apply_A(x_true)
    sig = synth.noise_scale(float(np.vdot(y0, y0).real), y0.size, 20.0)
    y = (y0 + sig * synth.unit_noise(y0.shape, seed=10)).astype(np.complex64)
    L, _ = op32.lipschitz(max_iter=400, rtol=1e-7, seed=1, safety=1e-3)
    yd = to_dev(y)
    x32 = to_host(op32.fista(yd, -0.05, L, 150))
    xh = to_host(oph.fista(yd, -0.05, L, 150))

    def nmse_db(x):
        return 10 * np.log10(np.linalg.norm(x - x_true) ** 2 / np.linalg.norm(x_true) ** 2)

    assert nmse_db(x32) < -1.0
    assert abs(nmse_db(xh) - nmse_db(x32)) <= 0.1
    # the top magnitudes sit on the same voxels
    top32 = set(np.argsort(np.abs(x32).ravel())[-6:])
    toph = set(np.argsort(np.abs(xh).ravel())[-6:])
    assert top32 == toph


def test_bf16_operator_info_and_table_bytes(sfs):
    params = geom_params(Nx=12, Ny=12, Nz=40, dz=0.15e-3, Nt=256)
    go = oracle_geometry(params)
    idx = O.select_indices(go, O.SEL_RANDOM, 16, True, 3)
    g = sfs.Geometry(**params)
    info = {m: sfs.Operator.from_indices(g, idx, precision=sfs.PRECISION_NAMES[m]).info
            for m in ("fp32", "bf16", "bf16x2", "fp16", "fp16x2")}
    # 16-bit table: No orbits x ceil(Nz / 32) blocks x U rows x 128 B per part
    No = info["bf16"]["Nslot"] // info["bf16"]["GS"]
    assert info["bf16"]["table_bytes"] == No * 2 * info["bf16"]["U"] * 128
    assert info["bf16x2"]["table_bytes"] == 2 * info["bf16"]["table_bytes"]
    assert info["fp16"]["table_bytes"] == info["bf16"]["table_bytes"]
    assert info["fp16x2"]["table_bytes"] == info["bf16x2"]["table_bytes"]
    with pytest.raises(sfs.SfsError):
        sfs.Operator.from_indices(g, idx, precision=17)


@pytest.mark.parametrize("mode", ["bf16", "fp16", "tf32x3"])
def test_16bit_noalloc_adjoint_equals_adjoint(sfs, mode):
    """sfs_apply_AH_noalloc on a tensor-core operator: 16-bit (spectra in the
    static scratch, so the adjoint reads them through a tensor map encoded for
    that array; FP16 also takes its spectra scale from the operator's maxima)
    and TF32X3 (its bulk copies read the scratch directly)."""
    params = geom_params(Nx=12, Ny=10, Nz=36, dz=0.15e-3, Nt=256)
    g, op, go, idx = make_pair(sfs, params, mode, M=12, seed=5)
    import torch
    rng = np.random.default_rng(6)
    y = to_dev(crandn(rng, g.S, 12))
    a = to_host(op.apply_AH(y))
    xb = torch.empty(op.shape_x, dtype=torch.complex64, device="cuda")
    sfs.sfs_apply_AH_noalloc(op.handle, y.data_ptr(), xb.data_ptr(),
                             torch.cuda.current_stream().cuda_stream)
    assert np.array_equal(a, to_host(xb))


@pytest.mark.parametrize("mode", ["fp16", "fp16x2", "bf16"])
def test_16bit_results_scale_with_the_input(sfs, mode):
    """The spectra scale is a power of two taken from the data, so scaling the
    input by 2^k scales A x and A^H y by exactly 2^k (bit for bit) while FP16
    alone spans only 2^-24 .. 2^16; inputs near 1e-25 and 1e25 stay within
    the mode's tolerance of the oracle.  (Scales stay where no FP32 value of
    the chain over- or underflows, so that the FP32 FFTs scale exactly too.)"""
    params = geom_params(Nx=12, Ny=10, Nz=36, dz=0.15e-3, Nt=256)
    g, op, go, idx = make_pair(sfs, params, mode, M=12, seed=13)
    A = O.dense_A(go, idx)
    rng = np.random.default_rng(14)
    x = crandn(rng, g.Nz, g.Ny, g.Nx)
    y = crandn(rng, g.S, 12)
    ya = to_host(op.apply_A(to_dev(x)))
    xa = to_host(op.apply_AH(to_dev(y)))
    for k in (-60, -30, 30, 60):
        c = 2.0 ** k
        assert np.array_equal(to_host(op.apply_A(to_dev(x * c))), ya * c)
        assert np.array_equal(to_host(op.apply_AH(to_dev(y * c))), xa * c)
    tol, _ = TOL[mode]
    for c in (1e-25, 1e25):
        yc = to_host(op.apply_A(to_dev(x * c)))
        xc = to_host(op.apply_AH(to_dev(y * c)))
        assert rel_err(yc, A @ (x * c).ravel()) <= tol
        assert rel_err(xc, A.conj().T @ (y * c).ravel()) <= tol


@pytest.mark.parametrize("mode", ["fp16", "fp16x2"])
def test_fp16_batched_scenes_take_their_own_scale(sfs, mode):
    """Five scenes 10^-12 .. 10^12 apart in one batched call (one contraction
    launch serves four of them): each scene within the tolerance of the
    oracle, which a scale shared by the group would break for all but the
    largest scene."""
    params = geom_params(Nx=10, Ny=8, Nz=40, dz=0.15e-3, Nt=256)
    g, op, go, idx = make_pair(sfs, params, mode, M=10, seed=15)
    A = O.dense_A(go, idx)
    rng = np.random.default_rng(16)
    scales = np.array([1e-12, 1e-6, 1.0, 1e6, 1e12])
    x = crandn(rng, 5, g.Nz, g.Ny, g.Nx) * scales[:, None, None, None]
    y = crandn(rng, 5, g.S, 10) * scales[:, None, None]
    yb = to_host(op.apply_A_batched(to_dev(x)))
    xb = to_host(op.apply_AH_batched(to_dev(y)))
    tol, _ = TOL[mode]
    for b in range(5):
        assert rel_err(yb[b], A @ x[b].ravel()) <= tol
        assert rel_err(xb[b], A.conj().T @ y[b].ravel()) <= tol
