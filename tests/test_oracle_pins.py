"""Pins of the FP64 oracle to facts other than itself (CPU only).

Each test fixes one part of the oracle by something the paper or the
mathematics determines independently: a worked example printed in the paper,
a brute-force time-domain simulation, a numerical Fourier integral, a library
SVD, optimality conditions, or structural identities.
"""
import math
import os

import numpy as np
import pytest

import oracle as O
import synth

HERE = os.path.dirname(os.path.abspath(__file__))


def small_geom(Nx=5, Ny=4, Nz=6, Nt=64, theta=0.0, dz=0.15e-3):
    return O.Geometry(Nx=Nx, Ny=Ny, dx=0.5e-3, dy=0.5e-3, Nz=Nz, z0=10e-3,
                      dz=dz, c=5900.0, fs=40e6, Nt=Nt, fc=5e6, frac_bw=0.7,
                      theta=theta)


def crandn(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


# ---------------------------------------------------------------- pulse ---

def test_pulse_spectrum_is_fourier_integral_of_pulse():
    """H(f) against a trapezoid Fourier integral of h(t) (Sec. VI pulse)."""
    fc, alpha = 5e6, O.pulse_alpha(5e6, 0.7)
    t = np.linspace(-12.0 / alpha, 12.0 / alpha, 200001)
    h = O.pulse_time(t, fc, alpha)
    for f in (0.0, 2e6, 4.1e6, 5e6, 6.3e6, 9e6):
        num = np.trapezoid(h * np.exp(-2j * np.pi * f * t), t)
        ref = O.pulse_spectrum(f, fc, alpha)
        assert abs(num - ref) <= 1e-9 * abs(O.pulse_spectrum(fc, fc, alpha))


def test_pulse_alpha_gives_requested_bandwidth():
    """|H| falls to one half at fc +- 0.35 fc for 70 % fractional bandwidth."""
    fc = 5e6
    alpha = O.pulse_alpha(fc, 0.7)
    peak = O.pulse_spectrum(fc, fc, alpha)
    for f in (fc - 0.35 * fc, fc + 0.35 * fc):
        assert O.pulse_spectrum(f, fc, alpha) / peak == pytest.approx(0.5, rel=1e-12)


# ----------------------------------------------------------------- band ---

@pytest.mark.parametrize("name", ["line2d", "vol32", "vol64"])
def test_band_matches_closed_form_width(name):
    """Bins with |H(f_k)| >= 10^(-b/20) peak lie within (alpha/pi)
    sqrt(b ln10 / 20) of fc; count them from that closed form."""
    w = synth.WORKLOADS[name]
    g = O.Geometry(**synth.geometry_params(name))
    k_lo, k_hi, b = O.candidate_band(g, w["M"])
    # first rung whose band holds M bins
    kstar_peak = round(g.fc * g.Nt / g.fs)
    for rung in O.BAND_LADDER_DB:
        half = g.alpha / math.pi * math.sqrt(rung * math.log(10) / 20.0)
        ks = [k for k in range(g.Nt // 2 + 1)
              if abs(k * g.fs / g.Nt - g.fc) <= half]
        if len(ks) >= w["M"]:
            assert (k_lo, k_hi, b) == (ks[0], ks[-1], rung)
            break
    assert k_lo <= kstar_peak <= k_hi
    assert k_hi - k_lo + 1 >= w["M"]


def test_band_sizes_of_workloads():
    """The reading that widens the band to 20 dB gives |C| = 41/81/163."""
    sizes = []
    for name in ("line2d", "vol32", "vol64"):
        g = O.Geometry(**synth.geometry_params(name))
        k_lo, k_hi, b = O.candidate_band(g, synth.WORKLOADS[name]["M"])
        sizes.append((k_hi - k_lo + 1, b))
    assert sizes == [(41, 20.0), (81, 20.0), (163, 20.0)]


# ------------------------------------------------------------ selection ---

def test_selection_invariants():
    g = small_geom(Nx=6, Ny=5, Nt=256)
    M = 9
    k_lo, k_hi, _ = O.candidate_band(g, M)
    for strat in (O.SEL_RANDOM, O.SEL_CONTIGUOUS, O.SEL_EQUISPACED):
        for per in (True, False):
            idx = O.select_indices(g, strat, M, per, seed=42)
            assert idx.shape == (g.S, M) and idx.dtype == np.int32
            assert np.all(np.diff(idx, axis=1) > 0)          # distinct, ascending
            assert idx.min() >= k_lo and idx.max() <= k_hi
            if strat != O.SEL_RANDOM or not per:
                assert np.all(idx == idx[0])                  # shared set


def test_contiguous_is_centred_on_peak_and_equispaced_spread():
    g = small_geom(Nt=512)
    M = 16
    k_lo, k_hi, _ = O.candidate_band(g, M)
    c = O.select_indices(g, O.SEL_CONTIGUOUS, M, False, 0)[0]
    peak = int(np.argmax(O.pulse_spectrum(g.bin_freq(np.arange(257)), g.fc, g.alpha)))
    assert np.all(np.diff(c) == 1) and c[0] <= peak <= c[-1]
    assert abs((c[0] + c[-1]) / 2 - peak) <= 0.5
    e = O.select_indices(g, O.SEL_EQUISPACED, M, False, 0)[0]
    gaps = np.diff(e)
    assert gaps.max() - gaps.min() <= 1                       # even spacing
    # the M points cut C into M cells of nearly equal size, one point each
    n = k_hi - k_lo + 1
    cells = ((e - k_lo) * M) // n
    assert np.array_equal(cells, np.arange(M))


def test_maximal_set_holds_the_largest_pulse_magnitudes():
    """Phi_max (Sec. III-A): the M bins with the largest |H(f_k)| of the
    pinned pulse spectrum (ties to the lower bin), shared by all positions."""
    g = small_geom(Nx=4, Ny=3, Nt=512)
    k = np.arange(g.Nt // 2 + 1)
    mag = np.abs(O.pulse_spectrum(g.bin_freq(k), g.fc, g.alpha))
    for M in (1, 2, 9, 40):
        idx = O.select_indices(g, O.SEL_MAXIMAL, M, True, 3)
        assert np.all(idx == idx[0])
        ref = np.sort(np.lexsort((k, -mag))[:M])
        assert np.array_equal(idx[0], ref)
        # a contiguous run around the peak bin fc Nt / fs = 64
        assert np.all(np.diff(idx[0]) == 1) and idx[0][0] <= 64 <= idx[0][-1]


def test_energy_draw_follows_the_pulse_energy():
    """Phi_nrg (Sec. III-A): a single draw picks bin k with probability
    q_k = |H(f_k)| / sum |H| (chi-square over 20000 streams, p > 1e-4);
    larger draws are distinct, ascending, reproducible per seed and vary per
    position (Phi_nrg,f)."""
    from scipy.stats import chi2
    g = small_geom(Nx=5, Ny=4, Nt=64)
    e, w = O.pulse_weights(g)
    k = np.arange(g.Nt // 2 + 1)
    q = np.abs(O.pulse_spectrum(g.bin_freq(k), g.fc, g.alpha))
    q = q / q.sum()
    T = 20000
    counts = np.zeros(len(k))
    for t in range(T):
        counts[O.energy_subset(w, 1, O.SplitMix64(t * 7919 + 1))[0]] += 1
    expect = T * q
    keep = expect >= 5
    stat = float((((counts - expect) ** 2) / expect)[keep].sum()) + float(
        ((counts[~keep].sum() - expect[~keep].sum()) ** 2) / max(expect[~keep].sum(), 1e-9))
    assert chi2.sf(stat, keep.sum()) > 1e-4
    a = O.select_indices(g, O.SEL_ENERGY, 6, True, 11)
    assert np.all(np.diff(a, axis=1) > 0)
    assert np.array_equal(a, O.select_indices(g, O.SEL_ENERGY, 6, True, 11))
    assert len({tuple(r) for r in a}) > g.S // 2
    b = O.select_indices(g, O.SEL_ENERGY, 6, False, 11)
    assert np.all(b == b[0])
    assert all(w[i] > 0 for i in a.ravel())


def test_random_selection_reproducible_and_position_dependent():
    g = small_geom(Nx=8, Ny=8, Nt=256)
    a = O.select_indices(g, O.SEL_RANDOM, 8, True, 7)
    b = O.select_indices(g, O.SEL_RANDOM, 8, True, 7)
    c = O.select_indices(g, O.SEL_RANDOM, 8, True, 8)
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    assert len({tuple(r) for r in a}) > g.S // 2


def test_random_subset_uniform_chi_square():
    """Marginal and pairwise inclusion frequencies of the M-subset draw over
    20000 streams match the uniform-subset values (chi-square, p > 1e-4)."""
    from scipy.stats import chi2
    n, M, T = 12, 4, 20000
    counts = np.zeros(n)
    pairs = np.zeros((n, n))
    for s in range(T):
        sub = O.random_subset(n, M, O.SplitMix64(12345 ^ ((s * 0x9E3779B97F4A7C15) % 2**64)))
        counts[sub] += 1
        for i in sub:
            for j in sub:
                if i < j:
                    pairs[i, j] += 1
    e1 = T * M / n
    stat1 = ((counts - e1) ** 2 / e1).sum()
    assert chi2.sf(stat1, n - 1) > 1e-4
    e2 = T * M * (M - 1) / (n * (n - 1))
    iu = np.triu_indices(n, 1)
    stat2 = ((pairs[iu] - e2) ** 2 / e2).sum()
    assert chi2.sf(stat2, len(iu[0]) - 1) > 1e-4


# ------------------------------------------------------- dense operator ---

@pytest.mark.parametrize("name", ["line2d", "vol32", "vol64"])
def test_time_gate_holds_every_echo(name):
    """Time-gate reading (t0 is not given for the workloads): t0 lies on the
    sample grid, at least three envelope widths 1/alpha before the earliest
    echo (the closest voxel straight below a transducer) and within one sample
    of that bound; the window t0 .. t0 + Nt/fs reaches three widths past the
    latest echo (the deepest voxel at the far corner), so no echo wraps."""
    g = O.Geometry(**synth.geometry_params(name))
    n0 = g.t0 * g.fs
    assert abs(n0 - round(n0)) <= 1e-6
    first = 2.0 * g.z0 / g.c - 3.0 / g.alpha
    assert first - 1.0 / g.fs < g.t0 <= first
    zmax = g.z0 + (g.Nz - 1) * g.dz
    last = O.time_of_flight(0.0, 0.0, (g.Nx - 1) * g.dx, (g.Ny - 1) * g.dy, zmax, g.c) + 3.0 / g.alpha
    assert g.t0 + g.Nt / g.fs >= last


def test_dense_A_equals_dft_of_time_domain_echo():
    """A x at the kept bins equals the direct DFT of the brute-force simulated
    A-scan of Eq. (2) (periodically folded), for random scatterers."""
    g = small_geom(Nx=4, Ny=3, Nz=10, Nt=128)
    rng = np.random.default_rng(3)
    idx = O.select_indices(g, O.SEL_RANDOM, 12, True, 5)
    xv, yv, zv = g.voxel_xyz()
    vs = rng.choice(g.V, 6, replace=False)
    amps = crandn(rng, 6)
    x = np.zeros(g.V, complex)
    x[vs] = amps
    y = O.dense_A(g, idx) @ x
    for s in range(g.S):
        b = O.time_domain_ascan(g, s, xv[vs], yv[vs], zv[vs], amps)
        ref = O.dft_bins(b, idx[s])
        got = y[s * 12:(s + 1) * 12]
        assert np.linalg.norm(got - ref) <= 1e-10 * np.linalg.norm(ref)


def test_dense_A_with_directivity_equals_time_domain_echo():
    g = small_geom(Nx=4, Ny=3, Nz=10, Nt=128, theta=math.radians(30))
    rng = np.random.default_rng(4)
    idx = O.select_indices(g, O.SEL_RANDOM, 12, True, 6)
    xv, yv, zv = g.voxel_xyz()
    vs = rng.choice(g.V, 5, replace=False)
    amps = crandn(rng, 5)
    x = np.zeros(g.V, complex)
    x[vs] = amps
    y = O.dense_A(g, idx) @ x
    for s in (0, 5, 11):
        b = O.time_domain_ascan(g, s, xv[vs], yv[vs], zv[vs], amps)
        ref = O.dft_bins(b, idx[s])
        assert np.linalg.norm(y[s * 12:(s + 1) * 12] - ref) <= 1e-10 * np.linalg.norm(ref)


def test_directivity_depends_on_the_angle_only():
    """Directivity reading of Sec. VI (the printed form is not dimensionless):
    the characteristic is a function of the angle atan(r / z) between the
    beam axis and the scatterer alone, equal to 1 straight below the
    transducer and to 1/e at the beam half-angle theta, at every depth and
    lateral direction; theta = 0 switches it off.  The echo pins above use
    the same routine on both sides, so this is its independent pin."""
    th = math.radians(25.0)
    for z in (5e-3, 12e-3, 30e-3):
        assert O.directivity(1e-3, 2e-3, 1e-3, 2e-3, z, th) == 1.0
        r = z * math.tan(th)
        for dx, dy in ((r, 0.0), (0.0, -r), (r / math.sqrt(2.0), r / math.sqrt(2.0))):
            assert O.directivity(1e-3 + dx, 2e-3 + dy, 1e-3, 2e-3, z, th) == pytest.approx(math.exp(-1.0), rel=1e-12)
        a = O.directivity(0.3 * z, 0.0, 0.0, 0.0, z, th)
        b = O.directivity(0.6 * z, 0.0, 0.0, 0.0, 2.0 * z, th)
        assert 0.0 < a < 1.0 and a == pytest.approx(b, rel=1e-12)
    assert O.directivity(1e-3, 0.0, 0.0, 0.0, 10e-3, 0.0) == 1.0


def test_A_cols_equal_time_domain_echo_of_one_scatterer():
    """Column v of A is the kept-bin DFT of the simulated echo of a unit
    scatterer at voxel v, at every position (directivity on); the columns
    also equal the dense A's (a swapped voxel index or axis breaks both)."""
    g = small_geom(Nx=4, Ny=3, Nz=6, Nt=128, theta=math.radians(25))
    idx = O.select_indices(g, O.SEL_RANDOM, 7, True, 8)
    xv, yv, zv = g.voxel_xyz()
    vox = np.array([0, 5, 17, 40, g.V - 1])
    C = O.A_cols(g, idx, vox)
    assert C.shape == (g.S * 7, vox.size)
    for j, v in enumerate(vox):
        for s in range(g.S):
            b = O.time_domain_ascan(g, s, xv[[v]], yv[[v]], zv[[v]], np.ones(1))
            ref = O.dft_bins(b, idx[s])
            assert np.linalg.norm(C[s * 7:(s + 1) * 7, j] - ref) <= 1e-10 * np.linalg.norm(ref)
    np.testing.assert_allclose(C, O.dense_A(g, idx)[:, vox], rtol=0, atol=1e-12 * np.abs(C).max())


def test_single_scatterer_below_position_closed_form():
    """A scatterer at depth z straight below the transducer: the echo is the
    pulse delayed by 2z/c, so bin k holds fs H(f_k) e^{-j 2 pi f_k (2z/c - t0)}."""
    g = small_geom(Nx=3, Ny=3, Nz=4, Nt=64)
    idx = O.select_indices(g, O.SEL_CONTIGUOUS, 6, False, 0)
    s, iz = 4, 2
    v = (iz * g.Ny + 1) * g.Nx + 1            # (ix, iy) = (1, 1) = scan pos 4
    col = O.dense_A(g, idx)[s * 6:(s + 1) * 6, v]
    f = g.bin_freq(idx[s])
    z = g.z0 + iz * g.dz
    ref = g.fs * O.pulse_spectrum(f, g.fc, g.alpha) * np.exp(-2j * np.pi * f * (2 * z / g.c - g.t0))
    np.testing.assert_allclose(col, ref, rtol=1e-13)


def test_lateral_shift_invariance():
    """Moving scatterer and transducer together leaves the data unchanged
    (Theorem 2, Sec. IV-B), for a shared bin set."""
    g = small_geom(Nx=5, Ny=4, Nz=3, Nt=64)
    idx = O.select_indices(g, O.SEL_RANDOM, 5, False, 9)
    A = O.dense_A(g, idx).reshape(g.S, 5, g.Nz, g.Ny, g.Nx)
    # s = (iy, ix); shift by (+1, +2)
    for (iy, ix) in [(0, 0), (1, 1), (2, 2)]:
        for (vy, vx) in [(0, 1), (2, 0), (1, 2)]:
            a = A[iy * g.Nx + ix, :, :, vy, vx]
            b = A[(iy + 1) * g.Nx + ix + 2, :, :, vy + 1, vx + 2]
            np.testing.assert_allclose(a, b, rtol=1e-12)


# ------------------------------------------------- Toeplitz structure ---

def test_multilevel_toeplitz_matches_printed_example():
    rows = []
    with open(os.path.join(HERE, "golden", "toeplitz_T22.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            rows.append([tuple(int(v) for v in e.split(",")) for e in line.split()])
    t = np.array([[10 * a + b for b in range(1, 4)] for a in range(1, 4)])
    T = O.multilevel_toeplitz(t, (2, 2))
    expect = np.array([[10 * a + b for (a, b) in r] for r in rows])
    assert np.array_equal(T, expect)


def test_dense_lateral_blocks_are_2level_toeplitz_of_generators():
    """Each (bin, depth) block of A for a shared set is the 2-level Toeplitz
    matrix T_{(Ny,Nx),2}(h_{k,z}) of Sec. IV-B built from the generator."""
    g = small_geom(Nx=4, Ny=3, Nz=3, Nt=64)
    idx = O.select_indices(g, O.SEL_EQUISPACED, 3, False, 0)
    A = O.dense_A(g, idx).reshape(g.S, 3, g.Nz, g.S)     # rows s, bin m, iz, lateral
    for m in range(3):
        for iz in range(g.Nz):
            h = O.lateral_generator(g, int(idx[0, m]), iz)
            T = O.multilevel_toeplitz(h, (g.Ny, g.Nx))
            np.testing.assert_allclose(A[:, m, iz, :], T, rtol=1e-12, atol=0)


# ------------------------------------------------- fast transform ---

@pytest.mark.parametrize("shape", [(7, 1, 9), (5, 4, 6), (6, 6, 5)])
@pytest.mark.parametrize("strategy", [O.SEL_RANDOM, O.SEL_CONTIGUOUS])
def test_lateral_fft_operator_equals_dense(shape, strategy):
    Nx, Ny, Nz = shape
    g = small_geom(Nx=Nx, Ny=Ny, Nz=Nz, Nt=128)
    idx = O.select_indices(g, strategy, 7, True, 11)
    A = O.dense_A(g, idx)
    op = O.LateralFFTOperator(g, idx)
    rng = np.random.default_rng(1)
    x = crandn(rng, g.V)
    y = crandn(rng, g.S * 7)
    ya = A @ x
    np.testing.assert_allclose(op.apply_A(x).ravel(), ya, rtol=0,
                               atol=1e-12 * np.abs(ya).max())
    xa = A.conj().T @ y
    np.testing.assert_allclose(op.apply_AH(y).ravel(), xa, rtol=0,
                               atol=1e-12 * np.abs(xa).max())


def test_adjoint_identity_structured():
    g = small_geom(Nx=8, Ny=7, Nz=9, Nt=256)
    idx = O.select_indices(g, O.SEL_RANDOM, 10, True, 3)
    op = O.LateralFFTOperator(g, idx)
    rng = np.random.default_rng(2)
    x = crandn(rng, g.Nz, g.Ny, g.Nx)
    y = crandn(rng, g.S, 10)
    lhs = np.vdot(y, op.apply_A(x))
    rhs = np.vdot(op.apply_AH(y), x)
    assert abs(lhs - rhs) <= 1e-13 * abs(lhs)


# ------------------------------------------------------- Lipschitz ---

def test_power_iteration_matches_svd_and_frobenius_bounds():
    g = small_geom(Nx=4, Ny=4, Nz=8, Nt=32)
    M = 3
    idx = O.select_indices(g, O.SEL_RANDOM, M, True, 21)
    A = O.dense_A(g, idx)
    smax2 = np.linalg.svd(A, compute_uv=False)[0] ** 2
    op = O.LateralFFTOperator(g, idx)
    est, it = O.power_iteration(op.apply_A, op.apply_AH, (g.Nz, g.Ny, g.Nx), 5,
                                max_iter=5000, rtol=1e-14)
    assert est == pytest.approx(smax2, rel=1e-9)
    fro2 = np.linalg.norm(A) ** 2
    assert fro2 / min(A.shape) <= smax2 <= fro2


# ----------------------------------------------------------- FISTA ---

def _small_problem(seed=0, M=8, Nz=10):
    g = small_geom(Nx=6, Ny=5, Nz=Nz, Nt=128)
    idx = O.select_indices(g, O.SEL_RANDOM, M, True, seed + 1)
    op = O.LateralFFTOperator(g, idx)
    x_true = synth.scene((g.Nz, g.Ny, g.Nx), 3, "uniform", seed=seed)
    y = op.apply_A(x_true)
    L, _ = O.power_iteration(op.apply_A, op.apply_AH, (g.Nz, g.Ny, g.Nx), 3,
                             max_iter=3000, rtol=1e-13)
    return g, op, x_true, y, L


def test_fista_zero_when_lambda_at_least_max_correlation():
    g, op, x_true, y, L = _small_problem()
    lam = float(np.abs(op.apply_AH(y)).max()) * 1.000001
    x = O.fista(op.apply_A, op.apply_AH, y, lam, L * 1.001, 20)
    assert np.all(x == 0)
    x = O.fista(op.apply_A, op.apply_AH, y, lam * 0.9, L * 1.001, 20)
    assert np.any(x != 0)


def test_fista_reaches_lasso_kkt_point():
    """After many iterations the iterate satisfies the LASSO optimality
    conditions of 1/2||Ax-y||^2 + lam||x||_1: on the support
    A^H(Ax-y) = -lam x/|x|, elsewhere |A^H(Ax-y)| <= lam."""
    g, op, x_true, y, L = _small_problem(seed=4)
    rng = np.random.default_rng(9)
    y = y + 0.02 * np.abs(y).max() * crandn(rng, *y.shape)
    lam = 0.1 * float(np.abs(op.apply_AH(y)).max())
    x = O.fista(op.apply_A, op.apply_AH, y, lam, L * 1.001, 6000)
    grad = op.apply_AH(op.apply_A(x) - y)
    on = np.abs(x) > 0
    assert on.any()
    # first-order method: 6000 iterations reach the optimum to ~1e-4 lam;
    # a step or threshold off by a factor 2 misses it by O(lam)
    np.testing.assert_allclose(grad[on], -lam * x[on] / np.abs(x[on]), atol=1e-3 * lam)
    assert np.abs(grad[~on]).max() <= lam * (1 + 1e-3)


def test_fista_rate_bound():
    """F(x_k) - F* <= 2 L ||x_0 - x*||^2 / (k+1)^2 (Beck-Teboulle)."""
    g, op, x_true, y, L = _small_problem(seed=5)
    lam = 0.05 * float(np.abs(op.apply_AH(y)).max())
    Lf = L * 1.001
    x_star = O.fista(op.apply_A, op.apply_AH, y, lam, Lf, 8000)
    F_star = O.lasso_objective(op.apply_A, y, lam, x_star)
    hist = []
    O.fista(op.apply_A, op.apply_AH, y, lam, Lf, 60, history=hist)
    r0 = float(np.vdot(x_star, x_star).real)
    for k, Fk in enumerate(hist, start=1):
        assert Fk - F_star <= 2 * Lf * r0 / (k + 1) ** 2 + 1e-9 * abs(F_star)


def test_fista_recovers_isolated_scatterers_noiseless():
    """Noiseless data of isolated scatterers (>= 4 voxels apart), small mu:
    the D largest magnitudes sit exactly on the true positions."""
    g = small_geom(Nx=10, Ny=10, Nz=16, Nt=256)
    idx = O.select_indices(g, O.SEL_RANDOM, 16, True, 77)
    op = O.LateralFFTOperator(g, idx)
    x_true = synth.scene((g.Nz, g.Ny, g.Nx), 4, "unit", seed=13, min_sep=4)
    y = op.apply_A(x_true)
    L, _ = O.power_iteration(op.apply_A, op.apply_AH, x_true.shape, 1,
                             max_iter=2000, rtol=1e-12)
    lam = O.lambda_from_mu(op.apply_AH, y, 0.02)
    x = O.fista(op.apply_A, op.apply_AH, y, lam, L * 1.001, 400)
    top = np.argsort(np.abs(x).ravel())[-4:]
    assert set(top.tolist()) == set(np.nonzero(x_true.ravel())[0].tolist())


def test_soft_threshold_special_cases():
    z = np.array([0, 3 + 4j, 0.5j, -2.0])
    out = O.soft_threshold(z, 1.0)
    np.testing.assert_allclose(out, [0, (3 + 4j) * 0.8, 0, -1.0], atol=1e-15)
    beta, _ = O.fista_momentum(4)
    assert beta[0] == 0.0 and np.all(np.diff(beta) > 0)


# -------------------------------------------------- FISTA with backtracking ---

def test_backtracking_without_backtracks_is_fista():
    """L0 at or above ||A||^2: f is L0-smooth, so every first trial is
    accepted and the iterates are FISTA's with L = L0, bit for bit."""
    g, op, x_true, y, L = _small_problem(seed=6)
    lam = 0.05 * float(np.abs(op.apply_AH(y)).max())
    hist = []
    xb = O.fista_backtracking(op.apply_A, op.apply_AH, y, lam, L * 1.5, 2.0, 40, L_history=hist)
    xf = O.fista(op.apply_A, op.apply_AH, y, lam, L * 1.5, 40)
    assert hist == [L * 1.5] * 40
    assert np.array_equal(xb, xf)


def test_backtracking_step_bounds_and_rate():
    """From a crude lower bound: L_k never falls, never exceeds eta ||A||^2,
    and F(x_k) - F* <= 2 eta ||A||^2 ||x*||^2 / (k+1)^2 (Beck-Teboulle's
    bound for the backtracking variant)."""
    g, op, x_true, y, L = _small_problem(seed=7)
    lam = 0.05 * float(np.abs(op.apply_AH(y)).max())
    eta = 1.7
    hist = []
    O.fista_backtracking(op.apply_A, op.apply_AH, y, lam, L / 500.0, eta, 80, L_history=hist)
    assert hist[0] > L / 500.0                     # it did backtrack
    assert all(b >= a for a, b in zip(hist, hist[1:]))
    assert max(hist) <= eta * L * (1 + 1e-9)
    x_star = O.fista(op.apply_A, op.apply_AH, y, lam, L * 1.001, 8000)
    F_star = O.lasso_objective(op.apply_A, y, lam, x_star)
    r0 = float(np.vdot(x_star, x_star).real)
    for k in (10, 40, 80):
        xk = O.fista_backtracking(op.apply_A, op.apply_AH, y, lam, L / 500.0, eta, k)
        Fk = O.lasso_objective(op.apply_A, y, lam, xk)
        assert Fk - F_star <= 2 * eta * L * r0 / (k + 1) ** 2 + 1e-9 * abs(F_star)


def _golden_splitmix():
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "splitmix64_seed1234567.txt")
    return [int(l) for l in open(path) if l.strip() and not l.startswith("#")]


def test_splitmix64_matches_published_outputs():
    """The oracle's generator reproduces the published first outputs from
    state 1234567, and its increment is the odd integer floor(2^64 / phi)
    (the golden-ratio gamma of SplitMix64), computed here in exact integers."""
    gold = _golden_splitmix()
    s = O.SplitMix64(1234567)
    assert [s.next() for _ in gold] == gold
    gamma = (math.isqrt(5 << 128) - (1 << 64)) // 2       # floor(2^64 (sqrt(5) - 1) / 2)
    assert gamma == O.sfs_oracle._GOLDEN and gamma % 2 == 1


def test_fista_resumed_from_its_state_equals_one_run():
    """The iteration state (gamma_{K+1}, x_K, t_{K+1}) carries Algorithm 1
    across calls: 17 + 13 resumed iterations equal 30 in one run exactly,
    and restarting the momentum at t = 1 instead (a warm start from x_K)
    does not."""
    g = O.Geometry(Nx=4, Ny=4, dx=0.5e-3, dy=0.5e-3, Nz=6, z0=10e-3, dz=0.15e-3, c=5900.0,
                   fs=40e6, Nt=64, fc=5e6, frac_bw=0.7, theta=0.0)
    idx = O.select_indices(g, O.SEL_RANDOM, 6, True, 3)
    op = O.LateralFFTOperator(g, idx)
    x_true = synth.scene((g.Nz, g.Ny, g.Nx), 3, "uniform", seed=4)
    y = op.apply_A(x_true)
    L = O.power_iteration(op.apply_A, op.apply_AH, x_true.shape, 1, max_iter=400, rtol=1e-12)[0] * 1.001
    lam = 0.05 * np.abs(op.apply_AH(y)).max()
    x30 = O.fista(op.apply_A, op.apply_AH, y, lam, L, 30)
    x17, st = O.fista(op.apply_A, op.apply_AH, y, lam, L, 17, return_state=True)
    assert st[2] > 1.0 and np.array_equal(st[1], x17)
    x_res = O.fista(op.apply_A, op.apply_AH, y, lam, L, 13, resume=st)
    assert np.array_equal(x_res, x30)
    x_warm = O.fista(op.apply_A, op.apply_AH, y, lam, L, 13, x0=x17)
    assert np.linalg.norm(x_warm - x30) > 1e-6 * np.linalg.norm(x30)
