"""Pins of the Rademacher-mixing oracle (oracle/mixing_oracle.py; Phi_s =
S_s F Sigma_s, Sec. II-B and III-A)."""
import numpy as np

import oracle as O
from oracle import mixing_oracle as X
import synth


def geom(Nx=5, Ny=4, Nz=6, Nt=128):
    return O.Geometry(Nx=Nx, Ny=Ny, dx=0.5e-3, dy=0.5e-3, Nz=Nz, z0=10e-3, dz=0.15e-3,
                      c=5900.0, fs=40e6, Nt=Nt, fc=5e6, frac_bw=0.7, theta=0.0)


def band_of(g, M):
    lo, hi, _ = O.candidate_band(g, M)
    return np.arange(lo, hi + 1)


def crandn(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def test_mixing_matrix_is_the_time_domain_definition():
    """Inverse DFT, sign flips, DFT and selection (numpy's own transforms)
    against the spectral mixing matrix, for random xi and band data."""
    rng = np.random.default_rng(1)
    for Nt in (64, 128, 96):
        band = np.arange(Nt // 8, Nt // 3)
        kept = np.sort(rng.choice(np.arange(Nt // 2 + 1), 9, replace=False))
        xi = synth.rademacher((Nt,), seed=Nt)
        B = crandn(rng, band.size)
        ref = X.mix_time_domain(B, xi, kept, band, Nt)
        np.testing.assert_allclose(X.mixing_matrix(xi, kept, band, Nt) @ B, ref, rtol=1e-12, atol=1e-12)


def test_no_mixing_is_plain_selection():
    """xi = 1: Xi = Nt delta, so the mixed operator is the unmixed one."""
    g = geom()
    idx = O.select_indices(g, O.SEL_RANDOM, 5, True, 2)
    band = band_of(g, 5)
    op = X.MixedOperator(g, band, idx, np.ones((g.S, g.Nt)))
    ref = O.LateralFFTOperator(g, idx)
    rng = np.random.default_rng(3)
    x = crandn(rng, g.Nz, g.Ny, g.Nx)
    y = crandn(rng, g.S, 5)
    np.testing.assert_allclose(op.apply_A(x), ref.apply_A(x), rtol=1e-10, atol=1e-10 * np.abs(ref.apply_A(x)).max())
    np.testing.assert_allclose(op.apply_AH(y), ref.apply_AH(y), rtol=1e-10,
                               atol=1e-10 * np.abs(ref.apply_AH(y)).max())


def test_mixed_operator_equals_dense_and_is_adjoint():
    g = geom()
    idx = O.select_indices(g, O.SEL_RANDOM, 6, True, 4)
    band = band_of(g, 6)
    xi = synth.rademacher((g.S, g.Nt), seed=5)
    op = X.MixedOperator(g, band, idx, xi)
    A = X.dense_A_mixed(g, band, idx, xi)
    rng = np.random.default_rng(6)
    x = crandn(rng, g.Nz, g.Ny, g.Nx)
    y = crandn(rng, g.S, 6)
    ya = op.apply_A(x)
    np.testing.assert_allclose(ya.ravel(), A @ x.ravel(), rtol=1e-10, atol=1e-10 * np.abs(ya).max())
    xa = op.apply_AH(y)
    np.testing.assert_allclose(xa.ravel(), A.conj().T @ y.ravel(), rtol=1e-10, atol=1e-10 * np.abs(xa).max())
    assert abs(np.vdot(y, ya) - np.vdot(xa, x)) <= 1e-10 * np.linalg.norm(y) * np.linalg.norm(ya)
    # mixing spreads the band bins into every kept coefficient
    assert np.count_nonzero(np.abs(op.Mix) > 1e-12) > 0.9 * op.Mix.size


def test_full_mixing_is_unitary():
    """Keeping every bin of an Nt-bin spectrum, F Sigma F^-1 with Sigma^2 = I
    is unitary: the mixing matrix over all bins has orthonormal columns."""
    for Nt in (32, 50):
        xi = synth.rademacher((Nt,), seed=Nt + 1)
        allk = np.arange(Nt)
        Mx = X.mixing_matrix(xi, allk, allk, Nt)
        np.testing.assert_allclose(Mx.conj().T @ Mx, np.eye(Nt), atol=1e-12)
