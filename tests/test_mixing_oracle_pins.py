"""Pins of the Rademacher-mixing oracle (oracle/mixing_oracle.py; Phi_s =
S_s F Sigma_s, Sec. II-B and III-A)."""
import math

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
    op = X.MixedOperator(g, idx, np.ones((g.S, g.Nt)))
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
    xi = synth.rademacher((g.S, g.Nt), seed=5)
    op = X.MixedOperator(g, idx, xi)
    A = X.dense_A_mixed(g, idx, xi)
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


def scatterer_scene(g, n, seed):
    """n distinct voxels with complex amplitudes: (x, voxel coordinates, amps)."""
    rng = np.random.default_rng(seed)
    vox = rng.choice(g.V, n, replace=False)
    amps = rng.uniform(0.5, 1.0, n) * np.exp(2j * np.pi * rng.uniform(size=n))
    x = np.zeros(g.V, dtype=np.complex128)
    x[vox] = amps
    xv, yv, zv = g.voxel_xyz()
    return x.reshape(g.Nz, g.Ny, g.Nx), xv[vox], yv[vox], zv[vox], amps


def literal_chain(g, idx, xi, xv, yv, zv, amps):
    """Eq. (2) echoes sampled on the receive window (periodic fold), times
    xi_s, direct DFT, kept bins: y_s = S_s F Sigma_s b_s term by term."""
    out = np.empty(idx.shape, dtype=np.complex128)
    for s in range(g.S):
        b = O.time_domain_ascan(g, s, xv, yv, zv, amps)
        out[s] = O.dft_bins(xi[s] * b, idx[s])
    return out


def test_mixed_operator_is_the_time_domain_chain():
    """The paper's chain on brute-force A-scans: every bin of the A-scan
    enters each kept coefficient, the bins above Nt/2 as negative
    frequencies.  Agreement to 1e-10 pins the full-spectrum sum (a dropped
    bin range, a wrong sign of the negative frequencies or a transposed
    mixing index would each fail it)."""
    for Nt, M, seed in ((128, 6, 1), (256, 8, 2)):
        g = geom(Nx=5, Ny=4, Nz=6, Nt=Nt)
        idx = O.select_indices(g, O.SEL_RANDOM, M, True, seed)
        xi = synth.rademacher((g.S, g.Nt), seed=seed + 10)
        x, xv, yv, zv, amps = scatterer_scene(g, 4, seed + 20)
        ref = literal_chain(g, idx, xi, xv, yv, zv, amps)
        got = X.MixedOperator(g, idx, xi).apply_A(x)
        assert np.linalg.norm(got - ref) <= 1e-10 * np.linalg.norm(ref)


def test_band_limited_spectrum_is_not_the_model():
    """Mixing only the candidate band's bins (the 20 dB rung of the
    selection) is a different operator: off by more than 1 % on the same
    chain, so the pin above separates the two."""
    g = geom(Nx=5, Ny=4, Nz=6, Nt=128)
    idx = O.select_indices(g, O.SEL_RANDOM, 6, True, 1)
    xi = synth.rademacher((g.S, g.Nt), seed=11)
    x, xv, yv, zv, amps = scatterer_scene(g, 4, 21)
    ref = literal_chain(g, idx, xi, xv, yv, zv, amps)
    cut = X.MixedOperator(g, idx, xi, band=band_of(g, 6)).apply_A(x)
    assert np.linalg.norm(cut - ref) > 1e-2 * np.linalg.norm(ref)


def test_spectrum_truncated_at_140_dB_is_within_1e6():
    """Bins whose pulse magnitude |H(f_k)| lies more than 140 dB below the
    peak carry a fraction erfc(sqrt(2 ln 1e7)) ~ 1e-15 of the pulse energy
    (Gaussian spectrum of Sec. VI), so dropping them changes A_mix and
    A_mix^H by far less than 1e-6 relative.  Checked on the full-spectrum
    operator with random data for two record lengths."""
    for Nt, M in ((128, 6), (256, 8)):
        g = geom(Nx=5, Ny=4, Nz=6, Nt=Nt)
        k = X.full_band(Nt)
        mag = O.pulse_spectrum(g.bin_freq(k), g.fc, g.alpha)
        band = k[mag >= 1e-7 * mag.max()]
        assert band.size < Nt and np.all(np.diff(band) == 1)     # one run of bins
        assert math.erfc(math.sqrt(2 * math.log(1e7))) < 1e-14
        idx = O.select_indices(g, O.SEL_RANDOM, M, True, 3)
        xi = synth.rademacher((g.S, g.Nt), seed=Nt)
        full = X.MixedOperator(g, idx, xi)
        cut = X.MixedOperator(g, idx, xi, band=band)
        rng = np.random.default_rng(Nt)
        x = crandn(rng, g.Nz, g.Ny, g.Nx)
        y = crandn(rng, g.S, M)
        yf = full.apply_A(x)
        assert np.linalg.norm(cut.apply_A(x) - yf) <= 1e-6 * np.linalg.norm(yf)
        xf = full.apply_AH(y)
        assert np.linalg.norm(cut.apply_AH(y) - xf) <= 1e-6 * np.linalg.norm(xf)
