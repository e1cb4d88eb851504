"""Pins of the FP64 Cramer-Rao bound oracle (oracle/crb_oracle.py, Sec. VI).

Each pin is fixed by something other than the oracle's own formulas: the
dense operator (itself pinned to the simulated time-domain echo), finite
differences of the data model, the textbook delay bound of a single
A-scan, and properties every Cramer-Rao bound has.
"""
import math

import numpy as np

import oracle as O
from oracle import crb_oracle as C


def geom(Nx=6, Ny=5, Nz=6, Nt=128, theta=0.0):
    return O.Geometry(Nx=Nx, Ny=Ny, dx=0.5e-3, dy=0.5e-3, Nz=Nz, z0=10e-3, dz=0.15e-3,
                      c=5900.0, fs=40e6, Nt=Nt, fc=5e6, frac_bw=0.7, theta=theta)


def test_scatterer_data_at_a_voxel_is_the_dense_column():
    g = geom(theta=math.radians(30))
    idx = O.select_indices(g, O.SEL_RANDOM, 7, True, 3)
    xv, yv, zv = g.voxel_xyz()
    for v in (0, 17, 101, g.V - 1):
        b = C.scatterer_data(g, idx, (xv[v], yv[v], zv[v]), 0.7, 0.4)
        col = O.A_cols(g, idx, [v])[:, 0] * 0.7 * np.exp(0.4j)
        np.testing.assert_allclose(b, col, rtol=1e-12, atol=1e-12 * np.abs(col).max())


def test_jacobian_equals_finite_differences_of_the_data():
    """Each column of D = d b / d u against central differences of b, with
    and without directivity, at an off-grid position (a wrong sign, factor
    2 / c or directivity derivative breaks it)."""
    for theta in (0.0, math.radians(25)):
        g = geom(theta=theta)
        idx = O.select_indices(g, O.SEL_RANDOM, 9, True, 4)
        p = np.array([1.13e-3, 0.87e-3, 10.4e-3])
        amp, ph = 0.8, -0.6
        D = C.data_jacobian(g, idx, p, amp, ph, "xyzap")
        for i, q in enumerate("xyzap"):
            if q in "xyz":
                h = 1e-8
                e = np.zeros(3)
                e["xyz".index(q)] = h
                fd = (C.scatterer_data(g, idx, p + e, amp, ph) - C.scatterer_data(g, idx, p - e, amp, ph)) / (2 * h)
            elif q == "a":
                h = 1e-6
                fd = (C.scatterer_data(g, idx, p, amp + h, ph) - C.scatterer_data(g, idx, p, amp - h, ph)) / (2 * h)
            else:
                h = 1e-6
                fd = (C.scatterer_data(g, idx, p, amp, ph + h) - C.scatterer_data(g, idx, p, amp, ph - h)) / (2 * h)
            assert np.linalg.norm(D[:, i] - fd) <= 1e-6 * np.linalg.norm(fd), (theta, q)


def test_single_ascan_depth_bound_is_the_delay_bound():
    """One A-scan straight above the scatterer, no directivity, u = (z, a,
    phi): C_z = sigma^2 c^2 / (8 (sum w w_k^2 - (sum w w_k)^2 / sum w)) with
    w = |b_k|^2 = (a fs H(f_k))^2 and w_k = 2 pi f_k, the delay bound scaled
    by (dz / dtau)^2 = (c / 2)^2."""
    g = geom(Nx=1, Ny=1, Nz=4, Nt=256)
    idx = O.select_indices(g, O.SEL_RANDOM, 20, True, 5)
    amp, sigma2 = 1.3, 0.25
    c, J = C.crb(g, idx, (0.0, 0.0, 12e-3), amp, 0.2, sigma2, "zap")
    f = g.bin_freq(idx[0])
    w = (amp * g.fs * O.pulse_spectrum(f, g.fc, g.alpha)) ** 2
    om = 2 * np.pi * f
    ref = sigma2 * g.c ** 2 / (8 * (np.sum(w * om ** 2) - np.sum(w * om) ** 2 / np.sum(w)))
    assert np.isnan(c[0]) and np.isnan(c[1])
    assert abs(c[2] - ref) <= 1e-9 * ref
    # a is decoupled from z and phi
    assert abs(J[0, 1]) <= 1e-9 * math.sqrt(J[0, 0] * J[1, 1])
    assert abs(J[1, 2]) <= 1e-9 * math.sqrt(J[1, 1] * J[2, 2])


def test_bound_scales_with_noise_and_amplitude_and_ignores_phase():
    g = geom(theta=math.radians(20))
    idx = O.select_indices(g, O.SEL_RANDOM, 8, True, 6)
    p = (1.2e-3, 1.0e-3, 10.5e-3)
    c0, _ = C.crb(g, idx, p, 1.0, 0.0, 1.0)
    c1, _ = C.crb(g, idx, p, 1.0, 1.1, 4.0)
    c2, _ = C.crb(g, idx, p, 2.0, -0.3, 1.0)
    np.testing.assert_allclose(c1, 4 * c0, rtol=1e-9)
    np.testing.assert_allclose(c2, c0 / 4, rtol=1e-9)
    assert np.all(np.isfinite(c0)) and np.all(c0 > 0)


def test_more_bins_never_raise_the_bound():
    """Every position keeps a superset of bins: the Fisher information grows
    by a positive semidefinite term, so each coordinate's bound can only
    fall (the text's C_{N_t} <= C)."""
    g = geom(Nt=128)
    full = O.select_indices(g, O.SEL_RANDOM, 16, True, 7)
    rng = np.random.default_rng(8)
    sub = np.sort(np.stack([rng.choice(row, 6, replace=False) for row in full]), axis=1)
    p = (1.4e-3, 0.9e-3, 10.3e-3)
    cf, Jf = C.crb(g, full, p, 1.0, 0.0, 1.0)
    cs, Js = C.crb(g, sub, p, 1.0, 0.0, 1.0)
    assert np.all(cf <= cs * (1 + 1e-12))
    assert np.linalg.eigvalsh(Jf - Js).min() >= -1e-9 * np.abs(Jf).max()
