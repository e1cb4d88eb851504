"""Pins of the learned-ISTA oracle (oracle/lista_oracle.py) to facts other
than itself (CPU only): a library correlation, the adjoint identity of the
convolution pair, Algorithm 1's ISTA step as computed by the FISTA oracle,
and central finite differences of the loss."""
import numpy as np
import pytest

import oracle as O
from oracle import lista_oracle as LO
import synth


def small_geom(Nx=4, Ny=3, Nz=5, Nt=32):
    return O.Geometry(Nx=Nx, Ny=Ny, dx=0.5e-3, dy=0.5e-3, Nz=Nz, z0=10e-3, dz=0.15e-3,
                      c=5900.0, fs=40e6, Nt=Nt, fc=5e6, frac_bw=0.7, theta=0.0)


def test_conv3d_equals_scipy_correlate():
    ndimage = pytest.importorskip("scipy.ndimage")
    rng = np.random.default_rng(0)
    u = rng.standard_normal((2, 5, 4, 6))
    W = rng.standard_normal((3, 2, 3, 3, 3))
    b = rng.standard_normal(3)
    out = LO.conv3d(u, W, b)
    ref = np.stack([sum(ndimage.correlate(u[i], W[o, i], mode="constant", cval=0.0) for i in range(2)) + b[o]
                    for o in range(3)])
    np.testing.assert_allclose(out, ref, rtol=1e-12, atol=1e-12)


def test_conv3d_transpose_and_weight_grad_are_adjoints():
    rng = np.random.default_rng(1)
    u = rng.standard_normal((2, 4, 5, 3))
    W = rng.standard_normal((8, 2, 3, 3, 3))
    g = rng.standard_normal((8, 4, 5, 3))
    lhs = float((LO.conv3d(u, W) * g).sum())
    assert lhs == pytest.approx(float((u * LO.conv3d_transpose(g, W)).sum()), rel=1e-12)
    dW, db = LO.conv3d_weight_grad(g, u)
    assert lhs == pytest.approx(float((W * dW).sum()), rel=1e-12)
    assert np.allclose(db, g.sum(axis=(1, 2, 3)))


def test_zero_prox_network_is_ista():
    """W = b = 0, eta_l = 1 (step 1/L), theta_l = lambda/(sigma L): the network is
    `layers` ISTA steps, i.e. warm-started single-iteration FISTA steps."""
    g = small_geom()
    idx = O.select_indices(g, O.SEL_RANDOM, 4, True, 3)
    A = O.dense_A(g, idx)
    fA = lambda v: (A @ np.ravel(v)).reshape(g.S, 4)
    fAH = lambda r: (A.conj().T @ np.ravel(r)).reshape(g.Nz, g.Ny, g.Nx)
    rng = np.random.default_rng(2)
    y = rng.standard_normal((g.S, 4)) + 1j * rng.standard_normal((g.S, 4))
    L = float(np.linalg.svd(A, compute_uv=False)[0] ** 2) * 1.01
    lam = 0.1 * float(np.abs(fAH(y)).max())
    sigma = float(np.abs(fAH(y)).max()) / L
    layers = 5
    p = np.zeros(layers * LO.PER_LAYER)
    for l in range(layers):
        p[l * LO.PER_LAYER] = 1.0
        p[l * LO.PER_LAYER + 1] = lam / (sigma * L)
    x_net, _ = LO.forward(fA, fAH, y, p, layers, L)
    x = np.zeros((g.Nz, g.Ny, g.Nx), complex)
    for _ in range(layers):
        x = O.fista(fA, fAH, y, lam, L, 1, x0=x)
    np.testing.assert_allclose(x_net, x, rtol=1e-12, atol=1e-12 * np.abs(x).max())
    assert np.abs(x).max() > 0


def test_backward_matches_central_differences():
    g = small_geom()
    idx = O.select_indices(g, O.SEL_RANDOM, 4, True, 5)
    A = O.dense_A(g, idx)
    fA = lambda v: (A @ np.ravel(v)).reshape(g.S, 4)
    fAH = lambda r: (A.conj().T @ np.ravel(r)).reshape(g.Nz, g.Ny, g.Nx)
    rng = np.random.default_rng(6)
    x_true = synth.scene((g.Nz, g.Ny, g.Nx), 3, "uniform", seed=4)
    y = fA(x_true) + 0.05 * (rng.standard_normal((g.S, 4)) + 1j * rng.standard_normal((g.S, 4)))
    L = float(np.linalg.svd(A, compute_uv=False)[0] ** 2) * 1.01
    layers = 2
    p = LO.init_params(layers, L, 0.05, rng, w_scale=0.1)
    p[1::LO.PER_LAYER][:layers] = 0.02
    # positive first-layer biases: some ReLUs on, some off
    p[LO.PER_LAYER - 2 - 2 * LO.C_HID * 27 - LO.C_HID:LO.PER_LAYER - 2 - 2 * LO.C_HID * 27] = 0.05

    def loss(q):
        x, _ = LO.forward(fA, fAH, y, q, layers, L)
        return LO.nmse_loss(x, x_true)[0]

    x, cache = LO.forward(fA, fAH, y, p, layers, L)
    _, gx = LO.nmse_loss(x, x_true)
    grad = LO.backward(fA, fAH, p, layers, cache, gx)
    # eta, theta of both layers, and a sample of weights and biases
    picks = [0, 1, LO.PER_LAYER, LO.PER_LAYER + 1]
    picks += list(rng.choice(np.arange(2, LO.PER_LAYER), 16, replace=False))
    picks += list(LO.PER_LAYER + rng.choice(np.arange(2, LO.PER_LAYER), 16, replace=False))
    for i in picks:
        h = 1e-4 * abs(p[i]) if p[i] != 0 else 1e-6
        qp, qm = p.copy(), p.copy()
        qp[i] += h
        qm[i] -= h
        fd = (loss(qp) - loss(qm)) / (2 * h)
        assert grad[i] == pytest.approx(fd, rel=1e-5, abs=1e-9 * np.abs(grad).max()), i


def test_nmse_loss_gradient():
    rng = np.random.default_rng(3)
    x = rng.standard_normal(7) + 1j * rng.standard_normal(7)
    t = rng.standard_normal(7) + 1j * rng.standard_normal(7)
    l, g = LO.nmse_loss(x, t)
    assert l == pytest.approx(np.sum(np.abs(x - t) ** 2) / np.sum(np.abs(t) ** 2))
    e = np.zeros(7, complex)
    e[2] = 1e-7
    assert (LO.nmse_loss(x + e, t)[0] - l) / 1e-7 == pytest.approx(g[2].real, rel=1e-5)
    assert (LO.nmse_loss(x + 1j * e, t)[0] - l) / 1e-7 == pytest.approx(g[2].imag, rel=1e-5)
