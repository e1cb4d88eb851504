"""Learned unrolled ISTA on the GPU against its FP64 oracle.

Convolution weights are rounded to FP16 before both sides see them (the GPU
uses FP16 weights with FP32 accumulation), so the comparison isolates the
FP32 arithmetic: forward within 1e-4 relative after three layers, parameter
gradients within 1e-3 relative (norm over each parameter group).  The
autograd wrapper is checked against finite differences, and a short
training run must beat the same number of FISTA iterations.
"""
import numpy as np
import pytest

import oracle as O
from oracle import lista_oracle as LO
import synth
from tests._common import crandn, ensure_built, geom_params, oracle_geometry, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    ensure_built()
    import torch
    from paper_2012_04534_gb300 import lista, sfs
    torch.cuda.init()
    return sfs, lista


def to_dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.complex64)).cuda()


def to_host(t):
    import torch
    torch.cuda.synchronize()
    return t.cpu().numpy().astype(np.complex128)


def fp16_weights(p, layers):
    """Round the convolution weights to FP16 (eta, theta and biases stay FP32)."""
    p = np.asarray(p, dtype=np.float32).copy()
    for l in range(layers):
        o = l * LO.PER_LAYER
        for a, n in ((2, 432), (2 + 432 + 8, 432)):
            p[o + a:o + a + n] = p[o + a:o + a + n].astype(np.float16).astype(np.float32)
    return p


def problem(sfs, Nx=8, Ny=8, Nz=12, Nt=128, M=8, B=3, seed=1):
    params = geom_params(Nx=Nx, Ny=Ny, Nz=Nz, dz=0.15e-3, Nt=Nt)
    go = oracle_geometry(params)
    idx = O.select_indices(go, O.SEL_RANDOM, M, True, seed)
    g = sfs.Geometry(**params)
    op = sfs.Operator.from_indices(g, idx)
    ref = O.LateralFFTOperator(go, idx)
    xs, ys = [], []
    for b in range(B):
        xt = synth.scene(op.shape_x, 4, "uniform", seed=seed * 10 + b)
        y0 = ref.apply_A(xt)
        sig = synth.noise_scale(float(np.vdot(y0, y0).real), y0.size, 20.0)
        xs.append(xt)
        ys.append((y0 + sig * synth.unit_noise(y0.shape, seed=seed * 20 + b)).astype(np.complex64))
    L, _ = O.power_iteration(ref.apply_A, ref.apply_AH, op.shape_x, 1, max_iter=300, rtol=1e-9)
    return op, ref, np.stack(xs), np.stack(ys), L * 1.001


def test_lista_forward_and_backward_match_oracle(mods):
    sfs, lista = mods
    op, ref, xt, y, L = problem(sfs)
    layers, B = 3, y.shape[0]
    rng = np.random.default_rng(4)
    p = LO.init_params(layers, L, 0.05, rng, w_scale=0.1)
    p[2 + 432:2 + 432 + 8] = 0.05          # first-layer biases: some ReLUs on, some off
    p = fp16_weights(p, layers)
    net = lista.LISTA(op, layers, 4, L)
    net.set_params(p)
    assert np.array_equal(net.get_params(), p)
    x = net.forward(to_dev(y))
    loss, gx = net.nmse(x, to_dev(xt))
    gp = net.backward(gx).cpu().numpy().astype(np.float64)
    xg = to_host(x)
    # oracle: per scene forward, NMSE gradient of the batch mean, backward
    gref = np.zeros(p.size)
    lref = 0.0
    for b in range(B):
        xo, cache = LO.forward(ref.apply_A, ref.apply_AH, y[b].astype(np.complex128), p.astype(np.float64),
                               layers, L)
        assert rel_err(xg[b], xo) <= 1e-4
        lb, gb = LO.nmse_loss(xo, xt[b])
        lref += lb / B
        gref += LO.backward(ref.apply_A, ref.apply_AH, p.astype(np.float64), layers, cache, gb / B)
    assert loss == pytest.approx(lref, rel=1e-4)
    # gradients, group by group (eta, theta, W1, b1, W2, b2 of every layer)
    groups = [(0, 1), (1, 2), (2, 434), (434, 442), (442, 874), (874, 876)]
    for l in range(layers):
        o = l * LO.PER_LAYER
        for a, e in groups:
            r, gg = gref[o + a:o + e], gp[o + a:o + e]
            assert np.linalg.norm(gg - r) <= 1e-3 * np.linalg.norm(r) + 1e-12, (l, a)


def test_lista_autograd_function_matches_finite_differences(mods):
    import torch
    sfs, lista = mods
    op, ref, xt, y, L = problem(sfs, B=2, seed=3)
    layers = 2
    rng = np.random.default_rng(5)
    p = LO.init_params(layers, L, 0.05, rng, w_scale=0.1)
    # nonzero first-convolution biases keep the ReLU inputs of voxels where
    # s = 0 away from the kink at 0, where a finite difference is one-sided
    for l in range(layers):
        p[l * LO.PER_LAYER + 434:l * LO.PER_LAYER + 442] = 0.05
    p = fp16_weights(p, layers)
    net = lista.LISTA(op, layers, 2, L)
    yd, td = to_dev(y), to_dev(xt)
    pt = torch.from_numpy(p).cuda().requires_grad_(True)
    x = lista.lista_apply(net, pt, yd)
    loss = ((x - td).abs() ** 2).sum() / (td.abs() ** 2).sum()
    loss.backward()
    grad = pt.grad.detach().cpu().numpy().astype(np.float64)

    def f(q):
        with torch.no_grad():
            xq = lista.lista_apply(net, torch.from_numpy(q.astype(np.float32)).cuda(), yd)
            return float((((xq - td).abs() ** 2).sum() / (td.abs() ** 2).sum()).item())

    # eta, theta and the biases (FP32 parameters: steps are not rounded away)
    for i in [0, 1, 434, 436, 874, 875, LO.PER_LAYER, LO.PER_LAYER + 1, LO.PER_LAYER + 874]:
        h = 1e-2 * abs(p[i]) if p[i] != 0 else 1e-3
        qp, qm = p.astype(np.float64).copy(), p.astype(np.float64).copy()
        qp[i] += h
        qm[i] -= h
        fd = (f(qp) - f(qm)) / (2 * h)
        assert grad[i] == pytest.approx(fd, rel=2e-2, abs=1e-3 * np.abs(grad).max()), i


def test_trained_lista_beats_fista_with_as_many_iterations(mods):
    """Four layers trained for 150 Adam steps on scenes from the forward model
    (4 scatterers, 20 dB) reach a lower NMSE on held-out scenes than FISTA
    with 4 iterations (the same number of A and A^H applies), and than the
    untrained network it started from (ISTA with zero convolutions)."""
    import torch
    sfs, lista = mods
    op, ref, _, _, L = problem(sfs, B=1, seed=7)
    layers, B = 4, 8
    net = lista.LISTA(op, layers, B, L)
    rng = np.random.default_rng(8)
    p = LO.init_params(layers, L, 0.05, rng, w_scale=0.0)
    net.set_params(p)

    def batch(seed):
        xs, ys = [], []
        for b in range(B):
            xt = synth.scene(op.shape_x, 4, "uniform", seed=seed * 100 + b)
            y0 = ref.apply_A(xt)
            sig = synth.noise_scale(float(np.vdot(y0, y0).real), y0.size, 20.0)
            xs.append(xt)
            ys.append((y0 + sig * synth.unit_noise(y0.shape, seed=seed * 100 + 50 + b)).astype(np.complex64))
        return to_dev(np.stack(ys)), to_dev(np.stack(xs))

    y_eval, x_eval = batch(9999)
    loss0, _ = net.nmse(net.forward(y_eval), x_eval, with_grad=False)
    for step in range(1, 151):
        yb, xb = batch(step)
        x = net.forward(yb)
        _, gx = net.nmse(x, xb)
        g = net.backward(gx)
        net.adam(g, 2e-3 if step < 100 else 5e-4, step)
    loss1, _ = net.nmse(net.forward(y_eval), x_eval, with_grad=False)
    xf = op.fista_batched(y_eval, -0.05, L, layers)
    lf, _ = net.nmse(xf, x_eval, with_grad=False)
    assert loss1 < loss0
    assert loss1 < lf
