"""FISTA with backtracking (sfs_fista_backtracking, Sec. IV-C) against the
FP64 oracle's fista_backtracking: the same sequence of accepted L_k and the
final iterate within the FISTA bar (1e-4)."""
import numpy as np
import pytest

import oracle as O
import synth
from tests._common import ensure_built, geom_params, oracle_geometry, rel_err

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


def problem(sfs, Nx=10, Ny=9, Nz=16, Nt=256, M=10, seed=3):
    params = geom_params(Nx=Nx, Ny=Ny, Nz=Nz, dz=0.15e-3, Nt=Nt)
    go = oracle_geometry(params)
    idx = O.select_indices(go, O.SEL_RANDOM, M, True, seed)
    g = sfs.Geometry(**params)
    op = sfs.Operator.from_indices(g, idx)
    op._geom = g
    ref = O.LateralFFTOperator(go, idx)
    xt = synth.scene((Nz, Ny, Nx), 4, "uniform", seed=seed + 1)
    y0 = ref.apply_A(xt)
    sig = synth.noise_scale(float(np.vdot(y0, y0).real), y0.size, 20.0)
    y = (y0 + sig * synth.unit_noise(y0.shape, seed=seed + 2)).astype(np.complex64).astype(complex)
    L, _ = O.power_iteration(ref.apply_A, ref.apply_AH, xt.shape, 1, max_iter=500, rtol=1e-10)
    return op, ref, y, L


@pytest.mark.parametrize("L0_frac,eta", [(1.5, 2.0), (1e-3, 2.0), (1e-2, 1.5)])
def test_backtracking_matches_oracle(sfs, L0_frac, eta):
    op, ref, y, L = problem(sfs)
    lam = O.lambda_from_mu(ref.apply_AH, y, 0.05)
    hist = []
    x_ref = O.fista_backtracking(ref.apply_A, ref.apply_AH, y, lam, L * L0_frac, eta, 60, L_history=hist)
    xg, hg = op.fista_backtracking(to_dev(y), lam, L * L0_frac, eta, 60)
    np.testing.assert_allclose(hg, hist, rtol=1e-12)
    assert max(hg) <= eta * L * 1.0001
    assert rel_err(to_host(xg), x_ref) <= 1e-4


def test_backtracking_mu_rule_and_no_backtracks_equal_fista(sfs):
    """lambda by the mu rule on the device; with L0 above ||A||^2 no trial is
    rejected and the iterate equals sfs_fista's with L = L0."""
    op, ref, y, L = problem(sfs, seed=7)
    yd = to_dev(y)
    xg, hg = op.fista_backtracking(yd, -0.05, 1.2 * L, 2.0, 40)
    assert np.all(hg == 1.2 * L)
    xf = op.fista(yd, -0.05, 1.2 * L, 40)
    assert rel_err(to_host(xg), to_host(xf)) <= 1e-5


def test_backtracking_invalid_arguments(sfs):
    op, ref, y, L = problem(sfs, Nx=4, Ny=4, Nz=4, Nt=128, M=4, seed=9)
    yd = to_dev(y)
    for L0, eta in ((0.0, 2.0), (1.0, 1.0), (-1.0, 2.0)):
        with pytest.raises(sfs.SfsError):
            op.fista_backtracking(yd, 0.1, L0, eta, 5)
