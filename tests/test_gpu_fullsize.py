"""GPU parity at the workloads' full sizes, through the C ABI, against the
FP64 lateral-FFT oracle (threaded over the host cores; its results do not
depend on the thread count).

  * 32 x 32 scan, 32 x 32 x 128 voxels (Nt 512, M 64 random bins per
    position): FISTA after 200 and after 300 iterations within 1e-4, same
    L and lambda on both sides.
  * the same 32 x 32 workload measured through Rademacher mixing (every
    position its own xi_s and bins): A_mix and A_mix^H within 1e-5 of the
    oracle that mixes all 512 bins of each A-scan, and 30 mixed FISTA
    iterations within 1e-4.
  * 64 x 64 scan, 64 x 64 x 256 voxels (Nt 1024, M 128, 128 x 128 lateral
    planes, 723 MB folded table): one whole A x and A^H y in FP32 (1e-5 in
    norm, 1e-4 of the oracle's largest entry element-wise), BF16 and FP16
    (their unit roundoff in norm, 8 u element-wise), and 20 FISTA iterations
    in FP32 within 1e-4.

The 64 x 64 oracle holds a 10.8 GB complex128 table; those tests are
skipped when the host has less than 48 GB available, so that they can never
drive it out of memory.
"""
import os

import numpy as np
import pytest

import oracle as O
import synth
from tests._common import crandn, ensure_built, oracle_geometry, rel_err

pytestmark = pytest.mark.gpu

TOL_OP = 1e-5
TOL_FISTA = 1e-4
MODE_TOL = {"fp32": (TOL_OP, 10 * TOL_OP), "bf16": (2.0 ** -8, 8 * 2.0 ** -8),
            "fp16": (2.0 ** -11, 8 * 2.0 ** -11)}
WORKERS = max(1, min(16, os.cpu_count() or 1))


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


def mem_available_gb():
    try:
        with open("/proc/meminfo") as fh:
            for line in fh:
                if line.startswith("MemAvailable:"):
                    return int(line.split()[1]) / 2 ** 20
    except OSError:
        pass
    return 0.0


def noisy_measurements(ref, x_true, snr_db, seed):
    y0 = ref.apply_A(x_true)
    sig = synth.noise_scale(float(np.vdot(y0, y0).real), y0.size, snr_db)
    return (y0 + sig * synth.unit_noise(y0.shape, seed=seed)).astype(np.complex64).astype(complex)


def test_vol32_fista_200_and_300_iterations(sfs):
    w = synth.WORKLOADS["vol32"]
    params = synth.geometry_params("vol32")
    go = oracle_geometry(params)
    g = sfs.Geometry(**params)
    op = sfs.Operator.select(g, sfs.SFS_SEL_RANDOM, w["M"], True, 1001)
    idx = O.select_indices(go, O.SEL_RANDOM, w["M"], True, 1001)
    assert np.array_equal(op.idx, idx)
    ref = O.LateralFFTOperator(go, idx, workers=WORKERS)
    x_true = synth.scene((g.Nz, g.Ny, g.Nx), w["n_scatter"], w["amp"], seed=1001)
    y = noisy_measurements(ref, x_true, w["snr_db"], 5)
    L, _ = op.lipschitz(max_iter=300, rtol=1e-6, seed=2, safety=1e-3)
    lam = O.lambda_from_mu(ref.apply_AH, y, w["mu"])
    x200, st = O.fista(ref.apply_A, ref.apply_AH, y, lam, L, 200, return_state=True)
    x300 = O.fista(ref.apply_A, ref.apply_AH, y, lam, L, 100, resume=st)
    assert np.abs(x300).max() > 0
    assert rel_err(to_host(op.fista(to_dev(y), lam, L, 200)), x200) <= TOL_FISTA
    assert rel_err(to_host(op.fista(to_dev(y), lam, L, 300)), x300) <= TOL_FISTA
    # the mu rule on the device, over the workload's 300 iterations
    assert rel_err(to_host(op.fista(to_dev(y), -w["mu"], L, 300)), x300) <= TOL_FISTA


@pytest.fixture(scope="module")
def vol64():
    if mem_available_gb() < 48:
        pytest.skip("the 64 x 64 x 256 oracle needs about 20 GB of host memory")
    w = synth.WORKLOADS["vol64"]
    params = synth.geometry_params("vol64")
    go = oracle_geometry(params)
    idx = O.select_indices(go, O.SEL_RANDOM, w["M"], True, 1002)
    ref = O.LateralFFTOperator(go, idx, workers=WORKERS)
    rng = np.random.default_rng(33)
    x = synth.scene((go.Nz, go.Ny, go.Nx), None, "uniform", seed=5, p_bernoulli=1e-4)
    x = x + 0.01 * crandn(rng, go.Nz, go.Ny, go.Nx)
    y = crandn(rng, go.S, w["M"])
    return dict(w=w, params=params, go=go, idx=idx, ref=ref, x=x, y=y,
                Ax=ref.apply_A(x), AHy=ref.apply_AH(y))


@pytest.mark.parametrize("mode", list(MODE_TOL))
def test_vol64_whole_A_and_AH(sfs, vol64, mode):
    g = sfs.Geometry(**vol64["params"])
    op = sfs.Operator.from_indices(g, vol64["idx"], precision=sfs.PRECISION_NAMES[mode])
    tol, tol_el = MODE_TOL[mode]
    ya = to_host(op.apply_A(to_dev(vol64["x"])))
    xa = to_host(op.apply_AH(to_dev(vol64["y"])))
    ry, rx = vol64["Ax"], vol64["AHy"]
    assert rel_err(ya, ry) <= tol
    assert rel_err(xa, rx) <= tol
    assert np.abs(ya - ry).max() <= tol_el * np.abs(ry).max()
    assert np.abs(xa - rx).max() <= tol_el * np.abs(rx).max()


def test_vol64_fista_20_iterations(sfs, vol64):
    w, ref = vol64["w"], vol64["ref"]
    g = sfs.Geometry(**vol64["params"])
    op = sfs.Operator.from_indices(g, vol64["idx"])
    x_true = synth.scene(op.shape_x, None, w["amp"], seed=1002, p_bernoulli=w["p_bernoulli"])
    y = noisy_measurements(ref, x_true, w["snr_db"], 6)
    L, _ = op.lipschitz(max_iter=300, rtol=1e-6, seed=2, safety=1e-3)
    lam = O.lambda_from_mu(ref.apply_AH, y, w["mu"])
    x_ref = O.fista(ref.apply_A, ref.apply_AH, y, lam, L, 20)
    assert np.abs(x_ref).max() > 0
    assert rel_err(to_host(op.fista(to_dev(y), lam, L, 20)), x_ref) <= TOL_FISTA


def test_vol32_mixing_full_size(sfs):
    from oracle import mixing_oracle as X
    w = synth.WORKLOADS["vol32"]
    params = synth.geometry_params("vol32")
    go = oracle_geometry(params)
    g = sfs.Geometry(**params)
    idx = O.select_indices(go, O.SEL_RANDOM, w["M"], True, 1001)
    xi = synth.rademacher((go.S, go.Nt), seed=1001 + 4242)
    mx = sfs.Mixing.create(g, idx, xi)
    mx.band._geom = g
    ref = X.MixedOperator(go, idx, xi, workers=WORKERS)
    rng = np.random.default_rng(41)
    x = crandn(rng, go.Nz, go.Ny, go.Nx)
    y = crandn(rng, go.S, w["M"])
    assert rel_err(to_host(mx.apply_A(to_dev(x))), ref.apply_A(x)) <= TOL_OP
    assert rel_err(to_host(mx.apply_AH(to_dev(y))), ref.apply_AH(y)) <= TOL_OP
    x_true = synth.scene((go.Nz, go.Ny, go.Nx), w["n_scatter"], w["amp"], seed=1001)
    ym = noisy_measurements(ref, x_true, w["snr_db"], 7)
    L, _ = mx.lipschitz(max_iter=300, rtol=1e-6, seed=3, safety=1e-3)
    lam = O.lambda_from_mu(ref.apply_AH, ym, w["mu"])
    x_ref = O.fista(ref.apply_A, ref.apply_AH, ym, lam, L, 30)
    assert np.abs(x_ref).max() > 0
    assert rel_err(to_host(mx.fista(to_dev(ym), lam, L, 30)), x_ref) <= TOL_FISTA
