"""Rademacher mixing (sfs_mixing_*, Phi_s = S_s F Sigma_s) on the GPU against
the FP64 mixing oracle, which mixes every one of the Nt bins of each A-scan:
A_mix, A_mix^H and FISTA at the FP32 bars of the plain operator (1e-5 for
the applies, 1e-4 for 100 FISTA iterations).  The library sums over the
bins within 140 dB of the pulse peak (sfs_mixing_band)."""
import numpy as np
import pytest

import oracle as O
from oracle import mixing_oracle as X
import synth
from tests._common import crandn, ensure_built, geom_params, oracle_geometry, rel_err

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


def build(sfs, params, M, seed, xi=None, precision=None):
    go = oracle_geometry(params)
    idx = O.select_indices(go, O.SEL_RANDOM, M, True, seed)
    if xi is None:
        xi = synth.rademacher((go.S, go.Nt), seed=seed + 1)
    g = sfs.Geometry(**params)
    mx = sfs.Mixing.create(g, idx, xi, precision=precision)
    mx.band._geom = g
    ref = X.MixedOperator(go, idx, xi)
    return mx, ref, go, idx, mx.band.idx[0], xi


@pytest.mark.parametrize("case", [
    (10, 8, 12, 128, 6),     # area scan
    (24, 1, 20, 256, 8),     # line scan
    (12, 12, 33, 256, 20),   # square scan, ragged depth
])
def test_mixed_apply_matches_oracle(sfs, case):
    Nx, Ny, Nz, Nt, M = case
    params = geom_params(Nx=Nx, Ny=Ny, Nz=Nz, dz=0.15e-3, Nt=Nt)
    mx, ref, go, idx, band, xi = build(sfs, params, M, 3)
    rng = np.random.default_rng(4)
    x = crandn(rng, Nz, Ny, Nx)
    y = crandn(rng, go.S, M)
    ya = to_host(mx.apply_A(to_dev(x)))
    xa = to_host(mx.apply_AH(to_dev(y)))
    assert rel_err(ya, ref.apply_A(x)) <= 1e-5
    assert rel_err(xa, ref.apply_AH(y)) <= 1e-5


def test_no_mixing_equals_the_plain_operator(sfs):
    params = geom_params(Nx=9, Ny=7, Nz=10, dz=0.15e-3, Nt=128)
    go = oracle_geometry(params)
    mx, ref, go, idx, band, xi = build(sfs, params, 5, 6, xi=np.ones((go.S, go.Nt), dtype=np.int8))
    op = sfs.Operator.from_indices(mx.band.geom, idx)
    rng = np.random.default_rng(7)
    x = to_dev(crandn(rng, go.Nz, go.Ny, go.Nx))
    y = to_dev(crandn(rng, go.S, 5))
    assert rel_err(to_host(mx.apply_A(x)), to_host(op.apply_A(x))) <= 1e-5
    assert rel_err(to_host(mx.apply_AH(y)), to_host(op.apply_AH(y))) <= 1e-5


def test_mixed_fista_and_lipschitz_match_oracle(sfs):
    """100 FISTA iterations on a noisy 3-scatterer scene measured through
    the mixed model: the GPU iterate within 1e-4 of the FP64 one (same L and
    lambda), and sfs_lipschitz_mixed within 1e-3 of the oracle's L."""
    params = geom_params(Nx=10, Ny=10, Nz=16, dz=0.15e-3, Nt=256)
    mx, ref, go, idx, band, xi = build(sfs, params, 8, 9)
    xt = synth.scene((go.Nz, go.Ny, go.Nx), 3, "uniform", seed=10)
    y0 = ref.apply_A(xt)
    sig = synth.noise_scale(float(np.vdot(y0, y0).real), y0.size, 20.0)
    y = (y0 + sig * synth.unit_noise(y0.shape, seed=11)).astype(np.complex64).astype(complex)
    L, _ = O.power_iteration(ref.apply_A, ref.apply_AH, xt.shape, 1, max_iter=500, rtol=1e-10)
    Lg, ok = mx.lipschitz(max_iter=500, rtol=1e-8, seed=3, safety=0.0)
    assert ok and abs(Lg - L) <= 1e-3 * L
    L *= 1.001
    lam = O.lambda_from_mu(ref.apply_AH, y, 0.05)
    x_ref = O.fista(ref.apply_A, ref.apply_AH, y, lam, L, 100)
    x_gpu = to_host(mx.fista(to_dev(y), lam, L, 100))
    assert np.abs(x_ref).max() > 0
    assert rel_err(x_gpu, x_ref) <= 1e-4
    # the mu rule on the device gives the same iterate
    x_mu = to_host(mx.fista(to_dev(y), -0.05, L, 100))
    assert rel_err(x_mu, x_ref) <= 1e-4


def test_mixing_invalid_arguments(sfs):
    params = geom_params(Nx=6, Ny=5, Nz=4, dz=0.15e-3, Nt=128)
    go = oracle_geometry(params)
    g = sfs.Geometry(**params)
    idx = O.select_indices(go, O.SEL_RANDOM, 4, True, 1)
    plain = sfs.Operator.from_indices(g, idx)   # rows differ: not a band operator
    with pytest.raises(sfs.SfsError):
        sfs.Mixing(plain, idx, synth.rademacher((go.S, go.Nt), seed=2))
    band = sfs.Mixing.band_bins(g)
    bop = sfs.Operator.from_indices(g, np.tile(band, (go.S, 1)))
    bad = synth.rademacher((go.S, go.Nt), seed=3)
    bad[0, 0] = 0
    with pytest.raises(sfs.SfsError):
        sfs.Mixing(bop, idx, bad)
    # a band operator that misses bins of the 140 dB run (here the
    # selection's candidate band only) is rejected
    lo, hi, _ = O.candidate_band(go, 4)
    narrow = sfs.Operator.from_indices(g, np.tile(np.arange(lo, hi + 1, dtype=np.int32), (go.S, 1)))
    with pytest.raises(sfs.SfsError) as ei:
        sfs.Mixing(narrow, idx, synth.rademacher((go.S, go.Nt), seed=4))
    assert ei.value.status == sfs.SFS_ERR_INVALID_ARG
    # a wider band (every signed bin) is accepted and gives the same A_mix
    wide = sfs.Operator.from_indices(g, np.tile(X.full_band(go.Nt).astype(np.int32), (go.S, 1)))
    xi = synth.rademacher((go.S, go.Nt), seed=5)
    m1, m2 = sfs.Mixing(bop, idx, xi), sfs.Mixing(wide, idx, xi)
    x = to_dev(crandn(np.random.default_rng(6), go.Nz, go.Ny, go.Nx))
    assert rel_err(to_host(m1.apply_A(x)), to_host(m2.apply_A(x))) <= 1e-6


@pytest.mark.parametrize("mode,tol", [("bf16", 2.0 ** -8), ("fp16", 2.0 ** -11)])
def test_mixing_over_a_16bit_band_operator(sfs, mode, tol):
    """The band operator on the tensor cores (16-bit table, FP16 with its
    per-scene scales): A_mix and A_mix^H within the mode's bar of the FP64
    mixing oracle."""
    params = geom_params(Nx=12, Ny=10, Nz=24, dz=0.15e-3, Nt=256)
    mx, ref, go, idx, band, xi = build(sfs, params, 8, 12, precision=sfs.PRECISION_NAMES[mode])
    rng = np.random.default_rng(14)
    x = crandn(rng, go.Nz, go.Ny, go.Nx)
    y = crandn(rng, go.S, 8)
    assert rel_err(to_host(mx.apply_A(to_dev(x))), ref.apply_A(x)) <= tol
    assert rel_err(to_host(mx.apply_AH(to_dev(y))), ref.apply_AH(y)) <= tol
