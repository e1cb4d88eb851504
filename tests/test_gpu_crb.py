"""sfs_crb (Sec. VI) on the GPU against the FP64 Cramer-Rao oracle.

Both sides are FP64; they differ in summation order and in how J is formed
(the library sums |b|^2-weighted coefficient products per row, the oracle
forms D and D^H D), so bounds and information agree to 1e-9 relative.
"""
import math

import numpy as np
import pytest

import oracle as O
from oracle import crb_oracle as C
from tests._common import ensure_built, geom_params, oracle_geometry

pytestmark = pytest.mark.gpu
MASK = {"xyz": 7, "xz": 5, "z": 4}


@pytest.fixture(scope="module")
def sfs():
    ensure_built()
    import torch
    from paper_2012_04534_gb300 import sfs as mod
    torch.cuda.init()
    return mod


def check(sfs, params, sets, pos, amp, sigma2, coords):
    g = sfs.Geometry(**params)
    go = oracle_geometry(params)
    idx = np.stack(sets).astype(np.int32)
    c, J = g.crb(idx, pos, amp, 0.3, sigma2, MASK[coords])
    order = coords + "ap"
    for t, ix in enumerate(sets):
        ref_c, ref_J = C.crb(go, ix, pos, amp, 0.3, sigma2, order)
        for q in "xyz":
            i = "xyz".index(q)
            if q in coords:
                assert abs(c[t, i] - ref_c[i]) <= 1e-9 * ref_c[i], (t, q)
            else:
                assert np.isnan(c[t, i])
        sel = ["xyzap".index(q) for q in order]
        got = J[t][np.ix_(sel, sel)]
        assert np.abs(got - ref_J).max() <= 1e-9 * np.abs(ref_J).max()
    return c


@pytest.mark.parametrize("theta_deg", [0.0, 30.0])
def test_crb_area_scan_strategies_match_oracle(sfs, theta_deg):
    params = geom_params(Nx=9, Ny=7, Nz=8, dz=0.15e-3, Nt=256, theta=math.radians(theta_deg))
    go = oracle_geometry(params)
    sets = [O.select_indices(go, O.SEL_RANDOM, 6, True, 1),
            O.select_indices(go, O.SEL_RANDOM, 6, False, 2),
            O.select_indices(go, O.SEL_CONTIGUOUS, 6, False, 0),
            O.select_indices(go, O.SEL_EQUISPACED, 6, False, 0),
            O.select_indices(go, O.SEL_MAXIMAL, 6, False, 0),
            O.select_indices(go, O.SEL_ENERGY, 6, True, 3)]
    check(sfs, params, sets, (2.1e-3, 1.35e-3, 10.6e-3), 0.9, 0.5, "xyz")


def test_crb_line_scan_and_single_ascan(sfs):
    params = geom_params(Nx=16, Ny=1, Nz=8, dz=0.15e-3, Nt=256, theta=math.radians(20))
    go = oracle_geometry(params)
    check(sfs, params, [O.select_indices(go, O.SEL_RANDOM, 5, True, 4)], (3.3e-3, 0.0, 11e-3), 1.0, 1.0, "xz")
    params = geom_params(Nx=1, Ny=1, Nz=8, dz=0.15e-3, Nt=512)
    go = oracle_geometry(params)
    check(sfs, params, [O.select_indices(go, O.SEL_RANDOM, 12, True, 5),
                        O.select_indices(go, O.SEL_MAXIMAL, 12, True, 0)], (0.0, 0.0, 12e-3), 1.0, 1.0, "z")


def test_crb_full_size_scan_and_more_bins(sfs):
    """A 32 x 32 scan (4096 rows per set at M = 4 ... 65536 at M = 64) with
    directivity: parity with the oracle, and the bound never rises when every
    position keeps more bins (the full band gives the smallest)."""
    params = geom_params(Nx=32, Ny=32, Nz=8, dz=0.15e-3, Nt=512, theta=math.radians(30))
    go = oracle_geometry(params)
    pos = (7.75e-3, 7.75e-3, 20e-3)
    full = O.select_indices(go, O.SEL_RANDOM, 64, True, 9)
    rng = np.random.default_rng(10)
    sub16 = np.sort(np.stack([rng.choice(r, 16, replace=False) for r in full]), axis=1)
    sub4 = np.sort(np.stack([rng.choice(r, 4, replace=False) for r in sub16]), axis=1)
    c64 = check(sfs, params, [full], pos, 1.0, 1.0, "xyz")
    c16 = check(sfs, params, [sub16], pos, 1.0, 1.0, "xyz")
    c4 = check(sfs, params, [sub4], pos, 1.0, 1.0, "xyz")
    assert np.all(c64[0] <= c16[0]) and np.all(c16[0] <= c4[0])


def test_crb_invalid_arguments(sfs):
    params = geom_params(Nx=1, Ny=1, Nz=4, dz=0.15e-3, Nt=128)
    g = sfs.Geometry(**params)
    go = oracle_geometry(params)
    idx = O.select_indices(go, O.SEL_RANDOM, 6, True, 1)
    with pytest.raises(sfs.SfsError):   # a single A-scan cannot locate x1, y1
        g.crb(idx, (0.0, 0.0, 11e-3), mask=7)
    with pytest.raises(sfs.SfsError):
        g.crb(idx, (0.0, 0.0, 11e-3), amp=0.0, mask=4)
    with pytest.raises(sfs.SfsError):
        g.crb(idx, (0.0, 0.0, -1e-3), mask=4)
    bad = idx.copy()
    bad[0, 1] = bad[0, 0]
    with pytest.raises(sfs.SfsError):
        g.crb(bad, (0.0, 0.0, 11e-3), mask=4)
