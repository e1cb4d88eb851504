"""CPU tests of the C-ABI library: it loads, exports every symbol the header
declares, and its host-side logic (geometry validation, integer frequency
selection) agrees with the oracle.  No device work is requested."""
import math
import os
import re

import numpy as np
import pytest

import oracle as O
import synth
from tests._common import ensure_built, geom_params, oracle_geometry

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def sfs():
    ensure_built()
    from paper_2012_04534_gb300 import sfs as mod
    mod.lib()
    return mod


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "sfs.h")).read()
    return set(re.findall(r"^(?:int|const char\*)\s+(sfs_\w+)\s*\(", text, re.M))


def test_library_exports_every_declared_symbol(sfs):
    names = declared_symbols()
    assert len(names) >= 15
    assert names == set(sfs.EXPORTS)
    L = sfs.lib()
    for n in names:
        assert hasattr(L, n), n
    assert "sm_103a" in sfs.sfs_version()


def test_grouped_order_setter(sfs):
    """sfs_set_grouped_order takes the three documented orders and refuses
    any other value (host logic, no device work)."""
    for bad in (-1, 3, 100):
        with pytest.raises(sfs.SfsError) as ei:
            sfs.set_grouped_order(bad)
        assert ei.value.status == sfs.SFS_ERR_INVALID_ARG
    for order in (sfs.SFS_GROUPED_LARGEST_FIRST, sfs.SFS_GROUPED_NO_PRIORITY, sfs.SFS_GROUPED_CHEAPEST_FIRST):
        sfs.set_grouped_order(order)


def test_grouped_argument_lists_must_match(sfs):
    """The grouped and persistent solves take one y, one L (and one x) per
    operator; lists of other lengths are refused before anything reaches
    the library."""
    ops = [object(), object()]
    for ys, Ls, xs in (([object()], [1.0, 1.0], None), ([object()] * 2, [1.0], None),
                       ([object()] * 2, [1.0, 1.0], [object()])):
        for persistent in (False, True):
            with pytest.raises(ValueError):
                sfs.fista_grouped(ops, ys, Ls, -0.05, 5, xs=xs, persistent=persistent)


def test_geometry_validation(sfs):
    ok = geom_params(Nx=8, Ny=8, Nz=4, dz=1e-4, Nt=64)
    g = sfs.Geometry(**ok)
    assert g.handle
    for bad in (dict(Nx=0), dict(Nz=-1), dict(Nt=1), dict(c=0.0), dict(fs=-1.0),
                dict(Nx=65, Ny=65), dict(Nx=600, Ny=1), dict(theta=2.0), dict(dz=0.0)):
        p = dict(ok)
        p.update(bad)
        with pytest.raises(sfs.SfsError) as ei:
            sfs.Geometry(**p)
        assert ei.value.status == sfs.SFS_ERR_INVALID_ARG


@pytest.mark.parametrize("name", ["line2d", "vol32", "vol64"])
@pytest.mark.parametrize("strategy", [O.SEL_RANDOM, O.SEL_CONTIGUOUS, O.SEL_EQUISPACED])
def test_host_selection_bit_exact_with_oracle(sfs, name, strategy):
    w = synth.WORKLOADS[name]
    params = synth.geometry_params(name)
    g = sfs.Geometry(**params)
    go = O.Geometry(**params)
    for per in (True, False):
        idx, band = g.select_indices(strategy, w["M"], per, seed=2024)
        ref = O.select_indices(go, strategy, w["M"], per, seed=2024)
        assert idx.dtype == np.int32
        assert np.array_equal(idx, ref)
        k_lo, k_hi, _ = O.candidate_band(go, w["M"])
        assert band == (k_lo, k_hi)


@pytest.mark.parametrize("name", ["line2d", "vol32", "vol64"])
@pytest.mark.parametrize("strategy", [O.SEL_MAXIMAL, O.SEL_ENERGY])
def test_host_knowledge_based_selection_bit_exact_with_oracle(sfs, name, strategy):
    """Phi_max and Phi_nrg(,f) (Sec. III-A): the host sets equal the oracle's
    bit for bit, shared and per position, for several seeds and M."""
    params = synth.geometry_params(name)
    g = sfs.Geometry(**params)
    go = O.Geometry(**params)
    for M in (1, 7, synth.WORKLOADS[name]["M"]):
        for per in (True, False):
            for seed in (0, 99, 2**63 + 11):
                idx, _ = g.select_indices(strategy, M, per, seed=seed)
                assert np.array_equal(idx, O.select_indices(go, strategy, M, per, seed=seed))


def test_host_selection_many_seeds_and_sizes(sfs):
    for (Nx, Ny, Nt, M) in [(5, 3, 128, 7), (1, 1, 64, 1), (9, 1, 256, 20), (4, 4, 512, 40)]:
        p = geom_params(Nx=Nx, Ny=Ny, Nz=3, dz=1e-4, Nt=Nt)
        g = sfs.Geometry(**p)
        go = oracle_geometry(p)
        for seed in (0, 1, 2**63 + 5, 12345678901234):
            idx, _ = g.select_indices(O.SEL_RANDOM, M, True, seed)
            assert np.array_equal(idx, O.select_indices(go, O.SEL_RANDOM, M, True, seed))


def test_band_too_narrow(sfs):
    g = sfs.Geometry(**geom_params(Nx=4, Ny=4, Nz=2, dz=1e-4, Nt=64))
    with pytest.raises(sfs.SfsError) as ei:
        g.select_indices(O.SEL_RANDOM, 30, True, 0)
    assert ei.value.status == sfs.SFS_ERR_BAND_TOO_NARROW
    with pytest.raises(sfs.SfsError) as ei:
        g.select_indices(O.SEL_RANDOM, 0, True, 0)
    assert ei.value.status == sfs.SFS_ERR_INVALID_ARG
    with pytest.raises(sfs.SfsError) as ei:
        g.select_indices(7, 3, True, 0)
    assert ei.value.status == sfs.SFS_ERR_INVALID_ARG


def test_null_handles_rejected(sfs):
    L = sfs.lib()
    assert L.sfs_apply_A(None, None, None, None) == sfs.SFS_ERR_INVALID_ARG
    assert "null" in L.sfs_last_error().decode()
    assert L.sfs_fista(None, None, 0.0, 1.0, 1, None, None, 0, None, None) == sfs.SFS_ERR_INVALID_ARG
    assert L.sfs_operator_from_indices(None, 1, None, None) == sfs.SFS_ERR_INVALID_ARG
    assert L.sfs_destroy_operator(None) == sfs.SFS_OK


@pytest.mark.parametrize("name", ["line2d", "vol32", "vol64"])
def test_mixing_band_is_the_140_dB_run_of_the_pulse(sfs, name):
    """sfs_mixing_band (host only) equals the run of signed bins -Nt/2 < k <=
    Nt/2 whose oracle pulse magnitude |H(k fs/Nt)| is within 140 dB of the
    peak, and it reaches into the negative frequencies."""
    from oracle import mixing_oracle as X
    params = synth.geometry_params(name)
    g = sfs.Geometry(**params)
    go = O.Geometry(**params)
    k = X.full_band(go.Nt)
    mag = O.pulse_spectrum(go.bin_freq(k), go.fc, go.alpha)
    ref = k[mag >= 10 ** (-140.0 / 20) * mag.max()]
    got = sfs.Mixing.band_bins(g)
    assert np.array_equal(got, ref)
    assert got[0] < 0 < got[-1] <= go.Nt // 2


def test_host_random_draw_uses_the_published_splitmix64_stream(sfs):
    """The C++ host selection keys position 0's stream with the seed itself,
    so a shared RANDOM set with seed 1234567 consumes the published outputs
    (tests/golden/splitmix64_seed1234567.txt): partial Fisher-Yates over the
    candidate band with j = i + floor(hi32(u_i) (|C| - i) / 2^32)."""
    path = os.path.join(ROOT, "tests", "golden", "splitmix64_seed1234567.txt")
    gold = [int(l) for l in open(path) if l.strip() and not l.startswith("#")]
    params = synth.geometry_params("vol32")
    g = sfs.Geometry(**params)
    M = len(gold)
    idx, (lo, hi) = g.select_indices(sfs.SFS_SEL_RANDOM, M, False, 1234567)
    n = hi - lo + 1
    perm = list(range(n))
    for i, u in enumerate(gold):
        j = i + (((u >> 32) * (n - i)) >> 32)
        perm[i], perm[j] = perm[j], perm[i]
    expect = np.array(sorted(lo + v for v in perm[:M]), dtype=np.int32)
    assert np.array_equal(idx[0], expect)
    assert all(np.array_equal(r, expect) for r in idx)
