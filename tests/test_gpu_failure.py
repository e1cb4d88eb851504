"""Failure handling on the GPU without faulting it.

The contraction kernels' waits on their bulk-copy barriers are bounded; a
wait that runs out sets the operator's error flag, drains the copies already
in flight and returns.  A tiny limit forces that path; the status must be
reported and the operator must work again once the limit is restored.
"""
import math

import numpy as np
import pytest

import oracle as O
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


@pytest.mark.parametrize("precision", ["fp32", "tf32x3", "bf16", "bf16x2", "fp16"])
def test_forced_wait_timeout_is_reported_and_recoverable(sfs, precision):
    """Every contraction kernel family: CUDA cores, tf32 tensor cores, and the
    TMA-fed 16-bit tensor-core kernels (one and two table parts)."""
    import torch
    params = geom_params(Nx=32, Ny=32, Nz=128, dz=0.15e-3, Nt=512)
    g = sfs.Geometry(**params)
    op = sfs.Operator.select(g, O.SEL_RANDOM, 64, True, 3,
                             precision=sfs.PRECISION_NAMES[precision])
    rng = np.random.default_rng(0)
    x = to_dev(crandn(rng, *op.shape_x))
    y = to_dev(crandn(rng, *op.shape_y))
    ref_y = op.apply_A(x).cpu().numpy()
    ref_x = op.apply_AH(y).cpu().numpy()
    assert op.check_status() == sfs.SFS_OK
    # each warp's first wait is on a barrier nothing arrives at: it runs out
    # after 2 ms, sets the flag, drains the real copies and returns
    op.set_wait_timeout_ns(2_000_000)
    op.inject_wait_timeout(True)
    op.apply_A(x)
    assert op.check_status() == sfs.SFS_ERR_TIMEOUT
    op.apply_AH(y)
    assert op.check_status() == sfs.SFS_ERR_TIMEOUT
    with pytest.raises(sfs.SfsError) as ei:
        op.max_abs_AH(y)                 # synchronising calls report it too
    assert ei.value.status == sfs.SFS_ERR_TIMEOUT
    with pytest.raises(sfs.SfsError) as ei:
        op.fista(y, -0.05, 1e8, 3, obj_hist=True)
    assert ei.value.status == sfs.SFS_ERR_TIMEOUT
    op.check_status()                    # clear
    op.inject_wait_timeout(False)
    op.set_wait_timeout_ns(2_000_000_000)
    ya = op.apply_A(x).cpu().numpy()
    xa = op.apply_AH(y).cpu().numpy()
    assert op.check_status() == sfs.SFS_OK
    assert rel_err(ya, ref_y) <= 1e-6 and rel_err(xa, ref_x) <= 1e-6
    torch.cuda.synchronize()


def test_invalid_wait_limit_and_non_finite_input(sfs):
    import torch
    g = sfs.Geometry(**geom_params(Nx=8, Ny=8, Nz=16, dz=0.15e-3, Nt=128))
    op = sfs.Operator.select(g, O.SEL_RANDOM, 6, True, 1)
    with pytest.raises(sfs.SfsError):
        op.set_wait_timeout_ns(0)
    y = torch.zeros(op.shape_y, dtype=torch.complex64, device="cuda")
    y[3, 2] = float("nan")
    with pytest.raises(sfs.SfsError) as ei:
        op.max_abs_AH(y)
    assert ei.value.status == sfs.SFS_ERR_NON_FINITE
    # the mu rule on the device flags a non-finite lambda
    op.fista(y, -0.05, 1e8, 2)
    assert op.check_status() == sfs.SFS_ERR_NON_FINITE
    assert op.check_status() == sfs.SFS_OK


def test_partial_sum_adjoint_and_two_depth_blocks(sfs):
    """Nz = 160 on a 32 x 32 scan: the forward sums two depth blocks and the
    (tile, 32-depth) segments outnumber the resident grid, so the adjoint
    leaves partial sums that the update planes add."""
    params = geom_params(Nx=32, Ny=32, Nz=160, dz=0.12e-3, Nt=128)
    g = sfs.Geometry(**params)
    op = sfs.Operator.select(g, O.SEL_RANDOM, 6, True, 21)
    go = oracle_geometry(params)
    idx = O.select_indices(go, O.SEL_RANDOM, 6, True, 21)
    assert np.array_equal(op.idx, idx)
    ref = O.LateralFFTOperator(go, idx)
    rng = np.random.default_rng(7)
    x = crandn(rng, *op.shape_x)
    y = crandn(rng, *op.shape_y)
    assert rel_err(op.apply_A(to_dev(x)).cpu().numpy(), ref.apply_A(x)) <= 1e-5
    assert rel_err(op.apply_AH(to_dev(y)).cpu().numpy(), ref.apply_AH(y)) <= 1e-5
    # the 128-row contraction slabs: 71 tiles x 5 blocks of 32 depths > 2 x 152 CTAs
    assert (op.info["Nslot"] // 64) * math.ceil(160 / 32) > 304
