"""sfs_apply_AH_noalloc against sfs_apply_AH, called through the C ABI.

The no-allocation entry point serves callers that must not allocate device
memory once running (fixed-latency acquisition loops, host frameworks that
own all device memory); it keeps its intermediate data in the library's
static device array.  This file is collected last so that a failure here
does not hide any other test, and it passes alone in a fresh process too.
"""
import ctypes

import numpy as np
import pytest

import oracle as O
from tests._common import crandn, ensure_built, geom_params, rel_err

pytestmark = pytest.mark.gpu

TOL_OP = 1e-5


@pytest.fixture(scope="module")
def sfs():
    ensure_built()
    import torch
    from paper_2012_04534_gb300 import sfs as mod
    torch.cuda.init()
    return mod


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


@pytest.mark.parametrize("shape", [(32, 32, 128, 512, 64), (12, 10, 20, 128, 12), (32, 1, 64, 256, 32)])
def test_noalloc_matches_apply_AH_twice(sfs, shape):
    import torch
    Nx, Ny, Nz, Nt, M = shape
    g = sfs.Geometry(**geom_params(Nx=Nx, Ny=Ny, Nz=Nz, dz=0.15e-3, Nt=Nt))
    op = sfs.Operator.select(g, O.SEL_RANDOM, M, True, 17)
    rng = np.random.default_rng(5)
    st = torch.cuda.current_stream()
    sp = ctypes.c_void_p(st.cuda_stream)
    outs = []
    for call in range(2):  # two calls in a row share (and reuse) the static scratch
        y = torch.from_numpy(crandn(rng, *op.shape_y).astype(np.complex64)).cuda()
        ref = op.apply_AH(y)
        x = torch.full(op.shape_x, float("nan"), dtype=torch.complex64, device="cuda")
        sfs.sfs_apply_AH_noalloc(op.handle, _ptr(y), _ptr(x), sp)
        torch.cuda.synchronize()
        a, b = x.cpu().numpy(), ref.cpu().numpy()
        assert np.all(np.isfinite(a))
        assert rel_err(a, b) <= TOL_OP
        outs.append(a)
    assert not np.array_equal(outs[0], outs[1])  # different inputs, no stale result


def test_noalloc_rejects_operator_beyond_static_maximum(sfs):
    import torch
    # 64 x 64 scan, 256 depths: 163 bins x 16384 wavenumbers of spectra alone
    # need 21 MiB, plus >= 512 partial-sum slots of 64 KiB: more than 32 MiB
    g = sfs.Geometry(**geom_params(Nx=64, Ny=64, Nz=256, dz=0.15e-3, Nt=1024))
    op = sfs.Operator.select(g, O.SEL_RANDOM, 128, True, 1)
    y = torch.zeros(op.shape_y, dtype=torch.complex64, device="cuda")
    x = torch.zeros(op.shape_x, dtype=torch.complex64, device="cuda")
    rc = sfs.lib().sfs_apply_AH_noalloc(op.handle, _ptr(y), _ptr(x),
                                        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == sfs.SFS_ERR_INVALID_ARG
    msg = sfs.lib().sfs_last_error().decode()
    assert "static maximum" in msg and str(32 << 20) in msg
