"""Learned unrolled ISTA on the library's kernels (include/sfs.h, sfs_lista_*).

Marshalling only: the forward, the backward, the loss and the Adam step run
in libsfs's CUDA kernels.  ``LISTA`` wraps one network; ``LISTAFunction``
exposes it to torch.autograd with the parameters as a differentiable input.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import sfs

PER_LAYER = 876


def _lib():
    L = sfs.lib()
    if not getattr(L, "_lista_sig", False):
        vp, i32, f32 = ctypes.c_void_p, ctypes.c_int, ctypes.c_float
        P = ctypes.POINTER
        sig = {
            "sfs_lista_create": [vp, i32, i32, ctypes.c_double, P(vp)],
            "sfs_lista_destroy": [vp],
            "sfs_lista_info": [vp, P(ctypes.c_int32), P(ctypes.c_int32)],
            "sfs_lista_set_params": [vp, P(ctypes.c_float)],
            "sfs_lista_get_params": [vp, P(ctypes.c_float)],
            "sfs_lista_load_params_dev": [vp, vp, vp],
            "sfs_lista_forward": [vp, i32, vp, vp, vp],
            "sfs_lista_backward": [vp, i32, vp, vp, vp],
            "sfs_lista_nmse": [vp, i32, vp, vp, vp, P(ctypes.c_double), vp],
            "sfs_lista_adam": [vp, vp, f32, f32, f32, f32, i32, vp],
        }
        for name, args in sig.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = ctypes.c_int
        L._lista_sig = True
    return L


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def _stream(device):
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


class LISTA:
    """Network of `layers` layers on operator `op` (Lipschitz constant L) for
    up to `max_batch` scenes."""

    def __init__(self, op: "sfs.Operator", layers: int, max_batch: int, L: float):
        self.op = op
        self.layers = layers
        self.max_batch = max_batch
        self.L = float(L)
        h = ctypes.c_void_p()
        sfs._check(_lib().sfs_lista_create(op.handle, layers, max_batch, self.L, ctypes.byref(h)))
        self.handle = h
        self.nparams = layers * PER_LAYER

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        assert p.size == self.nparams
        sfs._check(_lib().sfs_lista_set_params(self.handle, p.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))

    def get_params(self):
        p = np.zeros(self.nparams, dtype=np.float32)
        sfs._check(_lib().sfs_lista_get_params(self.handle, p.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))
        return p

    def load_params(self, t):
        """Parameters from a contiguous float32 CUDA tensor."""
        assert t.is_cuda and t.numel() == self.nparams and t.is_contiguous()
        sfs._check(_lib().sfs_lista_load_params_dev(self.handle, _ptr(t), _stream(t.device)))

    def forward(self, y, out=None):
        import torch
        B = int(y.shape[0])
        x = torch.empty((B,) + self.op.shape_x, dtype=torch.complex64, device=y.device) if out is None else out
        sfs._dev_ptr(y, B * self.op.S * self.op.M, "y")
        sfs._dev_ptr(x, B * self.op.V, "x")
        sfs._check(_lib().sfs_lista_forward(self.handle, B, _ptr(y), _ptr(x), _stream(y.device)))
        return x

    def backward(self, grad_x):
        import torch
        B = int(grad_x.shape[0])
        g = torch.empty(self.nparams, dtype=torch.float32, device=grad_x.device)
        sfs._dev_ptr(grad_x, B * self.op.V, "grad_x")
        sfs._check(_lib().sfs_lista_backward(self.handle, B, _ptr(grad_x), _ptr(g), _stream(grad_x.device)))
        return g

    def nmse(self, x, x_true, with_grad=True):
        import torch
        B = int(x.shape[0])
        g = torch.empty_like(x) if with_grad else None
        loss = ctypes.c_double()
        sfs._check(_lib().sfs_lista_nmse(self.handle, B, _ptr(x), _ptr(x_true), _ptr(g) if g is not None else None,
                                         ctypes.byref(loss), _stream(x.device)))
        return loss.value, g

    def adam(self, grad, lr, step, beta1=0.9, beta2=0.999, eps=1e-8):
        sfs._check(_lib().sfs_lista_adam(self.handle, _ptr(grad), float(lr), float(beta1), float(beta2),
                                         float(eps), int(step), _stream(grad.device)))

    def close(self):
        h, self.handle = getattr(self, "handle", None), None
        if h:
            _lib().sfs_lista_destroy(h)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _autograd_function():
    import torch

    class LISTAFunction(torch.autograd.Function):
        """x = network(params, y) with d/d params by the library's backward."""

        @staticmethod
        def forward(ctx, params, y, net):
            net.load_params(params.detach().contiguous())
            x = net.forward(y)
            ctx.net = net
            return x

        @staticmethod
        def backward(ctx, grad_x):
            # autograd hands the conjugate-Wirtinger form of a real loss's
            # gradient for complex outputs, which for a real loss equals
            # dL/dRe x + i dL/dIm x
            g = ctx.net.backward(grad_x.contiguous())
            return g, None, None

    return LISTAFunction


def lista_apply(net: LISTA, params, y):
    """Differentiable network output (params: float32 CUDA tensor)."""
    return _autograd_function().apply(params, y, net)
