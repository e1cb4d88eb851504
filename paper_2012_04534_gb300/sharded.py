"""Bin-sharded A, A^H, Lipschitz constant and FISTA over several GPUs (one
process per GPU).

The kept-bin union is cut into one contiguous run per rank
(sfs_shard_run); rank j builds the generator table (Theorem 2) of its run
only (sfs_operator_shard), so a table that does not fit one GPU is spread
over the ranks.  The runs partition the rows of A (Eq. (10)/(11)), hence

    A^H (A x - y) = sum_j A_j^H (A_j x - y),

and one FISTA iteration (Algorithm 1) is: every rank forms its partial
gradient with its own kernels (sfs_normal_residual, no exchange), one
all-reduce (sum) of the V voxel values joins them, and every rank applies
the same elementwise update (sfs_prox_momentum) to its replica of x and
gamma.  The forward A x needs no exchange: each rank writes the rows of its
bins.  The only collective is that all-reduce (NCCL on GPUs), per
iteration, per adjoint and per power-iteration step.

This module is argument marshalling and control flow: the arithmetic runs in
libsfs kernels; `allreduce` is the caller's collective (None on one rank).
A rank may also hold several shards (for instance to check the split on one
GPU): their partials are added before the collective.
"""
from __future__ import annotations

import math
from typing import Callable, List, Optional

from . import sfs


def torch_allreduce(group=None) -> Callable:
    """In-place sum of a complex64 tensor over the default (or given)
    torch.distributed process group."""
    import torch
    import torch.distributed as dist

    def run(t):
        dist.all_reduce(torch.view_as_real(t), op=dist.ReduceOp.SUM, group=group)
    return run


class GpuShard:
    """One shard operator on this process's GPU and the device vector
    operations the sharded solver needs."""

    def __init__(self, op: "sfs.Operator"):
        self.op = op
        self.V, self.S, self.M = op.V, op.S, op.M
        self.shape_x, self.shape_y = op.shape_x, op.shape_y

    @classmethod
    def build(cls, geom, idx, nshards, shard, precision=sfs.SFS_PREC_FP32):
        return cls(sfs.Operator.shard(geom, idx, nshards, shard, precision))

    def zeros(self, shape):
        import torch
        return torch.zeros(shape, dtype=torch.complex64, device="cuda:%d" % self.op.device)

    def apply_A_into(self, x, y):
        self.op.apply_A(x, out=y)

    def apply_AH(self, y):
        return self.op.apply_AH(y)

    def normal_residual(self, x, y, out):
        return self.op.normal_residual(x, y, out=out)

    def prox_momentum(self, x, gamma, grad, lam, L, beta):
        sfs.prox_momentum(x, gamma, grad, lam, L, beta)

    def sumsq(self, v):
        return self.op.vec_sumsq(v)

    def max_abs(self, v):
        return self.op.vec_max_abs(v)

    def scale(self, v, a):
        sfs.vec_scale(v, a)

    def randn(self, v, seed):
        sfs.vec_randn(v, seed)

    def add(self, a, b):
        """a += b (summing shards held by one process)."""
        a += b


class ShardedSolver:
    """The solver over this process's shards (usually one) and a collective.

    shards: backends with the methods of GpuShard, all of the same geometry
    and index set; allreduce(t): in-place sum of t over the ranks (None for a
    single process)."""

    def __init__(self, shards: List, allreduce: Optional[Callable] = None):
        if not shards:
            raise ValueError("at least one shard")
        self.shards = list(shards)
        self.allreduce = allreduce
        s0 = self.shards[0]
        self.V, self.S, self.M = s0.V, s0.S, s0.M
        self.shape_x, self.shape_y = s0.shape_x, s0.shape_y

    # sum of this process's partials, then over the ranks
    def _reduce(self, parts):
        acc = parts[0]
        for p in parts[1:]:
            self.shards[0].add(acc, p)
        if self.allreduce is not None:
            self.allreduce(acc)
        return acc

    def apply_A(self, x):
        """y = A x: every shard writes the rows of its bins; the sum over the
        ranks assembles y (the rows are disjoint)."""
        parts = []
        for sh in self.shards:
            y = sh.zeros(self.shape_y)
            sh.apply_A_into(x, y)
            parts.append(y)
        return self._reduce(parts)

    def apply_AH(self, y):
        """x = A^H y = sum_j A_j^H y."""
        return self._reduce([sh.apply_AH(y) for sh in self.shards])

    def gradient(self, x, y, out=None):
        """A^H (A x - y): partial gradients, then one sum."""
        parts = []
        for i, sh in enumerate(self.shards):
            buf = out if (i == 0 and out is not None) else sh.zeros(self.shape_x)
            parts.append(sh.normal_residual(x, y, buf))
        return self._reduce(parts)

    def lipschitz(self, max_iter=300, rtol=1e-6, seed=0, safety=1e-3):
        """L >= sigma_max^2 by power iteration on A^H A (Sec. IV-C): every
        rank draws the same start vector, each step one partial A_j^H A_j v
        per shard and one all-reduce; the estimate is ||A^H A v|| with
        ||v|| = 1.  Returns (L, converged)."""
        sh = self.shards[0]
        v = sh.zeros(self.shape_x)
        sh.randn(v, seed)
        sh.scale(v, 1.0 / math.sqrt(sh.sumsq(v)))
        zero_y = sh.zeros(self.shape_y)
        prev, est = -1.0, 0.0
        for _ in range(max_iter):
            w = self.gradient(v, zero_y)
            est = math.sqrt(sh.sumsq(w))
            if not math.isfinite(est) or est <= 0.0:
                raise sfs.SfsError(sfs.SFS_ERR_NON_FINITE, "power iteration met a zero or non-finite vector")
            sh.scale(w, 1.0 / est)
            v = w
            if prev > 0 and abs(est - prev) <= rtol * est:
                return est * (1.0 + safety), True
            prev = est
        return est * (1.0 + safety), False

    def fista(self, y, lam, L, iters, x=None):
        """Algorithm 1 with the sharded gradient: x_0 = gamma_1 = 0 (or x),
        t_1 = 1; lam < 0 means lam = -lam ||A^H y||_inf.  Every rank ends
        with the same x_K."""
        sh = self.shards[0]
        if lam < 0:
            lam = -lam * sh.max_abs(self.apply_AH(y))
        xk = sh.zeros(self.shape_x) if x is None else x
        gamma = xk.clone()
        grad = sh.zeros(self.shape_x)
        t = 1.0
        for _ in range(iters):
            g = self.gradient(gamma, y, out=grad)
            tn = 0.5 * (1.0 + math.sqrt(1.0 + 4.0 * t * t))
            sh.prox_momentum(xk, gamma, g, lam, L, (t - 1.0) / tn)
            t = tn
        return xk
