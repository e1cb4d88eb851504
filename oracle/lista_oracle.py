"""FP64 CPU oracle of the learned unrolled ISTA network (forward, analytic
backward, loss).

TEST INFRASTRUCTURE ONLY, under the same rules as sfs_oracle (only tests/,
__graft_entry__.smoke() and bench.py's CPU legs may use it; it never imports
the product library).

The paper reconstructs with ISTA/FISTA only (Sec. IV-A, Algorithm 1); the
unrolled network is the learned extension of that iteration that the
workloads ask for.  Each layer l keeps Algorithm 1's gradient step and
complex soft threshold with its own learned step eta_l and threshold
theta_l, and adds a residual 3-D convolutional proximal block:

    g_l     = A^H (A x_l - y_n)                    gradient of 1/2||A x - y_n||^2
    z_l     = x_l - (eta_l / L) g_l
    s_l     = tau_{theta_l}(z_l)                    complex soft threshold
    h_l     = W1_l * [Re s_l, Im s_l] + b1_l        8 channels, 3x3x3
    x_{l+1} = s_l + (W2_l * relu(h_l) + b2_l)       2 channels read as re, im

with x_0 = 0, y_n = y / sigma, sigma = ||A^H y||_inf / L (L the operator's
Lipschitz constant, so that ||A^H y_n||_inf = L and the layer variables are
O(1) whatever the data's scale), output x = sigma x_L.  "*" is the 3-D
cross-correlation with zero padding: (W * u)[o](z, y, x) =
sum_{i, dz, dy, dx} W[o][i][dz][dy][dx] u[i](z + dz - 1, y + dy - 1, x + dx - 1).

Parameters of layer l, flat in this order (876 numbers):
eta, theta, W1 (8, 2, 3, 3, 3), b1 (8), W2 (2, 8, 3, 3, 3), b2 (2).  Both
eta (step in units of 1/L) and theta are O(1), like the other parameters.

Parity status (tests/test_lista_oracle_pins.py): conv3d is pinned by
scipy.ndimage.correlate; the forward with zero convolutions and eta = 1,
theta = lambda/(sigma L) is pinned by L single-iteration warm-started
FISTA steps of sfs_oracle.fista (which are ISTA steps); the analytic
backward is pinned by central finite differences of the loss.
"""
from __future__ import annotations

from typing import Callable, List

import numpy as np

C_HID = 8
KS = 3
PER_LAYER = 2 + C_HID * 2 * 27 + C_HID + 2 * C_HID * 27 + 2


def split_params(p, layers: int):
    """Flat parameter vector -> list of per-layer dicts."""
    p = np.asarray(p, dtype=np.float64)
    assert p.size == layers * PER_LAYER
    out = []
    for l in range(layers):
        q = p[l * PER_LAYER:(l + 1) * PER_LAYER]
        o = 0
        eta, theta = q[0], q[1]
        o = 2
        W1 = q[o:o + C_HID * 2 * 27].reshape(C_HID, 2, KS, KS, KS)
        o += C_HID * 2 * 27
        b1 = q[o:o + C_HID]
        o += C_HID
        W2 = q[o:o + 2 * C_HID * 27].reshape(2, C_HID, KS, KS, KS)
        o += 2 * C_HID * 27
        b2 = q[o:o + 2]
        out.append(dict(eta=eta, theta=theta, W1=W1, b1=b1, W2=W2, b2=b2))
    return out


def conv3d(u, W, b=None):
    """3-D cross-correlation with zero padding (definition in the header).
    u: [Cin][Nz][Ny][Nx] real, W: [Cout][Cin][3][3][3], b: [Cout] or None."""
    u = np.asarray(u, dtype=np.float64)
    cin, nz, ny, nx = u.shape
    cout = W.shape[0]
    up = np.zeros((cin, nz + 2, ny + 2, nx + 2))
    up[:, 1:-1, 1:-1, 1:-1] = u
    out = np.zeros((cout, nz, ny, nx))
    for dz in range(KS):
        for dy in range(KS):
            for dx in range(KS):
                sl = up[:, dz:dz + nz, dy:dy + ny, dx:dx + nx]
                out += np.einsum("oi,izyx->ozyx", W[:, :, dz, dy, dx], sl)
    if b is not None:
        out += np.asarray(b)[:, None, None, None]
    return out


def conv3d_transpose(gout, W):
    """Adjoint of conv3d in its input: gin[i](v) = sum_{o, t} W[o][i][t] gout[o](v - t + 1)."""
    gout = np.asarray(gout, dtype=np.float64)
    cout, nz, ny, nx = gout.shape
    cin = W.shape[1]
    gp = np.zeros((cout, nz + 2, ny + 2, nx + 2))
    gp[:, 1:-1, 1:-1, 1:-1] = gout
    gin = np.zeros((cin, nz, ny, nx))
    for dz in range(KS):
        for dy in range(KS):
            for dx in range(KS):
                # v - t + 1 for t = (dz, dy, dx): the padded index 2 - dz ...
                sl = gp[:, 2 - dz:2 - dz + nz, 2 - dy:2 - dy + ny, 2 - dx:2 - dx + nx]
                gin += np.einsum("oi,ozyx->izyx", W[:, :, dz, dy, dx], sl)
    return gin


def conv3d_weight_grad(gout, u):
    """dW[o][i][t] = sum_v gout[o](v) u[i](v + t - 1); db[o] = sum_v gout[o](v)."""
    cin, nz, ny, nx = u.shape
    up = np.zeros((cin, nz + 2, ny + 2, nx + 2))
    up[:, 1:-1, 1:-1, 1:-1] = u
    dW = np.zeros((gout.shape[0], cin, KS, KS, KS))
    for dz in range(KS):
        for dy in range(KS):
            for dx in range(KS):
                sl = up[:, dz:dz + nz, dy:dy + ny, dx:dx + nx]
                dW[:, :, dz, dy, dx] = np.einsum("ozyx,izyx->oi", gout, sl)
    return dW, gout.sum(axis=(1, 2, 3))


def soft(z, theta):
    """Complex soft threshold tau_theta (Algorithm 1; sgn z = z/|z|, 0 at 0)."""
    mag = np.abs(z)
    return np.where(mag > theta, z * (1.0 - theta / np.where(mag > 0, mag, 1.0)), 0.0)


def forward(apply_A: Callable, apply_AH: Callable, y, params, layers: int, L: float):
    """Network output x and the cache of every layer's inputs for backward."""
    P = split_params(params, layers)
    y = np.asarray(y, dtype=np.complex128)
    sigma = float(np.abs(apply_AH(y)).max()) / L
    yn = y / sigma
    x = np.zeros_like(apply_AH(yn))
    cache = []
    for q in P:
        g = apply_AH(apply_A(x) - yn)
        z = x - (q["eta"] / L) * g
        s = soft(z, q["theta"])
        sc = np.stack([s.real, s.imag])
        h = conv3d(sc, q["W1"], q["b1"])
        r = conv3d(np.maximum(h, 0.0), q["W2"], q["b2"])
        cache.append(dict(x=x, g=g, z=z, s=s, h=h))
        x = s + (r[0] + 1j * r[1])
    return sigma * x, dict(layers=cache, sigma=sigma, L=L)


def backward(apply_A: Callable, apply_AH: Callable, params, layers: int, cache, grad_x):
    """Gradient of a real loss with respect to the flat parameters, given its
    gradient grad_x = dLoss/dRe x + i dLoss/dIm x at the output."""
    P = split_params(params, layers)
    sigma = cache["sigma"]
    gx = sigma * np.asarray(grad_x, dtype=np.complex128)   # d/d x_L
    grads = [None] * layers
    for l in reversed(range(layers)):
        q, c = P[l], cache["layers"][l]
        # residual conv block
        go = np.stack([gx.real, gx.imag])
        a = np.maximum(c["h"], 0.0)
        dW2, db2 = conv3d_weight_grad(go, a)
        gh = conv3d_transpose(go, q["W2"]) * (c["h"] > 0)
        sc = np.stack([c["s"].real, c["s"].imag])
        dW1, db1 = conv3d_weight_grad(gh, sc)
        gsc = conv3d_transpose(gh, q["W1"])
        gs = gx + (gsc[0] + 1j * gsc[1])
        # soft threshold: for |z| > theta, s = (|z| - theta) u with u = z/|z|
        z = c["z"]
        r = np.abs(z)
        act = r > q["theta"]
        rs = np.where(act, r, 1.0)
        u = np.where(act, z / rs, 0.0)
        ug = (np.conj(u) * gs).real
        gz = np.where(act, (1.0 - q["theta"] / rs) * gs + (q["theta"] / rs) * u * ug, 0.0)
        dtheta = -float(np.where(act, ug, 0.0).sum())
        # gradient step z = x - (eta / L) A^H (A x - y_n)
        L = cache["L"]
        deta = -float((np.conj(c["g"]) * gz).real.sum()) / L
        gx = gz - (q["eta"] / L) * apply_AH(apply_A(gz))
        grads[l] = np.concatenate([[deta, dtheta], dW1.ravel(), db1, dW2.ravel(), db2])
    return np.concatenate(grads)


def nmse_loss(x, x_true):
    """||x - x_true||^2 / ||x_true||^2 and its gradient (dRe + i dIm)."""
    x = np.asarray(x, dtype=np.complex128)
    x_true = np.asarray(x_true, dtype=np.complex128)
    den = float(np.vdot(x_true, x_true).real)
    d = x - x_true
    return float(np.vdot(d, d).real) / den, 2.0 * d / den


def init_params(layers: int, L: float, mu: float, rng, w_scale: float = 0.02):
    """eta_l = 1 (step 1/L), theta_l = mu (lambda = mu ||A^H y_n||_inf = mu L,
    so lambda / L = mu in the normalised units), small random convolution
    weights, zero biases.  (L is kept in the signature for symmetry with
    forward; the initial values do not depend on it.)"""
    p = []
    for _ in range(layers):
        W1 = w_scale * rng.standard_normal(C_HID * 2 * 27)
        W2 = w_scale * rng.standard_normal(2 * C_HID * 27)
        p.append(np.concatenate([[1.0, mu], W1, np.zeros(C_HID), W2, np.zeros(2)]))
    return np.concatenate(p)
