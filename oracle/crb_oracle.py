"""FP64 CPU oracle of the Cramer-Rao bound on the location of one scatterer
(Sec. VI, "Asymptotic performance").

TEST INFRASTRUCTURE ONLY, under the same rules as sfs_oracle (only tests/,
__graft_entry__.smoke() and bench.py's CPU legs may use it; it never imports
the product library).

Model.  One scatterer at the continuous position p = (x1, y1, z1) (z1 the
depth below the scan plane) with complex amplitude a e^{j phi}.  Its data at
the kept bins, Eq. (4) with Sigma = I (so Phi is the selection S):
    b[s, m] = a e^{j phi} fs H(f_k) g_s(p) exp(-j 2 pi f_k (tau_s(p) - t0)),
    k = idx[s, m],  tau_s = (2/c) R_s,  R_s = |p - (x_s, y_s, 0)|.
With white circular Gaussian noise of variance sigma^2 the Slepian-Bangs
Fisher information of u = (x1, y1, z1, a, phi) is (Eq. "fim")
    J = (2 / sigma^2) Re{ D^H D },  D = d b / d u^T,
and the bound on the location is the diagonal of the upper-left 3 x 3 block
of J^{-1} (the text computes that block by a Schur complement, which is the
block inverse written out).

Derivatives (Sec. VI), with the readings taken where the text is garbled:
    d b / d a   = b / a,    d b / d phi = j b,
    d b / d p   = b (d ln g / d p - j 2 pi f_k d tau / d p),
    d tau / d x1 = (2/c) (x1 - x_s) / R_s, likewise y1; d tau / d z1 = (2/c) z1 / R_s
        (the text prints c0/2; tau = 2 R / c gives 2/c),
    ln g = -r^2 / (z1 tan theta)^2, r^2 = (x1 - x_s)^2 + (y1 - y_s)^2 (the
        directivity reading of sfs_oracle.directivity), so
        d ln g / d x1 = -2 (x1 - x_s) / (z1 tan theta)^2 and
        d ln g / d z1 = 2 r^2 / (z1^3 tan^2 theta) (the printed z-derivative
        has a minus between the squares and no factor 2); theta = 0: g = 1.
`params` restricts u to a subset (a line scan cannot see y1, a single A-scan
neither x1 nor y1); excluded coordinates report NaN.

Parity status (tests/test_crb_oracle_pins.py): scatterer_data is pinned to
the dense operator's columns at voxel positions; data_jacobian to central
finite differences of scatterer_data; the bound to the closed-form delay
bound of a single A-scan, to its scaling in sigma^2 and a, and to its
monotonicity under adding measurements.
"""
from __future__ import annotations

import math

import numpy as np

from .sfs_oracle import Geometry, directivity, pulse_spectrum, time_of_flight

PARAMS = "xyzap"


def scatterer_data(g: Geometry, idx, p, amp: float, phase: float):
    """b of one scatterer at the continuous position p, flat [S*M] (row s*M + m)."""
    idx = np.asarray(idx)
    M = idx.shape[1]
    s, m = np.divmod(np.arange(idx.size), M)
    f = g.bin_freq(idx[s, m])
    xs, ys = g.scan_xy()
    xs, ys = xs[s], ys[s]
    x1, y1, z1 = (float(v) for v in p)
    tau = time_of_flight(xs, ys, x1, y1, z1, g.c)
    gd = directivity(xs, ys, x1, y1, z1, g.theta)
    return (amp * np.exp(1j * phase) * g.fs * pulse_spectrum(f, g.fc, g.alpha) * gd
            * np.exp(-2j * np.pi * f * (tau - g.t0)))


def data_jacobian(g: Geometry, idx, p, amp: float, phase: float, params: str = PARAMS):
    """D = d b / d u^T for u restricted to `params` (letters of "xyzap"), [S*M][len(params)]."""
    idx = np.asarray(idx)
    M = idx.shape[1]
    s, m = np.divmod(np.arange(idx.size), M)
    f = g.bin_freq(idx[s, m])
    xs, ys = g.scan_xy()
    xs, ys = xs[s], ys[s]
    x1, y1, z1 = (float(v) for v in p)
    b = scatterer_data(g, idx, p, amp, phase)
    R = np.sqrt((x1 - xs) ** 2 + (y1 - ys) ** 2 + z1 ** 2)
    dtau = {"x": (2.0 / g.c) * (x1 - xs) / R, "y": (2.0 / g.c) * (y1 - ys) / R,
            "z": (2.0 / g.c) * z1 / R}
    if g.theta > 0.0:
        w2 = (z1 * math.tan(g.theta)) ** 2
        r2 = (x1 - xs) ** 2 + (y1 - ys) ** 2
        dlng = {"x": -2.0 * (x1 - xs) / w2, "y": -2.0 * (y1 - ys) / w2,
                "z": 2.0 * r2 / (z1 ** 3 * math.tan(g.theta) ** 2)}
    else:
        dlng = {"x": 0.0 * R, "y": 0.0 * R, "z": 0.0 * R}
    cols = []
    for q in params:
        if q in "xyz":
            cols.append(b * (dlng[q] - 2j * np.pi * f * dtau[q]))
        elif q == "a":
            cols.append(b / amp)
        elif q == "p":
            cols.append(1j * b)
        else:
            raise ValueError(q)
    return np.stack(cols, axis=1)


def fisher_information(g: Geometry, idx, p, amp: float, phase: float, sigma2: float,
                       params: str = PARAMS):
    """J = (2 / sigma^2) Re{D^H D} over `params` (Eq. "fim")."""
    D = data_jacobian(g, idx, p, amp, phase, params)
    return (2.0 / sigma2) * np.real(D.conj().T @ D)


def crb(g: Geometry, idx, p, amp: float, phase: float, sigma2: float, params: str = PARAMS):
    """(c, J): c = [C_x, C_y, C_z], the diagonal of the location block of
    J^{-1} (m^2; NaN for coordinates outside `params`), and J over `params`."""
    J = fisher_information(g, idx, p, amp, phase, sigma2, params)
    Ji = np.linalg.inv(J)
    c = np.full(3, np.nan)
    for i, q in enumerate(params):
        if q in "xyz":
            c["xyz".index(q)] = Ji[i, i]
    return c, J
