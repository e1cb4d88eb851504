"""Helpers shared by the GPU parity tests: builds the library, makes both
sides' operators from one geometry dict, and compares complex arrays."""
import numpy as np

import oracle as O
import synth

GEOM_BASE = dict(dx=0.5e-3, dy=0.5e-3, z0=10e-3, c=5900.0, fs=40e6, fc=5e6, frac_bw=0.7,
                 theta=0.0)


def geom_params(**kw):
    p = dict(GEOM_BASE)
    p.update(kw)
    return p


def oracle_geometry(params):
    kw = {k: params[k] for k in synth.GEOM_KEYS if k in params}
    if "t0" in params:
        kw["t0"] = params["t0"]
    return O.Geometry(**kw)


def rel_err(a, b):
    a = np.asarray(a, dtype=np.complex128).ravel()
    b = np.asarray(b, dtype=np.complex128).ravel()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def crandn(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def ensure_built():
    from paper_2012_04534_gb300 import build
    return build.build()
