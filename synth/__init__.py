"""Seeded synthetic inputs: workload recipes, scatterer scenes and noise.

This package is the only code that the CUDA library's tests/bench and the
FP64 oracle both use.  It holds geometry parameters, random scene draws and
unit-variance noise only: none of the method's arithmetic (no operator, no
selection rule, no solver).  Scaling the noise to an SNR needs ||A x||, which
each caller computes with its own operator.

Workloads (the measured scenes stand in for the paper's steel specimen,
whose data are not available; shapes follow the paper's simulation setup of
Sec. VII-A / Table III, scaled to the sizes below):
  line2d  2-D pulse-echo line scan: 32 positions at 0.5 mm, 32 x 64 voxels
          (0.15 mm depth pitch from 10 mm), Nt = 256, M = 32 random bins per
          position, 3 unit-magnitude scatterers, 20 dB SNR, 200 iterations
  vol32   3-D: 32 x 32 scan at 0.5 mm, 32 x 32 x 128 voxels (10-29 mm),
          Nt = 512, M = 64 bins per position, 10 scatterers with U(0.5, 1)
          magnitudes and uniform phase, 20 dB SNR, 300 iterations
  vol64   3-D large: 64 x 64 scan, 64 x 64 x 256 voxels, Nt = 1024,
          M = 128, Bernoulli(1e-4) support, 30 dB SNR
All use a Gabor pulse with fc = 5 MHz, 70 % fractional bandwidth,
fs = 40 MHz, c = 5900 m/s and lambda = 0.05 ||A^H y||_inf.
"""
from __future__ import annotations

import math

import numpy as np

BASE = dict(dx=0.5e-3, dy=0.5e-3, z0=10e-3, c=5900.0, fs=40e6, fc=5e6,
            frac_bw=0.7, theta=0.0)

WORKLOADS = {
    "line2d": dict(BASE, Nx=32, Ny=1, Nz=64, dz=0.15e-3, Nt=256, M=32,
                   n_scatter=3, amp="unit", snr_db=20.0, iters=200, mu=0.05),
    "vol32": dict(BASE, Nx=32, Ny=32, Nz=128, dz=19e-3 / 128, Nt=512, M=64,
                  n_scatter=10, amp="uniform", snr_db=20.0, iters=300, mu=0.05),
    "vol64": dict(BASE, Nx=64, Ny=64, Nz=256, dz=0.15e-3, Nt=1024, M=128,
                  n_scatter=None, p_bernoulli=1e-4, amp="uniform",
                  snr_db=30.0, iters=300, mu=0.05),
}

GEOM_KEYS = ("Nx", "Ny", "dx", "dy", "Nz", "z0", "dz", "c", "fs", "Nt", "fc",
             "frac_bw", "theta")

# Learned unrolled ISTA: the vol32 geometry with M = 64 random bins, 16
# layers; training and evaluation scenes with 1-20 scatterers of U(0.5, 1)
# magnitude and uniform phase, SNR uniform in 10-30 dB.
LEARNED = dict(workload="vol32", layers=16, n_scatter=(1, 20), snr_db=(10.0, 30.0), amp="uniform")


# Serving mix: scenes of independent geometries, each drawn uniformly from
# scan grids {16, 32, 48, 64}^2, depths {64, 128, 256} and M {32, 64, 128}
# (0.5 mm pitch, 0.15 mm depth pitch from 10 mm); Nt is the larger of the
# record length that the line2d / vol32 / vol64 workloads pair with M
# (256 for 32 bins, 512 for 64, 1024 for 128) and the one they pair with the
# depth count (256 for 64 depths, 512 for 128, 1024 for 256).  Scenes: 10
# scatterers, U(0.5, 1) magnitudes and uniform phase, 20 dB SNR.
SERVING = dict(grids=(16, 32, 48, 64), depths=(64, 128, 256), Ms=(32, 64, 128), n_scatter=10,
               snr_db=20.0, iters=200)


# Cramer-Rao study: the simulation setup of Sec. VII-A's parameter table
# (50 x 50 scan at 0.5 mm, c = 5920 m/s, fs = 20 MHz, fc = 3.2 MHz, 30 deg
# directivity; its pulse-width entry is garbled, 65 % fractional bandwidth
# is the reading), Nt = 512, one scatterer 33.3 mm below the scan centre as
# in Sec. VI; n_f kept bins per position.
CRB = dict(params=dict(Nx=50, Ny=50, dx=0.5e-3, dy=0.5e-3, Nz=50, z0=29.6e-3, dz=0.15e-3, c=5920.0,
                       fs=20e6, Nt=512, fc=3.2e6, frac_bw=0.65, theta=math.radians(30.0)),
           pos=(12.25e-3, 12.25e-3, 33.3e-3), n_f=(1, 2, 4, 8, 16, 32), trials=50)


# Run-time sweep of one forward apply (the shapes of Sec. V's run-time
# figure): Nz = Nt over a ladder at the widest area scan the lateral FFT
# engine holds (64 x 64; the figure uses 100 x 100), and Nx = Ny over a
# ladder at Nz = 5 (Nt = 256).  M = max(1, Nt / 16) random bins per position
# (fewer where the band is narrower), one scene of 10 scatterers.
SWEEP = dict(nz_nt=(16, 32, 64, 128, 256, 512), nxy_at_nz=64, nxy=(8, 16, 24, 32, 40, 48, 56, 64), nz=5,
             nt_for_nxy=256)


def serving_classes():
    """All (grid, depth, M, Nt) classes of the serving mix."""
    out = []
    for n in SERVING["grids"]:
        for nz in SERVING["depths"]:
            for M in SERVING["Ms"]:
                nt = max({32: 256, 64: 512, 128: 1024}[M], {64: 256, 128: 512, 256: 1024}[nz])
                out.append((n, nz, M, nt))
    return out


def serving_params(cls):
    n, nz, M, nt = cls
    return dict(BASE, Nx=n, Ny=n, Nz=nz, dz=0.15e-3, Nt=nt)


def serving_draw(count, seed):
    """Class index of each of `count` scenes (uniform over the classes)."""
    rng = np.random.default_rng(seed)
    return rng.integers(0, len(serving_classes()), count)


def learned_draw(shape, seed):
    """One training / evaluation scene of the LEARNED recipe: (x, snr_db)."""
    rng = np.random.default_rng(seed + 7777)
    n = int(rng.integers(LEARNED["n_scatter"][0], LEARNED["n_scatter"][1] + 1))
    snr = float(rng.uniform(*LEARNED["snr_db"]))
    return scene(shape, n, LEARNED["amp"], seed=seed), snr


def geometry_params(name_or_dict):
    """Geometry fields of a workload (a dict usable by both sides)."""
    w = WORKLOADS[name_or_dict] if isinstance(name_or_dict, str) else name_or_dict
    return {k: w[k] for k in GEOM_KEYS}


def scene(shape, n_scatter=None, amp="uniform", seed=0, p_bernoulli=None,
          min_sep=0):
    """Sparse complex reflectivity x of shape (Nz, Ny, Nx), complex128.

    n_scatter distinct voxels drawn uniformly (or a Bernoulli(p) support when
    p_bernoulli is given); magnitudes 1 ("unit") or U(0.5, 1) ("uniform");
    phases U[0, 2 pi).  min_sep > 0 keeps every pair of scatterers at least
    that many voxels apart along some axis (Chebyshev distance)."""
    rng = np.random.default_rng(seed)
    Nz, Ny, Nx = shape
    V = Nz * Ny * Nx
    x = np.zeros(V, dtype=np.complex128)
    if p_bernoulli is not None:
        support = np.nonzero(rng.random(V) < p_bernoulli)[0]
    else:
        chosen = []
        tries = 0
        while len(chosen) < n_scatter:
            v = int(rng.integers(V))
            tries += 1
            if tries > 100000:
                raise RuntimeError("cannot place scatterers with min_sep")
            iz, rem = divmod(v, Ny * Nx)
            iy, ix = divmod(rem, Nx)
            ok = True
            for w in chosen:
                jz, r2 = divmod(w, Ny * Nx)
                jy, jx = divmod(r2, Nx)
                if w == v or max(abs(iz - jz), abs(iy - jy), abs(ix - jx)) < min_sep:
                    ok = False
                    break
            if ok:
                chosen.append(v)
        support = np.array(sorted(chosen), dtype=np.int64)
    n = support.size
    mag = np.ones(n) if amp == "unit" else rng.uniform(0.5, 1.0, n)
    phase = rng.uniform(0.0, 2.0 * math.pi, n)
    x[support] = mag * np.exp(1j * phase)
    return x.reshape(shape)


def rademacher(shape, seed=0):
    """Independent uniform draws from {-1, +1} (int8): the mixing sequences
    xi of Sec. III-A's random sampling."""
    rng = np.random.default_rng(seed)
    return (2 * rng.integers(0, 2, size=shape) - 1).astype(np.int8)


def unit_noise(shape, seed=0):
    """Circular complex Gaussian noise with E|n|^2 = 1, complex128."""
    rng = np.random.default_rng(seed)
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / math.sqrt(2.0)


def noise_scale(clean_energy: float, n_meas: int, snr_db: float) -> float:
    """Standard deviation sigma with sigma^2 = ||y_clean||^2 / (n_meas 10^(snr/10))."""
    return math.sqrt(clean_energy / (n_meas * 10.0 ** (snr_db / 10.0)))


def seeds(base: int):
    """Derived seeds of one run: scene, selection, noise, power iteration."""
    return dict(scene=base, select=base * 7919 + 1, noise=base * 104729 + 2,
                power=base * 1299709 + 3)
