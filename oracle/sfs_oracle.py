"""FP64 CPU oracle for the sub-sampled Fourier SAFT operator, its adjoint,
FISTA with complex soft thresholding and the power-iteration Lipschitz bound.

TEST INFRASTRUCTURE ONLY.  This package is the independent checker of the
CUDA library.  Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s
CPU-baseline and reference legs may import it, plus the two checks bench.py
reports beside its studies, outside every timed region: the index sets of
the strategy study compared with the oracle's bit for bit, and the precision
study's errors against FP64.  The product library never
imports, links or executes anything under ``oracle/``, and nothing here
imports the product library.  The only code the two sides share is the
seeded input generator package ``synth`` (scenes, noise), which holds none
of the method's arithmetic.

Everything is plain numpy in float64 / complex128.  Each function cites the
passage of Kirchhof et al., "Frequency Sub-Sampling of Ultrasound
Non-Destructive Measurements: Acquisition, Reconstruction and Performance"
(arXiv 2012.04534) that it follows.  Where the paper is silent or garbled
the reading taken is stated in the docstring.

Layouts (the reading of the conflicting vectorisation orders of Sec. II-A):
  * reflectivity x: complex [Nz][Ny][Nx], x fastest; voxel v = (iz*Ny+iy)*Nx+ix
  * measurements y: complex [S][M], scan position s = iy*Nx + ix, the M bins
    of a position in ascending order
  * dense operator A: row s*M + m, column v

Parity status of each function (what pins it, in tests/test_oracle_pins.py):
  pulse_spectrum      pinned: numerical Fourier integral of pulse_time
  dense_A / A_rows    pinned: DFT of the brute-force time-domain echo
                      simulation (time_domain_ascan), closed form below a
                      single scatterer, lateral shift invariance
  A_cols              pinned: DFT of the simulated echo of one unit
                      scatterer per column, equal to dense_A's columns
  multilevel_toeplitz pinned: the worked 2-level example printed in Sec. IV-B
  LateralFFTOperator  pinned: equal to dense_A / dense_A^H to 1e-12
  power_iteration     pinned: numpy SVD on tiny grids, Frobenius bounds
  fista_backtracking  pinned: with L0 >= ||A||^2 it never backtracks and equals
                      fista, L_k <= eta ||A||^2 and nondecreasing, the
                      Beck-Teboulle rate bound with eta ||A||^2
  fista               pinned: lambda >= ||A^H y||_inf gives 0, KKT
                      certificate of the LASSO optimum, Beck-Teboulle rate
                      bound, exact support recovery of isolated scatterers
  select_indices      pinned: invariants (distinct, sorted, inside the band,
                      count M), closed-form contiguous / equispaced sets,
                      chi-square uniformity of the random draw
  SplitMix64          pinned: the published first five outputs from state
                      1234567 (tests/golden/splitmix64_seed1234567.txt) and
                      the increment floor(2^64 / phi) in exact integers
"""
from __future__ import annotations

import dataclasses
import math
from typing import Callable, Optional

import numpy as np

# --------------------------------------------------------------------------
# Pulse and geometry (Sec. II-A; pulse model of Sec. VI)
# --------------------------------------------------------------------------

SEL_RANDOM = 0
SEL_CONTIGUOUS = 1
SEL_EQUISPACED = 2
SEL_MAXIMAL = 3
SEL_ENERGY = 4

BAND_LADDER_DB = (6.0, 10.0, 20.0, 40.0)


def pulse_alpha(fc: float, frac_bw: float) -> float:
    """Gaussian envelope rate alpha of h(t) = exp(-alpha^2 t^2 + j 2 pi fc t).

    Sec. VI gives the pulse form but its alpha values, (0.65 fc)^2 in Table
    III, do not have units of 1/s.  Reading: ``frac_bw`` is the -6 dB
    full amplitude bandwidth as a fraction of fc, and -6 dB is taken as the
    amplitude ratio 1/2.  |H(f)| = exp(-pi^2 (f-fc)^2 / alpha^2) falls to 1/2 at
    f - fc = BW/2, so alpha = pi (BW/2) / sqrt(ln 2).
    """
    half_bw = 0.5 * frac_bw * fc
    return math.pi * half_bw / math.sqrt(math.log(2.0))


def pulse_time(t, fc: float, alpha: float):
    """Analytic Gaussian pulse h(t) = exp(-alpha^2 t^2) exp(j 2 pi fc t) (Sec. VI,
    pulse model used for the CRB and the simulations; the envelope is real so
    this is already the analytic signal h^(a) of Sec. II-A, Eq. (1))."""
    t = np.asarray(t, dtype=np.float64)
    return np.exp(-(alpha * t) ** 2) * np.exp(2j * np.pi * fc * t)


def pulse_spectrum(f, fc: float, alpha: float):
    """H(f) = int h(t) exp(-j 2 pi f t) dt for the pulse above (Eq. (4) uses the
    Fourier transform H of the pulse): (sqrt(pi)/alpha) exp(-pi^2 (f-fc)^2/alpha^2)."""
    f = np.asarray(f, dtype=np.float64)
    return (math.sqrt(math.pi) / alpha) * np.exp(-(math.pi * (f - fc) / alpha) ** 2)


@dataclasses.dataclass
class Geometry:
    """Scan grid G_2D and voxel grid G_3D of Sec. II-A.

    Scan positions (n_x dx, n_y dy, 0); voxels share the lateral grid and sit
    at depth z0 + n_z dz.  Sec. II-A ties dz to the sampling rate; the
    frequency-domain model allows any dz (Sec. V-B), which the workloads use.
    ``t0`` is the start of the receive window; NaN selects the automatic
    gate of ``auto_t0``.  ``theta`` = 0 turns the directivity g off (g = 1).
    """
    Nx: int
    Ny: int
    dx: float
    dy: float
    Nz: int
    z0: float
    dz: float
    c: float
    fs: float
    Nt: int
    fc: float
    frac_bw: float
    t0: float = float("nan")
    theta: float = 0.0

    def __post_init__(self):
        if math.isnan(self.t0):
            self.t0 = auto_t0(self)

    @property
    def alpha(self) -> float:
        return pulse_alpha(self.fc, self.frac_bw)

    @property
    def S(self) -> int:
        return self.Nx * self.Ny

    @property
    def V(self) -> int:
        return self.Nx * self.Ny * self.Nz

    def bin_freq(self, k):
        """Frequency of DFT bin k, f_k = k fs / Nt (0 <= k <= Nt/2)."""
        return np.asarray(k, dtype=np.float64) * self.fs / self.Nt

    def scan_xy(self):
        """Lateral coordinates of all S scan positions, s = iy*Nx + ix."""
        iy, ix = np.divmod(np.arange(self.S), self.Nx)
        return ix * self.dx, iy * self.dy

    def voxel_xyz(self):
        """Coordinates of all V voxels, v = (iz*Ny + iy)*Nx + ix."""
        v = np.arange(self.V)
        iz, rem = np.divmod(v, self.Nx * self.Ny)
        iy, ix = np.divmod(rem, self.Nx)
        return ix * self.dx, iy * self.dy, self.z0 + iz * self.dz


def auto_t0(g: Geometry) -> float:
    """Receive-window start when none is given.  The paper fixes t0 = 10 us for
    its own geometry (Table III); reading for other depths: the last sample
    instant at or before the earliest echo minus three envelope widths,
    t0 = floor((2 z0 / c - 3/alpha) fs) / fs."""
    alpha = pulse_alpha(g.fc, g.frac_bw)
    return math.floor((2.0 * g.z0 / g.c - 3.0 / alpha) * g.fs) / g.fs


def time_of_flight(xs, ys, xv, yv, zv, c: float):
    """tau = (2/c) sqrt((x - x_d)^2 + (y - y_d)^2 + z_d^2), Sec. II-A, Eq. (3)."""
    return (2.0 / c) * np.sqrt((xs - xv) ** 2 + (ys - yv) ** 2 + zv ** 2)


def directivity(xs, ys, xv, yv, zv, theta: float):
    """Transducer characteristic g of Sec. VI.  The printed form divides by
    (tan(theta) z_d^2)^2, which is not dimensionless; reading:
    g = exp(-r^2 / (z tan theta)^2), r the lateral distance.  theta = 0 gives
    g = 1 (the workloads run without directivity)."""
    if theta == 0.0:
        return np.ones(np.broadcast(xs, ys, xv, yv, zv).shape)
    r2 = (xs - xv) ** 2 + (ys - yv) ** 2
    return np.exp(-r2 / (zv * math.tan(theta)) ** 2)


# --------------------------------------------------------------------------
# Frequency band and the selection S (Sec. III-A, Table I)
# --------------------------------------------------------------------------

def candidate_band(g: Geometry, M: int):
    """Candidate bins C = [k_lo, k_hi] for the selection.

    Reading (the workloads ask for M bins "from the -6 dB band" although that
    band holds fewer than M bins): C = {0 <= k <= Nt/2 : |H(f_k)| >=
    10^(-b/20) max_k |H(f_k)|} for the first rung b of 6, 10, 20, 40 dB that
    holds at least M bins.  Returns (k_lo, k_hi, b); raises ValueError when
    even the 40 dB band is too narrow.
    """
    k = np.arange(g.Nt // 2 + 1)
    mag = np.abs(pulse_spectrum(g.bin_freq(k), g.fc, g.alpha))
    peak = mag.max()
    for b in BAND_LADDER_DB:
        inside = np.nonzero(mag >= peak * 10.0 ** (-b / 20.0))[0]
        if inside.size >= M:
            return int(inside[0]), int(inside[-1]), b
    raise ValueError("band too narrow for M=%d" % M)


_MASK64 = (1 << 64) - 1
_GOLDEN = 0x9E3779B97F4A7C15


class SplitMix64:
    """SplitMix64 (Steele, Lea and Flood, OOPSLA 2014; the 64-bit finaliser
    constants of Vigna's public-domain splitmix64), written in Python integers.
    The paper draws its random subsets without naming a generator; reading:
    this counter-based generator, implemented independently on each side."""

    def __init__(self, state: int):
        self.state = state & _MASK64

    def next(self) -> int:
        self.state = (self.state + _GOLDEN) & _MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK64
        return z ^ (z >> 31)


def random_subset(n_cand: int, M: int, stream: SplitMix64):
    """Uniform M-subset of range(n_cand) by a partial Fisher-Yates shuffle,
    returned ascending (Phi_rnd of Sec. III-A: uniform over all subsets of
    size n_f).  Draw j = i + floor(hi32(u) * (n_cand - i) / 2^32)."""
    perm = list(range(n_cand))
    for i in range(M):
        u = stream.next()
        j = i + (((u >> 32) * (n_cand - i)) >> 32)
        perm[i], perm[j] = perm[j], perm[i]
    return sorted(perm[:M])


def pulse_weights(g: Geometry):
    """Relative pulse magnitudes e_k = |H(f_k)| / max |H| =
    exp(-(pi (f_k - fc) / alpha)^2) of the bins k = 0..Nt/2 (the analytic
    pulse has no energy at negative frequencies), and the integer weights
    floor(2^24 e_k) of the energy-based draw."""
    e = []
    for k in range(g.Nt // 2 + 1):
        a = math.pi * (k * g.fs / g.Nt - g.fc) / g.alpha
        e.append(math.exp(-a * a))
    return e, [int(math.floor(v * 16777216.0)) for v in e]


def maximal_set(g: Geometry, M: int):
    """J_M of Sec. III-A (Phi_max): the M bins with the largest |hat h_n|,
    ties to the lower bin, ascending."""
    e, _ = pulse_weights(g)
    if M > len(e):
        raise ValueError("M exceeds the Nt/2 + 1 bins")
    return sorted(sorted(range(len(e)), key=lambda k: (-e[k], k))[:M])


def energy_subset(weights, M: int, stream: "SplitMix64"):
    """Random energy-based draw of Sec. III-A (Phi_nrg): M bins drawn one by
    one with probability proportional to the pulse energy q_i = |hat h_i| /
    ||hat h||_1 among the bins not yet drawn (drawn bins get weight 0 and the
    rest is renormalised).  Reading: integer weights floor(2^24 |H| / max|H|)
    and, per draw, r = floor(u W / 2^64) for the next 64-bit u and the
    remaining total W; the bin whose cumulative weight first exceeds r is
    drawn.  Returned ascending."""
    w = list(weights)
    if sum(1 for v in w if v > 0) < M:
        raise ValueError("fewer than M bins carry pulse energy")
    out = []
    for _ in range(M):
        W = sum(w)
        r = (stream.next() * W) >> 64
        c = 0
        for k, v in enumerate(w):
            c += v
            if c > r:
                out.append(k)
                w[k] = 0
                break
    return sorted(out)


def select_indices(g: Geometry, strategy: int, M: int, per_position: bool,
                   seed: int):
    """Selected bin indices idx[S][M] (int32, ascending per position).

    * RANDOM: uniform M-subset of the band C (Phi_rnd, Sec. III-A, without
      the mixing Sigma), drawn per position (Phi_rnd,f of Table I) from the
      stream seeded with seed XOR (s * 0x9E3779B97F4A7C15), or once with
      s = 0 and shared (Kronecker case of Sec. III-A) if not per_position.
    * CONTIGUOUS: M adjacent bins centred on round(fc Nt / fs), clamped into C.
    * EQUISPACED: idx_i = k_lo + floor((2i+1)|C| / (2M)).
    The last two are not in the paper; they are the workloads' comparison
    strategies, shared by all positions.
    * MAXIMAL: Phi_max (Sec. III-A), the M bins of largest pulse magnitude,
      shared by all positions.
    * ENERGY: Phi_nrg, or Phi_nrg,f when per_position (Sec. III-A, Table I),
      drawn by energy_subset from the same per-position streams as RANDOM.
    MAXIMAL and ENERGY draw from all bins 0..Nt/2, not from the band C.
    """
    S = g.S
    idx = np.empty((S, M), dtype=np.int32)
    if strategy == SEL_MAXIMAL:
        idx[:] = maximal_set(g, M)
        return idx
    if strategy == SEL_ENERGY:
        _, w = pulse_weights(g)
        rows = S if per_position else 1
        for s in range(rows):
            idx[s] = energy_subset(w, M, SplitMix64(seed ^ ((s * _GOLDEN) & _MASK64)))
        if not per_position:
            idx[:] = idx[0]
        return idx
    k_lo, k_hi, _ = candidate_band(g, M)
    n_cand = k_hi - k_lo + 1
    if strategy == SEL_RANDOM:
        rows = S if per_position else 1
        for s in range(rows):
            stream = SplitMix64(seed ^ ((s * _GOLDEN) & _MASK64))
            idx[s] = [k_lo + c for c in random_subset(n_cand, M, stream)]
        if not per_position:
            idx[:] = idx[0]
    elif strategy == SEL_CONTIGUOUS:
        # k* = round(fc Nt / fs) in integer arithmetic (round half up)
        kstar = int(math.floor(g.fc * g.Nt / g.fs + 0.5))
        start = min(max(kstar - M // 2, k_lo), k_hi - M + 1)
        idx[:] = np.arange(start, start + M)
    elif strategy == SEL_EQUISPACED:
        i = np.arange(M, dtype=np.int64)
        idx[:] = k_lo + ((2 * i + 1) * n_cand) // (2 * M)
    else:
        raise ValueError("unknown strategy %d" % strategy)
    return idx


# --------------------------------------------------------------------------
# Dense operator (Eq. (4), (8), (10), (11))
# --------------------------------------------------------------------------

def A_rows(g: Geometry, idx, rows):
    """Rows of the dense operator A = Phi H for Sigma = I.

    A[(s,m), v] = fs g(s,v) H(f_k) exp(-j 2 pi f_k (tau(s,v) - t0)), k = idx[s,m].
    This is Eq. (4) (frequency-domain echo of one scatterer) evaluated at the
    kept DFT bins: the unnormalised DFT e^{-j 2 pi k n / Nt} of the samples
    h(t0 + n/fs - tau) equals fs H(f_k) e^{-j 2 pi f_k (tau - t0)} up to the
    spectral aliasing of Sec. II-A's discussion, which the test against
    ``time_domain_ascan`` bounds.  ``rows`` are flat indices s*M + m.
    """
    rows = np.asarray(rows, dtype=np.int64)
    M = idx.shape[1]
    s, m = np.divmod(rows, M)
    k = idx[s, m].astype(np.float64)
    f = g.bin_freq(k)[:, None]
    xs, ys = g.scan_xy()
    xv, yv, zv = g.voxel_xyz()
    xs = xs[s][:, None]
    ys = ys[s][:, None]
    tau = time_of_flight(xs, ys, xv[None], yv[None], zv[None], g.c)
    gd = directivity(xs, ys, xv[None], yv[None], zv[None], g.theta)
    amp = g.fs * pulse_spectrum(f, g.fc, g.alpha) * gd
    return amp * np.exp(-2j * np.pi * f * (tau - g.t0))


def A_cols(g: Geometry, idx, voxels):
    """Columns of the same dense A (Eq. (4) at the kept bins, Sigma = I):
    A[:, v] for the flat voxel indices ``voxels`` (v = (z Ny + y) Nx + x),
    shape (S*M, len(voxels)).  With these, (A^H y)[v] = sum_r conj(A[r, v])
    y[r] is computable voxel by voxel on grids whose dense A does not fit."""
    voxels = np.asarray(voxels, dtype=np.int64)
    M = idx.shape[1]
    rows = np.arange(idx.size)
    s, m = np.divmod(rows, M)
    k = idx[s, m].astype(np.float64)
    f = g.bin_freq(k)[:, None]
    xs, ys = g.scan_xy()
    xv, yv, zv = g.voxel_xyz()
    xs = xs[s][:, None]
    ys = ys[s][:, None]
    xv, yv, zv = xv[voxels][None], yv[voxels][None], zv[voxels][None]
    tau = time_of_flight(xs, ys, xv, yv, zv, g.c)
    gd = directivity(xs, ys, xv, yv, zv, g.theta)
    amp = g.fs * pulse_spectrum(f, g.fc, g.alpha) * gd
    return amp * np.exp(-2j * np.pi * f * (tau - g.t0))


def dense_A(g: Geometry, idx):
    """The whole dense A, shape (S*M, V).  Small geometries only."""
    return A_rows(g, idx, np.arange(idx.size))


def time_domain_ascan(g: Geometry, s: int, xv, yv, zv, amps, wraps: int = 2):
    """Brute-force A-scan of Eq. (2): samples n = 0..Nt-1 at t = t0 + n/fs of
    sum_d a_d g h^(a)(t - tau_d), folded with period Nt (the DFT sees the
    periodic extension), over wraps p = -wraps..wraps periods."""
    xs, ys = g.scan_xy()
    n = np.arange(g.Nt)
    b = np.zeros(g.Nt, dtype=np.complex128)
    for xd, yd, zd, ad in zip(np.atleast_1d(xv), np.atleast_1d(yv),
                              np.atleast_1d(zv), np.atleast_1d(amps)):
        tau = time_of_flight(xs[s], ys[s], xd, yd, zd, g.c)
        gd = directivity(xs[s], ys[s], xd, yd, zd, g.theta)
        for p in range(-wraps, wraps + 1):
            t = g.t0 + (n + p * g.Nt) / g.fs
            b += ad * gd * pulse_time(t - tau, g.fc, g.alpha)
    return b


def dft_bins(b, k):
    """Direct (not fast) unnormalised DFT sum_n b[n] e^{-j 2 pi k n / Nt} at bins k
    (the F of Phi = S F Sigma, Sec. II-B)."""
    Nt = b.shape[-1]
    n = np.arange(Nt)
    k = np.asarray(k)
    W = np.exp(-2j * np.pi * np.outer(k, n) / Nt)
    return W @ b


# --------------------------------------------------------------------------
# Multilevel Toeplitz structure (Sec. IV-B, Definition and Theorem 2)
# --------------------------------------------------------------------------

def multilevel_toeplitz(t, n):
    """d-level Toeplitz matrix T_{n,d}(t) by the recursive definition of
    Sec. IV-B: block (i, j) of the outer level is T_{(1 + (i - j) mod
    (2 n_1 - 1), m), d-1}, i.e. generator index (i - j) mod (2 n_1 - 1) in
    0-based terms; the innermost level is an ordinary Toeplitz matrix with
    entry (i, j) = t[(i - j) mod (2 n - 1)].  ``t`` has shape
    (2 n_1 - 1, ..., 2 n_d - 1)."""
    t = np.asarray(t)
    n = tuple(n)
    if len(n) == 1:
        L = 2 * n[0] - 1
        i = np.arange(n[0])
        return t[(i[:, None] - i[None, :]) % L]
    L = 2 * n[0] - 1
    inner = [multilevel_toeplitz(t[a], n[1:]) for a in range(L)]
    bs = inner[0].shape[0]
    out = np.zeros((n[0] * bs, n[0] * bs), dtype=t.dtype)
    for i in range(n[0]):
        for j in range(n[0]):
            out[i * bs:(i + 1) * bs, j * bs:(j + 1) * bs] = inner[(i - j) % L]
    return out


def lateral_generator(g: Geometry, k: int, iz: int):
    """Generating element h_{k,z}[dy, dx] of the 2-level Toeplitz block of A
    for bin k and depth index iz (Theorem 2, Sec. IV-B: the block depends only
    on the lateral offset between scan position and voxel).  Offsets
    d = -(N-1)..N-1 are stored at index d mod (2N - 1), the layout of the
    recursive definition.  Shape (2Ny-1, 2Nx-1)."""
    Lx, Ly = 2 * g.Nx - 1, 2 * g.Ny - 1
    dx_i = np.arange(Lx)
    dx_i = np.where(dx_i < g.Nx, dx_i, dx_i - Lx)        # signed offsets
    dy_i = np.arange(Ly)
    dy_i = np.where(dy_i < g.Ny, dy_i, dy_i - Ly)
    DX = (dx_i * g.dx)[None, :]
    DY = (dy_i * g.dy)[:, None]
    z = g.z0 + iz * g.dz
    f = float(g.bin_freq(k))
    tau = time_of_flight(DX, DY, 0.0, 0.0, z, g.c)
    gd = directivity(DX, DY, 0.0, 0.0, z, g.theta)
    amp = g.fs * float(pulse_spectrum(f, g.fc, g.alpha))
    return amp * gd * np.exp(-2j * np.pi * f * (tau - g.t0))


class LateralFFTOperator:
    """Matrix-free A and A^H by the fast transform of Sec. IV-B (Algorithm 2):
    zero-pad each depth plane to (2Ny-1) x (2Nx-1), 2-D FFT, multiply by the
    FFT of each generator and sum over depth, inverse 2-D FFT, crop, select.

    With Sigma = I the time-domain generators followed by the 1-D DFT and the
    selection of Algorithm 2 collapse to the frequency-domain generators of
    Eq. (4) evaluated only at the kept bins; ``lateral_generator`` builds
    those.  The adjoint is the composition beta = beta_H o beta_Phi of
    Sec. IV-B.  Pinned against ``dense_A``.

    ``workers`` > 1 runs independent pieces on that many threads: the
    generator planes of different bins, the FFTs of different planes, and the
    depth sums of different lateral wavenumbers.  Every output element is
    computed by the same operations as with one worker, so the results are
    identical; only the wall time changes.
    """

    def __init__(self, g: Geometry, idx, workers: int = 1):
        self.g = g
        self.idx = np.asarray(idx, dtype=np.int32)
        self.M = self.idx.shape[1]
        self.bins = np.unique(self.idx)                    # union U, ascending
        self.Lx, self.Ly = 2 * g.Nx - 1, 2 * g.Ny - 1
        self.workers = max(1, int(workers))
        self._pool = None
        # Hhat[u, z] = FFT2 of the generator for bin U[u], depth z
        self.Hhat = np.empty((self.bins.size, g.Nz, self.Ly, self.Lx),
                             dtype=np.complex128)

        def build(us):
            for u in us:
                k = int(self.bins[u])
                for iz in range(g.Nz):
                    self.Hhat[u, iz] = np.fft.fft2(lateral_generator(g, k, iz))
        self._chunks(self.bins.size, build)
        # for each kept (s, m): which union entry
        self.u_of = np.searchsorted(self.bins, self.idx)  # [S][M]

    def _chunks(self, n, fn):
        """fn(range) over a split of range(n): inline for one worker, else on
        the operator's thread pool (numpy releases the GIL in these calls)."""
        if self.workers == 1 or n < 2:
            fn(range(n))
            return
        if self._pool is None:
            from concurrent.futures import ThreadPoolExecutor
            self._pool = ThreadPoolExecutor(self.workers)
        parts = [range(int(c[0]), int(c[-1]) + 1)
                 for c in np.array_split(np.arange(n), min(n, 4 * self.workers)) if c.size]
        list(self._pool.map(fn, parts))

    def _fft2(self, planes, inverse=False):
        out = np.empty(planes.shape, dtype=np.complex128)
        f = np.fft.ifft2 if inverse else np.fft.fft2

        def run(r):
            out[r.start:r.stop] = f(planes[r.start:r.stop])
        self._chunks(planes.shape[0], run)
        return out

    def _depth_sum(self, spec, adjoint):
        """Forward: sum_z Hhat[u, z] spec[z]; adjoint: sum_u conj(Hhat[u, z])
        spec[u]; both per lateral wavenumber (a, b)."""
        U, Nz = self.Hhat.shape[:2]
        out = np.empty(((Nz if adjoint else U), self.Ly, self.Lx), dtype=np.complex128)

        def run(r):
            a = slice(r.start, r.stop)
            if adjoint:
                out[:, a] = np.einsum("uzab,uab->zab", np.conj(self.Hhat[:, :, a]), spec[:, a])
            else:
                out[:, a] = np.einsum("uzab,zab->uab", self.Hhat[:, :, a], spec[:, a])
        self._chunks(self.Ly, run)
        return out

    def _pad(self, planes):
        out = np.zeros(planes.shape[:-2] + (self.Ly, self.Lx), dtype=np.complex128)
        out[..., :self.g.Ny, :self.g.Nx] = planes
        return out

    def apply_A(self, x):
        """y = A x.  x: [Nz][Ny][Nx] (or flat V) -> y: [S][M]."""
        g = self.g
        x = np.asarray(x, dtype=np.complex128).reshape(g.Nz, g.Ny, g.Nx)
        xh = self._fft2(self._pad(x))                                # [Nz][Ly][Lx]
        yh = self._depth_sum(xh, adjoint=False)                      # sum over depth
        yk = self._fft2(yh, inverse=True)[:, :g.Ny, :g.Nx].reshape(self.bins.size, g.S)
        s = np.arange(g.S)[:, None]
        return yk[self.u_of, s]                                      # select

    def apply_AH(self, y):
        """x = A^H y.  y: [S][M] -> x: [Nz][Ny][Nx]."""
        g = self.g
        y = np.asarray(y, dtype=np.complex128).reshape(g.S, self.M)
        r = np.zeros((self.bins.size, g.S), dtype=np.complex128)
        s = np.broadcast_to(np.arange(g.S)[:, None], y.shape)
        np.add.at(r, (self.u_of, s), y)                              # beta_Phi
        rh = self._fft2(self._pad(r.reshape(-1, g.Ny, g.Nx)))        # [U][Ly][Lx]
        # adjoint of crop(ifft2(Hhat * fft2(pad(.)))): crop(ifft2(conj(Hhat) *
        # fft2(pad(.)))) since ifft2 = fft2^H / (Lx Ly)
        xh = self._depth_sum(rh, adjoint=True)
        return self._fft2(xh, inverse=True)[:, :g.Ny, :g.Nx]


# --------------------------------------------------------------------------
# Solver (Sec. IV-A, Algorithm 1) and sigma_max (Sec. IV-C)
# --------------------------------------------------------------------------

def soft_threshold(z, alpha: float):
    """tau_alpha(z)_i = max(|z_i| - alpha, 0) sgn(z_i) (Algorithm 1), with the
    complex sign read as z/|z| and 0 at z = 0."""
    z = np.asarray(z, dtype=np.complex128)
    mag = np.abs(z)
    scale = np.where(mag > alpha, 1.0 - alpha / np.where(mag > 0, mag, 1.0), 0.0)
    return z * scale


def fista_momentum(iters: int, t1: float = 1.0):
    """Momentum coefficients beta_k = (t_k - 1)/t_{k+1},
    t_{k+1} = (1 + sqrt(1 + 4 t_k^2))/2 (Algorithm 1), for k = 1..iters from
    t_1 (1 for a fresh start).  Returns (beta, t_{iters+1})."""
    t = float(t1)
    out = np.empty(iters)
    for k in range(iters):
        t_next = 0.5 * (1.0 + math.sqrt(1.0 + 4.0 * t * t))
        out[k] = (t - 1.0) / t_next
        t = t_next
    return out, t


def fista(apply_A: Callable, apply_AH: Callable, y, lam: float, L: float,
          iters: int, x0=None, history: Optional[list] = None, resume=None,
          return_state: bool = False):
    """FISTA (Algorithm 1) for min 1/2 ||A x - y||^2 + lam ||x||_1.

    Readings of Algorithm 1: the printed step gamma - 2 s beta(phi(gamma) - y)
    with s = 1/sigma^2 is read as the 1/L step of the 1/2-scaled LASSO with
    threshold lam/L, L >= sigma_max^2; the printed momentum index
    gamma_{k+1} = a_k + ... (a_k - a_{k-1}) is read as the standard
    x_k + beta_k (x_k - x_{k-1}) with x_k the iterate just computed.
      x_0 given, gamma_1 = x_0, t_1 = 1
      x_k      = tau_{lam/L}(gamma_k - A^H(A gamma_k - y)/L)
      gamma_k+1 = x_k + beta_k (x_k - x_{k-1})
    Returns x_K.  ``history`` (if a list) receives F(x_k) per iteration.
    The iteration's whole state after K steps is (gamma_{K+1}, x_K,
    t_{K+1}): with return_state the call returns (x_K, state), and
    ``resume=state`` continues from it in place of x0.
    """
    y = np.asarray(y, dtype=np.complex128)
    if resume is not None:
        gamma0, x_prev, t1 = resume
        gamma = np.array(gamma0, dtype=np.complex128)
        x_prev = np.array(x_prev, dtype=np.complex128)
    else:
        if x0 is None:
            x_prev = np.zeros_like(np.asarray(apply_AH(y), dtype=np.complex128))
        else:
            x_prev = np.array(x0, dtype=np.complex128)
        gamma = x_prev.copy()
        t1 = 1.0
    beta, t_end = fista_momentum(iters, t1)
    for k in range(iters):
        grad = apply_AH(apply_A(gamma) - y)
        x = soft_threshold(gamma - grad / L, lam / L)
        gamma = x + beta[k] * (x - x_prev)
        x_prev = x
        if history is not None:
            r = apply_A(x) - y
            history.append(0.5 * np.vdot(r, r).real + lam * np.abs(x).sum())
    if return_state:
        return x_prev, (gamma, x_prev, t_end)
    return x_prev


def fista_backtracking(apply_A: Callable, apply_AH: Callable, y, lam: float, L0: float,
                       eta: float, iters: int, L_history: Optional[list] = None):
    """FISTA with backtracking (Sec. IV-C, "Backtracking": a lower bound
    sigma_low^2 = L0 and a factor eta > 1 instead of sigma_max; the method of
    the cited Beck-Teboulle paper).  With f(x) = 1/2 ||A x - y||^2, F = f +
    lam ||x||_1 and p_L(g) = tau_{lam/L}(g - grad f(g) / L), step k takes the
    smallest i >= 0 such that L' = eta^i L_{k-1} satisfies
        F(p_L'(gamma_k)) <= Q_L'(p_L'(gamma_k), gamma_k),
        Q_L(x, g) = f(g) + Re<x - g, grad f(g)> + L/2 ||x - g||^2 + lam ||x||_1,
    then L_k = L', x_k = p_{L_k}(gamma_k) and the momentum of Algorithm 1.
    Returns x_K; ``L_history`` (if a list) receives L_k per iteration."""
    y = np.asarray(y, dtype=np.complex128)
    x_prev = np.zeros_like(np.asarray(apply_AH(y), dtype=np.complex128))
    gamma = x_prev.copy()
    beta, _ = fista_momentum(iters)
    L = float(L0)

    def f(v):
        r = apply_A(v) - y
        return 0.5 * float(np.vdot(r, r).real)

    for k in range(iters):
        grad = apply_AH(apply_A(gamma) - y)
        fg = f(gamma)
        while True:
            x = soft_threshold(gamma - grad / L, lam / L)
            d = x - gamma
            q = fg + float(np.vdot(d, grad).real) + 0.5 * L * float(np.vdot(d, d).real)
            if f(x) <= q:     # the l1 terms of F and Q are equal and cancel
                break
            L *= eta
        gamma = x + beta[k] * (x - x_prev)
        x_prev = x
        if L_history is not None:
            L_history.append(L)
    return x_prev


def lasso_objective(apply_A: Callable, y, lam: float, x):
    r = apply_A(x) - y
    return 0.5 * float(np.vdot(r, r).real) + lam * float(np.abs(x).sum())


def power_iteration(apply_A: Callable, apply_AH: Callable, shape, seed: int,
                    max_iter: int = 500, rtol: float = 1e-12):
    """Largest eigenvalue of A^H A (= sigma_max^2), by the power method.

    Sec. IV-C computes sigma_max by ARPACK (Arnoldi); reading: plain power
    iteration on A^H A from a seeded complex Gaussian start, stopped when the
    Rayleigh quotient ||A v||^2 (||v|| = 1) changes by less than rtol.
    Returns (sigma_max^2 estimate, iterations used)."""
    rng = np.random.default_rng(seed)
    v = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    v /= np.linalg.norm(v)
    est = 0.0
    for it in range(1, max_iter + 1):
        Av = apply_A(v)
        new = float(np.vdot(Av, Av).real)
        w = apply_AH(Av)
        v = w / np.linalg.norm(w)
        if it > 1 and abs(new - est) <= rtol * new:
            return new, it
        est = new
    return est, max_iter


def lambda_from_mu(apply_AH: Callable, y, mu: float) -> float:
    """lambda = mu ||beta_{Phi H}(y)||_inf, Sec. VII."""
    return mu * float(np.abs(apply_AH(y)).max())


def nmse(x_hat, x_true) -> float:
    """||x_hat - x_true||^2 / ||x_true||^2."""
    d = np.asarray(x_hat).ravel() - np.asarray(x_true).ravel()
    return float(np.vdot(d, d).real / np.vdot(x_true, x_true).real)
