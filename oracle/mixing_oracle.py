"""FP64 CPU oracle of the compressed model with Rademacher mixing,
Phi_s = S_s F Sigma_s (Sec. II-B, Eq. "compressed_model" and
"general_compression"; Sec. III-A, random sampling with Sigma_s =
Diag{xi_s}, xi_s in {-1, 1}^Nt).

TEST INFRASTRUCTURE ONLY, under the same rules as sfs_oracle (only tests/,
__graft_entry__.smoke() and bench.py's CPU legs may use it; it never imports
the product library).

Definition.  y_s = S_s F Sigma_s b_s with b_s the Nt time samples of A-scan s
(Eq. (2)).  Sigma_s acts on those samples, so one kept coefficient depends on
every DFT bin of b_s, not only on the bins near the pulse's centre frequency.
With B_s = F b_s (all Nt bins) and Xi_s = F xi_s (F the unnormalised DFT,
F^-1 = F^H / Nt), the product xi_s . b_s has the spectrum (1/Nt) Xi_s (*) B_s
(circular convolution), so
    y_s[m] = (1/Nt) sum_{k=0}^{Nt-1} Xi_s[(k_m - k) mod Nt] B_s[k].
B_s[k] at every bin comes from the frequency-domain model of Eq. (4): the
sampled A-scan is periodic in frequency with period fs, and the pulse
spectrum is centred on +fc, so bin k is evaluated at the frequency of its
signed index k' in (-Nt/2, Nt/2] (k' = k - Nt above Nt/2): the bins above
Nt/2 are the negative frequencies k fs/Nt - fs.  ``full_band`` lists those
signed indices and ``MixedOperator`` evaluates B_s on them with the pinned
lateral-FFT operator.

A restricted ``band`` (signed bins) may be passed to evaluate the same sum
over a subset of bins, the truncation whose error the tests measure.

Parity status (tests/test_mixing_oracle_pins.py): MixedOperator.apply_A is
pinned to the literal chain of the definition on brute-force echoes
(time_domain_ascan of Eq. (2), sign flips, direct DFT, selection);
mixing_matrix to numpy's transforms; MixedOperator to the dense product of
those matrices with the pinned dense A, to the unmixed operator for xi = 1,
and to the adjoint identity; the full mixing over all bins to unitarity.
"""
from __future__ import annotations

import numpy as np

from .sfs_oracle import Geometry, LateralFFTOperator, A_rows


def full_band(Nt: int):
    """Signed indices of all Nt DFT bins, ascending: -Nt/2 < k <= Nt/2 (bin
    k + Nt for negative k)."""
    return np.arange(-((Nt - 1) // 2), Nt // 2 + 1, dtype=np.int64)


def mixing_matrix(xi, kept, band, Nt: int):
    """(1/Nt) Xi[(k_m - k_u) mod Nt] for one position: xi [Nt] of +-1, kept
    [M] and band [U] (signed) bin indices -> [M][U] complex."""
    Xi = np.fft.fft(np.asarray(xi, dtype=np.float64))
    kept = np.asarray(kept, dtype=np.int64)
    band = np.asarray(band, dtype=np.int64)
    return Xi[(kept[:, None] - band[None, :]) % Nt] / Nt


def mix_time_domain(B_band, xi, kept, band, Nt: int):
    """The definition itself on spectral data: place the band coefficients in
    an Nt-bin spectrum, inverse DFT, multiply by xi, DFT, select the kept
    bins."""
    spec = np.zeros(Nt, dtype=np.complex128)
    spec[np.asarray(band) % Nt] = B_band
    b = np.fft.ifft(spec)
    return np.fft.fft(np.asarray(xi, dtype=np.float64) * b)[np.asarray(kept)]


class MixedOperator:
    """A_mix = Mix o A_band: A_band evaluates every bin of `band` (default:
    all Nt bins of the A-scan, ``full_band``) at every position with the
    lateral-FFT oracle of Sec. IV-B (``workers`` threads, identical results),
    and Mix applies each position's mixing matrix.  idx: [S][M] kept bins,
    xi: [S][Nt] of +-1."""

    def __init__(self, g: Geometry, idx, xi, band=None, workers: int = 1):
        self.g = g
        self.band = full_band(g.Nt) if band is None else np.asarray(band, dtype=np.int64)
        self.idx = np.asarray(idx, dtype=np.int64)
        self.xi = np.asarray(xi, dtype=np.float64)
        S = g.S
        self.A_band = LateralFFTOperator(g, np.tile(self.band.astype(np.int32), (S, 1)), workers=workers)
        self.Mix = np.stack([mixing_matrix(self.xi[s], self.idx[s], self.band, g.Nt) for s in range(S)])

    def apply_A(self, x):
        yb = self.A_band.apply_A(x)                                   # [S][U]
        return np.einsum("smu,su->sm", self.Mix, yb)

    def apply_AH(self, y):
        rb = np.einsum("smu,sm->su", self.Mix.conj(), np.asarray(y, dtype=np.complex128))
        return self.A_band.apply_AH(rb)


def dense_A_mixed(g: Geometry, idx, xi, band=None):
    """Dense A_mix, rows s*M + m: each position's mixing matrix times the
    dense rows of A at the band bins (default all Nt).  Small geometries
    only."""
    band = full_band(g.Nt) if band is None else np.asarray(band, dtype=np.int64)
    idx = np.asarray(idx)
    S, M = idx.shape
    U = band.size
    full = A_rows(g, np.tile(band.astype(np.int32), (S, 1)), np.arange(S * U)).reshape(S, U, -1)
    out = np.empty((S * M, full.shape[2]), dtype=np.complex128)
    for s in range(S):
        out[s * M:(s + 1) * M] = mixing_matrix(xi[s], idx[s], band, g.Nt) @ full[s]
    return out
