"""FP64 CPU oracle of the compressed model with Rademacher mixing,
Phi_s = S_s F Sigma_s (Sec. II-B, Eq. "compressed_model"; Sec. III-A,
random sampling with Sigma_s = Diag{xi_s}, xi_s in {-1, 1}^Nt).

TEST INFRASTRUCTURE ONLY, under the same rules as sfs_oracle (only tests/,
__graft_entry__.smoke() and bench.py's CPU legs may use it; it never imports
the product library).

Reading.  Sigma_s acts on the time samples of the A-scan b_s, so one kept
coefficient depends on every bin of b_s.  The A-scan is taken band-limited
to the candidate band C of the selection (the bins the frequency-domain
model of Eq. (4) evaluates; outside C the pulse spectrum is negligible, in
the spirit of Sec. II-A's remark that the DFT is a valid proxy):
B_s[k] = (H a)_s at bin k for k in C, 0 elsewhere.  Then
    y_s = S_s F (xi_s . F^-1 B_s),
and, with Xi_s = F xi_s (F the unnormalised DFT, F^-1 = F^H / Nt),
    y_s[m] = (1/Nt) sum_{u in C} Xi_s[(k_m - k_u) mod Nt] B_s[k_u],
a per-position M x |C| mixing matrix applied to the band operator's data.
With xi_s = 1 the mixing is the plain selection.

Parity status (tests/test_mixing_oracle_pins.py): mixing_matrix is pinned
to the time-domain definition (numpy's inverse FFT, sign flips, FFT,
selection); MixedOperator to the dense product of those matrices with the
pinned dense A, to the unmixed operator for xi = 1, and to the adjoint
identity.
"""
from __future__ import annotations

import numpy as np

from .sfs_oracle import Geometry, LateralFFTOperator, A_rows


def mixing_matrix(xi, kept, band, Nt: int):
    """(1/Nt) Xi[(k_m - k_u) mod Nt] for one position: xi [Nt] of +-1, kept
    [M] and band [U] bin indices -> [M][U] complex."""
    Xi = np.fft.fft(np.asarray(xi, dtype=np.float64))
    kept = np.asarray(kept, dtype=np.int64)
    band = np.asarray(band, dtype=np.int64)
    return Xi[(kept[:, None] - band[None, :]) % Nt] / Nt


def mix_time_domain(B_band, xi, kept, band, Nt: int):
    """The definition itself: place the band coefficients in an Nt-bin
    spectrum, inverse DFT, multiply by xi, DFT, select the kept bins."""
    spec = np.zeros(Nt, dtype=np.complex128)
    spec[np.asarray(band)] = B_band
    b = np.fft.ifft(spec)
    return np.fft.fft(np.asarray(xi, dtype=np.float64) * b)[np.asarray(kept)]


class MixedOperator:
    """A_mix = Mix o A_band: A_band keeps every bin of `band` at every
    position (the lateral-FFT oracle of Sec. IV-B), Mix applies each
    position's mixing matrix.  idx: [S][M] kept bins, xi: [S][Nt] of +-1."""

    def __init__(self, g: Geometry, band, idx, xi):
        self.g = g
        self.band = np.asarray(band, dtype=np.int64)
        self.idx = np.asarray(idx, dtype=np.int64)
        self.xi = np.asarray(xi, dtype=np.float64)
        S = g.S
        self.A_band = LateralFFTOperator(g, np.tile(self.band.astype(np.int32), (S, 1)))
        self.Mix = np.stack([mixing_matrix(self.xi[s], self.idx[s], self.band, g.Nt) for s in range(S)])

    def apply_A(self, x):
        yb = self.A_band.apply_A(x)                                   # [S][U]
        return np.einsum("smu,su->sm", self.Mix, yb)

    def apply_AH(self, y):
        rb = np.einsum("smu,sm->su", self.Mix.conj(), np.asarray(y, dtype=np.complex128))
        return self.A_band.apply_AH(rb)


def dense_A_mixed(g: Geometry, band, idx, xi):
    """Dense A_mix, rows s*M + m: each position's mixing matrix times the
    dense rows of A at the band bins.  Small geometries only."""
    band = np.asarray(band, dtype=np.int64)
    idx = np.asarray(idx)
    S, M = idx.shape
    U = band.size
    full = A_rows(g, np.tile(band.astype(np.int32), (S, 1)), np.arange(S * U)).reshape(S, U, -1)
    out = np.empty((S * M, full.shape[2]), dtype=np.complex128)
    for s in range(S):
        out[s * M:(s + 1) * M] = mixing_matrix(xi[s], idx[s], band, g.Nt) @ full[s]
    return out
