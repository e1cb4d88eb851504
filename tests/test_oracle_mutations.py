"""Planted mistakes in the oracle (CPU only).

Each test swaps one oracle routine for a plausible wrong version of it (a
dropped factor, a flipped sign, an off-by-one index, a missing conjugate, a
transposed operand, the paper's garbled printed form where a reading was
taken) and checks that at least one of the oracle's pins in
test_oracle_pins.py then fails.  The pins are meant to fix every part of the
oracle by something other than the oracle itself; these tests show that they
do for the mistakes listed here.  The mistakes are planted with monkeypatch
in the oracle's own module, so they vanish after each test.
"""
import math

import numpy as np
import pytest

import oracle as O
import oracle.sfs_oracle as SO
import tests.test_oracle_pins as P


def plant(mp, name, fn):
    """Replace oracle routine `name` where the oracle calls it and where the
    pins call it."""
    mp.setattr(SO, name, fn)
    if hasattr(O, name):
        mp.setattr(O, name, fn)


def failing(pins):
    """Names of the pins (callables with their arguments) that fail."""
    out = []
    for pin in pins:
        fn, args = (pin[0], pin[1:]) if isinstance(pin, tuple) else (pin, ())
        try:
            fn(*args)
        except AssertionError:
            out.append(fn.__name__)
    return out


def assert_caught(pins):
    bad = failing(pins)
    assert bad, "no pin caught the planted mistake"


# ------------------------------------------------------------ pulse ---

def test_pulse_with_conjugated_carrier_is_caught(monkeypatch):
    def wrong(t, fc, alpha):
        t = np.asarray(t, dtype=np.float64)
        return np.exp(-(alpha * t) ** 2) * np.exp(-2j * np.pi * fc * t)
    plant(monkeypatch, "pulse_time", wrong)
    assert_caught([P.test_pulse_spectrum_is_fourier_integral_of_pulse,
                   P.test_dense_A_equals_dft_of_time_domain_echo])


def test_pulse_spectrum_without_its_scale_is_caught(monkeypatch):
    def wrong(f, fc, alpha):
        f = np.asarray(f, dtype=np.float64)
        return np.exp(-(math.pi * (f - fc) / alpha) ** 2)
    plant(monkeypatch, "pulse_spectrum", wrong)
    assert_caught([P.test_pulse_spectrum_is_fourier_integral_of_pulse,
                   P.test_dense_A_equals_dft_of_time_domain_echo])


def test_pulse_spectrum_mirrored_about_zero_is_caught(monkeypatch):
    def wrong(f, fc, alpha):
        f = np.asarray(f, dtype=np.float64)
        return (math.sqrt(math.pi) / alpha) * np.exp(-(math.pi * (f + fc) / alpha) ** 2)
    plant(monkeypatch, "pulse_spectrum", wrong)
    assert_caught([P.test_pulse_spectrum_is_fourier_integral_of_pulse,
                   P.test_pulse_alpha_gives_requested_bandwidth])


def test_pulse_alpha_without_the_log_factor_is_caught(monkeypatch):
    plant(monkeypatch, "pulse_alpha", lambda fc, frac_bw: math.pi * 0.5 * frac_bw * fc)
    assert_caught([P.test_pulse_alpha_gives_requested_bandwidth])


# ----------------------------------------- time of flight, directivity ---

def test_one_way_time_of_flight_is_caught(monkeypatch):
    """Both the dense A and the simulated echo call time_of_flight, so the
    echo pins cannot see this; the closed form below the transducer does."""
    plant(monkeypatch, "time_of_flight",
          lambda xs, ys, xv, yv, zv, c: (1.0 / c) * np.sqrt((xs - xv) ** 2 + (ys - yv) ** 2 + zv ** 2))
    assert_caught([P.test_dense_A_equals_dft_of_time_domain_echo,
                   P.test_single_scatterer_below_position_closed_form])


def test_dropped_directivity_is_caught(monkeypatch):
    plant(monkeypatch, "directivity",
          lambda xs, ys, xv, yv, zv, theta: np.ones(np.broadcast(xs, ys, xv, yv, zv).shape))
    assert_caught([P.test_dense_A_with_directivity_equals_time_domain_echo,
                   P.test_directivity_depends_on_the_angle_only])


def test_printed_directivity_form_is_caught(monkeypatch):
    """The form as printed, exp(-r^2 / (tan(theta) z^2)^2)."""
    def wrong(xs, ys, xv, yv, zv, theta):
        if theta == 0.0:
            return np.ones(np.broadcast(xs, ys, xv, yv, zv).shape)
        r2 = (xs - xv) ** 2 + (ys - yv) ** 2
        return np.exp(-r2 / (math.tan(theta) * zv ** 2) ** 2)
    plant(monkeypatch, "directivity", wrong)
    assert_caught([P.test_directivity_depends_on_the_angle_only])


# ------------------------------------------ dense operator and the DFT ---

def test_dense_A_without_the_time_gate_is_caught(monkeypatch):
    """A_rows evaluated as if the receive window started at t = 0."""
    import dataclasses
    orig = SO.A_rows
    plant(monkeypatch, "A_rows", lambda g, idx, rows: orig(dataclasses.replace(g, t0=0.0), idx, rows))
    assert_caught([P.test_dense_A_equals_dft_of_time_domain_echo])


def test_dft_with_the_wrong_sign_is_caught(monkeypatch):
    def wrong(b, k):
        n = np.arange(b.shape[-1])
        return np.exp(2j * np.pi * np.outer(np.asarray(k), n) / b.shape[-1]) @ b
    plant(monkeypatch, "dft_bins", wrong)
    assert_caught([P.test_dense_A_equals_dft_of_time_domain_echo])


def test_voxel_axes_swapped_is_caught(monkeypatch):
    """x and y voxel coordinates exchanged (on non-square grids)."""
    def wrong(self):
        v = np.arange(self.V)
        iz, rem = np.divmod(v, self.Nx * self.Ny)
        iy, ix = np.divmod(rem, self.Nx)
        return iy * self.dx, ix * self.dy, self.z0 + iz * self.dz
    monkeypatch.setattr(SO.Geometry, "voxel_xyz", wrong)
    assert_caught([P.test_lateral_shift_invariance,
                   (P.test_lateral_fft_operator_equals_dense, (5, 4, 6), O.SEL_RANDOM)])


# ----------------------------------------------- Toeplitz structure ---

def test_transposed_toeplitz_blocks_are_caught(monkeypatch):
    """Generator index (j - i) instead of (i - j) at every level."""
    def wrong(t, n):
        t = np.asarray(t)
        n = tuple(n)
        L = 2 * n[0] - 1
        if len(n) == 1:
            i = np.arange(n[0])
            return t[(i[None, :] - i[:, None]) % L]
        inner = [wrong(t[a], n[1:]) for a in range(L)]
        bs = inner[0].shape[0]
        out = np.zeros((n[0] * bs, n[0] * bs), dtype=t.dtype)
        for i in range(n[0]):
            for j in range(n[0]):
                out[i * bs:(i + 1) * bs, j * bs:(j + 1) * bs] = inner[(j - i) % L]
        return out
    plant(monkeypatch, "multilevel_toeplitz", wrong)
    assert_caught([P.test_multilevel_toeplitz_matches_printed_example])


# -------------------------------------------------- fast transform ---

def test_adjoint_without_the_conjugate_is_caught(monkeypatch):
    """The adjoint depth sum with Hhat instead of conj(Hhat) (an operand
    transposed but not conjugated)."""
    orig = SO.LateralFFTOperator._depth_sum

    def wrong(self, spec, adjoint):
        if not adjoint:
            return orig(self, spec, adjoint)
        saved = self.Hhat
        self.Hhat = np.conj(saved)
        try:
            return orig(self, spec, True)
        finally:
            self.Hhat = saved
    monkeypatch.setattr(SO.LateralFFTOperator, "_depth_sum", wrong)
    assert_caught([P.test_adjoint_identity_structured,
                   (P.test_lateral_fft_operator_equals_dense, (5, 4, 6), O.SEL_RANDOM)])


def test_padding_off_by_one_column_is_caught(monkeypatch):
    def wrong(self, planes):
        out = np.zeros(planes.shape[:-2] + (self.Ly, self.Lx), dtype=np.complex128)
        out[..., :self.g.Ny, 1:self.g.Nx + 1] = planes
        return out
    monkeypatch.setattr(SO.LateralFFTOperator, "_pad", wrong)
    assert_caught([(P.test_lateral_fft_operator_equals_dense, (5, 4, 6), O.SEL_RANDOM),
                   P.test_adjoint_identity_structured])


def test_generator_with_unsigned_offsets_is_caught(monkeypatch):
    """Lateral offsets taken as 0 .. 2N-2 instead of -(N-1) .. N-1 (the
    circular layout of Sec. IV-B read without its wrap)."""
    def wrong(g, k, iz):
        Lx, Ly = 2 * g.Nx - 1, 2 * g.Ny - 1
        DX = (np.arange(Lx) * g.dx)[None, :]
        DY = (np.arange(Ly) * g.dy)[:, None]
        z = g.z0 + iz * g.dz
        f = float(g.bin_freq(k))
        tau = SO.time_of_flight(DX, DY, 0.0, 0.0, z, g.c)
        gd = SO.directivity(DX, DY, 0.0, 0.0, z, g.theta)
        return g.fs * float(SO.pulse_spectrum(f, g.fc, g.alpha)) * gd * np.exp(-2j * np.pi * f * (tau - g.t0))
    plant(monkeypatch, "lateral_generator", wrong)
    assert_caught([(P.test_lateral_fft_operator_equals_dense, (5, 4, 6), O.SEL_RANDOM),
                   P.test_dense_lateral_blocks_are_2level_toeplitz_of_generators])


# --------------------------------------------------- solver and L ---

def test_soft_threshold_dropping_the_phase_is_caught(monkeypatch):
    def wrong(z, alpha):
        mag = np.abs(np.asarray(z, dtype=np.complex128))
        return np.maximum(mag - alpha, 0.0).astype(np.complex128)
    plant(monkeypatch, "soft_threshold", wrong)
    assert_caught([P.test_soft_threshold_special_cases])


def test_threshold_not_divided_by_L_is_caught(monkeypatch):
    """x_k = tau_lam(...) instead of tau_{lam/L}(...)."""
    orig = SO.fista
    plant(monkeypatch, "fista",
          lambda apply_A, apply_AH, y, lam, L, iters, **kw: orig(apply_A, apply_AH, y, lam * L, L, iters, **kw))
    assert_caught([P.test_fista_zero_when_lambda_at_least_max_correlation])


def test_momentum_one_step_late_is_caught(monkeypatch):
    """beta_k taken from t_{k+1}, t_{k+2} (the off-by-one of the printed
    momentum index)."""
    orig = SO.fista_momentum

    def wrong(iters, t1=1.0):
        b, _ = orig(iters + 1, t1)
        _, t_end = orig(iters, t1)
        return b[1:], t_end
    plant(monkeypatch, "fista_momentum", wrong)
    assert_caught([P.test_soft_threshold_special_cases])


def test_power_iteration_returning_sigma_is_caught(monkeypatch):
    orig = SO.power_iteration
    plant(monkeypatch, "power_iteration",
          lambda *a, **kw: (math.sqrt(orig(*a, **kw)[0]), orig(*a, **kw)[1]))
    assert_caught([P.test_power_iteration_matches_svd_and_frobenius_bounds])


# --------------------------------------------- selection and the band ---

def test_band_in_power_instead_of_amplitude_is_caught(monkeypatch):
    """The band rungs read as power decibels (10^(-b/10))."""
    def wrong(g, M):
        k = np.arange(g.Nt // 2 + 1)
        mag = np.abs(SO.pulse_spectrum(g.bin_freq(k), g.fc, g.alpha))
        for b in SO.BAND_LADDER_DB:
            inside = np.nonzero(mag >= mag.max() * 10.0 ** (-b / 10.0))[0]
            if inside.size >= M:
                return int(inside[0]), int(inside[-1]), b
        raise ValueError("band too narrow")
    plant(monkeypatch, "candidate_band", wrong)
    assert_caught([(P.test_band_matches_closed_form_width, "vol32"), P.test_band_sizes_of_workloads])


def test_fisher_yates_never_drawing_the_last_candidate_is_caught(monkeypatch):
    def wrong(n_cand, M, stream):
        perm = list(range(n_cand))
        for i in range(M):
            u = stream.next()
            j = i + (((u >> 32) * (n_cand - i - 1)) >> 32)
            perm[i], perm[j] = perm[j], perm[i]
        return sorted(perm[:M])
    plant(monkeypatch, "random_subset", wrong)
    assert_caught([P.test_random_subset_uniform_chi_square])


def test_splitmix64_with_a_wrong_constant_is_caught(monkeypatch):
    """One hexadecimal digit of the first finaliser multiplier changed."""
    mask = (1 << 64) - 1

    def wrong(self):
        self.state = (self.state + SO._GOLDEN) & mask
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B8) & mask
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & mask
        return z ^ (z >> 31)
    monkeypatch.setattr(SO.SplitMix64, "next", wrong)
    assert_caught([P.test_splitmix64_matches_published_outputs])


def test_contiguous_block_off_centre_is_caught(monkeypatch):
    """The contiguous block started at the peak bin instead of centred on it."""
    orig = SO.select_indices

    def wrong(g, strategy, M, per_position, seed):
        if strategy != SO.SEL_CONTIGUOUS:
            return orig(g, strategy, M, per_position, seed)
        k_lo, k_hi, _ = SO.candidate_band(g, M)
        kstar = int(math.floor(g.fc * g.Nt / g.fs + 0.5))
        start = min(max(kstar, k_lo), k_hi - M + 1)
        idx = np.empty((g.S, M), dtype=np.int32)
        idx[:] = np.arange(start, start + M)
        return idx
    plant(monkeypatch, "select_indices", wrong)
    assert_caught([P.test_contiguous_is_centred_on_peak_and_equispaced_spread])


# ---------------------------------------------------------- control ---

def test_unmutated_oracle_passes_the_same_pins():
    """Without a planted mistake every pin used above passes, so the
    failures above come from the mistakes."""
    assert failing([P.test_pulse_spectrum_is_fourier_integral_of_pulse,
                    P.test_pulse_alpha_gives_requested_bandwidth,
                    P.test_dense_A_equals_dft_of_time_domain_echo,
                    P.test_dense_A_with_directivity_equals_time_domain_echo,
                    P.test_single_scatterer_below_position_closed_form,
                    P.test_directivity_depends_on_the_angle_only,
                    P.test_lateral_shift_invariance,
                    P.test_multilevel_toeplitz_matches_printed_example,
                    P.test_dense_lateral_blocks_are_2level_toeplitz_of_generators,
                    (P.test_lateral_fft_operator_equals_dense, (5, 4, 6), O.SEL_RANDOM),
                    P.test_adjoint_identity_structured,
                    P.test_soft_threshold_special_cases,
                    P.test_fista_zero_when_lambda_at_least_max_correlation,
                    P.test_power_iteration_matches_svd_and_frobenius_bounds,
                    (P.test_band_matches_closed_form_width, "vol32"),
                    P.test_band_sizes_of_workloads,
                    P.test_random_subset_uniform_chi_square,
                    P.test_splitmix64_matches_published_outputs,
                    P.test_contiguous_is_centred_on_peak_and_equispaced_spread]) == []
