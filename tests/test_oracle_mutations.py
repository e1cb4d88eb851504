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


def test_time_gate_without_the_envelope_margin_is_caught(monkeypatch):
    """t0 at the earliest echo itself, without the three envelope widths."""
    plant(monkeypatch, "auto_t0", lambda g: math.floor((2.0 * g.z0 / g.c) * g.fs) / g.fs)
    assert_caught([(P.test_time_gate_holds_every_echo, "vol32")])


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


def test_maximal_set_by_smallest_magnitude_is_caught(monkeypatch):
    """Phi_max sorted the wrong way (the M weakest bins)."""
    def wrong(g, M):
        e, _ = SO.pulse_weights(g)
        return sorted(sorted(range(len(e)), key=lambda k: (e[k], k))[:M])
    plant(monkeypatch, "maximal_set", wrong)
    assert_caught([P.test_maximal_set_holds_the_largest_pulse_magnitudes])


def test_energy_draw_ignoring_the_weights_is_caught(monkeypatch):
    """Phi_nrg drawn uniformly among the bins with energy (q_k dropped)."""
    orig = SO.energy_subset
    plant(monkeypatch, "energy_subset",
          lambda weights, M, stream: orig([1 if v > 0 else 0 for v in weights], M, stream))
    assert_caught([P.test_energy_draw_follows_the_pulse_energy])


def test_equispaced_without_the_half_cell_is_caught(monkeypatch):
    """idx_i = k_lo + floor(i |C| / M): the points at the cells' left edges."""
    orig = SO.select_indices

    def wrong(g, strategy, M, per_position, seed):
        if strategy != SO.SEL_EQUISPACED:
            return orig(g, strategy, M, per_position, seed)
        k_lo, k_hi, _ = SO.candidate_band(g, M)
        i = np.arange(M, dtype=np.int64)
        idx = np.empty((g.S, M), dtype=np.int32)
        idx[:] = k_lo + (i * (k_hi - k_lo + 1)) // M
        return idx
    plant(monkeypatch, "select_indices", wrong)
    assert_caught([P.test_contiguous_is_centred_on_peak_and_equispaced_spread])


def test_fast_operator_gathering_the_neighbouring_bin_is_caught(monkeypatch):
    """The kept bin of (s, m) looked up one entry too far in the union
    (a searchsorted off by one), clamped to the union."""
    orig = SO.LateralFFTOperator.__init__

    def wrong(self, g, idx, workers=1):
        orig(self, g, idx, workers)
        self.u_of = np.minimum(self.u_of + 1, self.bins.size - 1)
    monkeypatch.setattr(SO.LateralFFTOperator, "__init__", wrong)
    assert_caught([(P.test_lateral_fft_operator_equals_dense, (5, 4, 6), O.SEL_RANDOM)])


def test_backtracking_with_the_test_inverted_is_caught(monkeypatch):
    """The step accepted when F exceeds the quadratic model (>= for <=)."""
    def wrong(apply_A, apply_AH, y, lam, L0, eta, iters, L_history=None):
        y = np.asarray(y, dtype=np.complex128)
        x_prev = np.zeros_like(np.asarray(apply_AH(y), dtype=np.complex128))
        gamma = x_prev.copy()
        beta, _ = SO.fista_momentum(iters)
        L = float(L0)

        def f(v):
            r = apply_A(v) - y
            return 0.5 * float(np.vdot(r, r).real)
        for k in range(iters):
            grad = apply_AH(apply_A(gamma) - y)
            fg = f(gamma)
            for _ in range(60):
                x = SO.soft_threshold(gamma - grad / L, lam / L)
                d = x - gamma
                q = fg + float(np.vdot(d, grad).real) + 0.5 * L * float(np.vdot(d, d).real)
                if f(x) >= q:
                    break
                L *= eta
            gamma = x + beta[k] * (x - x_prev)
            x_prev = x
            if L_history is not None:
                L_history.append(L)
        return x_prev
    plant(monkeypatch, "fista_backtracking", wrong)
    assert_caught([P.test_backtracking_without_backtracks_is_fista])


def test_resume_restarting_the_momentum_is_caught(monkeypatch):
    """A resumed FISTA run that restarts t at 1 instead of carrying t_{K+1}."""
    orig = SO.fista

    def wrong(apply_A, apply_AH, y, lam, L, iters, x0=None, history=None, resume=None,
              return_state=False):
        if resume is not None:
            resume = (resume[0], resume[1], 1.0)
        return orig(apply_A, apply_AH, y, lam, L, iters, x0=x0, history=history, resume=resume,
                    return_state=return_state)
    plant(monkeypatch, "fista", wrong)
    assert_caught([P.test_fista_resumed_from_its_state_equals_one_run])


# ---------------------------------------------------------- control ---

def test_unmutated_oracle_passes_the_same_pins():
    """Without a planted mistake every pin used above passes, so the
    failures above come from the mistakes."""
    assert failing([P.test_pulse_spectrum_is_fourier_integral_of_pulse,
                    P.test_pulse_alpha_gives_requested_bandwidth,
                    P.test_dense_A_equals_dft_of_time_domain_echo,
                    P.test_dense_A_with_directivity_equals_time_domain_echo,
                    P.test_single_scatterer_below_position_closed_form,
                    (P.test_time_gate_holds_every_echo, "vol32"),
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
                    P.test_contiguous_is_centred_on_peak_and_equispaced_spread,
                    P.test_maximal_set_holds_the_largest_pulse_magnitudes,
                    P.test_energy_draw_follows_the_pulse_energy,
                    P.test_backtracking_without_backtracks_is_fista,
                    P.test_fista_resumed_from_its_state_equals_one_run]) == []


# ------------------------------------------- Cramér-Rao bound oracle ---

import oracle.crb_oracle as CO  # noqa: E402
import tests.test_crb_oracle_pins as PC  # noqa: E402


def _jacobian(delay=lambda c: 2.0 / c, dlng_z_sign=1.0):
    """data_jacobian with the delay derivative's factor 2/c replaced by
    delay(c), or the sign of the directivity's depth derivative
    flipped: the two ways the paper's printed derivative can be misread."""
    def jac(g, idx, p, amp, phase, params=CO.PARAMS):
        idx = np.asarray(idx)
        M = idx.shape[1]
        s, m = np.divmod(np.arange(idx.size), M)
        f = g.bin_freq(idx[s, m])
        xs, ys = g.scan_xy()
        xs, ys = xs[s], ys[s]
        x1, y1, z1 = (float(v) for v in p)
        b = CO.scatterer_data(g, idx, p, amp, phase)
        R = np.sqrt((x1 - xs) ** 2 + (y1 - ys) ** 2 + z1 ** 2)
        k = delay(g.c)
        dtau = {"x": k * (x1 - xs) / R, "y": k * (y1 - ys) / R, "z": k * z1 / R}
        if g.theta > 0.0:
            w2 = (z1 * math.tan(g.theta)) ** 2
            r2 = (x1 - xs) ** 2 + (y1 - ys) ** 2
            dlng = {"x": -2.0 * (x1 - xs) / w2, "y": -2.0 * (y1 - ys) / w2,
                    "z": dlng_z_sign * 2.0 * r2 / (z1 ** 3 * math.tan(g.theta) ** 2)}
        else:
            dlng = {"x": 0.0 * R, "y": 0.0 * R, "z": 0.0 * R}
        cols = []
        for q in params:
            if q in "xyz":
                cols.append(b * (dlng[q] - 2j * np.pi * f * dtau[q]))
            elif q == "a":
                cols.append(b / amp)
            else:
                cols.append(1j * b)
        return np.stack(cols, axis=1)
    return jac


def test_unmutated_jacobian_copy_passes():
    """The copy used for the two mutations below, unmutated, passes the
    pins, so their failures come from the planted change."""
    mp = pytest.MonkeyPatch()
    try:
        mp.setattr(CO, "data_jacobian", _jacobian())
        assert failing([PC.test_jacobian_equals_finite_differences_of_the_data,
                        PC.test_single_ascan_depth_bound_is_the_delay_bound]) == []
    finally:
        mp.undo()


def test_crb_delay_derivative_with_c_over_2_is_caught(monkeypatch):
    """d tau / d x with c/2 where 2/c belongs (the printed form)."""
    monkeypatch.setattr(CO, "data_jacobian", _jacobian(delay=lambda c: 0.5 * c))
    assert_caught([PC.test_jacobian_equals_finite_differences_of_the_data])


def test_crb_directivity_depth_derivative_sign_is_caught(monkeypatch):
    monkeypatch.setattr(CO, "data_jacobian", _jacobian(dlng_z_sign=-1.0))
    assert_caught([PC.test_jacobian_equals_finite_differences_of_the_data])


def test_fisher_information_without_the_factor_2_is_caught(monkeypatch):
    orig = CO.fisher_information
    monkeypatch.setattr(CO, "fisher_information", lambda *a, **kw: 0.5 * orig(*a, **kw))
    assert_caught([PC.test_single_ascan_depth_bound_is_the_delay_bound])


def test_crb_from_the_inverted_diagonal_is_caught(monkeypatch):
    """1 / J_ii instead of (J^-1)_ii: ignores the coupling of depth and phase."""
    def wrong(g, idx, p, amp, phase, sigma2, params=CO.PARAMS):
        J = CO.fisher_information(g, idx, p, amp, phase, sigma2, params)
        c = np.full(3, np.nan)
        for i, q in enumerate(params):
            if q in "xyz":
                c["xyz".index(q)] = 1.0 / J[i, i]
        return c, J
    monkeypatch.setattr(CO, "crb", wrong)
    assert_caught([PC.test_single_ascan_depth_bound_is_the_delay_bound])


# ------------------------------------------------ Rademacher mixing ---

import oracle.mixing_oracle as XO  # noqa: E402
import tests.test_mixing_oracle_pins as PX  # noqa: E402


def test_mixing_matrix_with_transposed_index_is_caught(monkeypatch):
    """Xi[(k_u - k_m) mod Nt] instead of Xi[(k_m - k_u) mod Nt]."""
    def wrong(xi, kept, band, Nt):
        Xi = np.fft.fft(np.asarray(xi, dtype=np.float64))
        kept = np.asarray(kept, dtype=np.int64)
        band = np.asarray(band, dtype=np.int64)
        return Xi[(band[None, :] - kept[:, None]) % Nt] / Nt
    monkeypatch.setattr(XO, "mixing_matrix", wrong)
    assert_caught([PX.test_mixing_matrix_is_the_time_domain_definition,
                   PX.test_mixed_operator_is_the_time_domain_chain])


def test_mixing_matrix_without_1_over_Nt_is_caught(monkeypatch):
    orig = XO.mixing_matrix
    monkeypatch.setattr(XO, "mixing_matrix", lambda xi, kept, band, Nt: Nt * orig(xi, kept, band, Nt))
    assert_caught([PX.test_mixing_matrix_is_the_time_domain_definition, PX.test_no_mixing_is_plain_selection])


def test_mixing_over_the_nonnegative_half_spectrum_is_caught(monkeypatch):
    """The band-limited reading: only bins 0 .. Nt/2 of the A-scan enter
    the mixing, the negative frequencies dropped."""
    monkeypatch.setattr(XO, "full_band", lambda Nt: np.arange(0, Nt // 2 + 1, dtype=np.int64))
    assert_caught([PX.test_mixed_operator_is_the_time_domain_chain])


def test_mixed_adjoint_without_the_conjugate_is_caught(monkeypatch):
    def wrong(self, y):
        rb = np.einsum("smu,sm->su", self.Mix, np.asarray(y, dtype=np.complex128))
        return self.A_band.apply_AH(rb)
    monkeypatch.setattr(XO.MixedOperator, "apply_AH", wrong)
    assert_caught([PX.test_mixed_operator_equals_dense_and_is_adjoint])


# ------------------------------------------------- learned ISTA oracle ---

import oracle.lista_oracle as LO  # noqa: E402
import tests.test_lista_oracle_pins as PL  # noqa: E402


def test_conv3d_as_convolution_is_caught(monkeypatch):
    """The kernel flipped (a true convolution instead of the correlation)."""
    orig = LO.conv3d
    monkeypatch.setattr(LO, "conv3d", lambda u, W, b=None: orig(u, W[:, :, ::-1, ::-1, ::-1], b))
    assert_caught([PL.test_conv3d_equals_scipy_correlate])


def test_conv3d_transpose_with_unflipped_shift_is_caught(monkeypatch):
    """The adjoint convolution reading the same window as the forward."""
    def wrong(gout, W):
        cout, nz, ny, nx = gout.shape
        gp = np.zeros((cout, nz + 2, ny + 2, nx + 2))
        gp[:, 1:-1, 1:-1, 1:-1] = gout
        gin = np.zeros((W.shape[1], nz, ny, nx))
        for dz in range(3):
            for dy in range(3):
                for dx in range(3):
                    sl = gp[:, dz:dz + nz, dy:dy + ny, dx:dx + nx]
                    gin += np.einsum("oi,ozyx->izyx", W[:, :, dz, dy, dx], sl)
        return gin
    monkeypatch.setattr(LO, "conv3d_transpose", wrong)
    assert_caught([PL.test_conv3d_transpose_and_weight_grad_are_adjoints])


def test_lista_soft_threshold_without_the_phase_is_caught(monkeypatch):
    def wrong(z, theta):
        mag = np.abs(z)
        return np.where(mag > theta, mag - theta, 0.0).astype(np.complex128)
    monkeypatch.setattr(LO, "soft", wrong)
    assert_caught([PL.test_zero_prox_network_is_ista])


def test_lista_backward_without_the_normal_operator_is_caught(monkeypatch):
    """The gradient passed to the previous layer without the -(eta/L)
    A^H A term of the gradient step (apply_AH o apply_A treated as zero)."""
    orig = LO.backward

    def wrong(apply_A, apply_AH, params, layers, cache, grad_x):
        return orig(apply_A, lambda r: 0.0 * apply_AH(r), params, layers, cache, grad_x)
    monkeypatch.setattr(LO, "backward", wrong)
    assert_caught([PL.test_backward_matches_central_differences])


def test_unmutated_mixing_crb_and_lista_oracles_pass_the_same_pins():
    assert failing([PX.test_mixing_matrix_is_the_time_domain_definition,
                    PX.test_no_mixing_is_plain_selection,
                    PX.test_mixed_operator_is_the_time_domain_chain,
                    PX.test_mixed_operator_equals_dense_and_is_adjoint,
                    PC.test_jacobian_equals_finite_differences_of_the_data,
                    PC.test_single_ascan_depth_bound_is_the_delay_bound,
                    PL.test_conv3d_equals_scipy_correlate,
                    PL.test_conv3d_transpose_and_weight_grad_are_adjoints,
                    PL.test_zero_prox_network_is_ista,
                    PL.test_backward_matches_central_differences]) == []
