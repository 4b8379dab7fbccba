"""Pins for the FP64 oracle: checks against closed forms, library routines and brute force.

None of these re-type the oracle's own formulas: each compares the oracle with something the
mathematics or the physics fixes independently (numpy.fft, straight-ray traveltimes, energy
conservation, adjointness, Cholesky solves, shift invariance).  The mutation tests at the end
plant plausible mistakes in the oracle (on the CPU) and check that some pin catches each one.
"""

import math
import os

import numpy as np
import pytest
from scipy.ndimage import gaussian_filter1d

from oracle import lsm_oracle as O
from synth import linear_frequencies, ricker_spectrum, random_case, config_tiny

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _op(sv, shots=None):
    src = sv.src_ix if shots is None else sv.src_ix[shots]
    rec = sv.rec_ix if shots is None else sv.rec_ix[shots]
    return O.SplitStepOperator(sv.slowness, sv.dx, sv.dz, sv.freqs, sv.wavelet, src, rec)


def _envelope_peak(trace_w, omega, tmax, dt=2e-4):
    t = np.arange(0.0, tmax, dt)
    env = np.abs(np.exp(-1j * np.outer(t, omega)) @ trace_w)
    return t[np.argmax(env)]


# ---------------------------------------------------------------- transforms and wavelet


def test_dft_matches_numpy_fft():
    rng = np.random.default_rng(0)
    for nx in (8, 64, 96):
        u = rng.normal(size=(3, nx)) + 1j * rng.normal(size=(3, nx))
        np.testing.assert_allclose(u @ O.dft_matrix(nx).T, np.fft.fft(u, axis=-1), rtol=0,
                                   atol=1e-11 * nx)
        np.testing.assert_allclose(u @ O.idft_matrix(nx).T, np.fft.ifft(u, axis=-1), rtol=0,
                                   atol=1e-13 * nx)


def test_kx_axis_matches_fftfreq():
    for nx, dx in ((64, 10.0), (512, 8.0), (7, 3.0)):
        ref = 2 * math.pi * np.fft.fftfreq(nx, d=dx)
        kx = O.kx_axis(nx, dx)
        # fftfreq puts the Nyquist bin of an even nx on the negative side, as the oracle does
        np.testing.assert_allclose(kx, ref, rtol=1e-14, atol=1e-14)


def test_ricker_spectrum_is_fourier_transform_of_time_ricker():
    fp = 20.0
    dt = 1e-5
    t = np.arange(-0.25, 0.25 + dt / 2, dt)
    r = (1 - 2 * (math.pi * fp * t) ** 2) * np.exp(-((math.pi * fp * t) ** 2))
    f = np.array([1.0, 5.0, 12.5, 20.0, 33.3, 60.0])
    numeric = np.array([np.trapezoid(r * np.exp(-2j * math.pi * fi * t), t) for fi in f])
    np.testing.assert_allclose(ricker_spectrum(f, fp), numeric, rtol=1e-7, atol=1e-12)


# ---------------------------------------------------------------- one depth step


def _homogeneous_op(nx=64, nz=4, dx=10.0, dz=10.0, v=2000.0, freqs=(10.0, 25.0)):
    s = np.full((nz, nx), 1.0 / v)
    f = np.asarray(freqs, dtype=np.float64)
    return O.SplitStepOperator(s, dx, dz, f, ricker_spectrum(f), np.array([nx // 2]),
                               np.arange(nx)[None, :])


@pytest.mark.parametrize("k", [0, 1, 5, 31, 32, 40, 63])
def test_plane_wave_is_eigenvector_with_dispersion_phase(k):
    """Homogeneous medium: exp(i kx x) advances by exp(i kz dz), kz^2 = w^2/v^2 - kx^2."""
    nx, dx, dz, v = 64, 10.0, 10.0, 2000.0
    op = _homogeneous_op(nx=nx, dx=dx, dz=dz, v=v)
    x = np.arange(nx) * dx
    # physical wavenumber of grid mode k: the alias with the smallest |kx|
    kk = k if k < nx / 2 else k - nx
    kx = 2 * math.pi * kk / (nx * dx)
    u = np.exp(1j * kx * x)[None, :].repeat(op.nw, axis=0)
    out = op.propagate(u, 0)
    for iw, w in enumerate(op.omega):
        a = (w / v) ** 2 - kx ** 2
        lam = np.exp(1j * math.sqrt(a) * dz) if a >= 0 else np.exp(-math.sqrt(-a) * dz)
        np.testing.assert_allclose(out[iw], lam * u[iw], rtol=0, atol=1e-12)


def test_propagating_band_is_energy_preserving_in_heterogeneous_medium():
    sv = random_case(48, 6, 1, 3, seed=4)
    op = _op(sv)
    rng = np.random.default_rng(1)
    for j in range(op.nz):
        kmax = op.omega[:, None] * op.s.min()
        spec = rng.normal(size=(op.nw, op.nx)) + 1j * rng.normal(size=(op.nw, op.nx))
        spec[np.abs(op.kx)[None, :] >= 0.95 * kmax] = 0.0
        u = np.fft.ifft(spec, axis=-1)
        out = op.propagate(u, j)
        np.testing.assert_allclose(np.linalg.norm(out, axis=-1), np.linalg.norm(u, axis=-1),
                                   rtol=1e-12)


def test_step_adjoint_dot_product():
    sv = random_case(32, 5, 1, 4, seed=5)
    op = _op(sv)
    rng = np.random.default_rng(2)
    for j in range(op.nz):
        u = rng.normal(size=(op.nw, op.nx)) + 1j * rng.normal(size=(op.nw, op.nx))
        w = rng.normal(size=(op.nw, op.nx)) + 1j * rng.normal(size=(op.nw, op.nx))
        lhs = np.vdot(op.propagate(u, j), w)
        rhs = np.vdot(u, op.propagate_adjoint(w, j))
        assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


# ---------------------------------------------------------------- the operator A and A^T


def _dot_test_error(op, seed=3):
    rng = np.random.default_rng(seed)
    m = rng.normal(size=(op.nz, op.nx))
    d = rng.normal(size=(op.ns, op.nw, op.nrec)) + 1j * rng.normal(size=(op.ns, op.nw, op.nrec))
    lhs = O.real_dot(op.forward(m), d)
    rhs = O.real_dot(m, op.adjoint(d))
    return abs(lhs - rhs) / abs(lhs)


@pytest.mark.parametrize("case", [(32, 12, 3, 5), (64, 8, 2, 4), (24, 7, 4, 3)])
def test_dot_product_test_fp64(case):
    nx, nz, ns, nw = case
    op = _op(random_case(nx, nz, ns, nw, seed=nx + nz))
    assert _dot_test_error(op) < 1e-12


def test_dot_product_with_partial_receiver_spread():
    sv = random_case(32, 8, 3, 4, seed=11)
    rng = np.random.default_rng(0)
    rec = np.stack([np.sort(rng.choice(32, 20, replace=False)) for _ in range(3)])
    op = O.SplitStepOperator(sv.slowness, sv.dx, sv.dz, sv.freqs, sv.wavelet, sv.src_ix, rec)
    assert _dot_test_error(op) < 1e-12


def test_horner_equals_direct_sum_of_propagated_scatterers():
    """A m (Horner, bottom-up) == sum_j P_0...P_{j-1}(S_j m_j) evaluated term by term."""
    sv = random_case(16, 6, 2, 3, seed=7)
    op = _op(sv)
    m = sv.reflectivity
    shots = np.arange(op.ns)
    S = op.source_wavefield(shots)
    total = np.zeros((op.ns, op.nw, op.nx), dtype=complex)
    for j in range(op.nz):
        term = S[j] * m[j]
        for jj in range(j - 1, -1, -1):
            term = op.propagate(term, jj)
        total += term
    np.testing.assert_allclose(op.forward(m), op.record(total, shots), rtol=0,
                               atol=1e-12 * np.abs(total).max())


def test_point_diffractor_traveltime():
    """Homogeneous medium: the envelope of each trace peaks at the two-leg straight-ray time."""
    nx, nz, dx, dz, v = 128, 48, 10.0, 10.0, 2000.0
    f = linear_frequencies(5.0, 40.0, 64)
    xs, jd, xd = 40, 40, 64
    op = O.SplitStepOperator(np.full((nz, nx), 1 / v), dx, dz, f, ricker_spectrum(f),
                             np.array([xs]), np.arange(nx)[None, :])
    m = np.zeros((nz, nx))
    m[jd, xd] = 1.0
    d = op.forward(m)
    for xr in (20, 40, 64, 90, 110):
        tau = (math.hypot((xd - xs) * dx, jd * dz) + math.hypot((xd - xr) * dx, jd * dz)) / v
        tp = _envelope_peak(d[0, :, xr], op.omega, 1.5)
        assert abs(tp - tau) < 0.005 * tau, (xr, tau, tp)


def _vertical_times(op_cls=None):
    nx, nz, dx, dz = 256, 40, 10.0, 10.0
    f = linear_frequencies(5.0, 40.0, 64)
    vel = np.full((nz, nx), 2000.0)
    xx = np.arange(nx)
    vel[:, (xx >= 40) & (xx < 120)] = 1600.0
    vel = gaussian_filter1d(vel, 2, axis=1, mode="wrap")
    xs = np.array([80, 200])
    op = O.SplitStepOperator(1 / vel, dx, dz, f, ricker_spectrum(f), xs,
                             np.array([np.arange(nx)] * 2))
    m = np.zeros((nz, nx))
    m[30, :] = 1.0
    d = op.forward(m)
    out = []
    for i, x in enumerate(xs):
        t_ray = 2 * np.sum(1 / vel[:30, x]) * dz
        out.append((t_ray, _envelope_peak(d[i, :, x], op.omega, 1.0)))
    return out


def test_split_step_vertical_traveltime_in_laterally_varying_medium():
    """Zero-offset reflection time under a wide slow block equals 2 sum_j s(x, z_j) dz."""
    for t_ray, tp in _vertical_times():
        assert abs(tp - t_ray) < 0.01 * t_ray, (t_ray, tp)


def test_circular_shift_invariance_homogeneous():
    nx, nz = 64, 10
    f = linear_frequencies(5.0, 30.0, 6)
    s = np.tile((1.0 / np.linspace(1800, 2600, nz))[:, None], (1, nx))  # v(z): D_j == 1
    rng = np.random.default_rng(9)
    m = rng.normal(size=(nz, nx))
    shift = 11
    op_a = O.SplitStepOperator(s, 10.0, 10.0, f, ricker_spectrum(f), np.array([20]),
                               np.arange(nx)[None, :])
    op_b = O.SplitStepOperator(s, 10.0, 10.0, f, ricker_spectrum(f), np.array([20 + shift]),
                               np.arange(nx)[None, :])
    da = op_a.forward(m)
    db = op_b.forward(np.roll(m, shift, axis=1))
    np.testing.assert_allclose(db, np.roll(da, shift, axis=-1), rtol=0,
                               atol=1e-12 * np.abs(da).max())


# ---------------------------------------------------------------- solver


def _tiny_problem(seed=0, nx=8, nz=6, ns=3, nw=4):
    sv = random_case(nx, nz, ns, nw, seed=seed)
    op = _op(sv)
    d = op.forward(sv.reflectivity) + 0.05 * sv.noise()
    return op, d


def test_cg_matches_explicit_cholesky_solution():
    op, d = _tiny_problem()
    A = O.explicit_matrix(op)
    hess_norm = np.linalg.norm(np.real(A.conj().T @ A), 2)
    lam = 1e-2 * hess_norm
    m_chol = O.closed_form_solution(A, d, lam).reshape(op.nz, op.nx)
    m_cg, st = O.cg_window(op, np.arange(op.ns), d, lam, np.zeros((op.nz, op.nx)), 300,
                           tol=1e-13)
    assert st.rel_res <= 1e-13
    assert np.linalg.norm(m_cg - m_chol) <= 1e-9 * np.linalg.norm(m_chol)


def test_explicit_matrix_columns_match_operator():
    op, d = _tiny_problem(seed=1)
    A = O.explicit_matrix(op)
    rng = np.random.default_rng(4)
    m = rng.normal(size=(op.nz, op.nx))
    np.testing.assert_allclose(A @ m.ravel(), op.forward(m).ravel(), rtol=0,
                               atol=1e-12 * np.abs(A).max() * op.nz * op.nx)
    # A^T == Re A^H as a matrix
    np.testing.assert_allclose(np.real(A.conj().T @ d.ravel()), op.adjoint(d).ravel(), rtol=0,
                               atol=1e-11 * np.abs(d).max() * np.abs(A).max() * A.shape[0])


def test_warm_start_iterates_equal_textbook_cg_on_residual_system():
    """Eq. 11: CG from m_prev == m_prev + textbook CG on (H) dm = A^T(d - A m_prev) - lam m_prev."""
    op, d = _tiny_problem(seed=2)
    A = O.explicit_matrix(op)
    H = np.real(A.conj().T @ A)
    lam = 0.05 * np.linalg.norm(H, 2)
    H = H + lam * np.eye(H.shape[0])
    rng = np.random.default_rng(5)
    m_prev = rng.normal(size=(op.nz, op.nx))
    hist = []
    O.cg_window(op, np.arange(op.ns), d, lam, m_prev, 8, tol=0.0, history=hist)
    b = np.real(A.conj().T @ (d.ravel() - A @ m_prev.ravel())) - lam * m_prev.ravel()
    x = np.zeros_like(b)
    r = b.copy()
    p = r.copy()
    assert np.allclose(hist[0], m_prev)
    for it in range(1, 9):
        Hp = H @ p
        a = (r @ r) / (p @ Hp)
        x = x + a * p
        r_new = r - a * Hp
        p = r_new + (r_new @ r_new) / (r @ r) * p
        r = r_new
        np.testing.assert_allclose(hist[it].ravel(), m_prev.ravel() + x, rtol=0,
                                   atol=1e-9 * np.linalg.norm(m_prev))


def test_single_window_spanning_all_shots_is_full_solve():
    op, d = _tiny_problem(seed=3)
    lam = 1e-3 * float(np.abs(op.adjoint(d)).max())
    m_full, st_full = O.cg_window(op, np.arange(op.ns), d, lam, np.zeros((op.nz, op.nx)), 6)
    m_rls, stats = O.rls_solve(op, d, lam, op.ns, 1, 6)
    assert len(stats) == 1
    np.testing.assert_array_equal(m_rls, m_full)


def test_large_lambda_limit_is_scaled_adjoint():
    op, d = _tiny_problem(seed=4)
    A = O.explicit_matrix(op)
    lam = 1e7 * np.linalg.norm(np.real(A.conj().T @ A), 2)
    m, _ = O.cg_window(op, np.arange(op.ns), d, lam, np.zeros((op.nz, op.nx)), 20, tol=1e-14)
    b = op.adjoint(d)
    assert np.linalg.norm(lam * m - b) <= 1e-6 * np.linalg.norm(b)


def test_window_starts_golden():
    """Window schedules, including the paper's own 240-shot experiment (window 5, slide 3)."""
    with open(os.path.join(GOLDEN, "window_starts.txt")) as fh:
        rows = [ln.split("#")[0].strip() for ln in fh]
    rows = [r for r in rows if r]
    assert rows
    for row in rows:
        head, tail = row.split(":")
        ns, window, slide = (int(v) for v in head.split())
        expect = [int(v) for v in tail.split()]
        assert O.window_starts(ns, window, slide) == expect


def test_each_window_converges_to_its_own_exact_solution():
    """Tight-tolerance sliding solve: every window's image is that window's Eq. 4 solution."""
    op, d = _tiny_problem(seed=6, ns=5)
    lam = 0.02 * float(np.abs(op.adjoint(d)).max())
    window, slide = 3, 1
    starts = O.window_starts(op.ns, window, slide)
    m = np.zeros((op.nz, op.nx))
    for k, st in enumerate(starts):
        shots = np.arange(st, st + window)
        m, stat = O.cg_window(op, shots, d[shots], lam, m, 400, tol=1e-12)
        A = O.explicit_matrix(op, shots)
        exact = O.closed_form_solution(A, d[shots], lam).reshape(op.nz, op.nx)
        assert np.linalg.norm(m - exact) <= 1e-8 * np.linalg.norm(exact)


def test_warm_start_reduces_iterations_on_tiny_config():
    """Paper's claim (block-row section): warm starts cut CG iterations vs cold starts."""
    sv = config_tiny()
    op = _op(sv)
    clean = op.forward(sv.reflectivity)
    d = clean + sv.noise_pct * np.sqrt(np.mean(np.abs(clean) ** 2)) * sv.noise()
    lam = O.regularisation_from_adjoint(op, d)
    starts = O.window_starts(op.ns, sv.window, sv.slide)
    warm_its, cold_its = 0, 0
    m = np.zeros((op.nz, op.nx))
    for st in starts:
        shots = np.arange(st, st + sv.window)
        m, s1 = O.cg_window(op, shots, d[shots], lam, m, 100, tol=1e-2)
        _, s0 = O.cg_window(op, shots, d[shots], lam, np.zeros_like(m), 100, tol=1e-2)
        warm_its += s1.iters
        cold_its += s0.iters
    assert warm_its < cold_its


def test_reference_slowness_is_least_squares_constant_of_each_row():
    """The split-step reference slowness of depth row j is the constant that fits that row of the
    slowness best in least squares (library lstsq on a column of ones): the phase screen
    D_j = exp(i w (s - s_ref) dz) then has zero mean phase across x, which the operator's
    coefficient rows show directly."""
    sv = random_case(48, 10, 2, 3, seed=17)
    op = _op(sv)
    ones = np.ones((sv.nx, 1))
    for j in range(sv.nz):
        fit = np.linalg.lstsq(ones, op.s[j], rcond=None)[0][0]
        assert abs(op.sref[j] - fit) <= 1e-15 * abs(fit)
        _, dj = op.coefficients(j)
        assert np.all(np.abs(np.angle(dj).sum(axis=1)) <= 1e-9)


# ---------------------------------------------------------------- planted mistakes


def test_planted_wrong_phase_sign_fails_traveltime_pin(monkeypatch):
    good = O.phase_shift
    monkeypatch.setattr(O, "phase_shift", lambda *a: np.conj(good(*a)))
    with pytest.raises(AssertionError):
        test_point_diffractor_traveltime()


def test_planted_missing_split_step_fails_vertical_time_pin(monkeypatch):
    monkeypatch.setattr(O, "split_step", lambda w, s, sr, dz: np.ones((len(w), len(s)),
                                                                      dtype=complex))
    with pytest.raises(AssertionError):
        test_split_step_vertical_traveltime_in_laterally_varying_medium()


def test_planted_adjoint_without_conjugate_fails_dot_test(monkeypatch):
    def bad(self, u, j):
        phi, d = self.coefficients(j)
        return self._ifft(np.conj(phi) * self._fft(d * u))
    monkeypatch.setattr(O.SplitStepOperator, "propagate_adjoint", bad)
    op = _op(random_case(32, 8, 2, 4, seed=1))
    assert _dot_test_error(op) > 1e-6


def test_planted_unwrapped_kx_fails_plane_wave_pin(monkeypatch):
    monkeypatch.setattr(O, "kx_axis", lambda nx, dx: 2 * math.pi * np.arange(nx) / (nx * dx))
    with pytest.raises(AssertionError):
        test_plane_wave_is_eigenvector_with_dispersion_phase(40)


def test_planted_transposed_image_index_fails_shift_pin(monkeypatch):
    good = O.SplitStepOperator.forward

    def bad(self, m, shots=None):
        return good(self, np.roll(m, 1, axis=0) if m.ndim == 2 else m, shots)
    monkeypatch.setattr(O.SplitStepOperator, "forward", bad)
    op, d = _tiny_problem(seed=1)
    assert _dot_test_error(op) > 1e-6


def test_planted_minimum_reference_slowness_fails_least_squares_pin(monkeypatch):
    monkeypatch.setattr(O, "reference_slowness", lambda s: s.min(axis=1))
    with pytest.raises(AssertionError):
        test_reference_slowness_is_least_squares_constant_of_each_row()


def test_planted_unconjugated_inner_product_fails_cholesky_pin(monkeypatch):
    monkeypatch.setattr(O, "real_dot", lambda u, v: float(np.real(np.sum(u * v))))
    with pytest.raises(AssertionError):
        test_cg_matches_explicit_cholesky_solution()


# ---------------------------------------------------------------- gradients (autograd row)


def _gradient_problem(seed=3, nx=64, nz=32, ns=2, nw=6):
    """64 x 32 crop with a smooth slowness perturbation direction (Gaussian-smoothed N(0, 1e-5))."""
    sv = random_case(nx, nz, ns, nw, seed=seed)
    op = _op(sv)
    m = sv.reflectivity
    dobs = op.forward(m) + 0.1 * sv.noise()
    rng = np.random.default_rng(seed)
    from scipy.ndimage import gaussian_filter
    ds = gaussian_filter(rng.normal(0.0, 1e-5, size=m.shape), 2.0)
    return sv, op, m, dobs, ds


def _misfit(sv, sref, s, m, dobs):
    o = O.SplitStepOperator(s, sv.dx, sv.dz, sv.freqs, sv.wavelet, sv.src_ix, sv.rec_ix, sref=sref)
    return float(np.sum(np.abs(o.forward(m) - dobs) ** 2))


def test_slowness_gradient_matches_central_differences():
    """dL/ds (s_ref held fixed) against central differences of L = ||A(s) m - d||^2, h = 1e-3."""
    sv, op, m, dobs, ds = _gradient_problem()
    _, gs = O.born_gradients(op, m, 2.0 * (op.forward(m) - dobs))
    analytic = float(np.sum(gs * ds))
    for h, tol in ((1e-1, 1e-3), (1e-3, 1e-6)):
        fd = (_misfit(sv, op.sref, op.s + h * ds, m, dobs) - _misfit(sv, op.sref, op.s - h * ds, m, dobs)) / (2 * h)
        assert abs(fd - analytic) <= tol * abs(analytic), (h, fd, analytic)


def test_model_gradient_is_adjoint_and_matches_differences():
    sv, op, m, dobs, _ = _gradient_problem(seed=5, nx=32, nz=12)
    g = 2.0 * (op.forward(m) - dobs)
    gm, _ = O.born_gradients(op, m, g)
    np.testing.assert_allclose(gm, op.adjoint(g), rtol=0, atol=1e-12 * np.abs(gm).max())
    dm = np.random.default_rng(1).normal(size=m.shape)
    h = 1e-3
    fd = (np.sum(np.abs(op.forward(m + h * dm) - dobs) ** 2) - np.sum(np.abs(op.forward(m - h * dm) - dobs) ** 2)) / (2 * h)
    assert abs(fd - np.sum(gm * dm)) <= 1e-8 * abs(fd)


def test_planted_missing_source_adjoint_term_fails_gradient_pin(monkeypatch):
    """Dropping the mu (source-side) term of the slowness gradient is caught by the FD pin."""
    good = O.born_gradients

    def without_mu(op, m, g, shots=None):
        gm, gs = good(op, m, g, shots)
        shots = np.arange(op.ns) if shots is None else shots
        S = op.source_wavefield(shots)
        R = [op.inject(np.asarray(g, dtype=complex), shots)]
        for j in range(op.nz - 1):
            R.append(op.propagate_adjoint(R[-1], j))
        U = [None] * op.nz
        U[-1] = S[-1] * m[-1]
        for j in range(op.nz - 2, -1, -1):
            U[j] = S[j] * m[j] + op.propagate(U[j + 1], j)
        w = op.omega[None, :, None]
        gs2 = np.zeros_like(gs)
        for j in range(op.nz - 1):
            gs2[j] = np.real(1j * w * op.dz * np.conj(R[j]) * (U[j] - S[j] * m[j])).sum(axis=(0, 1))
        return gm, gs2
    monkeypatch.setattr(O, "born_gradients", without_mu)
    with pytest.raises(AssertionError):
        test_slowness_gradient_matches_central_differences()


# ---------------------------------------------------------------- preconditioned variant


def test_pcg_converges_to_cholesky_solution():
    op, d = _tiny_problem(seed=7)
    A = O.explicit_matrix(op)
    lam = 1e-2 * np.linalg.norm(np.real(A.conj().T @ A), 2)
    m_chol = O.closed_form_solution(A, d, lam).reshape(op.nz, op.nx)
    m_pcg, st = O.pcg_window(op, np.arange(op.ns), d, lam, np.zeros((op.nz, op.nx)), 300, tol=1e-13)
    assert st.rel_res <= 1e-13
    assert np.linalg.norm(m_pcg - m_chol) <= 1e-9 * np.linalg.norm(m_chol)


def test_pcg_iterates_equal_textbook_pcg_on_explicit_matrix():
    op, d = _tiny_problem(seed=8)
    A = O.explicit_matrix(op)
    H = np.real(A.conj().T @ A)
    lam = 0.05 * np.linalg.norm(H, 2)
    H = H + lam * np.eye(H.shape[0])
    shots = np.arange(op.ns)
    illum = O.illumination(op, shots).ravel()
    # the illumination is the diagonal of the source-side part, cross-checked by brute force
    S = op.source_wavefield(shots)
    assert np.allclose(illum, sum(np.abs(S[:, i, w, :].ravel()) ** 2 for i in range(op.ns) for w in range(op.nw)))
    minv = 1.0 / (illum + 1e-2 * illum.max())
    hist = []
    O.pcg_window(op, shots, d, lam, np.zeros((op.nz, op.nx)), 6, tol=0.0, precond_eps=1e-2, history=hist)
    b = np.real(A.conj().T @ d.ravel())
    x = np.zeros_like(b)
    r = b.copy()
    z = minv * r
    p = z.copy()
    for it in range(1, 7):
        Hp = H @ p
        a = (r @ z) / (p @ Hp)
        x = x + a * p
        r_new = r - a * Hp
        z_new = minv * r_new
        p = z_new + (r_new @ z_new) / (r @ z) * p
        r, z = r_new, z_new
        np.testing.assert_allclose(hist[it].ravel(), x, rtol=0, atol=1e-9 * np.linalg.norm(x))


def test_illumination_preconditioner_cuts_iterations_on_tiny_config():
    sv = config_tiny()
    op = _op(sv)
    clean = op.forward(sv.reflectivity)
    d = clean + sv.noise_pct * np.sqrt(np.mean(np.abs(clean) ** 2)) * sv.noise()
    lam = O.regularisation_from_adjoint(op, d)
    shots = np.arange(sv.window)
    _, plain = O.cg_window(op, shots, d[shots], lam, np.zeros((op.nz, op.nx)), 200, tol=1e-3)
    _, pre = O.pcg_window(op, shots, d[shots], lam, np.zeros((op.nz, op.nx)), 200, tol=1e-3)
    assert pre.iters < plain.iters
