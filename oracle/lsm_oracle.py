"""FP64 CPU oracle for block-row recursive least-squares migration (Kazemi & Sacchi).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or execute this
module: only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline / reference legs of
``bench.py`` use it.  It is deliberately plain and slow: every lateral transform is a naive DFT
written as a dense DFT matrix, every step is done in the order the method states, in float64,
vectorised only over the independent (shot, frequency) items.  It shares no code with the CUDA
path; the only thing both sides share is the seeded input generator package ``synth``.

What it computes, with the passage each part follows:

* Data model d = A m + n (Eq. 1) and adjoint migration m_hat = A^T d (Eq. 2), where A is the
  shot-profile de-migration operator built from the one-way wave equation with the split-step
  correction (Examples section).  The operator's details are not spelled out in the paper; the
  readings used here are:
    - lateral DFT  F u[k] = sum_x u[x] exp(-2 pi i k x / nx), inverse with 1/nx;
    - kx = 2 pi k / (nx dx) for k < nx/2, 2 pi (k - nx) / (nx dx) otherwise;
    - reference slowness s_ref(z_j) = mean over x of s(x, z_j);
    - phase shift Phi_j(kx) = exp(+i kz dz), kz = sqrt(w^2 s_ref^2 - kx^2) where that is real,
      and exp(-sqrt(kx^2 - w^2 s_ref^2) dz) for evanescent kx (time convention exp(-i w t));
    - split-step correction D_j(x) = exp(+i w (s(x, z_j) - s_ref(z_j)) dz);
    - one depth step P_j = D_j F^-1 Phi_j F, its adjoint P_j^H = F^-1 conj(Phi_j) F conj(D_j);
    - source S_0 = W(w) delta(x - x_s), S_{j+1} = P_j S_j;
    - A m = sum_j P_0 ... P_{j-1} (S_j * m_j), sampled at the receivers (depth 0);
    - A^T d: R_0 = receivers' data injected at depth 0, R_{j+1} = P_j^H R_j,
      m_j(x) = Re sum_{shots, w} conj(S_j(x)) R_j(x);
  A and A^T are exact adjoints under <u, v> = Re sum conj(u) v (real model, complex data).
* Damped least squares (Eq. 3) and its closed form (Eq. 4): explicit-matrix Cholesky on tiny
  grids, used to pin the iterative solver.
* Per-window CG on the normal equations (A_k^T A_k + lambda I) m = A_k^T d_k (Eq. 10), started
  from the previous window's image, which is the warm start of Eq. 11.
* The sliding window: windows of K consecutive shots, each step dropping the first `slide`
  shots and adding the next `slide` (the rank-K downdate/update of the block-row section).
  Window starts are 0, slide, 2 slide, ... while start + K <= ns, plus a final window at
  ns - K when the last one does not end at ns.  The result is the last window's image.
* Stopping rule (a threshold on the normal equation, Examples section) read as
  ||A_k^T (d_k - A_k m) - lambda m|| / ||A_k^T d_k|| <= tol.
* Preconditioned variant (`pcg_window`): the paper asks for preconditioners in each windowed
  setup without naming one; the reading is the diagonal source-illumination preconditioner.
* Gradients of a real loss of d = A(s) m with respect to m (= A^T g, Eq. 2) and to the slowness
  with the reference slowness held fixed (adjoint-state recursion, `born_gradients`).

Parity pins for every function live in tests/test_oracle_pins.py.  The operator conventions
above are readings (the paper prints no numbers or figures for them); they are pinned by
closed forms (plane-wave eigenvalues, point-diffractor traveltime, vertical traveltime through a
laterally varying medium, shift invariance), by the dot-product test and by library routines
(numpy.fft, Cholesky).
"""

from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


# --------------------------------------------------------------------------------------------
# Lateral transform (naive DFT) and wavenumber axis
# --------------------------------------------------------------------------------------------

def dft_matrix(nx: int) -> np.ndarray:
    """F[k, x] = exp(-2 pi i k x / nx): the naive forward DFT as a dense matrix."""
    k = np.arange(nx)
    return np.exp(-2j * math.pi * np.outer(k, k) / nx)


def idft_matrix(nx: int) -> np.ndarray:
    """F^-1[x, k] = exp(+2 pi i k x / nx) / nx."""
    k = np.arange(nx)
    return np.exp(2j * math.pi * np.outer(k, k) / nx) / nx


def kx_axis(nx: int, dx: float) -> np.ndarray:
    """kx_k = 2 pi k / (nx dx) for k < nx/2, 2 pi (k - nx) / (nx dx) otherwise."""
    k = np.arange(nx, dtype=np.float64)
    k = np.where(k < nx / 2.0, k, k - nx)
    return 2.0 * math.pi * k / (nx * dx)


def reference_slowness(slowness: np.ndarray) -> np.ndarray:
    """s_ref(z_j) = mean over x of s(x, z_j); slowness is [nz][nx]."""
    return slowness.mean(axis=1)


def phase_shift(omega: np.ndarray, sref_j: float, kx: np.ndarray, dz: float) -> np.ndarray:
    """Phi_j[w, k]: exp(+i kz dz) on the propagating band, exp(-|kz| dz) on the evanescent one."""
    kz2 = (np.asarray(omega)[:, None] * sref_j) ** 2 - kx[None, :] ** 2
    prop = kz2 >= 0.0
    root = np.sqrt(np.abs(kz2))
    return np.where(prop, np.exp(1j * root * dz), np.exp(-root * dz))


def split_step(omega: np.ndarray, s_j: np.ndarray, sref_j: float, dz: float) -> np.ndarray:
    """D_j[w, x] = exp(+i w (s(x, z_j) - s_ref(z_j)) dz)."""
    return np.exp(1j * np.asarray(omega)[:, None] * (s_j[None, :] - sref_j) * dz)


# --------------------------------------------------------------------------------------------
# Shot-profile split-step operator (Eq. 1 / Eq. 2, Examples section)
# --------------------------------------------------------------------------------------------

@dataclass
class Geometry:
    src_ix: np.ndarray   # [ns] source grid columns
    rec_ix: np.ndarray   # [ns][nrec] receiver grid columns


class SplitStepOperator:
    """De-migration A and migration A^T for one survey line, in float64.

    slowness: [nz][nx] in s/m; freqs_hz: [nw]; wavelet: [nw] complex source spectrum;
    src_ix: [ns]; rec_ix: [ns][nrec].
    """

    def __init__(self, slowness, dx, dz, freqs_hz, wavelet, src_ix, rec_ix, sref=None):
        self.s = np.asarray(slowness, dtype=np.float64)
        self.nz, self.nx = self.s.shape
        self.dx, self.dz = float(dx), float(dz)
        self.freqs = np.asarray(freqs_hz, dtype=np.float64)
        self.omega = 2.0 * math.pi * self.freqs
        self.wavelet = np.asarray(wavelet, dtype=np.complex128)
        self.geom = Geometry(np.asarray(src_ix, dtype=np.int64),
                             np.asarray(rec_ix, dtype=np.int64))
        self.F = dft_matrix(self.nx)
        self.Finv = idft_matrix(self.nx)
        self.kx = kx_axis(self.nx, self.dx)
        # the reference slowness may be held fixed at a background model's (for slowness gradients)
        self.sref = reference_slowness(self.s) if sref is None else np.asarray(sref, dtype=np.float64)

    @property
    def ns(self):
        return int(self.geom.src_ix.shape[0])

    @property
    def nw(self):
        return int(self.freqs.shape[0])

    @property
    def nrec(self):
        return int(self.geom.rec_ix.shape[1])

    def with_freqs(self, idx):
        """The same operator restricted to a subset of the frequency axis."""
        idx = np.asarray(idx)
        return SplitStepOperator(self.s, self.dx, self.dz, self.freqs[idx], self.wavelet[idx],
                                 self.geom.src_ix, self.geom.rec_ix, sref=self.sref)

    # lateral transforms on the last axis
    def _fft(self, u):
        return u @ self.F.T

    def _ifft(self, u):
        return u @ self.Finv.T

    def coefficients(self, j):
        """(Phi_j [nw][nx], D_j [nw][nx]) for depth row j."""
        phi = phase_shift(self.omega, self.sref[j], self.kx, self.dz)
        d = split_step(self.omega, self.s[j], self.sref[j], self.dz)
        return phi, d

    def propagate(self, u, j):
        """P_j u = D_j F^-1 (Phi_j F u); u is [..., nw, nx]."""
        phi, d = self.coefficients(j)
        return d * self._ifft(phi * self._fft(u))

    def propagate_adjoint(self, u, j):
        """P_j^H u = F^-1 (conj(Phi_j) F (conj(D_j) u))."""
        phi, d = self.coefficients(j)
        return self._ifft(np.conj(phi) * self._fft(np.conj(d) * u))

    def source_wavefield(self, shots):
        """S[j, i, w, x] for shots[i]: S_0 = W(w) delta_{x_s}, S_{j+1} = P_j S_j."""
        shots = np.asarray(shots)
        S = np.zeros((self.nz, len(shots), self.nw, self.nx), dtype=np.complex128)
        cur = np.zeros((len(shots), self.nw, self.nx), dtype=np.complex128)
        for i, sh in enumerate(shots):
            cur[i, :, self.geom.src_ix[sh]] = self.wavelet
        for j in range(self.nz):
            S[j] = cur
            if j + 1 < self.nz:
                cur = self.propagate(cur, j)
        return S

    def record(self, u0, shots):
        """Sample a depth-0 wavefield [ns_w, nw, nx] at each shot's receivers."""
        out = np.empty((len(shots), self.nw, self.nrec), dtype=np.complex128)
        for i, sh in enumerate(shots):
            out[i] = u0[i][:, self.geom.rec_ix[sh]]
        return out

    def inject(self, d, shots):
        """Adjoint of record: add each receiver's data into its grid column at depth 0."""
        u = np.zeros((len(shots), self.nw, self.nx), dtype=np.complex128)
        for i, sh in enumerate(shots):
            np.add.at(u[i], (slice(None), self.geom.rec_ix[sh]), d[i])
        return u

    def forward(self, m, shots=None):
        """d = A m for the given shots (Eq. 1 without noise), by Horner's rule from the bottom.

        U_{nz-1} = S_{nz-1} m_{nz-1};  U_j = S_j m_j + P_j U_{j+1};  d = U_0 at the receivers.
        This equals sum_j P_0 ... P_{j-1} (S_j m_j) (pinned by a brute-force test).
        """
        shots = np.arange(self.ns) if shots is None else np.asarray(shots)
        m = np.asarray(m, dtype=np.float64)
        S = self.source_wavefield(shots)
        U = S[self.nz - 1] * m[self.nz - 1]
        for j in range(self.nz - 2, -1, -1):
            U = S[j] * m[j] + self.propagate(U, j)
        return self.record(U, shots)

    def adjoint(self, d, shots=None):
        """m = A^T d for the given shots (Eq. 2): cross-correlation imaging condition."""
        shots = np.arange(self.ns) if shots is None else np.asarray(shots)
        S = self.source_wavefield(shots)
        R = self.inject(np.asarray(d, dtype=np.complex128), shots)
        m = np.zeros((self.nz, self.nx))
        for j in range(self.nz):
            m[j] = np.real(np.conj(S[j]) * R).sum(axis=(0, 1))
            if j + 1 < self.nz:
                R = self.propagate_adjoint(R, j)
        return m


# --------------------------------------------------------------------------------------------
# Gradients of a real loss L(d), d = A(s) m, with respect to m and to the slowness s
# --------------------------------------------------------------------------------------------

def born_gradients(op, m, g, shots=None):
    """(dL/dm, dL/ds) for d = A(s) m given g = dL/dRe(d) + i dL/dIm(d) at the receivers.

    The reference slowness s_ref is held fixed (only the split-step factor D_j depends on s), so
    dD_j(x)/ds_j(x) = i w dz D_j(x) and dP_j u = i w dz ds_j . (P_j u).  Adjoint-state recursion:
      R_0 = injected g, R_{j+1} = P_j^H R_j;
      U_{nz-1} = S_{nz-1} m_{nz-1}, U_j = S_j m_j + P_j U_{j+1};
      mu_{nz} = 0, mu_j = m_j R_j + P_j^H mu_{j+1};
      dL/dm_j = Re sum conj(S_j) R_j                      (= A^T g, Eq. 2);
      dL/ds_j = Re sum i w dz [conj(R_j) (U_j - S_j m_j) + conj(mu_{j+1}) S_{j+1}]
    summed over shots and frequencies.  Pinned by central finite differences of the oracle's
    forward operator with the same fixed s_ref.
    """
    shots = np.arange(op.ns) if shots is None else np.asarray(shots)
    m = np.asarray(m, dtype=np.float64)
    S = op.source_wavefield(shots)
    nz = op.nz
    R = np.empty_like(S)
    cur = op.inject(np.asarray(g, dtype=np.complex128), shots)
    for j in range(nz):
        R[j] = cur
        if j + 1 < nz:
            cur = op.propagate_adjoint(cur, j)
    U = np.empty_like(S)
    U[nz - 1] = S[nz - 1] * m[nz - 1]
    for j in range(nz - 2, -1, -1):
        U[j] = S[j] * m[j] + op.propagate(U[j + 1], j)
    w = op.omega[None, :, None]
    grad_m = np.zeros((nz, op.nx))
    grad_s = np.zeros((nz, op.nx))
    mu = np.zeros_like(S[0])
    for j in range(nz - 1, -1, -1):
        grad_m[j] = np.real(np.conj(S[j]) * R[j]).sum(axis=(0, 1))
        if j + 1 < nz:
            term = np.conj(R[j]) * (U[j] - S[j] * m[j]) + np.conj(mu) * S[j + 1]
            grad_s[j] = np.real(1j * w * op.dz * term).sum(axis=(0, 1))
        mu_next = mu
        mu = m[j] * R[j] + (op.propagate_adjoint(mu_next, j) if j + 1 < nz else 0.0)
    return grad_m, grad_s


# --------------------------------------------------------------------------------------------
# Damped least squares: closed form (Eq. 4) and CG on the normal equations (Eq. 10, Eq. 11)
# --------------------------------------------------------------------------------------------

def real_dot(u, v) -> float:
    """<u, v> = Re sum conj(u) v."""
    return float(np.real(np.vdot(u, v)))


def explicit_matrix(op: SplitStepOperator, shots=None) -> np.ndarray:
    """Columns A e_i for every model cell (probe by unit vectors): complex [N][M]."""
    shots = np.arange(op.ns) if shots is None else np.asarray(shots)
    M = op.nz * op.nx
    cols = []
    for i in range(M):
        e = np.zeros(M)
        e[i] = 1.0
        cols.append(op.forward(e.reshape(op.nz, op.nx), shots).ravel())
    return np.stack(cols, axis=1)


def closed_form_solution(Amat: np.ndarray, d: np.ndarray, lam: float) -> np.ndarray:
    """m = (A^T A + lambda I)^-1 A^T d (Eq. 4) by Cholesky, with A^T = Re A^H."""
    H = np.real(Amat.conj().T @ Amat) + lam * np.eye(Amat.shape[1])
    rhs = np.real(Amat.conj().T @ d.ravel())
    L = np.linalg.cholesky(H)
    y = np.linalg.solve(L, rhs)
    return np.linalg.solve(L.T, y)


@dataclass
class WindowStats:
    start: int
    iters: int
    rel_res0: float
    rel_res: float
    n_forward: int
    n_adjoint: int


def cg_window(op, shots, d_k, lam, m0, max_iter, tol=0.0, history=None):
    """CG on (A_k^T A_k + lambda I) m = A_k^T d_k from m0 (Eq. 10, warm start of Eq. 11).

    Stops before an iteration once ||A_k^T(d_k - A_k m) - lambda m|| / ||A_k^T d_k|| <= tol,
    or after max_iter iterations.  Scalars and vectors are float64.
    Returns (m, WindowStats).  If ``history`` is a list, each iterate m is appended.
    """
    b = op.adjoint(d_k, shots)
    nb = math.sqrt(real_dot(b, b))
    m = np.array(m0, dtype=np.float64, copy=True)
    r = d_k - op.forward(m, shots)
    s = op.adjoint(r, shots) - lam * m
    p = s.copy()
    gamma = real_dot(s, s)
    rel0 = math.sqrt(gamma) / nb if nb > 0 else 0.0
    rel = rel0
    nfwd, nadj = 1, 2
    it = 0
    if history is not None:
        history.append(m.copy())
    while it < max_iter and not (rel <= tol):
        q = op.forward(p, shots)
        nfwd += 1
        delta = real_dot(q, q) + lam * real_dot(p, p)
        alpha = gamma / delta
        m = m + alpha * p
        r = r - alpha * q
        s = op.adjoint(r, shots) - lam * m
        nadj += 1
        gamma_new = real_dot(s, s)
        beta = gamma_new / gamma
        p = s + beta * p
        gamma = gamma_new
        it += 1
        rel = math.sqrt(gamma) / nb if nb > 0 else 0.0
        if history is not None:
            history.append(m.copy())
    return m, WindowStats(int(shots[0]), it, rel0, rel, nfwd, nadj)


def illumination(op, shots):
    """Source illumination of a window: sum over its shots and frequencies of |S_j(x)|^2, [nz][nx]."""
    S = op.source_wavefield(np.asarray(shots))
    return np.sum(np.abs(S) ** 2, axis=(1, 2))


def pcg_window(op, shots, d_k, lam, m0, max_iter, tol=0.0, precond_eps=1e-2, history=None):
    """Preconditioned CG on (A_k^T A_k + lambda I) m = A_k^T d_k from m0 (block-row section: the
    paper asks for preconditioners that cluster the windowed Hessian's spectrum; reading: the
    diagonal source-illumination preconditioner M = illum + eps max(illum)).

    Standard PCG with z = M^-1 s: q = A p; alpha = s.z / (||q||^2 + lambda ||p||^2); m += alpha p;
    r -= alpha q; s = A^T r - lambda m; z = M^-1 s; beta = s_new.z_new / s.z; p = z + beta p.
    The stopping rule uses the unpreconditioned ||s|| / ||A_k^T d_k||, as cg_window does.
    """
    b = op.adjoint(d_k, shots)
    nb = math.sqrt(real_dot(b, b))
    illum = illumination(op, shots)
    minv = 1.0 / (illum + precond_eps * illum.max())
    m = np.array(m0, dtype=np.float64, copy=True)
    r = d_k - op.forward(m, shots)
    s = op.adjoint(r, shots) - lam * m
    z = minv * s
    p = z.copy()
    gamma = real_dot(s, z)
    rel0 = math.sqrt(real_dot(s, s)) / nb if nb > 0 else 0.0
    rel = rel0
    nfwd, nadj, it = 1, 2, 0
    if history is not None:
        history.append(m.copy())
    while it < max_iter and not (rel <= tol):
        q = op.forward(p, shots)
        nfwd += 1
        delta = real_dot(q, q) + lam * real_dot(p, p)
        alpha = gamma / delta
        m = m + alpha * p
        r = r - alpha * q
        s = op.adjoint(r, shots) - lam * m
        nadj += 1
        z = minv * s
        gamma_new = real_dot(s, z)
        p = z + (gamma_new / gamma) * p
        gamma = gamma_new
        it += 1
        rel = math.sqrt(real_dot(s, s)) / nb if nb > 0 else 0.0
        if history is not None:
            history.append(m.copy())
    return m, WindowStats(int(shots[0]), it, rel0, rel, nfwd, nadj)


def window_starts(ns: int, window: int, slide: int):
    """Starts 0, slide, 2 slide, ... while start + window <= ns; then ns - window if needed."""
    if window > ns:
        raise ValueError("window longer than the survey")
    starts = list(range(0, ns - window + 1, slide))
    if starts[-1] + window < ns:
        starts.append(ns - window)
    return starts


def rls_solve(op, d, lam, window, slide, max_iter, tol=0.0, m0=None, first_window=0,
              n_windows=None, precond_eps=None):
    """Block-row recursive LS migration: CG per sliding window, warm-started (Eq. 10, Eq. 11).

    d is [ns][nw][nrec]; returns (image of the last window solved, [WindowStats]).  With
    precond_eps set, each window uses pcg_window (illumination preconditioner) instead.
    """
    starts = window_starts(op.ns, window, slide)
    m = np.zeros((op.nz, op.nx)) if m0 is None else np.array(m0, dtype=np.float64)
    last = len(starts) if n_windows is None else min(len(starts), first_window + n_windows)
    stats = []
    for k in range(first_window, last):
        shots = np.arange(starts[k], starts[k] + window)
        if precond_eps is None:
            m, st = cg_window(op, shots, d[shots], lam, m, max_iter, tol)
        else:
            m, st = pcg_window(op, shots, d[shots], lam, m, max_iter, tol, precond_eps)
        stats.append(st)
    return m, stats


def regularisation_from_adjoint(op, d, scale=1e-3):
    """lambda = scale * max |A^T d| over all shots."""
    return scale * float(np.max(np.abs(op.adjoint(d))))
