"""Seeded synthetic surveys standing in for the paper's Marmousi experiment (Examples section).

The paper images Marmousi data (240 shots, 25 m interval, 20 Hz Ricker, off-end spread).  That
dataset is not available, so every workload here is synthetic and seeded.  The recipes:

* tiny (64 x 32, 10 m): v(z) linear 1500 -> 2500 m/s; three flat reflectors at depth indices
  8, 16, 24 with amplitudes 0.1, -0.08, 0.12 and a point diffractor of 0.1 at (x=32, z=20);
  8 shots; 32 frequencies 5-30 Hz; 1 % noise (seed 0); window 4 shots, slide 2.
* realistic (512 x 256, 8 m): six random smooth interfaces (seed 1) separating layers whose
  velocity rises from 1500 to 4000 m/s, Gaussian-smoothed (sigma = 3 cells), clipped to
  [1500, 4000], plus four Gaussian anomalies of +-300 m/s with sigma = 40 m; reflectivity with
  5 % nonzeros drawn from N(0, 0.1) (seed 2) plus three dipping layers (dips 5-20 degrees,
  amplitudes 0.05-0.1); 96 shots; 128 frequencies 3-40 Hz; 2 % noise; window 16, slide 8.
* precision (1024 x 512, 6 m): the realistic construction, 192 shots, 256 frequencies 3-60 Hz.
* midsize (128 x 64, 8 m): the realistic construction, 16 shots, 32 frequencies 3-40 Hz,
  window 8, slide 4, CG to 1e-3 (the tolerance-stopped solve the oracle can still run).
* batching: eight lines with nx in {256, 384, 512, 640, 768, 896, 1024, 1024}, nz = nx / 2,
  shots U{64..200}, frequencies U{96..192}, window U{4..32}, slide = ceil(window / 2) (seed 3);
  the reduced form keeps each line's first three windows of shots and every other frequency.

Shots sit at grid columns floor((i + 1/2) nx / ns); receivers at every grid column.  The
frequency axis is linear with both ends included.  The wavelet is the zero-phase spectrum of a
Ricker wavelet with the paper's 20 Hz peak frequency.  Noise is returned as unit circular complex
Gaussian samples; callers scale it by pct * rms|A m| once the clean data exist.

Nothing here implements the migration operator or the solver.
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
from scipy.ndimage import gaussian_filter


def linear_frequencies(f_lo: float, f_hi: float, nw: int) -> np.ndarray:
    """Frequencies f_i = f_lo + i (f_hi - f_lo) / (nw - 1) in Hz, both ends included."""
    if nw == 1:
        return np.array([f_lo], dtype=np.float64)
    return f_lo + np.arange(nw, dtype=np.float64) * (f_hi - f_lo) / (nw - 1)


def ricker_spectrum(freq_hz: np.ndarray, f_peak: float = 20.0) -> np.ndarray:
    """Zero-phase Ricker spectrum W(f) = (2 / sqrt(pi)) f^2 / f_p^3 exp(-f^2 / f_p^2).

    This is the Fourier transform (convention exp(-2 pi i f t)) of the time-domain Ricker
    wavelet r(t) = (1 - 2 pi^2 f_p^2 t^2) exp(-pi^2 f_p^2 t^2); the paper's source has
    f_p = 20 Hz (Examples section).  Returned as complex128 with zero imaginary part.
    """
    f = np.asarray(freq_hz, dtype=np.float64)
    w = (2.0 / math.sqrt(math.pi)) * f * f / f_peak**3 * np.exp(-(f * f) / (f_peak * f_peak))
    return w.astype(np.complex128)


def centred_shots(nx: int, ns: int) -> np.ndarray:
    """Shot columns floor((i + 1/2) nx / ns), i = 0..ns-1, as int32."""
    return np.floor((np.arange(ns) + 0.5) * nx / ns).astype(np.int32)


def full_spread_receivers(nx: int, ns: int) -> np.ndarray:
    """Receivers at every grid column for every shot: int32 array [ns][nx]."""
    return np.tile(np.arange(nx, dtype=np.int32), (ns, 1))


def unit_complex_noise(shape, seed: int) -> np.ndarray:
    """Circular complex Gaussian samples with E|n|^2 = 1 (numpy default_rng(seed))."""
    rng = np.random.default_rng(seed)
    re = rng.standard_normal(shape)
    im = rng.standard_normal(shape)
    return (re + 1j * im) / math.sqrt(2.0)


@dataclass
class Survey:
    """One 2D survey line: grid, model, geometry, frequency axis and solver settings.

    Layouts: velocity/slowness/reflectivity are [nz][nx] (a depth row is contiguous);
    src_ix is [ns]; rec_ix is [ns][nrec]; freqs and wavelet are [nw].  Data arrays built from a
    survey are [ns][nw][nrec] complex.
    """

    name: str
    nx: int
    nz: int
    dx: float
    dz: float
    velocity: np.ndarray
    reflectivity: np.ndarray
    src_ix: np.ndarray
    rec_ix: np.ndarray
    freqs: np.ndarray
    wavelet: np.ndarray
    noise_pct: float
    noise_seed: int
    window: int
    slide: int
    cg_tol: float
    cg_iters: int
    extra: dict = field(default_factory=dict)

    @property
    def slowness(self) -> np.ndarray:
        return 1.0 / self.velocity

    @property
    def ns(self) -> int:
        return int(self.src_ix.shape[0])

    @property
    def nw(self) -> int:
        return int(self.freqs.shape[0])

    @property
    def nrec(self) -> int:
        return int(self.rec_ix.shape[1])

    def data_shape(self):
        return (self.ns, self.nw, self.nrec)

    def noise(self) -> np.ndarray:
        return unit_complex_noise(self.data_shape(), self.noise_seed)


def _layered_velocity(nx, nz, dx, dz, rng, n_interfaces=6, v_top=1500.0, v_bottom=4000.0,
                      smooth_cells=3.0, n_anomalies=4, anomaly_amp=300.0, anomaly_sigma_m=40.0):
    x = np.arange(nx) * dx
    depth = nz * dz
    width = nx * dx
    # interface depths: sorted random means with smooth lateral undulation
    means = np.sort(rng.uniform(0.08, 0.92, n_interfaces)) * depth
    zgrid = np.arange(nz)[:, None] * dz
    layer_v = np.linspace(v_top, v_bottom, n_interfaces + 1)
    layer_v[1:-1] += rng.uniform(-0.25, 0.25, n_interfaces - 1) * (layer_v[1] - layer_v[0])
    v = np.full((nz, nx), layer_v[0])
    for i, zm in enumerate(means):
        undulation = np.zeros(nx)
        for _ in range(3):
            amp = rng.uniform(0.0, 0.03) * depth
            wavelength = rng.uniform(0.3, 1.5) * width
            phase = rng.uniform(0.0, 2.0 * math.pi)
            undulation += amp * np.sin(2.0 * math.pi * x / wavelength + phase)
        zi = zm + undulation
        v = np.where(zgrid >= zi[None, :], layer_v[i + 1], v)
    v = gaussian_filter(v, smooth_cells, mode="nearest")
    v = np.clip(v, v_top, v_bottom)
    xx = np.arange(nx)[None, :] * dx
    zz = np.arange(nz)[:, None] * dz
    for _ in range(n_anomalies):
        xc = rng.uniform(0.1, 0.9) * width
        zc = rng.uniform(0.15, 0.85) * depth
        sign = 1.0 if rng.uniform() < 0.5 else -1.0
        v = v + sign * anomaly_amp * np.exp(-((xx - xc) ** 2 + (zz - zc) ** 2)
                                            / (2.0 * anomaly_sigma_m ** 2))
    return v


def _sparse_dipping_reflectivity(nx, nz, dx, dz, rng, density=0.05, sigma=0.1, n_dipping=3):
    m = np.zeros((nz, nx))
    mask = rng.uniform(size=(nz, nx)) < density
    m[mask] = rng.normal(0.0, sigma, int(mask.sum()))
    x = np.arange(nx) * dx
    for _ in range(n_dipping):
        dip = math.radians(rng.uniform(5.0, 20.0)) * (1.0 if rng.uniform() < 0.5 else -1.0)
        amp = rng.uniform(0.05, 0.1) * (1.0 if rng.uniform() < 0.5 else -1.0)
        z0 = rng.uniform(0.2, 0.8) * nz * dz
        zline = z0 + math.tan(dip) * (x - 0.5 * nx * dx)
        jz = np.rint(zline / dz).astype(int)
        ok = (jz >= 0) & (jz < nz)
        m[jz[ok], np.nonzero(ok)[0]] += amp
    return m


def config_tiny() -> Survey:
    """Plain method, tiny: 64 x 32 grid, 8 shots, 32 frequencies, window 4, slide 2."""
    nx, nz, dx, dz, ns, nw = 64, 32, 10.0, 10.0, 8, 32
    vz = 1500.0 + 1000.0 * np.arange(nz) / (nz - 1)
    vel = np.tile(vz[:, None], (1, nx))
    m = np.zeros((nz, nx))
    for jz, a in ((8, 0.1), (16, -0.08), (24, 0.12)):
        m[jz, :] = a
    m[20, 32] += 0.1
    freqs = linear_frequencies(5.0, 30.0, nw)
    return Survey("tiny", nx, nz, dx, dz, vel, m, centred_shots(nx, ns),
                  full_spread_receivers(nx, ns), freqs, ricker_spectrum(freqs), 0.01, 0,
                  window=4, slide=2, cg_tol=0.0, cg_iters=10)


def _realistic_like(name, nx, nz, dx, dz, ns, f_lo, f_hi, nw, window, slide, seed_v=1,
                    seed_m=2, noise_seed=0, noise_pct=0.02) -> Survey:
    vel = _layered_velocity(nx, nz, dx, dz, np.random.default_rng(seed_v))
    m = _sparse_dipping_reflectivity(nx, nz, dx, dz, np.random.default_rng(seed_m))
    freqs = linear_frequencies(f_lo, f_hi, nw)
    return Survey(name, nx, nz, dx, dz, vel, m, centred_shots(nx, ns),
                  full_spread_receivers(nx, ns), freqs, ricker_spectrum(freqs), noise_pct,
                  noise_seed, window=window, slide=slide, cg_tol=1e-3, cg_iters=200)


def config_realistic() -> Survey:
    """Plain method, realistic: 512 x 256 at 8 m, 96 shots, 128 frequencies 3-40 Hz, K=16, S=8."""
    return _realistic_like("realistic", 512, 256, 8.0, 8.0, 96, 3.0, 40.0, 128, 16, 8)


def config_precision() -> Survey:
    """Precision workload: 1024 x 512 at 6 m, 192 shots, 256 frequencies 3-60 Hz."""
    return _realistic_like("precision", 1024, 512, 6.0, 6.0, 192, 3.0, 60.0, 256, 16, 8)


def config_midsize() -> Survey:
    """The realistic construction at 128 x 64 (8 m), 16 shots, 32 frequencies 3-40 Hz, window 8,
    slide 4, CG to 1e-3: small enough for the FP64 oracle to run the whole tolerance-stopped
    sliding solve (three windows of a few dozen iterations each)."""
    return _realistic_like("midsize", 128, 64, 8.0, 8.0, 16, 3.0, 40.0, 32, 8, 4)


def config_precision_subsample(nx: int = 128) -> Survey:
    """The precision workload's construction (6 m grid, 3-60 Hz) subsampled to nx x 64, 6 shots,
    10 frequencies: small enough for the FP64 oracle, used to compare the transform precisions."""
    return _realistic_like("precision-subsample", nx, 64, 6.0, 6.0, 6, 3.0, 60.0, 10, 3, 2)


def config_batching_lines():
    """Eight independent lines of the batching workload (seed 3)."""
    rng = np.random.default_rng(3)
    out = []
    for i, nx in enumerate((256, 384, 512, 640, 768, 896, 1024, 1024)):
        ns = int(rng.integers(64, 201))
        nw = int(rng.integers(96, 193))
        window = int(rng.integers(4, 33))
        slide = (window + 1) // 2
        out.append(_realistic_like(f"line{i}", nx, nx // 2, 8.0, 8.0, ns, 3.0, 40.0, nw, window,
                                   slide, seed_v=10 + i, seed_m=20 + i, noise_seed=30 + i))
    return out


def config_batching_lines_reduced(max_windows: int = 3, freq_stride: int = 2):
    """The batching workload cut down for a bounded benchmark: the same eight lines (widths, nz,
    window K, slide, velocity, reflectivity and noise seeds), each keeping only the shots of its
    first `max_windows` windows and every `freq_stride`-th frequency of its axis."""
    out = []
    for sv in config_batching_lines():
        keep = min(sv.ns, sv.window + (max_windows - 1) * sv.slide)
        sv.src_ix = centred_shots(sv.nx, keep)
        sv.rec_ix = full_spread_receivers(sv.nx, keep)
        sv.freqs = sv.freqs[::freq_stride].copy()
        sv.wavelet = ricker_spectrum(sv.freqs)
        sv.name = sv.name + "-reduced"
        out.append(sv)
    return out


def random_case(nx: int, nz: int, ns: int, nw: int, seed: int, dx: float = 10.0,
                dz: float = 10.0, f_lo: float = 5.0, f_hi: float = 30.0,
                heterogeneous: bool = True) -> Survey:
    """Small random survey for parity tests: smooth random v(x, z), random reflectivity."""
    rng = np.random.default_rng(seed)
    if heterogeneous:
        vel = 1500.0 + 1500.0 * gaussian_filter(rng.uniform(size=(nz, nx)), 2.0, mode="wrap")
        vel = vel + 400.0 * np.arange(nz)[:, None] / max(nz - 1, 1)
    else:
        vel = np.full((nz, nx), 2000.0)
    m = rng.normal(0.0, 0.1, (nz, nx))
    freqs = linear_frequencies(f_lo, f_hi, nw)
    return Survey(f"random{seed}", nx, nz, dx, dz, vel, m, centred_shots(nx, ns),
                  full_spread_receivers(nx, ns), freqs, ricker_spectrum(freqs), 0.01, seed + 1,
                  window=max(1, ns // 2), slide=max(1, ns // 4), cg_tol=0.0, cg_iters=5)
