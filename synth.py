"""Seeded synthetic scans shaped like the ptychography workloads of
arXiv:1602.01448 (Sec. 3.1 simulations, Sec. 3.2 experiment, Fig. 3).

This module only draws random numbers and lays out geometry: objects, probes,
scan positions, initial guesses and photon noise applied to intensities that
the caller computes. It holds none of the solver's arithmetic (no transform,
no projection, no overlap sum), so that both the FP64 oracle and the CUDA path
can take their inputs from it without sharing any of the method.

Conventions shared by both sides:
  * complex images are complex128 here (callers cast to complex64 for the GPU);
  * positions are int32 (row, col) top-left corners of each m x m frame, on the
    integer grid of Sec. 2.1 (x_(i) = (r mu', r nu'));
  * every generator takes an explicit ``numpy.random.Generator`` or seed.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

try:  # scipy is present on both machines; keep a plain fallback anyway
    from scipy.ndimage import gaussian_filter as _gaussian_filter
except Exception:  # pragma: no cover
    _gaussian_filter = None


def _rng(seed) -> np.random.Generator:
    if isinstance(seed, np.random.Generator):
        return seed
    return np.random.default_rng(seed)


def _smooth(field: np.ndarray, sigma: float) -> np.ndarray:
    """Periodic Gaussian smoothing of a real 2D field (data generation only)."""
    if _gaussian_filter is not None:
        return _gaussian_filter(field, sigma=sigma, mode="wrap")
    ny, nx = field.shape  # pragma: no cover - fallback path
    ky = np.fft.fftfreq(ny)[:, None]
    kx = np.fft.fftfreq(nx)[None, :]
    g = np.exp(-2.0 * (math.pi * sigma) ** 2 * (ky ** 2 + kx ** 2))
    return np.real(np.fft.ifft2(np.fft.fft2(field) * g))


def random_object(shape, seed, amp_range=(0.8, 1.0), phase_sigma=4.0,
                  phase_range=(-math.pi / 2, math.pi / 2)) -> np.ndarray:
    """Complex transmission: amplitude U[amp_range], phase a Gaussian-smoothed
    white-noise field linearly rescaled to ``phase_range``."""
    rng = _rng(seed)
    ny, nx = shape
    amp = rng.uniform(amp_range[0], amp_range[1], size=(ny, nx))
    ph = _smooth(rng.standard_normal((ny, nx)), phase_sigma)
    lo, hi = ph.min(), ph.max()
    ph = phase_range[0] + (ph - lo) * (phase_range[1] - phase_range[0]) / max(hi - lo, 1e-300)
    return amp * np.exp(1j * ph)


def aperture_probe(m: int, radius: float, edge_phase: float = 0.5) -> np.ndarray:
    """Circular aperture of ``radius`` px centred in an m x m frame with a
    quadratic phase reaching ``edge_phase`` rad at the rim."""
    yy, xx = np.mgrid[0:m, 0:m].astype(np.float64)
    rho2 = (yy - m / 2) ** 2 + (xx - m / 2) ** 2
    inside = rho2 <= radius ** 2
    return np.where(inside, np.exp(1j * edge_phase * rho2 / radius ** 2), 0.0).astype(np.complex128)


def gaussian_probe(m: int, sigma: float, seed, phase_coeff: float = 1.0,
                   degree: int = 3) -> np.ndarray:
    """Gaussian amplitude (``sigma`` px) with a random low-order polynomial
    phase (total degree <= ``degree``, coefficients uniform in +-phase_coeff rad
    on coordinates normalised to [-1, 1])."""
    rng = _rng(seed)
    yy, xx = np.mgrid[0:m, 0:m].astype(np.float64)
    u = (xx - m / 2) / (m / 2)
    v = (yy - m / 2) / (m / 2)
    amp = np.exp(-((xx - m / 2) ** 2 + (yy - m / 2) ** 2) / (2.0 * sigma ** 2))
    phase = np.zeros((m, m))
    for i in range(degree + 1):
        for j in range(degree + 1 - i):
            if i + j == 0:
                continue
            phase += rng.uniform(-phase_coeff, phase_coeff) * u ** i * v ** j
    return amp * np.exp(1j * phase)


def perturb_probe(w: np.ndarray, seed, rel: float = 0.1, sigma: float = 4.0) -> np.ndarray:
    """Initial probe guess w * (1 + rel * xi), xi a smoothed complex Gaussian
    field normalised to unit RMS."""
    rng = _rng(seed)
    m = w.shape[0]
    xi = _smooth(rng.standard_normal((m, m)), sigma) + 1j * _smooth(rng.standard_normal((m, m)), sigma)
    xi /= np.sqrt(np.mean(np.abs(xi) ** 2))
    return w * (1.0 + rel * xi)


def raster_positions(rows: int, cols: int, step: int, m: int, shape, seed=None,
                     jitter: int = 1) -> np.ndarray:
    """rows x cols raster with integer jitter drawn uniformly from
    {-jitter..jitter}, centred in the object.  Returns int32 (K, 2)."""
    rng = _rng(0 if seed is None else seed)
    ny, nx = shape
    ext_y = (rows - 1) * step + m
    ext_x = (cols - 1) * step + m
    oy = (ny - ext_y) // 2
    ox = (nx - ext_x) // 2
    iy, ix = np.meshgrid(np.arange(rows), np.arange(cols), indexing="ij")
    pos = np.stack([oy + iy * step, ox + ix * step], axis=-1).reshape(-1, 2)
    if jitter:
        pos = pos + rng.integers(-jitter, jitter + 1, size=pos.shape)
    return pos.astype(np.int32)


def fermat_positions(count: int, spacing: float, m: int, shape) -> np.ndarray:
    """Fermat spiral r_k = c sqrt(k), theta_k = k * 137.508 deg with c chosen so
    each point owns ``spacing``^2 px^2, centred, rounded to integers."""
    ny, nx = shape
    c = spacing / math.sqrt(math.pi)
    k = np.arange(count, dtype=np.float64)
    r = c * np.sqrt(k)
    th = np.deg2rad(137.508) * k
    cy = ny / 2 - m / 2
    cx = nx / 2 - m / 2
    pos = np.stack([np.rint(cy + r * np.sin(th)), np.rint(cx + r * np.cos(th))], axis=-1)
    return pos.astype(np.int32)


def poisson_intensities(intensity: np.ndarray, photons: float, seed) -> np.ndarray:
    """Scale every frame to ``photons`` counts in total, draw Poisson counts and
    scale back, so the noisy intensities stay on the model scale."""
    rng = _rng(seed)
    inten = np.asarray(intensity, dtype=np.float64)
    tot = inten.reshape(inten.shape[0], -1).sum(axis=1)
    scale = np.where(tot > 0, photons / np.maximum(tot, 1e-300), 0.0)[:, None, None]
    counts = rng.poisson(inten * scale)
    return np.where(scale > 0, counts / np.maximum(scale, 1e-300), 0.0)


@dataclasses.dataclass
class Scan:
    """One synthetic scan: the truth, the geometry and the starting guesses."""
    name: str
    obj: np.ndarray          # ground-truth object psi_0 (ny, nx) complex128
    probe: np.ndarray        # true illumination w (m, m) complex128
    pos: np.ndarray          # int32 (K, 2)
    wrap: bool
    photons: float | None    # None = noiseless
    psi_init: np.ndarray     # psi^(0)
    probe_init: np.ndarray   # w^(0)
    n_iter: int
    probe_every: int
    seed: int

    @property
    def m(self) -> int:
        return self.probe.shape[0]

    @property
    def K(self) -> int:
        return self.pos.shape[0]

    @property
    def shape(self):
        return self.obj.shape


def scan_small_raster(seed: int = 1) -> Scan:
    """100 frames of 64^2 on a 10x10 raster (step 12, +-1 px jitter) over a
    256^2 object; aperture probe r=16; noiseless; known probe; 100 iterations."""
    rng = _rng(seed)
    shape = (256, 256)
    m = 64
    obj = random_object(shape, rng)
    probe = aperture_probe(m, 16.0, 0.5)
    pos = raster_positions(10, 10, 12, m, shape, rng, jitter=1)
    return Scan("raster-100x64-obj256", obj, probe, pos, False, None,
                np.ones(shape, np.complex128), probe.copy(), 100, 0, seed)


def scan_fermat(seed: int = 2, count: int = 2500, m: int = 128, n: int = 1024,
                photons: float = 1e6) -> Scan:
    """Fermat spiral of ``count`` points at 10 px mean spacing, Gaussian probe
    sigma=20 px with random low-order phase, Poisson noise, probe refinement
    every 2nd iteration starting from a 10% perturbed probe, 300 iterations."""
    rng = _rng(seed)
    shape = (n, n)
    obj = random_object(shape, rng)
    probe = gaussian_probe(m, 20.0 * m / 128.0, rng)
    pos = fermat_positions(count, 10.0, m, shape)
    psi0 = rng.uniform(0.0, 1.0, size=shape).astype(np.complex128)
    w0 = perturb_probe(probe, rng, 0.1)
    return Scan(f"fermat-{count}x{m}-obj{n}", obj, probe, pos, False, photons,
                psi0, w0, 300, 2, seed)


def scan_large_raster(seed: int = 3, side: int = 100, m: int = 256, n: int = 3072,
                      step: int = 24, photons: float = 1e8) -> Scan:
    """side x side raster (step 24 +-1) of 256^2 frames over a 3072^2 object."""
    rng = _rng(seed)
    shape = (n, n)
    obj = random_object(shape, rng)
    probe = gaussian_probe(m, 20.0 * m / 128.0, rng)
    pos = raster_positions(side, side, step, m, shape, rng, jitter=1)
    psi0 = rng.uniform(0.0, 1.0, size=shape).astype(np.complex128)
    return Scan(f"raster-{side * side}x{m}-obj{n}", obj, probe, pos, False, photons,
                psi0, probe.copy(), 100, 0, seed)


def scan_wrapped_raster(seed: int = 4, side: int = 40, m: int = 128, n: int = 512,
                        step: int = 10, photons: float | None = 1e6) -> Scan:
    """40x40 raster (step 10) of 128^2 frames over a 512^2 object; the scan
    spans more than the object so indices wrap periodically."""
    rng = _rng(seed)
    shape = (n, n)
    obj = random_object(shape, rng)
    probe = gaussian_probe(m, 20.0 * m / 128.0, rng)
    iy, ix = np.meshgrid(np.arange(side), np.arange(side), indexing="ij")
    pos = np.stack([iy * step, ix * step], axis=-1).reshape(-1, 2).astype(np.int32)
    psi0 = np.ones(shape, np.complex128)
    return Scan(f"wrapped-raster-{side * side}x{m}-obj{n}", obj, probe, pos, True, photons,
                psi0, probe.copy(), 200, 0, seed)


def scan_tiny(seed: int = 5, m: int = 16, n: int = 32, rows: int = 2, cols: int = 4,
              step: int = 4, wrap: bool = False) -> Scan:
    """8 frames of 16^2 on a 2x4 raster over a 32^2 object (finite-difference
    sized instance)."""
    rng = _rng(seed)
    shape = (n, n)
    obj = random_object(shape, rng, phase_sigma=2.0)
    probe = gaussian_probe(m, m / 5.0, rng)
    pos = raster_positions(rows, cols, step, m, shape, rng, jitter=0)
    return Scan(f"tiny-{rows * cols}x{m}-obj{n}", obj, probe, pos, wrap, None,
                np.ones(shape, np.complex128), probe.copy(), 20, 0, seed)


def scan_batch_member(seed: int, m: int, count: int) -> Scan:
    """One scan of a batch: raster of side ceil(sqrt(count)) with step
    round(0.1875 m), object = scan extent + 64 px, Poisson 10^U[5,7]."""
    rng = _rng(seed)
    side = int(math.ceil(math.sqrt(count)))
    step = int(round(0.1875 * m))
    ext = (side - 1) * step + m + 2
    n = ext + 64
    shape = (n, n)
    obj = random_object(shape, rng)
    probe = gaussian_probe(m, 20.0 * m / 128.0, rng)
    pos = raster_positions(side, side, step, m, shape, rng, jitter=1)[:count]
    photons = float(10.0 ** rng.uniform(5.0, 7.0))
    return Scan(f"batch-{count}x{m}-obj{n}", obj, probe, pos, False, photons,
                np.ones(shape, np.complex128), probe.copy(), 100, 0, seed)


def random_frames(K: int, m: int, seed) -> np.ndarray:
    """Unstructured complex Gaussian frames for operator-level tests."""
    rng = _rng(seed)
    return (rng.standard_normal((K, m, m)) + 1j * rng.standard_normal((K, m, m))) / math.sqrt(2.0)


def random_amplitudes(K: int, m: int, seed) -> np.ndarray:
    """Non-negative amplitudes with a Rayleigh-like spread."""
    rng = _rng(seed)
    return np.abs(rng.standard_normal((K, m, m)) + 1j * rng.standard_normal((K, m, m)))
