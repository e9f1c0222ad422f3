"""Seeded synthetic inputs shared by the CUDA library's tests/benchmarks and the
FP64 oracle.

This module holds none of the registration method's arithmetic: no transport,
no band-limited expansion or projection, no regulariser.  It only draws
images, smooth warps and coefficient arrays from a seed.  Both sides of every
parity comparison receive the same arrays from here (the CUDA side in float32 /
complex64, the oracle the same rounded values widened to float64 / complex128).

Workload stand-ins (the paper registers NIREP brains resampled to 180x210x180,
which are not available here):

* ``blob_pair``      -- template = 6 isotropic Gaussians (centres uniform in the
  inner 60% of the grid, widths 2-5 voxels, amplitudes 0.3-1.0); target = the
  same blobs evaluated at x - u(x) for a smooth random periodic displacement u
  with a prescribed maximum length.
* ``phantom_pair``   -- brain-like phantom of three nested ellipsoidal tissue
  classes (intensities 0.2 / 0.5 / 0.8 outer to inner, semi-axes 0.40 / 0.30 /
  0.18 of the grid jittered +-10% per axis), periodic Gaussian blur of 1 voxel
  and N(0, 0.01^2) noise; the target is the same phantom evaluated at x - u(x).
* ``uneven_pairs``   -- the many-pair batching workload: grids drawn from
  {64^3, 96^3, 128^3, 160x192x160}, bands from {16^3, 24^3, 32^3}, maximum warp
  uniform in [3, 8] voxels, one phantom seed per pair.
* ``random_coefficients`` -- complex Gaussian band coefficients with a
  smoothness decay (1 + |k|^2)^-1, scaled so that sum_k |v_c(k)| equals a given
  bound; that bound caps the spatial velocity of every component.
"""

from __future__ import annotations

import numpy as np


def _rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(np.random.SeedSequence(int(seed)))


def _grid(n):
    return np.indices(tuple(n), dtype=np.float64)


def smooth_displacement(n, seed: int, max_disp: float, modes: int = 8,
                        kmax: int = 2) -> np.ndarray:
    """Random periodic displacement u (3, N1, N2, N3), sum of `modes` sinusoids of
    integer frequency |k_d| <= kmax, scaled so that max_x |u(x)| = max_disp."""
    rng = _rng(seed)
    x = _grid(n)
    u = np.zeros((3,) + tuple(n))
    for _ in range(modes):
        k = rng.integers(-kmax, kmax + 1, size=3)
        if not k.any():
            k[rng.integers(0, 3)] = 1
        phase = sum(2.0 * np.pi * k[a] * x[a] / n[a] for a in range(3))
        phase = phase + rng.uniform(0, 2 * np.pi)
        amp = rng.normal(size=3)
        u += amp[:, None, None, None] * np.sin(phase)[None]
    norm = np.sqrt(np.sum(u * u, axis=0)).max()
    if max_disp == 0.0 or norm == 0.0:
        return np.zeros_like(u)
    return u * (max_disp / norm)


def _periodic_delta(y: np.ndarray, c: float, N: int) -> np.ndarray:
    """Minimum-image difference y - c on a periodic axis of length N."""
    return (y - c + 0.5 * N) % N - 0.5 * N


def _blobs_at(y, n, centres, widths, amps) -> np.ndarray:
    out = np.zeros(tuple(n))
    for c, s, a in zip(centres, widths, amps):
        r2 = sum(_periodic_delta(y[d], c[d], n[d]) ** 2 for d in range(3))
        out += a * np.exp(-0.5 * r2 / (s * s))
    return out


def blob_pair(n, seed: int, max_disp: float = 2.0, count: int = 6):
    """Template of `count` Gaussians and its warp by a smooth displacement.
    Returns (I0, I1, u) in float64."""
    rng = _rng(seed)
    n = tuple(int(v) for v in n)
    centres = [rng.uniform(0.2, 0.8, size=3) * np.array(n) for _ in range(count)]
    widths = rng.uniform(2.0, 5.0, size=count)
    amps = rng.uniform(0.3, 1.0, size=count)
    x = _grid(n)
    u = smooth_displacement(n, seed + 7919, max_disp)
    I0 = _blobs_at(x, n, centres, widths, amps)
    I1 = _blobs_at(x - u, n, centres, widths, amps)
    return I0, I1, u


def _periodic_blur(img: np.ndarray, sigma: float) -> np.ndarray:
    if sigma <= 0:
        return img
    freqs = np.meshgrid(*[np.fft.fftfreq(N) for N in img.shape], indexing="ij")
    f2 = sum(f * f for f in freqs)
    return np.real(np.fft.ifftn(np.fft.fftn(img) * np.exp(-2.0 * (np.pi * sigma) ** 2 * f2)))


def _phantom_at(y, n, centre, radii) -> np.ndarray:
    """Nested ellipsoids: 0.2 in the outer shell, 0.5 in the middle, 0.8 inside."""
    out = np.zeros(tuple(n))
    for r, step in zip(radii, (0.2, 0.3, 0.3)):
        q = sum((_periodic_delta(y[d], centre[d], n[d]) / r[d]) ** 2 for d in range(3))
        out += step * (q <= 1.0)
    return out


def phantom_pair(n, seed: int, max_disp: float = 6.0, noise: float = 0.01,
                 blur: float = 1.0):
    """Brain-like phantom and its warp by a smooth displacement.
    Returns (I0, I1, u) in float64."""
    rng = _rng(seed)
    n = tuple(int(v) for v in n)
    N = np.array(n, dtype=np.float64)
    base = (0.40, 0.30, 0.18)
    radii = [b * N * rng.uniform(0.9, 1.1, size=3) for b in base]
    centre = 0.5 * N + rng.uniform(-0.02, 0.02, size=3) * N
    x = _grid(n)
    u = smooth_displacement(n, seed + 7919, max_disp)
    I0 = _periodic_blur(_phantom_at(x, n, centre, radii), blur)
    I1 = _periodic_blur(_phantom_at(x - u, n, centre, radii), blur)
    I0 = I0 + rng.normal(0.0, noise, size=n)
    I1 = I1 + rng.normal(0.0, noise, size=n)
    return I0, I1, u


def centred(B: int) -> np.ndarray:
    """Integer frequency labels -B/2 .. B/2-1 used to shape the coefficient spectrum."""
    return np.arange(B) - B // 2


def random_coefficients(band, seed: int, bound: float) -> np.ndarray:
    """Complex Gaussian coefficients (3, B1, B2, B3), complex128, decaying as
    (1 + |k|^2)^-1, scaled so that sum_k |v_c(k)| = bound for every component."""
    rng = _rng(seed)
    shape = (3,) + tuple(int(b) for b in band)
    z = rng.normal(size=shape) + 1j * rng.normal(size=shape)
    k2 = sum(np.meshgrid(*[centred(b) ** 2 for b in band], indexing="ij"))
    z *= (1.0 / (1.0 + k2))[None]
    l1 = np.abs(z).reshape(3, -1).sum(axis=1)
    return z * (bound / l1)[:, None, None, None]


UNEVEN_GRIDS = ((64, 64, 64), (96, 96, 96), (128, 128, 128), (160, 192, 160))
UNEVEN_BANDS = ((16, 16, 16), (24, 24, 24), (32, 32, 32))


def uneven_pairs(npairs: int, seed: int) -> list:
    """Shapes of a batch of independent registration pairs: per pair a dict
    with ``n`` (grid), ``band``, ``max_disp`` (voxels) and ``seed`` (its
    phantom_pair seed)."""
    rng = _rng(seed)
    out = []
    for p in range(npairs):
        out.append(dict(n=UNEVEN_GRIDS[int(rng.integers(len(UNEVEN_GRIDS)))],
                        band=UNEVEN_BANDS[int(rng.integers(len(UNEVEN_BANDS)))],
                        max_disp=float(rng.uniform(3.0, 8.0)), seed=int(seed) * 1000 + p))
    return out


def phantom_pair_f32(n, seed: int, max_disp: float):
    """phantom_pair rounded to float32 (I0, I1): a picklable task for a process
    pool that prepares many pairs."""
    I0, I1, _ = phantom_pair(tuple(n), seed, max_disp=max_disp)
    return I0.astype(np.float32), I1.astype(np.float32)


def random_direction(band, seed: int) -> np.ndarray:
    """i.i.d. complex normal coefficients (3, B1, B2, B3), complex128, unit 2-norm."""
    rng = _rng(seed)
    shape = (3,) + tuple(int(b) for b in band)
    z = rng.normal(size=shape) + 1j * rng.normal(size=shape)
    return z / np.sqrt(np.sum(np.abs(z) ** 2))


def as_device_inputs(*arrays):
    """Round to the CUDA library's precision (float32 / complex64) and return the
    pairs (rounded, rounded widened back to float64 / complex128) so that both
    sides of a comparison see bit-identical inputs."""
    out = []
    for a in arrays:
        if np.iscomplexobj(a):
            lo = np.ascontiguousarray(a, dtype=np.complex64)
            out.append((lo, lo.astype(np.complex128)))
        else:
            lo = np.ascontiguousarray(a, dtype=np.float32)
            out.append((lo, lo.astype(np.float64)))
    return out
