"""Seeded synthetic inputs for NLINV (radial real-time MRI, Sec. 3).

This module only draws numbers: a numerical phantom, smooth coil sensitivity maps, a rasterised radial sampling
pattern and unit complex noise.  It holds none of the reconstruction's arithmetic (no Fourier transform, no
Sobolev weight, no forward model), so both the CPU oracle and the CUDA path can take their inputs from it.

Conventions shared with the rest of the package:

* a grid of side ``n`` (twice the image matrix, Sec. 3.2) is stored row-major in natural FFT order: index ``i``
  holds the signed coordinate ``g(i) = ((i + n/2) mod n) - n/2``, so the origin sits at index 0;
* the field of view Omega is the centred square ``-fov <= g < fov`` in both axes (``fov = n/4`` by default, the
  un-oversampled image of Sec. 3.2);
* complex arrays are ``complex128`` here; callers cast to ``complex64`` for the GPU.

Every generator takes a ``numpy.random.Generator`` so that one seed fixes a whole workload.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


def rng_for(seed: int) -> np.random.Generator:
    """The generator used for every workload: PCG64 with a fixed integer seed."""
    return np.random.Generator(np.random.PCG64(int(seed)))


def signed_coords(n: int) -> np.ndarray:
    """Signed pixel (or k-space) coordinate of each natural-order index: ``((i + n/2) mod n) - n/2``."""
    i = np.arange(n)
    return (i + n // 2) % n - n // 2


def phantom(n: int, fov: int, rng: np.random.Generator, n_ellipses: int = 8) -> np.ndarray:
    """Sum of random ellipses inside Omega with a smooth phase (<= 0.3 rad), peak magnitude 1, zero outside Omega.

    Units are fractions of the field-of-view width ``2*fov``.  Centres lie within 0.3 FOV of the middle, semi-axes
    are 0.05..0.4 FOV, rotations uniform in [0, pi), intensities uniform in [0.1, 1].
    """
    g = signed_coords(n).astype(np.float64)
    u1 = g[:, None] / (2.0 * fov)           # row coordinate in FOV units
    u2 = g[None, :] / (2.0 * fov)           # column coordinate in FOV units
    img = np.zeros((n, n), dtype=np.float64)
    for _ in range(n_ellipses):
        r = 0.3 * np.sqrt(rng.uniform())
        phi = rng.uniform(0.0, 2.0 * np.pi)
        cx, cy = r * np.cos(phi), r * np.sin(phi)
        ax, ay = rng.uniform(0.05, 0.4, size=2)
        th = rng.uniform(0.0, np.pi)
        amp = rng.uniform(0.1, 1.0)
        d1, d2 = u1 - cy, u2 - cx
        e1 = (d2 * np.cos(th) + d1 * np.sin(th)) / ax
        e2 = (-d2 * np.sin(th) + d1 * np.cos(th)) / ay
        img = img + amp * ((e1 * e1 + e2 * e2) <= 1.0)
    inside = ((g >= -fov) & (g < fov))
    support = inside[:, None] & inside[None, :]
    img = np.where(support, img, 0.0)
    peak = img.max()
    if peak > 0:
        img = img / peak
    k1, k2 = rng.uniform(0.5, 1.5, size=2)
    p0 = rng.uniform(0.0, 2.0 * np.pi)
    phase = 0.3 * np.sin(2.0 * np.pi * (k1 * u1 + k2 * u2) + p0)
    return (img * np.exp(1j * phase)).astype(np.complex128)


def coil_maps(n: int, ncoils: int, fov: int, rng: np.random.Generator) -> np.ndarray:
    """Smooth Gaussian coil sensitivities centred on a circle: ``exp(-|u - p_j|^2 / (2 s^2)) * exp(i phi_j)``.

    ``p_j = 0.5 FOV (cos 2 pi j/J, sin 2 pi j/J)``, ``s = 0.35 FOV``, ``phi_j`` uniform; defined on the whole grid.
    Shape ``(ncoils, n, n)``.
    """
    g = signed_coords(n).astype(np.float64)
    u1 = g[:, None] / (2.0 * fov)
    u2 = g[None, :] / (2.0 * fov)
    s = 0.35
    out = np.empty((ncoils, n, n), dtype=np.complex128)
    phases = rng.uniform(0.0, 2.0 * np.pi, size=ncoils)
    for j in range(ncoils):
        px = 0.5 * np.cos(2.0 * np.pi * j / ncoils)
        py = 0.5 * np.sin(2.0 * np.pi * j / ncoils)
        d2 = (u2 - px) ** 2 + (u1 - py) ** 2
        out[j] = np.exp(-d2 / (2.0 * s * s)) * np.exp(1j * phases[j])
    return out


def radial_mask(n: int, spokes: int, rotation: float = 0.0) -> np.ndarray:
    """0/1 sampling pattern of ``spokes`` full-diameter radial spokes rasterised onto the ``n`` x ``n`` grid.

    Spoke ``s`` has angle ``pi s / spokes + rotation``.  Its samples are ``t (cos, sin)`` for
    ``t = -n/2, -n/2 + 1/2, ..., n/2 - 1/2``; each is rounded to the nearest grid point with ``floor(v + 1/2)`` and
    kept when ``-n/2 <= v < n/2``.  Returned as ``uint8`` in natural order (row = ky, column = kx).
    """
    m = np.zeros((n, n), dtype=np.uint8)
    t = np.arange(-n, n) * 0.5
    for s in range(spokes):
        th = np.pi * s / spokes + rotation
        kx = np.floor(t * np.cos(th) + 0.5).astype(np.int64)
        ky = np.floor(t * np.sin(th) + 0.5).astype(np.int64)
        ok = (kx >= -n // 2) & (kx < n // 2) & (ky >= -n // 2) & (ky < n // 2)
        m[ky[ok] % n, kx[ok] % n] = 1
    return m


def frame_rotation(frame: int, spokes: int, turns: int = 5) -> float:
    """Angle offset of frame ``frame`` in a real-time series: ``frame * 2 pi / (spokes * turns)`` (mod pi)."""
    return float(np.mod(frame * 2.0 * np.pi / (spokes * turns), np.pi))


def unit_noise(shape, rng: np.random.Generator) -> np.ndarray:
    """Complex Gaussian noise with E|n|^2 = 1 (real and imaginary parts N(0, 1/2))."""
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) * np.sqrt(0.5)


def noise_sigma(mean_sampled_power: float, snr_db: float) -> float:
    """Noise standard deviation for a given mean signal power on the sampled points and an SNR in dB."""
    return float(np.sqrt(mean_sampled_power / (10.0 ** (snr_db / 10.0))))


def random_complex(shape, rng: np.random.Generator) -> np.ndarray:
    """Standard complex normal array (used for operator-level parity tests)."""
    return unit_noise(shape, rng)


def initial_guess(n: int, ncoils: int) -> np.ndarray:
    """Single-frame start value x_0 = (rho = 1 on every pixel, chat_j = 0), shape ``(1 + J, n, n)``."""
    x = np.zeros((1 + ncoils, n, n), dtype=np.complex128)
    x[0] = 1.0
    return x


@dataclass(frozen=True)
class Workload:
    """One NLINV workload: grid side, coils, spokes and solver schedule."""
    name: str
    n: int
    ncoils: int
    spokes: int
    newton_steps: int
    cg_iters: int
    frames: int = 1
    alpha0: float = 1.0
    alpha_q: float = 0.5
    sobolev_a: float = 220.0
    sobolev_l: float = 32.0
    snr_db: float = 30.0
    seed: int = 1000
    extra: dict = field(default_factory=dict)

    @property
    def fov(self) -> int:
        return self.n // 4


# Shapes of the paper's real-time radial workloads (Sec. 3.2: matrix 192-384 on a 2x grid, 8-12 virtual coils).
WORKLOADS = {
    "single_64": Workload("single frame, 64x64 grid, 4 coils, 16 spokes", 64, 4, 16, 7, 30, seed=1001),
    "grad_256": Workload("single frame with gradient, 256x256 grid, 8 coils, 25 spokes", 256, 8, 25, 8, 40, seed=1002),
    "realtime_384": Workload("real-time series, 384x384 grid, 10 coils, 13 spokes, 200 frames", 384, 10, 13, 7, 30,
                             frames=200, seed=1003),
    "precision_512": Workload("512x512 grid, 16 coils, 32 spokes", 512, 16, 32, 8, 30, seed=1005),
}


def uneven_batch_shapes(nframes: int = 64, seed: int = 1004):
    """The uneven batch workload: per frame a grid side from {128, 192, 256, 320, 384}, 4..16 coils and 9..31
    spokes, drawn from one seeded generator.  Returns [(n, ncoils, spokes)]."""
    rng = rng_for(seed)
    sides = [128, 192, 256, 320, 384]
    return [(int(sides[rng.integers(0, 5)]), int(rng.integers(4, 17)), int(rng.integers(9, 32)))
            for _ in range(nframes)]


@dataclass
class Frame:
    """Synthetic ground truth and sampling for one frame (image-domain truth, no k-space data)."""
    rho: np.ndarray        # (n, n) complex, zero outside Omega
    coils: np.ndarray      # (J, n, n) complex, image-domain sensitivities
    mask: np.ndarray       # (n, n) uint8
    noise: np.ndarray      # (J, n, n) unit complex noise


def make_frame(n: int, ncoils: int, spokes: int, seed: int, frame: int = 0, fov: int | None = None,
               turns: int = 5) -> Frame:
    """Ground truth, radial mask and unit noise for one frame; the object and coils are fixed over a series,
    only the spoke rotation and the noise change with ``frame``."""
    fov = n // 4 if fov is None else fov
    rng = rng_for(seed)
    rho = phantom(n, fov, rng)
    coils = coil_maps(n, ncoils, fov, rng)
    mask = radial_mask(n, spokes, frame_rotation(frame, spokes, turns))
    noise = unit_noise((ncoils, n, n), rng_for(seed * 7919 + frame))
    return Frame(rho=rho, coils=coils, mask=mask, noise=noise)
