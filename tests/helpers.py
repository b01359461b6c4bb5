"""Shared test helpers: library build, tensor conversion and the noisy synthetic data of the workloads."""
from __future__ import annotations

import numpy as np

import oracle.nlinv_oracle as O
from paper_1301_1215_gb300 import synth


def ensure_built() -> str:
    from paper_1301_1215_gb300.build import build
    return build()


def rel(a, b) -> float:
    a, b = np.asarray(a), np.asarray(b)
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def noisy_data(n: int, J: int, spokes: int, seed: int, snr_db: float = 30.0, frame: int = 0, fov=None):
    """Oracle setup, frame, and data y = P FFT(M rho c_j) + noise at the given SNR on the sampled points."""
    fov = n // 4 if fov is None else fov
    s = O.Setup(n, J, fov)
    fr = synth.make_frame(n, J, spokes, seed=seed, frame=frame, fov=fov)
    y0 = O.simulate(s, fr.mask, fr.rho, fr.coils)
    power = float(np.sum(np.abs(y0) ** 2) / (fr.mask.sum() * J))
    y = y0 + fr.mask * synth.noise_sigma(power, snr_db) * fr.noise
    return s, fr, y
