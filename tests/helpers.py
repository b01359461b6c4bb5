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


GOLDEN_512 = __import__("os").path.join(__import__("os").path.dirname(__import__("os").path.abspath(__file__)),
                                        "golden", "precision_512.npz")


def precision_512_errors(torch, tensor_dft: bool):
    """The 512 x 512, 16-coil, 32-spoke frame (8 Newton x 30 CG) on the GPU against the oracle's run stored by
    tests/golden/make_precision_512.py: per iterate the relative L2 error on the stored structured sample (rho on
    Omega at every 4th pixel, the central 8 x 8 k-space block of every chat_j), the residual norms, and the final
    rho on Omega and display image.  Returns a dict of the errors."""
    from paper_1301_1215_gb300.nlinv import Nlinv
    g = np.load(GOLDEN_512)
    n, J, spokes, seed, newton, cg = (int(v) for v in g["meta"])
    fr = synth.make_frame(n, J, spokes, seed=seed)
    s = O.Setup(n, J, n // 4)
    y0 = O.simulate(s, fr.mask, fr.rho, fr.coils)
    power = float(np.sum(np.abs(y0) ** 2) / (fr.mask.sum() * J))
    y = (y0 + fr.mask * synth.noise_sigma(power, 30.0) * fr.noise).astype(np.complex64)
    dev = torch.device("cuda")
    ty = torch.from_numpy(y).to(dev)
    tm = torch.from_numpy(fr.mask).to(dev)
    with Nlinv(n, J, newton_steps=newton, cg_iters=cg, tensor_dft=tensor_dft) as ctx:
        xN, ck = ctx.reconstruct_checkpoints(ty, tm)
        _, resid = ctx.reconstruct(ty, tm, resid=True)
        img = ctx.image(xN).cpu().numpy()
        ck = ck.cpu().numpy()
    idx = g["sample_index"]
    steps = [rel(ck[k].ravel()[idx], g["samples"][k]) for k in range(newton + 1)]
    h = n // 2
    rho = np.fft.fftshift(ck[-1][0])[h - n // 4: h + n // 4, h - n // 4: h + n // 4]
    return {"per_step_sample": steps, "rho_omega": rel(rho, g["rho_omega"]), "image": rel(img, g["image"]),
            "resid_gpu": list(resid), "resid_oracle": [float(v) for v in g["resid"]],
            "resid_rel": [abs(a - b) / b for a, b in zip(resid, g["resid"])]}
