"""Writes tests/golden/precision_512.npz: the CPU oracle's Gauss-Newton run on the 512 x 512, 16-coil, 32-spoke
frame (8 Newton steps x 30 CG iterations, alpha_0 = 1 halved per step), the precision workload.

Calls nothing but the oracle (and the seeded input generator).  The run takes several minutes of CPU, so the GPU
test reads its results from this file instead of recomputing them.  Stored (all from the oracle):
  resid        |y - F x_n| for n = 0..8 (complex128 arithmetic)
  rho_omega    rho of the final iterate on Omega, centred (256 x 256, complex64)
  image        the display image rho * sqrt(sum_j |c_j|^2) of the final iterate on Omega, centred (complex64)
  samples      per iterate x_0..x_8 a fixed structured sample (complex64): rho on Omega at every 4th pixel of
               each axis, and the central 8 x 8 k-space block of every chat_j (where the coil coefficients
               carry their energy)
  sample_index flat indices of those samples in the (1 + J) x n x n unknown
Usage: python tests/golden/make_precision_512.py
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle.nlinv_oracle as O  # noqa: E402
from paper_1301_1215_gb300 import synth  # noqa: E402

N, J, SPOKES, SEED, NEWTON, CG = 512, 16, 32, 1005, 8, 30


def problem():
    """Data of the frame, as the GPU sees it (rounded to complex64)."""
    s = O.Setup(N, J, N // 4)
    fr = synth.make_frame(N, J, SPOKES, seed=SEED)
    y0 = O.simulate(s, fr.mask, fr.rho, fr.coils)
    power = float(np.sum(np.abs(y0) ** 2) / (fr.mask.sum() * J))
    y = y0 + fr.mask * synth.noise_sigma(power, 30.0) * fr.noise
    return s, fr.mask, y.astype(np.complex64).astype(np.complex128)


def sample_index():
    g = O.signed_index(N)
    om = np.nonzero((g >= -N // 4) & (g < N // 4))[0]            # Omega rows / columns, natural order
    om_c = om[np.argsort(g[om])][::4]                             # every 4th, in signed order
    rho = (om_c[:, None] * N + om_c[None, :]).ravel()
    k = np.nonzero((g >= -4) & (g < 4))[0]
    k = k[np.argsort(g[k])]
    blk = (k[:, None] * N + k[None, :]).ravel()
    coils = [(1 + j) * N * N + blk for j in range(J)]
    return np.concatenate([rho] + coils).astype(np.int64)


def main():
    t0 = time.time()
    s, mask, y = problem()
    xs, alphas = O.irgnm_path(s, mask, y, synth.initial_guess(N, J), None, NEWTON, CG)
    resid = [O.residual(s, mask, y, x)[1] for x in xs]
    idx = sample_index()
    samples = np.stack([x.ravel()[idx] for x in xs]).astype(np.complex64)
    xf = xs[-1]
    h = N // 2
    rho_omega = np.fft.fftshift(xf[0])[h - N // 4: h + N // 4, h - N // 4: h + N // 4].astype(np.complex64)
    image = O.image(s, xf).astype(np.complex64)
    out = os.path.join(HERE, "precision_512.npz")
    np.savez_compressed(out, resid=np.array(resid), rho_omega=rho_omega, image=image, samples=samples,
                        sample_index=idx, alphas=np.array(alphas),
                        meta=np.array([N, J, SPOKES, SEED, NEWTON, CG], dtype=np.int64))
    print(f"wrote {out} in {time.time() - t0:.0f} s; resid {['%.6g' % r for r in resid]}")


if __name__ == "__main__":
    main()
