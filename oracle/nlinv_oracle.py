"""CPU oracle for the NLINV hot path (Schaetz & Uecker, Sec. 3.1, Eq. 2 and Eq. 3, Table 1).

TEST INFRASTRUCTURE ONLY.  This module is the slow, plain, complex128 statement of what the GPU library computes.
Only the test suite, the package smoke check and the benchmark's CPU-baseline leg may import it; the library never
does, and it shares no code with the CUDA path.

Every step follows the paper's order and notation, with numpy's FFT (pocketfft, double precision) as the one
library primitive.  Where the paper leaves a detail open, the reading taken here is stated at the function:

* grid arrays are in natural FFT order (origin at index 0), row-major, one ``n`` x ``n`` plane per coil;
* the unknown is ``x = (rho, chat_1 .. chat_J)``, an array of shape ``(1 + J, n, n)``;
* the 2D Fourier transform is unitary (``FFT^-1 = FFT^H``);
* the Sobolev weight of ``W`` is ``w(k) = (1 + a |k|^2)^(-l/2)`` with ``|k|`` in cycles per grid width,
  ``k_i = g(i)/n`` in ``[-1/2, 1/2)``;
* Omega is the centred square ``-fov <= g < fov`` (the un-oversampled image of a 2x grid, Sec. 3.2);
* CG runs a fixed number of iterations from ``dx = 0`` and stops early only at the rounding floor of the
  single-precision arithmetic the method runs in (Sec. 3.2): ``|r| <= 2^-24 |b|`` (the unit roundoff of FP32),
  ``Re<p, A p> <= 0`` or a non-finite value -- none of which occurs in exact arithmetic for the positive definite
  system before the solution is reached; once stopped, the rest of that solve leaves dx unchanged;
* ``alpha_n = max(alpha_0 q^n, alpha_min)``; a single frame regularises toward its start value.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass(frozen=True)
class Setup:
    """Static problem description: grid side, coil count, field of view and Sobolev parameters."""
    n: int
    ncoils: int
    fov: int
    a: float = 220.0
    l: float = 32.0


# ---------------------------------------------------------------------------------------------------------------
# Building blocks of Eq. 2
# ---------------------------------------------------------------------------------------------------------------

def signed_index(n: int) -> np.ndarray:
    """g(i) = ((i + n/2) mod n) - n/2: the signed coordinate held by natural-order index i."""
    i = np.arange(n)
    return (i + n // 2) % n - n // 2


def sobolev_weight(n: int, a: float, l: float) -> np.ndarray:
    """Weight of the weighted Fourier transform W (Sec. 3.1): w(k) = (1 + a |k|^2)^(-l/2), k = g/n per axis."""
    k = signed_index(n) / n
    k2 = k[:, None] ** 2 + k[None, :] ** 2
    return (1.0 + a * k2) ** (-l / 2.0)


def omega_mask(n: int, fov: int) -> np.ndarray:
    """M_Omega of Eq. 2 as a 0/1 array: the centred square -fov <= g < fov in both axes."""
    g = signed_index(n)
    inside = ((g >= -fov) & (g < fov)).astype(np.float64)
    return inside[:, None] * inside[None, :]


def fft2u(a: np.ndarray) -> np.ndarray:
    """Unitary 2D DFT over the last two axes: X[k] = (1/n) sum_x a[x] exp(-2 pi i k.x / n)."""
    return np.fft.fft2(a, axes=(-2, -1), norm="ortho")


def ifft2u(a: np.ndarray) -> np.ndarray:
    """Inverse (= adjoint) of fft2u."""
    return np.fft.ifft2(a, axes=(-2, -1), norm="ortho")


def inner(u: np.ndarray, v: np.ndarray) -> complex:
    """Scalar product <u, v> = sum conj(u) v over every entry (Table 1's "A.B")."""
    return complex(np.vdot(u.ravel(), v.ravel()))


def Wi(s: Setup, chat: np.ndarray) -> np.ndarray:
    """W^-1 of Eq. 2 applied to k-space coil coefficients: c = FFT^-1(w . chat)."""
    return ifft2u(sobolev_weight(s.n, s.a, s.l) * chat)


def WiH(s: Setup, u: np.ndarray) -> np.ndarray:
    """Adjoint of W^-1: w . FFT(u)."""
    return sobolev_weight(s.n, s.a, s.l) * fft2u(u)


# ---------------------------------------------------------------------------------------------------------------
# The operator F of Eq. 2, its derivative and adjoint (the three rows F, DF, DF^H of Table 1)
# ---------------------------------------------------------------------------------------------------------------

def coils(s: Setup, x: np.ndarray) -> np.ndarray:
    """Image-domain coil sensitivities c_j = W^-1 chat_j of the current estimate."""
    return Wi(s, x[1:])


def channel_sum(c: np.ndarray, z: np.ndarray) -> np.ndarray:
    """Channel summation of Table 1: sum_j conj(c_j) z_j."""
    return np.sum(np.conj(c) * z, axis=0)


def forward(s: Setup, mask: np.ndarray, x: np.ndarray) -> np.ndarray:
    """F(x)_j = P FFT(M rho c_j) with c_j = W^-1 chat_j (Eq. 2, applied right to left)."""
    M = omega_mask(s.n, s.fov)
    c = coils(s, x)
    return mask * fft2u(M * x[0] * c)


def derivative(s: Setup, mask: np.ndarray, x: np.ndarray, dx: np.ndarray, c: np.ndarray | None = None) -> np.ndarray:
    """DF_x dx: the Frechet derivative of F at x.  F is bilinear in (rho, chat), so
    DF_x(drho, dchat)_j = P FFT(M (drho c_j + rho W^-1 dchat_j)).  ``c`` = W^-1 chat of x, if already known."""
    M = omega_mask(s.n, s.fov)
    c = coils(s, x) if c is None else c
    dc = Wi(s, dx[1:])
    return mask * fft2u(M * (dx[0] * c + x[0] * dc))


def adjoint(s: Setup, mask: np.ndarray, x: np.ndarray, r: np.ndarray, c: np.ndarray | None = None) -> np.ndarray:
    """DF_x^H r: z_j = M FFT^-1(P r_j); image part sum_j conj(c_j) z_j (the channel summation of Table 1);
    coil part W^-H(conj(rho) z_j).  ``c`` = W^-1 chat of x, if already known."""
    M = omega_mask(s.n, s.fov)
    c = coils(s, x) if c is None else c
    z = M * ifft2u(mask * r)
    out = np.empty((1 + s.ncoils, s.n, s.n), dtype=np.complex128)
    out[0] = channel_sum(c, z)
    out[1:] = WiH(s, np.conj(x[0]) * z)
    return out


def normal(s: Setup, mask: np.ndarray, x: np.ndarray, d: np.ndarray, alpha: float,
           c: np.ndarray | None = None) -> np.ndarray:
    """Left-hand operator of Eq. 3: (DF^H DF + alpha I) d."""
    c = coils(s, x) if c is None else c
    return adjoint(s, mask, x, derivative(s, mask, x, d, c), c) + alpha * d


def simulate(s: Setup, mask: np.ndarray, rho: np.ndarray, coil_img: np.ndarray) -> np.ndarray:
    """Noiseless gridded data of the signal equation (Eq. 1) for image-domain coils: P FFT(M rho c_j)."""
    M = omega_mask(s.n, s.fov)
    return mask * fft2u(M * rho * coil_img)


def grid_radial(n: int, angles, samples: np.ndarray):
    """Interpolation of radial samples onto the n x n grid: the CPU pre-processing step of Sec. 3.1 that the paper
    leaves unspecified, read as nearest-neighbour gridding with averaging.  Sample i of spoke s lies at
    t_i (cos theta_s, sin theta_s), t_i = -n/2 + i/2 (i < 2n); each coordinate goes to the grid point floor(v + 1/2)
    and the sample is kept when both lie in [-n/2, n/2).  A grid point (row = ky, column = kx, natural order) holds
    the mean of its samples; the sampling pattern marks the points that received at least one.
    samples: (J, S, 2n).  Returns (y (J, n, n), mask (n, n) uint8)."""
    samples = np.asarray(samples, dtype=np.complex128)
    J = samples.shape[0]
    total = np.zeros((J, n, n), dtype=np.complex128)
    count = np.zeros((n, n), dtype=np.int64)
    for si, th in enumerate(angles):
        for i in range(2 * n):
            t = -n / 2 + 0.5 * i
            kx = int(np.floor(t * np.cos(th) + 0.5))
            ky = int(np.floor(t * np.sin(th) + 0.5))
            if -n // 2 <= kx < n // 2 and -n // 2 <= ky < n // 2:
                total[:, ky % n, kx % n] += samples[:, si, i]
                count[ky % n, kx % n] += 1
    hit = count > 0
    y = np.zeros_like(total)
    y[:, hit] = total[:, hit] / count[hit]
    return y, hit.astype(np.uint8)


def image(s: Setup, x: np.ndarray) -> np.ndarray:
    """Coil-combined image rho * sqrt(sum_j |c_j|^2) on Omega, centred (row i holds the signed coordinate i - fov):
    the customary NLINV output, which removes the rho -> s rho, c -> c / s ambiguity up to a phase.  The paper does
    not describe its post-processing; this is a reading."""
    full = x[0] * np.sqrt(np.sum(np.abs(coils(s, x)) ** 2, axis=0))
    shifted = np.fft.fftshift(full)
    h = s.n // 2
    return shifted[h - s.fov: h + s.fov, h - s.fov: h + s.fov]


# ---------------------------------------------------------------------------------------------------------------
# Conjugate gradients and the iteratively regularised Gauss-Newton method (Eq. 3)
# ---------------------------------------------------------------------------------------------------------------

# Rounding floor of CG: |r|^2 <= CG_FLOOR2 |b|^2 with 2^-24 the unit roundoff of the FP32 arithmetic (Sec. 3.2).
CG_FLOOR2 = 2.0 ** -48


def cg(apply_A, b: np.ndarray, iters: int, info: dict | None = None, floor2: float = CG_FLOOR2) -> np.ndarray:
    """Conjugate gradients for A dx = b, A Hermitian positive definite, from dx = 0, for a fixed count.

    Per iteration (Table 1, row CG: two scalar products): q = A p; alpha = |r|^2 / Re<p, q>; dx += alpha p;
    r -= alpha q; beta = |r_new|^2 / |r|^2; p = r + beta p.  Stops early only at the rounding floor of the
    single-precision method: |r|^2 <= floor2 |b|^2 (floor2 = CG_FLOOR2 = 2^-48, |r| at the FP32 unit roundoff
    relative to |b|; this includes b = 0), Re<p, q> <= 0, or a non-finite value.  No later iteration of this solve
    changes dx.  ``info``, if given, receives ``info["stop"]``: the index of the iteration that stopped, or -1 when
    all ``iters`` iterations ran.  ``floor2 = 0`` gives plain CG (stopping only at |r| = 0).
    """
    dx = np.zeros_like(b)
    r = b.copy()
    p = r.copy()
    rr = inner(r, r).real
    rr0 = rr
    if info is not None:
        info["stop"] = -1
    for it in range(iters):
        if not (rr > floor2 * rr0 and np.isfinite(rr)):
            if info is not None:
                info["stop"] = it
            break
        q = apply_A(p)
        pq = inner(p, q).real
        if not (pq > 0.0 and np.isfinite(pq)):
            if info is not None:
                info["stop"] = it
            break
        a = rr / pq
        dx = dx + a * p
        r = r - a * q
        rr_new = inner(r, r).real
        beta = rr_new / rr
        p = r + beta * p
        rr = rr_new
    return dx


def residual(s: Setup, mask: np.ndarray, y: np.ndarray, x: np.ndarray):
    """r = y - F(x) and its norm (Table 1, row F: one scalar product)."""
    r = y - forward(s, mask, x)
    return r, float(np.sqrt(inner(r, r).real))


def alpha_schedule(newton_steps: int, alpha0: float, q: float, alpha_min: float = 0.0) -> list:
    """alpha_n = max(alpha_0 q^n, alpha_min) for n = 0 .. newton_steps-1."""
    return [max(alpha0 * q ** k, alpha_min) for k in range(newton_steps)]


def irgnm(s: Setup, mask: np.ndarray, y: np.ndarray, x0: np.ndarray, xref: np.ndarray | None,
          newton_steps: int, cg_iters: int, alpha0: float = 1.0, q: float = 0.5, alpha_min: float = 0.0,
          cg_stops: list | None = None):
    """Iteratively regularised Gauss-Newton method (Eq. 3).

    For n = 0 .. newton_steps-1: b = DF^H(y - F x_n) - alpha_n (x_n - x_ref); solve
    (DF^H DF + alpha_n I) dx = b by ``cg_iters`` CG iterations; x_{n+1} = x_n + dx.
    ``xref=None`` regularises toward x0.  Returns x_N and the residual norms |y - F x_n| for n = 0 .. N.
    ``cg_stops``, if given, receives per Newton step the CG iteration that reached the rounding floor (-1: none).
    """
    x = np.array(x0, dtype=np.complex128, copy=True)
    xr = x.copy() if xref is None else np.asarray(xref, dtype=np.complex128)
    norms = []
    for alpha in alpha_schedule(newton_steps, alpha0, q, alpha_min):
        info = {}
        x, nr = newton_step(s, mask, y, x, xr, alpha, cg_iters, info)
        norms.append(nr)
        if cg_stops is not None:
            cg_stops.append(info["stop"])
    norms.append(residual(s, mask, y, x)[1])
    return x, norms


def newton_step(s: Setup, mask: np.ndarray, y: np.ndarray, x: np.ndarray, xr: np.ndarray, alpha: float,
                cg_iters: int, info: dict | None = None):
    """One step of Eq. 3: b = DF^H(y - F x) - alpha (x - x_ref), (DF^H DF + alpha I) dx = b by CG, x + dx.
    Returns the new iterate and |y - F x| at the old one (``info`` as for :func:`cg`)."""
    r0, nr = residual(s, mask, y, x)
    c = coils(s, x)
    b = adjoint(s, mask, x, r0, c) - alpha * (x - xr)
    dx = cg(lambda d: normal(s, mask, x, d, alpha, c), b, cg_iters, info)
    return x + dx, nr


def irgnm_path(s: Setup, mask: np.ndarray, y: np.ndarray, x0: np.ndarray, xref: np.ndarray | None,
               newton_steps: int, cg_iters: int, alpha0: float = 1.0, q: float = 0.5, alpha_min: float = 0.0):
    """irgnm with every iterate kept: returns [x_0 .. x_N] and [alpha_0 .. alpha_{N-1}] (the checkpoints that the
    gradient through the reconstruction needs)."""
    xs = [np.array(x0, dtype=np.complex128, copy=True)]
    xr = xs[0].copy() if xref is None else np.asarray(xref, dtype=np.complex128)
    alphas = alpha_schedule(newton_steps, alpha0, q, alpha_min)
    for alpha in alphas:
        xs.append(newton_step(s, mask, y, xs[-1], xr, alpha, cg_iters)[0])
    return xs, alphas


def irgnm_vjp(s: Setup, mask: np.ndarray, y: np.ndarray, xs, alphas, g: np.ndarray, cg_iters: int):
    """Gradient of a real loss L(x_N) through the Gauss-Newton iteration, from g = dL/dx_N, with every CG solve
    taken as exact (implicit differentiation of each Newton step; exact when CG has converged).  Gradients are
    with respect to the real inner product Re<u, v>: dL = Re<g, dx>.

    With A = DF^H DF + alpha I at x = x_n, the step dx = x_{n+1} - x_n and s = y - F(x) - DF_x dx, the Jacobian
    of x_{n+1} with respect to x_n is d -> A^-1 (DF_d^H s - DF_x^H DF_dx d), using that F is bilinear
    (DF_x d = DF_d x and DF_{x+d} = DF_x + DF_d).  Per step, backwards: u = A^-1 g (CG),
    dL/dy += DF_x u, dL/dx_ref += alpha u, and g <- DF_u^H s - DF_dx^H (DF_x u).
    Returns (dL/dy, dL/dx_0, dL/dx_ref); when the iteration regularises toward x_0, dL/dx_0 is the sum of the
    last two."""
    gy = np.zeros_like(np.asarray(y, dtype=np.complex128))
    gref = np.zeros_like(xs[0])
    g = np.array(g, dtype=np.complex128, copy=True)
    for k in reversed(range(len(alphas))):
        x, alpha = xs[k], alphas[k]
        dx = xs[k + 1] - x
        c = coils(s, x)
        u = cg(lambda d: normal(s, mask, x, d, alpha, c), g, cg_iters)
        v = derivative(s, mask, x, u, c)
        sres = y - forward(s, mask, x) - derivative(s, mask, x, dx, c)
        gy = gy + v
        gref = gref + alpha * u
        g = adjoint(s, mask, u, sres) - adjoint(s, mask, dx, v)
    return gy, g, gref


def realtime_series(s: Setup, masks, ys, x0: np.ndarray, newton_steps: int, cg_iters: int,
                    alpha0: float = 1.0, q: float = 0.5, alpha_min: float = 0.0):
    """Frame-sequential reconstruction with temporal regularisation (Sec. 3.2): frame k starts from, and is
    regularised toward, the result of frame k-1; frame 0 uses x0 for both."""
    out = []
    prev = np.array(x0, dtype=np.complex128, copy=True)
    for mask, y in zip(masks, ys):
        prev, _ = irgnm(s, mask, y, prev, prev, newton_steps, cg_iters, alpha0, q, alpha_min)
        out.append(prev)
    return out
