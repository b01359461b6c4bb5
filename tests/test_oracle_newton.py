"""Pins for the Gauss-Newton side of the oracle (Eq. 3): the alpha schedule, one Newton step as the minimiser of
its Tikhonov functional, a chain of Newton steps, and the rounding-floor rule of CG.

Each Newton step of Eq. 3 solves (DF^H DF + alpha_n I) dx = DF^H (y - F x_n) - alpha_n (x_n - x_ref), which is the
normal equation of  min_d |y - F x_n - J d|^2 + alpha_n |x_n + d - x_ref|^2  with J the (complex-linear) Jacobian
DF_{x_n}.  Here J is built column by column from the derivative (itself pinned by central differences), and the
minimiser is computed by dense linear algebra, independently of the oracle's adjoint, normal operator and CG."""
import numpy as np
import pytest

import oracle.nlinv_oracle as O
from paper_1301_1215_gb300 import synth


def rel(a, b):
    return np.linalg.norm(np.ravel(a - b)) / np.linalg.norm(np.ravel(b))


def test_alpha_schedule_halves_from_alpha0():
    # the real-time setting: alpha_0 = 1, halved every Newton step
    assert O.alpha_schedule(7, 1.0, 0.5) == [1.0, 0.5, 0.25, 0.125, 0.0625, 0.03125, 0.015625]
    assert O.alpha_schedule(1, 3.0, 0.5) == [3.0]


def test_alpha_schedule_floor():
    assert O.alpha_schedule(5, 1.0, 0.5, 0.1) == [1.0, 0.5, 0.25, 0.125, 0.1]
    assert O.alpha_schedule(3, 2.0, 1.0, 0.0) == [2.0, 2.0, 2.0]


def _tiny_system(seed, n=8, J=2, fov=2, spokes=3):
    s = O.Setup(n, J, fov)
    rng = synth.rng_for(seed)
    x = synth.random_complex((1 + J, n, n), rng)
    xref = synth.random_complex((1 + J, n, n), rng)
    y = synth.random_complex((J, n, n), rng) * synth.radial_mask(n, spokes)
    return s, synth.radial_mask(n, spokes), x, xref, y


def dense_jacobian(s, mask, x):
    """DF_x as a dense complex matrix, one column per unit vector of the unknown."""
    dim = (1 + s.ncoils) * s.n * s.n
    cols = []
    for i in range(dim):
        e = np.zeros(dim, complex)
        e[i] = 1.0
        cols.append(O.derivative(s, mask, x, e.reshape(1 + s.ncoils, s.n, s.n)).ravel())
    return np.stack(cols, axis=1)


def tikhonov_step(s, mask, y, x, xref, alpha):
    """x + argmin_d |y - F x - J d|^2 + alpha |x + d - xref|^2, by a dense solve."""
    Jm = dense_jacobian(s, mask, x)
    res = (y - O.forward(s, mask, x)).ravel()
    lhs = Jm.conj().T @ Jm + alpha * np.eye(Jm.shape[1])
    rhs = Jm.conj().T @ res - alpha * (x - xref).ravel()
    return x + np.linalg.solve(lhs, rhs).reshape(x.shape)


def test_jacobian_is_complex_linear_derivative():
    # the columns reproduce DF_x d for a random d (complex linearity: DF_x (i d) = i DF_x d)
    s, mask, x, _, _ = _tiny_system(41)
    Jm = dense_jacobian(s, mask, x)
    d = synth.random_complex(x.shape, synth.rng_for(42))
    assert rel(Jm @ d.ravel(), O.derivative(s, mask, x, d).ravel()) < 1e-12
    assert rel(Jm @ (1j * d).ravel(), 1j * O.derivative(s, mask, x, d).ravel()) < 1e-12


@pytest.mark.parametrize("alpha", [1.0, 0.125])
def test_newton_step_is_the_tikhonov_minimiser(alpha):
    s, mask, x, xref, y = _tiny_system(43)
    want = tikhonov_step(s, mask, y, x, xref, alpha)
    got, nr = O.newton_step(s, mask, y, x, xref, alpha, 600)
    assert rel(got, want) < 1e-6          # CG stops at the FP32 rounding floor, |r| <= 2^-24 |b|
    assert abs(nr - np.linalg.norm(y - O.forward(s, mask, x))) < 1e-12 * nr


def test_irgnm_chains_tikhonov_minimisers_with_halved_alpha():
    s, mask, x0, xref, y = _tiny_system(47)
    x = x0
    for alpha in (1.0, 0.5, 0.25):
        x = tikhonov_step(s, mask, y, x, xref, alpha)
    got, norms = O.irgnm(s, mask, y, x0, xref, 3, 600, alpha0=1.0, q=0.5)
    assert rel(got, x) < 1e-6
    assert len(norms) == 4


def test_planted_alpha_off_by_one_is_caught(monkeypatch):
    """A schedule that starts at alpha_0 q instead of alpha_0 must fail the chained-minimiser pin."""
    s, mask, x0, xref, y = _tiny_system(47)
    x = x0
    for alpha in (1.0, 0.5):
        x = tikhonov_step(s, mask, y, x, xref, alpha)
    good, _ = O.irgnm(s, mask, y, x0, xref, 2, 600)
    monkeypatch.setattr(O, "alpha_schedule",
                        lambda k, a0, q, amin=0.0: [max(a0 * q ** (i + 1), amin) for i in range(k)])
    bad, _ = O.irgnm(s, mask, y, x0, xref, 2, 600)
    assert rel(good, x) < 1e-6 and rel(bad, x) > 1e-3


def test_planted_regulariser_sign_is_caught():
    """b = DF^H r0 + alpha (x - x_ref) (a flipped sign) is not the minimiser."""
    s, mask, x, xref, y = _tiny_system(43)
    alpha = 0.5
    want = tikhonov_step(s, mask, y, x, xref, alpha)
    r0, _ = O.residual(s, mask, y, x)
    c = O.coils(s, x)
    b = O.adjoint(s, mask, x, r0, c) + alpha * (x - xref)
    bad = x + O.cg(lambda d: O.normal(s, mask, x, d, alpha, c), b, 600)
    assert rel(bad, want) > 1e-3


def test_cg_stops_at_the_floor_and_leaves_dx_unchanged():
    # A = 2 I: the first step is exact in binary arithmetic (alpha = 1/2), so |r|^2 is exactly 0 afterwards and
    # the solve stops at iteration 1 with dx = b / 2
    b = np.array([1.0, 2.0 - 1.0j], complex)
    info = {}
    dx = O.cg(lambda v: 2.0 * v, b, 10, info)
    assert info["stop"] == 1 and np.array_equal(dx, 0.5 * b)
    info1 = {}
    assert np.array_equal(O.cg(lambda v: 2.0 * v, b, 1, info1), dx) and info1["stop"] == -1


def test_cg_stops_at_the_fp32_roundoff_of_the_residual():
    # A = diag(1, 2), b = (1, t): the first step leaves r = b - a A b with a = |b|^2 / <b, A b>; for t = 2^-13 the
    # remaining |r|^2 / |b|^2 is about t^2 / 4 ~ 2^-28 (above the floor: the solve continues), for t = 2^-26 it is
    # about 2^-54 (below 2^-48: the solve stops at iteration 1).
    A = np.diag([1.0, 2.0]).astype(complex)
    assert O.CG_FLOOR2 == 2.0 ** -48
    for t, stop in ((2.0 ** -13, -1), (2.0 ** -26, 1)):
        b = np.array([1.0, t], complex)
        a = np.vdot(b, b).real / np.vdot(b, A @ b).real
        r = b - a * (A @ b)
        ratio = np.vdot(r, r).real / np.vdot(b, b).real
        assert (ratio <= O.CG_FLOOR2) == (stop == 1)
        info = {}
        O.cg(lambda v: A @ v, b, 2, info)
        assert info["stop"] == stop, (t, ratio)


def test_cg_stops_on_non_positive_curvature():
    # an indefinite A: the first direction has Re<p, A p> = 0, so the solve stops at iteration 0 with dx = 0
    A = np.diag([1.0, -1.0]).astype(complex)
    info = {}
    dx = O.cg(lambda v: A @ v, np.array([1.0, 1.0], complex), 5, info)
    assert info["stop"] == 0 and not dx.any()


@pytest.mark.parametrize("scale", [1e-12, 1e12])
def test_cg_floor_is_relative_to_the_right_hand_side(scale):
    # CG is scale-equivariant: b -> s b gives dx -> s dx in exact arithmetic, and a floor relative to |b| stops
    # on the same iteration (the scaled arithmetic rounds differently, hence the 1e-12 comparison)
    rng = synth.rng_for(29)
    B = synth.random_complex((12, 8), rng)
    A = B.conj().T @ B + 0.1 * np.eye(8)
    b = synth.random_complex((8,), rng)
    ref_info, info = {}, {}
    ref = O.cg(lambda v: A @ v, b, 8, ref_info)
    got = O.cg(lambda v: A @ v, scale * b, 8, info)
    assert info["stop"] == ref_info["stop"]
    assert np.linalg.norm(got / scale - ref) < 1e-12 * np.linalg.norm(ref)

