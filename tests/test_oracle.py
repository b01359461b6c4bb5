"""Pins for the CPU oracle: each check ties a piece of the oracle to something other than itself (a direct
definition on tiny grids, a library routine, a closed form, an invariant or the paper's Table 1)."""
import os

import numpy as np
import pytest

import oracle.nlinv_oracle as O
from paper_1301_1215_gb300 import synth

HERE = os.path.dirname(os.path.abspath(__file__))


def rel(a, b):
    return np.linalg.norm(np.ravel(a - b)) / np.linalg.norm(np.ravel(b))


def direct_dft2(a):
    """Unitary 2D DFT written out term by term (O(n^4)), natural index order."""
    n = a.shape[-1]
    out = np.zeros_like(a, dtype=np.complex128)
    for k1 in range(n):
        for k2 in range(n):
            acc = 0j
            for x1 in range(n):
                for x2 in range(n):
                    acc += a[x1, x2] * np.exp(-2j * np.pi * (k1 * x1 + k2 * x2) / n)
            out[k1, k2] = acc / n
    return out


# ----------------------------------------------------------------------------------------------------- FFT ----

@pytest.mark.parametrize("n", [2, 3, 4, 5, 6, 8, 12])
def test_fft_matches_direct_definition(n):
    a = synth.random_complex((n, n), synth.rng_for(n))
    assert rel(O.fft2u(a), direct_dft2(a)) < 1e-13
    assert rel(O.ifft2u(O.fft2u(a)), a) < 1e-13


def test_inverse_fft_is_adjoint_and_parseval():
    rng = synth.rng_for(7)
    a, b = synth.random_complex((3, 24, 24), rng), synth.random_complex((3, 24, 24), rng)
    assert abs(O.inner(O.fft2u(a), b) - O.inner(a, O.ifft2u(b))) < 1e-12 * np.linalg.norm(a) * np.linalg.norm(b)
    assert abs(np.linalg.norm(O.fft2u(a)) - np.linalg.norm(a)) < 1e-12 * np.linalg.norm(a)


def test_fft_of_delta_is_flat():
    n = 16
    d = np.zeros((n, n), complex)
    d[0, 0] = 1.0
    assert np.allclose(O.fft2u(d), 1.0 / n, atol=1e-15)


# ------------------------------------------------------------------------------------------ weight and mask ----

def test_signed_index_matches_fftshift():
    for n in (8, 9, 64):
        g = O.signed_index(n)
        assert np.array_equal(np.fft.fftshift(g), np.arange(n) - n // 2)


def test_sobolev_weight_properties():
    n = 64
    w = O.sobolev_weight(n, 220.0, 32.0)
    assert w[0, 0] == 1.0
    assert np.all(w > 0) and np.all(w <= 1.0)
    # even: w(k) = w(-k) in both axes
    idx = (-np.arange(n)) % n
    assert np.array_equal(w, w[idx][:, idx])
    # strictly decreasing with |k| along an axis, from DC to Nyquist
    axis = w[0, : n // 2 + 1]
    assert np.all(np.diff(axis) < 0) or np.all(np.diff(w[0, [0] + list(range(n // 2, n))[::-1]]) < 0)
    # a = 0 or l = 0 turn W into the plain transform
    assert np.array_equal(O.sobolev_weight(n, 0.0, 32.0), np.ones((n, n)))
    assert np.array_equal(O.sobolev_weight(n, 220.0, 0.0), np.ones((n, n)))
    # with l = 2 the reciprocal is 1 + a|k|^2: additive over the axes, unit step 1/n^2, Nyquist |k| = 1/2
    v = 1.0 / O.sobolev_weight(n, 1.0, 2.0) - 1.0
    assert np.allclose(v, v[:, :1] + v[:1, :], rtol=0, atol=1e-15)
    assert np.isclose(v[1, 0], 1.0 / n**2) and np.isclose(v[n // 2, 0], 0.25)


def test_omega_is_centred_square():
    for n, fov in [(16, 4), (64, 16), (80, 20), (12, 6)]:
        M = O.omega_mask(n, fov)
        assert M.sum() == (2 * fov) ** 2
        S = np.fft.fftshift(M)
        ref = np.zeros((n, n))
        ref[n // 2 - fov: n // 2 + fov, n // 2 - fov: n // 2 + fov] = 1
        assert np.array_equal(S, ref)


def test_Wi_delta_and_plain_case():
    s = O.Setup(16, 1, 4)
    d = np.zeros((1, 16, 16), complex)
    d[0, 0, 0] = 1.0
    assert np.allclose(O.Wi(s, d), 1.0 / 16, atol=1e-15)      # w(0) = 1: a constant map
    s0 = O.Setup(16, 2, 4, a=0.0)
    c = synth.random_complex((2, 16, 16), synth.rng_for(3))
    assert rel(O.Wi(s0, c), np.fft.ifft2(c, norm="ortho")) < 1e-14


def test_WiH_is_adjoint_of_Wi():
    s = O.Setup(24, 3, 6, a=5.0, l=4.0)
    rng = synth.rng_for(11)
    c, u = synth.random_complex((3, 24, 24), rng), synth.random_complex((3, 24, 24), rng)
    lhs, rhs = O.inner(O.Wi(s, c), u), O.inner(c, O.WiH(s, u))
    assert abs(lhs - rhs) < 1e-13 * abs(lhs)


# ---------------------------------------------------------------------------------------------- operators ----

def brute_forward(s, mask, x):
    """Eq. 2 evaluated term by term on a tiny grid: coils from the weighted inverse DFT of chat, then the DFT of
    rho c_j over the pixels of Omega, then the sampling pattern."""
    n = s.n
    g = [((i + n // 2) % n) - n // 2 for i in range(n)]
    inside = [(-s.fov <= g[i] < s.fov) for i in range(n)]

    def w(k1, k2):
        return (1.0 + s.a * ((g[k1] / n) ** 2 + (g[k2] / n) ** 2)) ** (-s.l / 2.0)

    y = np.zeros((s.ncoils, n, n), complex)
    for j in range(s.ncoils):
        c = np.zeros((n, n), complex)
        for p1 in range(n):
            for p2 in range(n):
                acc = 0j
                for k1 in range(n):
                    for k2 in range(n):
                        acc += w(k1, k2) * x[1 + j, k1, k2] * np.exp(2j * np.pi * (k1 * p1 + k2 * p2) / n)
                c[p1, p2] = acc / n
        for k1 in range(n):
            for k2 in range(n):
                acc = 0j
                for p1 in range(n):
                    for p2 in range(n):
                        if inside[p1] and inside[p2]:
                            acc += x[0, p1, p2] * c[p1, p2] * np.exp(-2j * np.pi * (k1 * p1 + k2 * p2) / n)
                y[j, k1, k2] = mask[k1, k2] * acc / n
    return y


@pytest.mark.parametrize("a,l", [(3.0, 4.0), (220.0, 32.0)])
def test_forward_matches_term_by_term_definition(a, l):
    s = O.Setup(8, 2, 2, a=a, l=l)
    rng = synth.rng_for(5)
    x = synth.random_complex((3, 8, 8), rng)
    mask = (rng.uniform(size=(8, 8)) < 0.5).astype(np.uint8)
    assert rel(O.forward(s, mask, x), brute_forward(s, mask, x)) < 1e-12


def test_forward_with_flat_coil_is_masked_fft():
    # a = 0 and chat = n delta_0 give c = 1 everywhere, so F(rho) = P FFT(M rho): a library transform.
    n, fov = 32, 8
    s = O.Setup(n, 1, fov, a=0.0)
    rng = synth.rng_for(9)
    x = np.zeros((2, n, n), complex)
    x[0] = synth.random_complex((n, n), rng)
    x[1, 0, 0] = n
    mask = synth.radial_mask(n, 6)
    M = O.omega_mask(n, fov)
    ref = mask * np.fft.fft2(M * x[0], norm="ortho")
    assert rel(O.forward(s, mask, x)[0], ref) < 1e-13
    r = synth.random_complex((1, n, n), rng)
    ref_adj = M * np.fft.ifft2(mask * r[0], norm="ortho")
    assert rel(O.adjoint(s, mask, x, r)[0], ref_adj) < 1e-13


def test_forward_reproduces_signal_equation_data():
    # chat = FFT(c_true) / w is the exact preimage of a known coil map, so F(rho, chat) equals the simulated data.
    n, J, fov = 32, 3, 8
    s = O.Setup(n, J, fov, a=4.0, l=2.0)
    fr = synth.make_frame(n, J, 8, seed=21)
    w = O.sobolev_weight(n, s.a, s.l)
    x = np.concatenate([fr.rho[None], O.fft2u(fr.coils) / w])
    assert rel(O.forward(s, fr.mask, x), O.simulate(s, fr.mask, fr.rho, fr.coils)) < 1e-12


def test_simulate_ignores_the_image_outside_omega():
    # Eq. 2 restricts the image to Omega (M_Omega) before the coil product, so the data of a rho that also has
    # content outside Omega equal those of its restriction to Omega, and differ from the unrestricted product's.
    n, J, fov = 32, 3, 8
    s = O.Setup(n, J, fov)
    rng = synth.rng_for(23)
    rho = synth.random_complex((n, n), rng)
    c = synth.random_complex((J, n, n), rng)
    mask = synth.radial_mask(n, 9)
    inside = O.omega_mask(n, fov)
    assert inside.sum() < n * n
    y = O.simulate(s, mask, rho, c)
    assert rel(y, O.simulate(s, mask, inside * rho, c)) < 1e-14
    assert rel(y, mask * np.fft.fft2(rho * c, norm="ortho")) > 0.1


def test_inner_product_conjugates_its_first_argument():
    # Table 1's scalar product <u, v> = sum conj(u) v, on values worked by hand
    assert O.inner(np.array([1j]), np.array([1.0])) == -1j
    assert O.inner(np.array([1.0, 2j]), np.array([3.0, 1.0])) == 3 - 2j
    assert O.inner(np.array([[2 - 1j]]), np.array([[1j]])) == (2 + 1j) * 1j


def setup_random(n=32, J=3, fov=8, seed=13):
    s = O.Setup(n, J, fov)
    rng = synth.rng_for(seed)
    x = synth.random_complex((1 + J, n, n), rng)
    d = synth.random_complex((1 + J, n, n), rng)
    r = synth.random_complex((J, n, n), rng)
    mask = synth.radial_mask(n, 7)
    return s, mask, x, d, r


@pytest.mark.parametrize("eps", [1e-3, 1.0, 30.0])
def test_derivative_equals_central_difference(eps):
    # F is bilinear in (rho, chat): the second-order terms cancel in a central difference for every eps.
    s, mask, x, d, _ = setup_random()
    fd = (O.forward(s, mask, x + eps * d) - O.forward(s, mask, x - eps * d)) / (2 * eps)
    assert rel(fd, O.derivative(s, mask, x, d)) < 1e-10


def test_one_sided_difference_has_closed_form_remainder():
    s, mask, x, d, _ = setup_random()
    eps = 0.5
    lhs = O.forward(s, mask, x + eps * d) - O.forward(s, mask, x)
    M = O.omega_mask(s.n, s.fov)
    rem = mask * O.fft2u(M * d[0] * O.Wi(s, d[1:]))
    assert rel(lhs, eps * O.derivative(s, mask, x, d) + eps * eps * rem) < 1e-12


def test_adjoint_identity():
    s, mask, x, d, r = setup_random(n=40, J=4, fov=10)
    lhs = O.inner(O.derivative(s, mask, x, d), r)
    rhs = O.inner(d, O.adjoint(s, mask, x, r))
    assert abs(lhs.real - rhs.real) < 1e-12 * abs(lhs) and abs(lhs.imag - rhs.imag) < 1e-12 * abs(lhs)


def dense_normal(s, mask, x, alpha):
    dim = (1 + s.ncoils) * s.n * s.n
    A = np.zeros((dim, dim), complex)
    for i in range(dim):
        e = np.zeros(dim, complex)
        e[i] = 1.0
        A[:, i] = O.normal(s, mask, x, e.reshape(1 + s.ncoils, s.n, s.n), alpha).ravel()
    return A


def test_normal_operator_is_hermitian_and_bounded_below():
    s = O.Setup(8, 2, 2)
    rng = synth.rng_for(17)
    x = synth.random_complex((3, 8, 8), rng)
    mask = synth.radial_mask(8, 3)
    alpha = 0.25
    A = dense_normal(s, mask, x, alpha)
    assert np.linalg.norm(A - A.conj().T) < 1e-12 * np.linalg.norm(A)
    ev = np.linalg.eigvalsh(0.5 * (A + A.conj().T))
    assert ev.min() > alpha * (1 - 1e-10)


# --------------------------------------------------------------------------------------------- CG, IRGNM ----

def test_cg_solves_small_hermitian_system():
    rng = synth.rng_for(19)
    B = synth.random_complex((30, 20), rng)
    A = B.conj().T @ B + np.eye(20)
    b = synth.random_complex(20, rng)
    dx = O.cg(lambda v: A @ v, b, 60, floor2=0.0)
    assert rel(dx, np.linalg.solve(A, b)) < 1e-10


def test_cg_on_dense_nlinv_system_matches_solve():
    s = O.Setup(8, 2, 2)
    rng = synth.rng_for(23)
    x = synth.random_complex((3, 8, 8), rng)
    mask = synth.radial_mask(8, 3)
    A = dense_normal(s, mask, x, 1.0)
    b = synth.random_complex((3, 8, 8), rng)
    dx = O.cg(lambda v: O.normal(s, mask, x, v, 1.0), b, 400, floor2=0.0)
    assert rel(dx.ravel(), np.linalg.solve(A, b.ravel())) < 1e-9
    # with the FP32 rounding floor the solve stops once |r| <= 2^-24 |b|: the solution to about that level
    info = {}
    dxf = O.cg(lambda v: O.normal(s, mask, x, v, 1.0), b, 400, info)
    assert 0 < info["stop"] < 400 and rel(dxf.ravel(), np.linalg.solve(A, b.ravel())) < 1e-6


def test_cg_zero_rhs_stays_zero():
    dx = O.cg(lambda v: 2.0 * v, np.zeros((2, 4, 4), complex), 5)
    assert not dx.any()


def test_cg_single_iteration_is_steepest_descent_step():
    rng = synth.rng_for(29)
    A = np.diag(np.arange(1.0, 9.0)).astype(complex)
    b = synth.random_complex(8, rng)
    dx = O.cg(lambda v: A @ v, b, 1)
    t = np.vdot(b, b).real / np.vdot(b, A @ b).real
    assert rel(dx, t * b) < 1e-14


def _noiseless(n, J, spokes, seed):
    s = O.Setup(n, J, n // 4)
    fr = synth.make_frame(n, J, spokes, seed=seed)
    return s, fr, O.simulate(s, fr.mask, fr.rho, fr.coils)


def test_irgnm_residual_non_increasing_on_noiseless_phantom():
    s, fr, y = _noiseless(32, 3, 12, seed=31)
    x0 = synth.initial_guess(32, 3)
    _, norms = O.irgnm(s, fr.mask, y, x0, None, 6, 20)
    assert all(b <= a * (1 + 1e-12) for a, b in zip(norms, norms[1:]))
    assert norms[-1] < 0.75 * norms[0]


def test_irgnm_fully_sampled_recovers_coil_images():
    n, J = 32, 3
    s = O.Setup(n, J, n // 4)
    fr = synth.make_frame(n, J, 12, seed=37)
    full = np.ones((n, n), np.uint8)
    y = O.simulate(s, full, fr.rho, fr.coils)
    M = O.omega_mask(n, s.fov)
    errs = []
    for steps in (4, 8, 16):
        x, _ = O.irgnm(s, full, y, synth.initial_guess(n, J), None, steps, 30)
        errs.append(rel(M * x[0] * O.coils(s, x), M * fr.rho * fr.coils))
    # the coil images rho c_j (invariant under rho -> s rho, c -> c / s) approach the truth as alpha_n shrinks
    assert errs[0] > errs[1] > errs[2] and errs[2] < 0.1


def test_realtime_series_chains_frames():
    n, J = 16, 2
    s = O.Setup(n, J, 4)
    frames = [synth.make_frame(n, J, 5, seed=41, frame=k) for k in range(3)]
    ys = [O.simulate(s, f.mask, f.rho, f.coils) for f in frames]
    out = O.realtime_series(s, [f.mask for f in frames], ys, synth.initial_guess(n, J), 2, 5)
    x1, _ = O.irgnm(s, frames[1].mask, ys[1], out[0], out[0], 2, 5)
    assert rel(out[1], x1) < 1e-14


# -------------------------------------------------------------------------------------------- Table 1 ----

def _table1():
    rows = {}
    with open(os.path.join(HERE, "golden", "table1_operator_breakdown.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                name, *vals = line.split()
                rows[name] = dict(zip(["fft", "elementwise", "channel_sum", "scalar_product", "gpu_sum"],
                                      map(int, vals)))
    return rows


def test_operator_breakdown_matches_table1(monkeypatch):
    counts = {"fft": 0, "dot": 0, "sum": 0}
    f, fi, dot, cs = O.fft2u, O.ifft2u, O.inner, O.channel_sum

    def count(key, fn):
        def wrapped(*a, **k):
            counts[key] += 1
            return fn(*a, **k)
        return wrapped

    monkeypatch.setattr(O, "fft2u", count("fft", f))
    monkeypatch.setattr(O, "ifft2u", count("fft", fi))
    monkeypatch.setattr(O, "inner", count("dot", dot))
    monkeypatch.setattr(O, "channel_sum", count("sum", cs))
    s, mask, x, d, r = setup_random(n=16, J=2, fov=4)
    c = O.coils(s, x)
    t1 = _table1()

    def measure(fn):
        for k in counts:
            counts[k] = 0
        fn()
        return dict(counts)

    got = measure(lambda: O.residual(s, mask, r, x))
    assert (got["fft"], got["dot"]) == (t1["F"]["fft"], t1["F"]["scalar_product"])
    got = measure(lambda: O.derivative(s, mask, x, d, c))
    assert (got["fft"], got["dot"], got["sum"]) == (t1["DF"]["fft"], 0, 0)
    got = measure(lambda: O.adjoint(s, mask, x, r, c))
    assert (got["fft"], got["sum"]) == (t1["DFH"]["fft"], t1["DFH"]["channel_sum"])
    # one CG iteration beyond its operator: apply_A is a plain diagonal scaling here
    b = synth.random_complex((3, 16, 16), synth.rng_for(1))
    diag = 1.0 + np.arange(b.size).reshape(b.shape)
    one = measure(lambda: O.cg(lambda v: diag * v, b, 1))
    two = measure(lambda: O.cg(lambda v: diag * v, b, 2))
    assert two["dot"] - one["dot"] == t1["CG"]["scalar_product"] and two["fft"] == t1["CG"]["fft"]


def test_image_of_flat_coils_is_centred_rho():
    # a = 0 and chat = n delta_0 / sqrt(J) per coil give |c_j| = 1/sqrt(J), so sqrt(sum |c_j|^2) = 1
    n, J, fov = 32, 2, 8
    s = O.Setup(n, J, fov, a=0.0)
    x = np.zeros((1 + J, n, n), complex)
    x[0] = synth.random_complex((n, n), synth.rng_for(91))
    x[1:, 0, 0] = n / np.sqrt(J)
    img = O.image(s, x)
    assert img.shape == (2 * fov, 2 * fov)
    ref = np.fft.fftshift(x[0])[n // 2 - fov: n // 2 + fov, n // 2 - fov: n // 2 + fov]
    assert rel(img, ref) < 1e-13
    # invariance: rho -> 2 rho, chat -> chat / 2 leaves the image unchanged
    y = x.copy()
    y[0] *= 2.0
    y[1:] /= 2.0
    assert rel(O.image(s, y), img) < 1e-13


# ------------------------------------------------------------------------ gradient through the reconstruction ----

def _vjp_problem(seed):
    """8x8 grid, 2 coils: the CG solves of Eq. 3 converge to rounding in 250 iterations, so the implicit
    gradient is the exact derivative of the iteration."""
    s = O.Setup(8, 2, 2)
    rng = synth.rng_for(seed)
    mask = synth.radial_mask(8, 3)
    x0 = synth.initial_guess(8, 2) + 0.1 * synth.random_complex((3, 8, 8), rng)
    xref = synth.initial_guess(8, 2) + 0.1 * synth.random_complex((3, 8, 8), rng)
    y = mask * synth.random_complex((2, 8, 8), rng)
    g = synth.random_complex((3, 8, 8), rng)
    return s, rng, mask, x0, xref, y, g


def _loss(s, mask, y, x0, xref, g, newton=2, cg_iters=250):
    x, _ = O.irgnm(s, mask, y, x0, xref, newton, cg_iters)
    return O.inner(g, x).real


@pytest.mark.parametrize("wrt", ["y", "x0", "xref"])
def test_irgnm_vjp_matches_central_differences(wrt):
    s, rng, mask, x0, xref, y, g = _vjp_problem(41)
    xs, alphas = O.irgnm_path(s, mask, y, x0, xref, 2, 250)
    assert np.allclose(xs[-1], O.irgnm(s, mask, y, x0, xref, 2, 250)[0], rtol=0, atol=1e-12)
    gy, gx0, gref = O.irgnm_vjp(s, mask, y, xs, alphas, g, 250)
    eps = 1e-6
    if wrt == "y":
        d = mask * synth.random_complex(y.shape, rng)
        fd = (_loss(s, mask, y + eps * d, x0, xref, g) - _loss(s, mask, y - eps * d, x0, xref, g)) / (2 * eps)
        grad = gy
    elif wrt == "x0":
        d = synth.random_complex(x0.shape, rng)
        fd = (_loss(s, mask, y, x0 + eps * d, xref, g) - _loss(s, mask, y, x0 - eps * d, xref, g)) / (2 * eps)
        grad = gx0
    else:
        d = synth.random_complex(xref.shape, rng)
        fd = (_loss(s, mask, y, x0, xref + eps * d, g) - _loss(s, mask, y, x0, xref - eps * d, g)) / (2 * eps)
        grad = gref
    assert abs(O.inner(grad, d).real - fd) <= 1e-6 * abs(fd)


def test_irgnm_vjp_with_start_as_reference_sums_both_paths():
    """A single frame regularises toward its start value: x_ref = x_0 moves with x_0."""
    s, rng, mask, x0, _, y, g = _vjp_problem(43)
    xs, alphas = O.irgnm_path(s, mask, y, x0, None, 2, 250)
    gy, gx0, gref = O.irgnm_vjp(s, mask, y, xs, alphas, g, 250)
    d = synth.random_complex(x0.shape, rng)
    eps = 1e-6
    fd = (_loss(s, mask, y, x0 + eps * d, None, g) - _loss(s, mask, y, x0 - eps * d, None, g)) / (2 * eps)
    assert abs(O.inner(gx0 + gref, d).real - fd) <= 1e-6 * abs(fd)


def test_irgnm_vjp_ignores_data_outside_the_mask():
    s, rng, mask, x0, xref, y, g = _vjp_problem(47)
    xs, alphas = O.irgnm_path(s, mask, y, x0, xref, 2, 250)
    gy = O.irgnm_vjp(s, mask, y, xs, alphas, g, 250)[0]
    assert not gy[:, mask == 0].any()


# ----------------------------------------------------------------------------------------------- gridding ----

@pytest.mark.parametrize("n,spokes,rot", [(16, 5, 0.0), (64, 16, 0.3), (96, 13, 1.1)])
def test_gridding_pattern_is_the_rasterised_mask(n, spokes, rot):
    """Two independent statements of the spoke rasterisation agree: the gridder's pattern and the input
    generator's sampling mask."""
    angles = [np.pi * k / spokes + rot for k in range(spokes)]
    rng = synth.rng_for(61)
    _, mask = O.grid_radial(n, angles, synth.random_complex((2, spokes, 2 * n), rng))
    assert np.array_equal(mask, synth.radial_mask(n, spokes, rot))


def test_gridding_of_one_horizontal_spoke_by_hand():
    """n = 8, one spoke at angle 0: t = -4, -3.5, ..., 3.5 round to kx = -4, -3, -3, -2, -2, ..., 3, 3 and 4 (dropped),
    so column k (-3..3) of row 0 holds the mean of samples 2k+7 and 2k+8, column -4 sample 0 alone."""
    rng = synth.rng_for(62)
    smp = synth.random_complex((2, 1, 16), rng)
    y, mask = O.grid_radial(8, [0.0], smp)
    want = np.zeros((2, 8, 8), complex)
    want[:, 0, (-4) % 8] = smp[:, 0, 0]
    for k in range(-3, 4):
        want[:, 0, k % 8] = 0.5 * (smp[:, 0, 2 * k + 7] + smp[:, 0, 2 * k + 8])
    assert np.allclose(y, want, rtol=0, atol=1e-15)
    assert mask.sum() == 8 and mask[0].all()


def test_gridding_of_identical_samples_is_that_value():
    angles = [np.pi * k / 7 for k in range(7)]
    smp = np.full((3, 7, 64), 0.25 - 0.5j)
    y, mask = O.grid_radial(32, angles, smp)
    assert np.allclose(y[:, mask == 1], 0.25 - 0.5j, rtol=0, atol=1e-15)
    assert not y[:, mask == 0].any()
