"""Property tests of the oracle over random small problems (grid side, coil count, field of view, Sobolev
parameters, sampling pattern): the identities that hold for any input, checked where hypothesis is available."""
import numpy as np
import pytest

import oracle.nlinv_oracle as O
from paper_1301_1215_gb300 import synth

hyp = pytest.importorskip("hypothesis")
from hypothesis import given, settings, strategies as st  # noqa: E402

problem = st.tuples(st.sampled_from([8, 12, 16]), st.integers(1, 3), st.integers(0, 10_000),
                    st.sampled_from([0.0, 1.0, 220.0]), st.sampled_from([0.0, 2.0, 32.0]))


def _setup(n, J, seed, a, l):
    rng = synth.rng_for(seed)
    fov = int(rng.integers(1, n // 2 + 1))
    s = O.Setup(n, J, fov, a, l)
    mask = (rng.random((n, n)) < 0.4).astype(np.uint8)
    x = synth.random_complex((1 + J, n, n), rng)
    return s, rng, mask, x


@settings(max_examples=25, deadline=None)
@given(problem)
def test_adjoint_identity_holds_for_any_problem(p):
    s, rng, mask, x = _setup(*p)
    d = synth.random_complex(x.shape, rng)
    r = synth.random_complex((s.ncoils, s.n, s.n), rng)
    lhs = O.inner(O.derivative(s, mask, x, d), r)
    rhs = O.inner(d, O.adjoint(s, mask, x, r))
    assert abs(lhs - rhs) <= 1e-11 * max(1.0, abs(lhs))


@settings(max_examples=25, deadline=None)
@given(problem, st.sampled_from([1e-3, 0.5, 3.0]))
def test_central_difference_is_exact_for_any_step(p, eps):
    """F is bilinear, so the central difference equals DF for every step size (up to rounding)."""
    s, rng, mask, x = _setup(*p)
    d = synth.random_complex(x.shape, rng)
    fd = (O.forward(s, mask, x + eps * d) - O.forward(s, mask, x - eps * d)) / (2 * eps)
    df = O.derivative(s, mask, x, d)
    assert np.linalg.norm(fd - df) <= 1e-9 * max(1.0, np.linalg.norm(df))


@settings(max_examples=25, deadline=None)
@given(problem, st.sampled_from([0.01, 1.0, 4.0]))
def test_normal_operator_is_hermitian_positive_definite(p, alpha):
    s, rng, mask, x = _setup(*p)
    u = synth.random_complex(x.shape, rng)
    v = synth.random_complex(x.shape, rng)
    Au, Av = O.normal(s, mask, x, u, alpha), O.normal(s, mask, x, v, alpha)
    assert abs(O.inner(u, Av) - np.conj(O.inner(v, Au))) <= 1e-10 * max(1.0, abs(O.inner(u, Av)))
    assert O.inner(u, Au).real >= alpha * O.inner(u, u).real * (1 - 1e-12)


@settings(max_examples=15, deadline=None)
@given(st.sampled_from([8, 16, 32]), st.integers(1, 6), st.floats(0.0, 3.0), st.integers(0, 10_000))
def test_gridding_is_linear_in_the_samples(n, spokes, rot, seed):
    rng = synth.rng_for(seed)
    angles = [np.pi * k / spokes + rot for k in range(spokes)]
    a = synth.random_complex((2, spokes, 2 * n), rng)
    b = synth.random_complex((2, spokes, 2 * n), rng)
    ya, ma = O.grid_radial(n, angles, a)
    yb, mb = O.grid_radial(n, angles, b)
    yab, mab = O.grid_radial(n, angles, 2.0 * a - 3.0j * b)
    assert np.array_equal(ma, mb) and np.array_equal(ma, mab)
    assert np.allclose(yab, 2.0 * ya - 3.0j * yb, rtol=0, atol=1e-12)
