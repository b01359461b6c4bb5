"""F as a torch.autograd.Function (backward = the DF^H kernel chain) on the 256 x 256, 8-coil, 25-spoke setting:
the gradient of |F(x) - y|^2 against the oracle's 2 DF^H (F x - y) and against central finite differences."""
import numpy as np
import pytest

import oracle.nlinv_oracle as O
from paper_1301_1215_gb300 import synth
from tests.helpers import ensure_built, noisy_data, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    ensure_built()
    import torch
    from paper_1301_1215_gb300.nlinv import Nlinv
    n, J = 256, 8
    s, fr, y = noisy_data(n, J, 25, 1002)
    rng = synth.rng_for(55)
    x = synth.initial_guess(n, J) + 0.1 * synth.random_complex((1 + J, n, n), rng)
    x, y = (a.astype(np.complex64).astype(np.complex128) for a in (x, y))
    op = Nlinv(n, J)
    dev = op.device
    t = lambda a: torch.from_numpy(a.astype(np.complex64)).to(dev)
    yield torch, op, s, fr, x, y, t
    op.close()


def _loss_and_grad(torch, op, x_t, m_t, y_t):
    from paper_1301_1215_gb300.autograd import forward
    xr = x_t.clone().requires_grad_(True)
    loss = (forward(op, xr, m_t) - y_t).abs().pow(2).sum()
    loss.backward()
    return loss.detach(), xr.grad.detach()


def test_gradient_matches_oracle_adjoint(setup):
    torch, op, s, fr, x, y, t = setup
    m_t = torch.from_numpy(fr.mask).to(op.device)
    _, g = _loss_and_grad(torch, op, t(x), m_t, t(y))
    ref = 2.0 * O.adjoint(s, fr.mask, x, O.forward(s, fr.mask, x) - y)
    assert rel(g.cpu().numpy(), ref) < 1e-5


def test_gradient_matches_central_differences(setup):
    torch, op, s, fr, x, y, t = setup
    m_t = torch.from_numpy(fr.mask).to(op.device)
    _, g = _loss_and_grad(torch, op, t(x), m_t, t(y))
    g = g.cpu().numpy().astype(np.complex128)
    rng = synth.rng_for(66)
    for _ in range(3):
        v = synth.random_complex(x.shape, rng)
        v /= np.linalg.norm(v)
        eps = 1e-2 * np.linalg.norm(x)
        def L(z):
            yz = op.forward(t(z), m_t).cpu().numpy().astype(np.complex128)
            return float(np.sum(np.abs(yz - y) ** 2))
        fd = (L(x + eps * v) - L(x - eps * v)) / (2 * eps)
        an = float(np.real(np.vdot(g, v)))
        assert abs(fd - an) <= 1e-3 * max(abs(an), 1e-3 * np.linalg.norm(g))


def test_output_requires_grad_and_gradient_is_finite(setup):
    torch, op, s, fr, x, y, t = setup
    from paper_1301_1215_gb300.autograd import forward
    m_t = torch.from_numpy(fr.mask).to(op.device)
    xr = t(x).requires_grad_(True)
    out = forward(op, xr, m_t)
    assert out.requires_grad and out.shape == (8, 256, 256)
    out.real.sum().backward()
    assert xr.grad is not None and torch.isfinite(torch.view_as_real(xr.grad)).all()
