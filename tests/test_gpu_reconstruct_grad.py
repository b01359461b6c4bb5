"""Gradients through the whole Gauss-Newton reconstruction (nlinv_reconstruct_checkpoints + nlinv_reconstruct_vjp,
wrapped as a torch.autograd.Function) against the oracle's checkpoints and implicit gradient (the oracle's gradient
is pinned by central differences on converged systems in test_oracle.py).  Each side runs its own forward path
from the same seeded inputs; no GPU value enters the oracle.

Bar: checkpoints within 1e-3 relative L2 of the oracle's iterates (the Gauss-Newton bar); gradients within 2e-3
(they add one FP32 CG solve per Newton step on top of the forward path)."""
import numpy as np
import pytest

import oracle.nlinv_oracle as O
from paper_1301_1215_gb300 import synth
from tests.helpers import ensure_built, noisy_data, rel

pytestmark = pytest.mark.gpu
NEWTON, CG = 3, 12


@pytest.fixture(scope="module")
def case():
    ensure_built()
    import torch
    from paper_1301_1215_gb300.nlinv import Nlinv
    n, J = 64, 4
    s, fr, y = noisy_data(n, J, 16, 1001)
    rng = synth.rng_for(71)
    x0 = synth.initial_guess(n, J) + 0.05 * synth.random_complex((1 + J, n, n), rng)
    xref = synth.initial_guess(n, J) + 0.05 * synth.random_complex((1 + J, n, n), rng)
    g = synth.random_complex((1 + J, n, n), rng)
    y, x0, xref, g = (a.astype(np.complex64).astype(np.complex128) for a in (y, x0, xref, g))
    op = Nlinv(n, J, newton_steps=NEWTON, cg_iters=CG)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a).astype(np.complex64)).to(op.device)
    m = torch.from_numpy(fr.mask).to(op.device)
    yield torch, op, s, fr, y, x0, xref, g, t, m
    op.close()


def test_checkpoints_are_the_gauss_newton_iterates(case):
    torch, op, s, fr, y, x0, xref, g, t, m = case
    xN, ck = op.reconstruct_checkpoints(t(y), m, t(x0), t(xref))
    xs, _ = O.irgnm_path(s, fr.mask, y, x0, xref, NEWTON, CG)
    ck = ck.cpu().numpy()
    assert np.array_equal(ck[0], x0.astype(np.complex64))
    for k in range(1, NEWTON + 1):
        assert rel(ck[k], xs[k]) < 1e-3
    assert np.array_equal(ck[-1], xN.cpu().numpy())
    # the same iterate as the plain (graph-replayed) reconstruction
    assert np.array_equal(xN.cpu().numpy(), op.reconstruct(t(y), m, t(x0), t(xref)).cpu().numpy())


def test_vjp_matches_oracle(case):
    torch, op, s, fr, y, x0, xref, g, t, m = case
    _, ck = op.reconstruct_checkpoints(t(y), m, t(x0), t(xref))
    gy, g0, gr = op.reconstruct_vjp(t(y), m, ck, t(g))
    xs, alphas = O.irgnm_path(s, fr.mask, y, x0, xref, NEWTON, CG)
    oy, o0, oref = O.irgnm_vjp(s, fr.mask, y, xs, alphas, g, CG)
    assert rel(gy.cpu().numpy(), oy) < 2e-3
    assert rel(g0.cpu().numpy(), o0) < 2e-3
    assert rel(gr.cpu().numpy(), oref) < 2e-3
    assert not gy.cpu().numpy()[:, fr.mask == 0].any()


def test_autograd_function_gives_the_vjp(case):
    torch, op, s, fr, y, x0, xref, g, t, m = case
    from paper_1301_1215_gb300.autograd import reconstruct
    yt, x0t, xrt = (t(a).requires_grad_(True) for a in (y, x0, xref))
    x = reconstruct(op, yt, m, x0t, xrt)
    loss = torch.real(torch.sum(torch.conj(t(g)) * x))      # Re<g, x_N>: its gradient with respect to x_N is g
    loss.backward()
    _, ck = op.reconstruct_checkpoints(t(y), m, t(x0), t(xref))
    gy, g0, gr = op.reconstruct_vjp(t(y), m, ck, t(g))
    assert torch.equal(yt.grad, gy) and torch.equal(x0t.grad, g0) and torch.equal(xrt.grad, gr)


def test_tied_reference_gradient_is_the_sum(case):
    """A single frame regularises toward its start value: the gradient with respect to that value carries both the
    start and the reference paths, as in the oracle."""
    torch, op, s, fr, y, x0, xref, g, t, m = case
    from paper_1301_1215_gb300.autograd import reconstruct
    x0t = t(x0).requires_grad_(True)
    x = reconstruct(op, t(y), m, x0t)
    torch.real(torch.sum(torch.conj(t(g)) * x)).backward()
    xs, alphas = O.irgnm_path(s, fr.mask, y, x0, None, NEWTON, CG)
    _, o0, oref = O.irgnm_vjp(s, fr.mask, y, xs, alphas, g, CG)
    assert rel(x0t.grad.cpu().numpy(), o0 + oref) < 2e-3
