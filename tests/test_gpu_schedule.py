"""GPU parity of the Gauss-Newton schedule's less common settings (Eq. 3) against the oracle: the regularisation
floored at alpha_min, other reduction factors (alpha_q = 0.3, and 1: alpha constant), a zero CG count (every
Newton step is then the identity: dx = 0), and whole reconstructions at fields of view other than n/4 (Omega
not filling whole column strips, and Omega = the whole grid), which run the general (not f = N/4) passes inside
the CG iteration.

Bar: final x within relative L2 1e-3 of the oracle; x bit-exact where the schedule leaves it unchanged; residual
norms |y - F x_n| within 1e-3 of |y| (the first of them: F x_0 = 0 for chat = 0).  That last bar follows from the
first: F is bilinear (F x = DF_x x / 2), so an iterate within a relative error e of the oracle's moves the residual
norm by up to about |DF_x| e |x|, a small multiple of e |y| near a fit.  The schedule with alpha_q = 0.3 takes alpha
down to 5e-3, where the scaling direction (rho, -chat) of the bilinear F -- a null direction of DF, held only by
alpha -- makes the late Newton steps ill-conditioned: the FP32 iterates then differ from the oracle's by 6e-4 (the
residual norms by 1.3e-4 of |y|), against 2e-8 with the other schedules."""
import numpy as np
import pytest

import oracle.nlinv_oracle as O
from paper_1301_1215_gb300 import synth
from tests.helpers import ensure_built, noisy_data, rel

pytestmark = pytest.mark.gpu
TOL_X = 1e-3


@pytest.fixture(scope="module")
def torch_cuda():
    ensure_built()
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return torch


def _t(torch, a):
    if a.dtype == np.uint8:
        return torch.from_numpy(np.ascontiguousarray(a)).cuda()
    return torch.from_numpy(np.ascontiguousarray(a.astype(np.complex64))).cuda()


def _run(torch, n, J, spokes, newton, cg, seed, fov=None, **sched):
    from paper_1301_1215_gb300.nlinv import Nlinv
    s, fr, y = noisy_data(n, J, spokes, seed, fov=fov)
    y = y.astype(np.complex64).astype(np.complex128)
    x0 = synth.initial_guess(n, J)
    o_sched = {"alpha0": sched.get("alpha0", 1.0), "q": sched.get("alpha_q", 0.5),
               "alpha_min": sched.get("alpha_min", 0.0)}
    stops = []
    xo, ro = O.irgnm(s, fr.mask, y, x0, None, newton, cg, cg_stops=stops, **o_sched)
    with Nlinv(n, J, newton_steps=newton, cg_iters=cg, fov=fov, **sched) as ctx:
        xg, rg = ctx.reconstruct(_t(torch, y), _t(torch, fr.mask), _t(torch, x0), resid=True)
        xg = xg.cpu().numpy()
        print("CG stops, oracle", stops, "GPU", ctx.cg_stops())
    return x0, xo, ro, xg, rg


@pytest.mark.parametrize("alpha0,alpha_q,alpha_min", [(1.0, 0.5, 0.1), (2.0, 0.3, 0.0), (0.25, 1.0, 0.0)])
def test_alpha_schedule_variants_match_oracle(torch_cuda, alpha0, alpha_q, alpha_min):
    # (1, 0.5, 0.1): alpha 1, 0.5, 0.25, 0.125, then floored at 0.1 for the last two steps
    assert O.alpha_schedule(6, alpha0, alpha_q, alpha_min)[-1] == (0.1 if alpha_min else alpha0 * alpha_q ** 5)
    _, xo, ro, xg, rg = _run(torch_cuda, 64, 4, 16, 6, 12, 2101, alpha0=alpha0, alpha_q=alpha_q,
                             alpha_min=alpha_min)
    print(f"alpha {alpha0}, {alpha_q}, {alpha_min}: rel x {rel(xg, xo):.3g}, residual differences / |y| "
          f"{max(abs(a - b) for a, b in zip(rg, ro)) / ro[0]:.3g}, last residual relative "
          f"{abs(rg[-1] - ro[-1]) / ro[-1]:.3g}")
    assert rel(xg, xo) < TOL_X
    assert np.allclose(rg, ro, rtol=0, atol=TOL_X * ro[0]), (rel(xg, xo), rg, ro)


def test_zero_cg_iterations_leave_x_unchanged(torch_cuda):
    x0, xo, ro, xg, rg = _run(torch_cuda, 64, 4, 16, 3, 0, 2102)
    assert np.array_equal(xo, x0)
    assert np.array_equal(xg, x0.astype(np.complex64))
    # every Newton step evaluates |y - F x_0|: the same norm each time, as in the oracle
    assert np.allclose(rg, ro, rtol=1e-4, atol=0)
    assert np.allclose(rg, rg[0], rtol=1e-6, atol=0)


@pytest.mark.parametrize("n,J,spokes,fov", [(96, 3, 14, 20), (64, 2, 16, 32), (160, 4, 20, 37)])
def test_field_of_view_variants_match_oracle(torch_cuda, n, J, spokes, fov):
    _, xo, ro, xg, rg = _run(torch_cuda, n, J, spokes, 4, 10, 2103 + n, fov=fov)
    assert rel(xg, xo) < TOL_X
    assert rel(xg[0], xo[0]) < TOL_X
    assert np.allclose(rg, ro, rtol=0, atol=TOL_X * ro[0]), (rel(xg, xo), rg, ro)
