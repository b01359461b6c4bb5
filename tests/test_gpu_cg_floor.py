"""The CG rounding floor on the GPU against the oracle's rule (both: the solve stops once |r| <= 2^-24 |b|,
Re<p, A p> <= 0 or a value is not finite, and no later iteration of that solve changes dx).

Small, well-conditioned systems run with many more CG iterations than they need, so that the FP32 solve reaches
its floor mid-solve; before the floor was latched, the iterations after it took steps along directions that were
no longer conjugate (and on the 16 x 16 case below diverged to inf).  Bar: the Gauss-Newton bar, 1e-3 on x and
1e-4 on the residual norms."""
import numpy as np
import pytest

import oracle.nlinv_oracle as O
from paper_1301_1215_gb300 import synth
from tests.helpers import ensure_built, noisy_data, rel

pytestmark = pytest.mark.gpu


def _t(torch, a):
    if a.dtype == np.uint8:
        return torch.from_numpy(np.ascontiguousarray(a)).cuda()
    return torch.from_numpy(np.ascontiguousarray(a.astype(np.complex64))).cuda()


@pytest.mark.parametrize("n,J,spokes,alpha0,newton,cg_iters", [
    (16, 1, 5, 1e-2, 2, 300),       # many more iterations than the 512 unknowns need
    (16, 2, 5, 1e-3, 2, 600),
    (64, 4, 16, 1.0, 7, 30),        # the small single-frame schedule: the FP32 solves reach the floor early
])
def test_floor_reached_and_result_matches_oracle(n, J, spokes, alpha0, newton, cg_iters):
    ensure_built()
    import torch
    from paper_1301_1215_gb300.nlinv import Nlinv
    s, fr, y = noisy_data(n, J, spokes, 91)
    y = y.astype(np.complex64).astype(np.complex128)
    x0 = synth.initial_guess(n, J)
    stops_o = []
    xo, ro = O.irgnm(s, fr.mask, y, x0, None, newton, cg_iters, alpha0=alpha0, cg_stops=stops_o)
    with Nlinv(n, J, newton_steps=newton, cg_iters=cg_iters, alpha0=alpha0) as ctx:
        xg, rg = ctx.reconstruct(_t(torch, y), _t(torch, fr.mask), _t(torch, x0), resid=True)
        stops_g = ctx.cg_stops()
    xg = xg.cpu().numpy()
    assert np.isfinite(xg).all()
    assert stops_g[0] >= 0, (stops_g, stops_o)             # the floor was reached on the GPU
    assert rel(xg, xo) < 1e-3, (stops_g, stops_o)
    assert np.allclose(rg, ro, rtol=1e-4, atol=0), (stops_g, stops_o)


def test_zero_right_hand_side_stops_at_the_first_iteration():
    ensure_built()
    import torch
    from paper_1301_1215_gb300.nlinv import Nlinv
    n, J = 32, 2
    x0 = synth.initial_guess(n, J)
    with Nlinv(n, J, newton_steps=3, cg_iters=5) as ctx:
        x = ctx.reconstruct(_t(torch, np.zeros((J, n, n), complex)), _t(torch, synth.radial_mask(n, 5)),
                            _t(torch, x0))
        assert ctx.cg_stops() == [0, 0, 0]
    stops = []
    O.irgnm(O.Setup(n, J, n // 4), synth.radial_mask(n, 5), np.zeros((J, n, n), complex), x0, None, 3, 5,
            cg_stops=stops)
    assert stops == [0, 0, 0]
    assert np.array_equal(x.cpu().numpy(), x0.astype(np.complex64))
