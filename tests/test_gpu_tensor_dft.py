"""The optional tensor-core path: radix-16 DFT stages as split-BF16, 3-pass contractions on tcgen05 (params
tensor_dft = 1), against the oracle.

Tolerances.  One stage keeps about 16 significant bits (hi*hi + hi*lo + lo*hi of bf16 halves, FP32 accumulation):
relative error ~2^-16 = 1.5e-5 per stage, against ~1e-7 for the FP32 butterflies.  An operator application runs
up to eight such stages (four 2D transforms, one radix-16 stage per 1D transform of a 256 or 512 grid), so the
operators are held to 1e-4 (not the FP32 operators' 1e-5); whole reconstructions to the Gauss-Newton bar, 1e-3."""
import numpy as np
import pytest

import oracle.nlinv_oracle as O
from paper_1301_1215_gb300 import synth
from tests.helpers import ensure_built, noisy_data, rel

pytestmark = pytest.mark.gpu
TOL_OP = 1e-4
TOL_X = 1e-3


def _t(torch, a):
    if a.dtype == np.uint8:
        return torch.from_numpy(np.ascontiguousarray(a)).cuda()
    return torch.from_numpy(np.ascontiguousarray(a.astype(np.complex64))).cuda()


@pytest.mark.parametrize("n,J,fov", [(256, 8, 64), (256, 3, 50), (512, 16, 128)])
def test_operators_with_tensor_core_stages_match_oracle(n, J, fov):
    ensure_built()
    import torch
    from paper_1301_1215_gb300.nlinv import Nlinv
    s = O.Setup(n, J, fov)
    rng = synth.rng_for(400 + n + J)
    x = synth.random_complex((1 + J, n, n), rng)
    d = synth.random_complex((1 + J, n, n), rng)
    r = synth.random_complex((J, n, n), rng)
    mask = synth.radial_mask(n, 21, 0.2)
    with Nlinv(n, J, fov=fov, tensor_dft=True) as ctx:
        tx, tm = _t(torch, x), _t(torch, mask)
        f = ctx.forward(tx, tm).cpu().numpy()
        df = ctx.derivative(tx, tm, _t(torch, d)).cpu().numpy()
        a = ctx.adjoint(tx, tm, _t(torch, r)).cpu().numpy()
        q = ctx.normal(tx, tm, _t(torch, d), 0.5).cpu().numpy()
    assert rel(f, O.forward(s, mask, x)) < TOL_OP
    assert rel(df, O.derivative(s, mask, x, d)) < TOL_OP
    assert rel(a, O.adjoint(s, mask, x, r)) < TOL_OP
    assert rel(q, O.normal(s, mask, x, d, 0.5)) < TOL_OP


def test_tensor_core_stages_are_not_the_fp32_stages():
    """The option really changes the arithmetic: results differ from the FP32 path at the split-BF16 level."""
    ensure_built()
    import torch
    from paper_1301_1215_gb300.nlinv import Nlinv
    n, J = 256, 4
    rng = synth.rng_for(17)
    x = _t(torch, synth.random_complex((1 + J, n, n), rng))
    m = _t(torch, synth.radial_mask(n, 21))
    with Nlinv(n, J) as c32, Nlinv(n, J, tensor_dft=True) as ctc:
        a = c32.forward(x, m).cpu().numpy()
        b = ctc.forward(x, m).cpu().numpy()
    assert 1e-8 < rel(b, a) < TOL_OP


def test_reconstruction_256_with_tensor_core_stages_matches_oracle():
    ensure_built()
    import torch
    from paper_1301_1215_gb300.nlinv import Nlinv
    n, J = 256, 8
    s, fr, y = noisy_data(n, J, 25, 1002)
    y = y.astype(np.complex64).astype(np.complex128)
    x0 = synth.initial_guess(n, J)
    xo, ro = O.irgnm(s, fr.mask, y, x0, None, 4, 20)
    outs = []
    for graph in (True, False):
        with Nlinv(n, J, newton_steps=4, cg_iters=20, tensor_dft=True, use_graph=graph) as ctx:
            xg, rg = ctx.reconstruct(_t(torch, y), _t(torch, fr.mask), _t(torch, x0), resid=True)
        outs.append(xg.cpu().numpy())
        assert rel(outs[-1], xo) < TOL_X
        assert np.allclose(rg, ro, rtol=1e-3)
    assert np.array_equal(outs[0], outs[1])      # graph replay and kernel-by-kernel launches agree bitwise


def test_precision_frame_512_with_tensor_core_stages():
    """The precision workload (512 x 512, 16 coils, 32 spokes, 8 Newton x 30 CG) with the radix-16 stages on the
    tensor cores, against the oracle's stored run: every Newton step's iterate (stored sample) and the final image
    within the Gauss-Newton bar."""
    ensure_built()
    import torch
    from tests.helpers import precision_512_errors
    e = precision_512_errors(torch, tensor_dft=True)
    assert max(e["per_step_sample"]) < TOL_X, e
    assert e["rho_omega"] < TOL_X and e["image"] < TOL_X, e
    assert max(e["resid_rel"]) < 1e-3, e
