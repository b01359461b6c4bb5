"""GPU parity of single operator applications (F, DF, DF^H, the normal operator of Eq. 3 and the data
simulation) against the complex128 oracle, on the same seeded inputs, through the C interface.

Bar: relative L2 error <= 1e-5 in FP32 complex.  Sizes span one tile up to the 384 x 384, 10-coil and
512 x 512, 16-coil workloads; fields of view that do not fill whole column strips give ragged tails, and
fov = n/2 (Omega = the whole grid) is the degenerate mask."""
import numpy as np
import pytest

import oracle.nlinv_oracle as O
from paper_1301_1215_gb300 import synth
from tests.helpers import ensure_built, rel

pytestmark = pytest.mark.gpu
TOL = 1e-5

CASES = [  # (n, J, fov)
    (16, 1, 4), (32, 3, 8), (48, 2, 12), (64, 4, 13), (80, 3, 20), (96, 2, 48), (128, 4, 32), (160, 2, 37),
    (192, 3, 48), (256, 8, 64), (320, 2, 80), (384, 10, 96), (512, 16, 128),
    (64, 64, 16), (512, 24, 128),      # the largest coil count the interface takes; more coils at the largest side
]


@pytest.fixture(scope="module")
def torch_cuda():
    ensure_built()
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return torch


def _t(torch, a, dev="cuda"):
    if a.dtype == np.uint8:
        return torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    return torch.from_numpy(np.ascontiguousarray(a.astype(np.complex64))).to(dev)


def _inputs(n, J, fov, seed):
    rng = synth.rng_for(seed)
    s = O.Setup(n, J, fov)
    x = synth.random_complex((1 + J, n, n), rng)
    d = synth.random_complex((1 + J, n, n), rng)
    r = synth.random_complex((J, n, n), rng)
    mask = synth.radial_mask(n, max(3, n // 8))
    # evaluate the oracle on exactly the values the GPU sees
    x, d, r = (a.astype(np.complex64).astype(np.complex128) for a in (x, d, r))
    return s, x, d, r, mask


@pytest.mark.parametrize("n,J,fov", CASES)
def test_operators_match_oracle(torch_cuda, n, J, fov):
    torch = torch_cuda
    from paper_1301_1215_gb300.nlinv import Nlinv
    s, x, d, r, mask = _inputs(n, J, fov, seed=1000 + n + J)
    with Nlinv(n, J, fov=fov) as ctx:
        tx, td, tr, tm = _t(torch, x), _t(torch, d), _t(torch, r), _t(torch, mask)
        c = O.coils(s, x)
        got = ctx.forward(tx, tm).cpu().numpy()
        assert rel(got, O.forward(s, mask, x)) < TOL
        got = ctx.derivative(tx, tm, td).cpu().numpy()
        assert rel(got, O.derivative(s, mask, x, d, c)) < TOL
        got = ctx.adjoint(tx, tm, tr).cpu().numpy()
        ref = O.adjoint(s, mask, x, r, c)
        assert rel(got, ref) < TOL
        assert rel(got[0], ref[0]) < TOL and rel(got[1:], ref[1:]) < TOL
        got = ctx.normal(tx, tm, td, 0.25).cpu().numpy()
        assert rel(got, O.normal(s, mask, x, d, 0.25, c)) < TOL


@pytest.mark.parametrize("n,J,fov", [(64, 4, 16), (384, 10, 96)])
def test_simulate_matches_oracle(torch_cuda, n, J, fov):
    torch = torch_cuda
    from paper_1301_1215_gb300.nlinv import Nlinv
    fr = synth.make_frame(n, J, 13, seed=5, fov=fov)
    s = O.Setup(n, J, fov)
    rho = fr.rho.astype(np.complex64).astype(np.complex128)
    coils = fr.coils.astype(np.complex64).astype(np.complex128)
    with Nlinv(n, J, fov=fov) as ctx:
        got = ctx.simulate(_t(torch, rho), _t(torch, coils), _t(torch, fr.mask)).cpu().numpy()
    assert rel(got, O.simulate(s, fr.mask, rho, coils)) < TOL


@pytest.mark.parametrize("n,J,fov", [(48, 2, 12), (384, 10, 96)])
def test_adjoint_identity_on_gpu(torch_cuda, n, J, fov):
    torch = torch_cuda
    from paper_1301_1215_gb300.nlinv import Nlinv
    s, x, d, r, mask = _inputs(n, J, fov, seed=7)
    with Nlinv(n, J, fov=fov) as ctx:
        tx, tm = _t(torch, x), _t(torch, mask)
        Fd = ctx.derivative(tx, tm, _t(torch, d)).cpu().numpy().astype(np.complex128)
        FHr = ctx.adjoint(tx, tm, _t(torch, r)).cpu().numpy().astype(np.complex128)
    lhs, rhs = np.vdot(Fd, r), np.vdot(d, FHr)
    assert abs(lhs - rhs) < 1e-5 * abs(lhs)


def test_sobolev_special_cases(torch_cuda):
    # a = 0 (w = 1) and a non-integer l/2 (the powf path) against the oracle
    torch = torch_cuda
    from paper_1301_1215_gb300.nlinv import Nlinv
    n, J, fov = 64, 2, 16
    for a, l in [(0.0, 32.0), (30.0, 3.0), (220.0, 0.0)]:
        s = O.Setup(n, J, fov, a=a, l=l)
        rng = synth.rng_for(3)
        x = synth.random_complex((1 + J, n, n), rng).astype(np.complex64).astype(np.complex128)
        mask = synth.radial_mask(n, 9)
        with Nlinv(n, J, fov=fov, sobolev_a=a, sobolev_l=l) as ctx:
            got = ctx.forward(_t(torch, x), _t(torch, mask)).cpu().numpy()
        assert rel(got, O.forward(s, mask, x)) < TOL, (a, l)


def test_empty_mask_and_zero_inputs(torch_cuda):
    torch = torch_cuda
    from paper_1301_1215_gb300.nlinv import Nlinv
    n, J = 32, 2
    s, x, d, r, _ = _inputs(n, J, 8, seed=9)
    empty = np.zeros((n, n), np.uint8)
    with Nlinv(n, J) as ctx:
        assert not ctx.forward(_t(torch, x), _t(torch, empty)).cpu().numpy().any()
        out = ctx.normal(_t(torch, x), _t(torch, empty), _t(torch, d), 0.5).cpu().numpy()
        assert rel(out, 0.5 * d) < 1e-6
        z = np.zeros_like(x)
        assert not ctx.forward(_t(torch, z), _t(torch, np.ones((n, n), np.uint8))).cpu().numpy().any()


def test_host_pointer_rejected_by_operators(torch_cuda):
    torch = torch_cuda
    import ctypes as C
    from paper_1301_1215_gb300 import _lib
    from paper_1301_1215_gb300.nlinv import Nlinv
    n, J = 32, 1
    with Nlinv(n, J) as ctx:
        xh = torch.zeros((2, n, n), dtype=torch.complex64)
        m = torch.ones((n, n), dtype=torch.uint8, device="cuda")
        y = torch.empty((1, n, n), dtype=torch.complex64, device="cuda")
        st = ctx._lib.nlinv_forward(ctx._h, C.c_void_p(xh.data_ptr()), C.c_void_p(m.data_ptr()),
                                    C.c_void_p(y.data_ptr()))
        assert st == _lib.EINVAL
        assert b"device pointer" in ctx._lib.nlinv_last_error(ctx._h)


@pytest.mark.parametrize("n,J,fov", [(64, 4, 13), (384, 10, 96)])
def test_image_matches_oracle(torch_cuda, n, J, fov):
    torch = torch_cuda
    from paper_1301_1215_gb300.nlinv import Nlinv
    s, x, d, r, mask = _inputs(n, J, fov, seed=99)
    with Nlinv(n, J, fov=fov) as ctx:
        got = ctx.image(_t(torch, x)).cpu().numpy()
    assert rel(got, O.image(s, x)) < TOL
