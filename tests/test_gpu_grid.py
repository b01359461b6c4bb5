"""GPU gridding of radial spokes (nlinv_gridder_create / nlinv_grid) against the oracle's nearest-neighbour gridding
with averaging: the sampling pattern bit for bit, the gridded data within FP32 rounding (at most a few samples are
averaged per grid point, so 1e-6 relative L2 leaves ample room)."""
import numpy as np
import pytest

import oracle.nlinv_oracle as O
from paper_1301_1215_gb300 import synth
from tests.helpers import ensure_built, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    ensure_built()
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return torch


@pytest.mark.parametrize("n,spokes,rot,J", [(64, 16, 0.3, 4), (96, 9, 0.0, 2),
                                            (384, 13, synth.frame_rotation(3, 13), 10)])
def test_gridding_matches_oracle(torch_cuda, n, spokes, rot, J):
    torch = torch_cuda
    from paper_1301_1215_gb300.nlinv import Gridder
    angles = [np.pi * k / spokes + rot for k in range(spokes)]
    dirs = [(np.cos(th), np.sin(th)) for th in angles]          # the same scalar calls the oracle makes
    rng = synth.rng_for(81)
    smp = synth.random_complex((J, spokes, 2 * n), rng).astype(np.complex64)
    yo, mo = O.grid_radial(n, angles, smp.astype(np.complex128))
    with Gridder(n, dirs) as g:
        y, m = g.grid(torch.from_numpy(smp).cuda())
        y, m = y.cpu().numpy(), m.cpu().numpy()
    assert np.array_equal(m, mo)
    assert np.array_equal(m, synth.radial_mask(n, spokes, rot))
    assert rel(y, yo) < 1e-6
    assert not y[:, m == 0].any()


def test_gridding_rejects_host_buffers(torch_cuda):
    torch = torch_cuda
    from paper_1301_1215_gb300 import _lib
    from paper_1301_1215_gb300.nlinv import Gridder
    with Gridder(16, [(1.0, 0.0)]) as g:
        smp = torch.zeros((1, 1, 32), dtype=torch.complex64)      # host tensor
        y = torch.zeros((1, 16, 16), dtype=torch.complex64, device="cuda")
        m = torch.zeros((16, 16), dtype=torch.uint8, device="cuda")
        st = g._lib.nlinv_grid(g._h, 1, _lib.C.c_void_p(smp.data_ptr()), _lib.C.c_void_p(y.data_ptr()),
                               _lib.C.c_void_p(m.data_ptr()))
        assert st == _lib.EINVAL
