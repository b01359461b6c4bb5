"""The allocation-free forward operator (nlinv_forward_noalloc) against the context-based nlinv_forward.

Callers that may not allocate device memory when they apply F -- a real-time loop that reserved its GPU memory up
front, or a host framework that owns every device allocation -- cannot create a context, so this entry point keeps
its scratch in a fixed file-scope device array.  Checked through the C interface on calls in a row against the
existing entry point, within the operator tolerance of the other GPU tests: calls with the same grid side but
other coil counts and fields of view (the tables written by the first call are reused, the buffers behind them
change size), then another grid side (the tables are rewritten); plus the size limit of the array.  This file is
collected last so that a failure here does not hide any other test."""
import ctypes as C

import numpy as np
import pytest

from paper_1301_1215_gb300 import synth
from tests.helpers import ensure_built, rel

pytestmark = pytest.mark.gpu
TOL = 1e-5


def _params(lib, _lib, n, J, fov):
    p = _lib.Params()
    assert lib.nlinv_default_params(C.byref(p), n, J) == _lib.OK
    p.fov = fov
    return p


def test_forward_noalloc_matches_forward_on_calls_in_a_row():
    ensure_built()
    import torch
    from paper_1301_1215_gb300 import _lib
    from paper_1301_1215_gb300.nlinv import Nlinv
    lib = _lib.load()
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = C.c_void_p(torch.cuda.current_stream(dev).cuda_stream)
    calls = [(64, 4, 13, 31), (64, 8, 16, 33), (64, 4, 16, 34), (384, 10, 96, 32), (384, 10, 96, 35)]
    for call, (n, J, fov, seed) in enumerate(calls):
        rng = synth.rng_for(seed)
        x = torch.from_numpy(synth.random_complex((1 + J, n, n), rng).astype(np.complex64)).to(dev)
        mask = torch.from_numpy(synth.radial_mask(n, 13, 0.1 * call)).to(dev)
        with Nlinv(n, J, fov=fov, device=dev) as ctx:
            ref = ctx.forward(x, mask).cpu().numpy()
        y = torch.full((J, n, n), complex(float("nan"), 0.0), dtype=torch.complex64, device=dev)
        st = lib.nlinv_forward_noalloc(C.byref(_params(lib, _lib, n, J, fov)), stream, C.c_void_p(x.data_ptr()),
                                       C.c_void_p(mask.data_ptr()), C.c_void_p(y.data_ptr()))
        assert st == _lib.OK, lib.nlinv_last_error(None)
        torch.cuda.synchronize()
        got = y.cpu().numpy()
        assert np.isfinite(got).all()
        assert rel(got, ref) < TOL, (call, n, J)


def test_forward_noalloc_rejects_sizes_beyond_its_scratch():
    ensure_built()
    import torch
    from paper_1301_1215_gb300 import _lib
    lib = _lib.load()
    n, J = 512, 16
    x = torch.zeros((1 + J, n, n), dtype=torch.complex64, device="cuda")
    m = torch.ones((n, n), dtype=torch.uint8, device="cuda")
    y = torch.zeros((J, n, n), dtype=torch.complex64, device="cuda")
    st = lib.nlinv_forward_noalloc(C.byref(_params(lib, _lib, n, J, n // 4)), None, C.c_void_p(x.data_ptr()),
                                   C.c_void_p(m.data_ptr()), C.c_void_p(y.data_ptr()))
    assert st == _lib.EINVAL
    assert b"static maximum" in lib.nlinv_last_error(None)
