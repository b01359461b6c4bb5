"""Host-side checks of the C interface: the library builds, loads and exports every declared entry point, and
argument validation answers before any CUDA call.  No GPU is used."""
import ctypes as C
import os
import re

import pytest

from tests.helpers import ensure_built

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    path = ensure_built()
    from paper_1301_1215_gb300 import _lib
    return _lib.load(path)


def declared_functions():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            text = open(os.path.join(ROOT, "include", h)).read()
            names += re.findall(r"NLINV_API\s+[\w\s\*]+?\b(nlinv_\w+)\s*\(", text)
    return names


def test_every_declared_function_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 13
    for n in names:
        assert hasattr(lib, n), f"{n} is declared in include/ but not exported"


def test_binding_covers_every_declared_function():
    from paper_1301_1215_gb300 import _lib
    assert set(declared_functions()) == set(_lib.SIGNATURES)


def test_supported_sizes(lib):
    for n in (16, 32, 48, 64, 80, 96, 128, 160, 192, 256, 320, 384, 512):
        assert lib.nlinv_supported_size(n) == 1
    for n in (0, 8, 100, 1000, 1024, -64):
        assert lib.nlinv_supported_size(n) == 0


def test_default_params(lib):
    from paper_1301_1215_gb300 import _lib
    p = _lib.Params()
    assert lib.nlinv_default_params(C.byref(p), 384, 10) == _lib.OK
    assert (p.n, p.ncoils, p.newton_steps, p.cg_iters, p.fov, p.use_graph) == (384, 10, 7, 30, 96, 1)
    assert (p.alpha0, p.alpha_q, p.alpha_min, p.sobolev_a, p.sobolev_l) == (1.0, 0.5, 0.0, 220.0, 32.0)
    assert lib.nlinv_default_params(None, 64, 4) == _lib.EINVAL


@pytest.mark.parametrize("field,value", [("n", 100), ("ncoils", 0), ("ncoils", 65), ("newton_steps", 0),
                                         ("newton_steps", 65), ("cg_iters", -1), ("cg_iters", 100001),
                                         ("alpha0", 0.0), ("alpha0", float("nan")), ("alpha0", float("inf")),
                                         ("alpha_q", 0.0), ("alpha_q", 1.5), ("alpha_min", -1.0),
                                         ("alpha_min", float("nan")), ("sobolev_a", -1.0), ("sobolev_a", float("nan")),
                                         ("sobolev_l", -1.0), ("sobolev_l", float("inf")), ("fov", 0), ("fov", 33),
                                         ("tensor_dft", 2), ("tensor_dft", 1)])
def test_create_rejects_bad_params_before_touching_cuda(lib, field, value):
    from paper_1301_1215_gb300 import _lib
    p = _lib.Params()
    lib.nlinv_default_params(C.byref(p), 64, 4)
    setattr(p, field, value)
    h = C.c_void_p()
    assert lib.nlinv_create(C.byref(p), None, C.byref(h)) == _lib.EINVAL
    assert not h.value
    assert lib.nlinv_last_error(None)


def test_null_context_is_rejected(lib):
    from paper_1301_1215_gb300 import _lib
    assert lib.nlinv_forward(None, None, None, None) == _lib.EINVAL
    assert lib.nlinv_reconstruct(None, None, None, None, None, None) == _lib.EINVAL
    assert lib.nlinv_wait(None, 0.0) == _lib.EINVAL
    assert lib.nlinv_destroy(None) == _lib.OK
    assert lib.nlinv_last_launch_count(None) == -1


def test_every_context_call_rejects_a_null_context(lib):
    """Each entry point that takes a context (or batch) answers a NULL one on the host, before any CUDA call."""
    from paper_1301_1215_gb300 import _lib
    E = _lib.EINVAL
    assert lib.nlinv_derivative(None, None, None, None, None) == E
    assert lib.nlinv_adjoint(None, None, None, None, None) == E
    assert lib.nlinv_normal(None, None, None, None, 1.0, None) == E
    assert lib.nlinv_image(None, None, None) == E
    assert lib.nlinv_simulate(None, None, None, None, None) == E
    assert lib.nlinv_reconstruct_checkpoints(None, None, None, None, None, None, None) == E
    assert lib.nlinv_reconstruct_vjp(None, None, None, None, None, 0, None, None, None) == E
    ms = (C.c_double * 6)()
    assert lib.nlinv_profile_cg(None, 1, ms) == E
    assert lib.nlinv_autotune(None, None, None, None, 3, None, None, 0) == E
    assert lib.nlinv_set_shapes(None, None) == E
    assert lib.nlinv_cg_stops(None, None, 0) == E
    assert lib.nlinv_batch_profile_cg(None, 1, ms) == E
    assert lib.nlinv_reconstruct_batch(None, 0, None) == E
    assert lib.nlinv_batch_launch_count(None) == -1
    assert lib.nlinv_batch_destroy(None) == _lib.OK


def test_gridder_create_rejects_bad_arguments_on_the_host(lib):
    from paper_1301_1215_gb300 import _lib
    d = (C.c_double * 2)(1.0, 0.0)
    h = C.c_void_p()
    assert lib.nlinv_gridder_create(7, 1, d, None, C.byref(h)) == _lib.EINVAL       # odd n
    assert lib.nlinv_gridder_create(4, 1, d, None, C.byref(h)) == _lib.EINVAL       # too small
    assert lib.nlinv_gridder_create(16, 0, d, None, C.byref(h)) == _lib.EINVAL      # no spokes
    assert lib.nlinv_gridder_create(16, 1, None, None, C.byref(h)) == _lib.EINVAL   # no directions
    nan = (C.c_double * 2)(float("nan"), 0.0)
    assert lib.nlinv_gridder_create(16, 1, nan, None, C.byref(h)) == _lib.EINVAL
    assert lib.nlinv_grid(None, 1, None, None, None) == _lib.EINVAL
    assert lib.nlinv_gridder_destroy(None) == _lib.OK


def test_batch_create_rejects_bad_arguments_on_the_host(lib):
    from paper_1301_1215_gb300 import _lib
    p = _lib.Params()
    lib.nlinv_default_params(C.byref(p), 64, 4)
    h = C.c_void_p()
    assert lib.nlinv_batch_create(C.byref(p), 0, None, None, C.byref(h)) == _lib.EINVAL
    assert lib.nlinv_batch_create(None, 1, None, None, C.byref(h)) == _lib.EINVAL
    assert lib.nlinv_batch_create(C.byref(p), 1, None, None, None) == _lib.EINVAL


def test_create_without_gpu_reports_cuda_error(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1301_1215_gb300 import _lib
    p = _lib.Params()
    lib.nlinv_default_params(C.byref(p), 64, 4)
    h = C.c_void_p()
    assert lib.nlinv_create(C.byref(p), None, C.byref(h)) == _lib.ECUDA
    assert b"cuda" in lib.nlinv_last_error(None).lower()


def test_binding_refuses_without_gpu():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1301_1215_gb300.nlinv import Nlinv
    with pytest.raises(RuntimeError):
        Nlinv(64, 4)


def test_every_kernel_waits_for_its_predecessor():
    # Passes are launched with programmatic stream serialisation, so each kernel must execute
    # griddepcontrol.wait (nlv::pdl_enter) before it reads what the kernel just before it wrote, and before
    # any store.  A kernel may stage inputs written two or more launches back before the wait, so the wait need
    # not be its first statement; it must be in the kernel's own body, or in row_pass_body, whose PRE form waits
    # inside its `enter` step (before the first round's stores).
    csrc = os.path.join(ROOT, "paper_1301_1215_gb300", "csrc")
    kernels = 0
    for name in os.listdir(csrc):
        if not name.endswith((".cu", ".cuh")):
            continue
        lines = open(os.path.join(csrc, name)).read().splitlines()
        for i, line in enumerate(lines):
            if "__global__" in line and "(" in line and line.rstrip().endswith("{"):
                j = i + 1
                while j < len(lines) and lines[j].rstrip() != "}":
                    j += 1
                body = "\n".join(lines[i + 1: j])
                kernels += 1
                waits = "pdl_enter()" in body or re.search(r"row_pass_body<[^>]*,\s*true>", body)
                assert waits, f"{name}:{i + 1} kernel never reaches pdl_enter()"
    assert kernels >= 10
    src = open(os.path.join(csrc, "kernels.cuh")).read()
    body = src[src.index("void row_pass_body("):src.index("__global__ void __launch_bounds__(kRowMaxThreads, "
                                                          "kRowCtasPerSM) row_pass(")]
    enter = body[body.index("auto enter = [&]"):]
    assert "pdl_enter();" in enter[:200]
    # the deferred wait of the early-load path comes before the first store of a round
    assert body.index("if (!waited)") < body.index("A.dst[")


def test_every_specialised_pass_has_batched_and_multi_side_forms():
    # A single-frame pass specialised for the standard field of view (SizeKernels::row_std / col_std) is mapped to
    # its batched form (row_std_batch / col_std_batch) and, with NLINV_BATCH_MULTI=1, to the multi-side kernel
    # (MultiKernels::row_std / col_std); a mode missing from either table would leave batches without a kernel.
    csrc = os.path.join(ROOT, "paper_1301_1215_gb300", "csrc")
    kern = open(os.path.join(csrc, "kernels.cuh")).read()
    body = kern[kern.index("template <int N1, int N2> SizeKernels make_size_kernels() {"):]
    body = body[:body.index("\n}\n")]
    multi = open(os.path.join(csrc, "batch_multi.cu")).read()
    for side in ("row", "col"):
        single = set(re.findall(rf"s\.{side}_std\[(\w+)\] =", body))
        batched = set(re.findall(rf"s\.{side}_std_batch\[(\w+)\] =", body))
        multi_std = set(re.findall(rf"m\.{side}_std\[(\w+)\] =", multi))
        assert single, side
        assert single == batched, (side, single ^ batched)
        assert single == multi_std, (side, single ^ multi_std)


def test_forward_noalloc_checks_its_arguments_on_the_host(lib):
    # every rejection below happens before the entry point asks CUDA for anything (the pointers are never read)
    from paper_1301_1215_gb300 import _lib
    E = _lib.EINVAL
    dummy = C.c_void_p(16)
    p = _lib.Params()
    lib.nlinv_default_params(C.byref(p), 64, 4)
    assert lib.nlinv_forward_noalloc(None, None, dummy, dummy, dummy) == E
    assert lib.nlinv_forward_noalloc(C.byref(p), None, None, dummy, dummy) == E
    assert lib.nlinv_forward_noalloc(C.byref(p), None, dummy, None, dummy) == E
    assert lib.nlinv_forward_noalloc(C.byref(p), None, dummy, dummy, None) == E
    for field, value in (("n", 100), ("ncoils", 0), ("fov", 0), ("fov", 33), ("sobolev_a", float("nan"))):
        q = _lib.Params()
        lib.nlinv_default_params(C.byref(q), 64, 4)
        setattr(q, field, value)
        assert lib.nlinv_forward_noalloc(C.byref(q), None, dummy, dummy, dummy) == E, field
    big = _lib.Params()
    lib.nlinv_default_params(C.byref(big), 512, 16)          # needs more than the static scratch array
    assert lib.nlinv_forward_noalloc(C.byref(big), None, dummy, dummy, dummy) == E
    assert b"static maximum" in lib.nlinv_last_error(None)
