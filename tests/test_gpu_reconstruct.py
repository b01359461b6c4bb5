"""GPU parity of the whole Gauss-Newton reconstruction (Eq. 3 with CG) against the oracle on the seeded
workloads, plus the real-time series, graph replay, host buffers and the host-visible failure paths.

Bar: final x within relative L2 1e-3 of the oracle; residual norms within 1e-4."""
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


def _compare(torch, n, J, spokes, newton, cg, seed):
    from paper_1301_1215_gb300.nlinv import Nlinv
    s, fr, y = noisy_data(n, J, spokes, seed)
    y = y.astype(np.complex64).astype(np.complex128)
    x0 = synth.initial_guess(n, J)
    xo, ro = O.irgnm(s, fr.mask, y, x0, None, newton, cg)
    with Nlinv(n, J, newton_steps=newton, cg_iters=cg) as ctx:
        xg, rg = ctx.reconstruct(_t(torch, y), _t(torch, fr.mask), _t(torch, x0), resid=True)
        xg = xg.cpu().numpy()
    assert rel(xg, xo) < TOL_X
    assert rel(xg[0], xo[0]) < TOL_X
    assert np.allclose(rg, ro, rtol=1e-4, atol=0)
    return xg


def test_single_frame_64(torch_cuda):
    _compare(torch_cuda, 64, 4, 16, 7, 30, seed=1001)


def test_single_frame_256(torch_cuda):
    _compare(torch_cuda, 256, 8, 25, 8, 40, seed=1002)


def test_realtime_frame_384(torch_cuda):
    _compare(torch_cuda, 384, 10, 13, 7, 30, seed=1003)


def test_precision_frame_512(torch_cuda):
    """512 x 512 grid, 16 coils, 32 spokes (the precision workload) on its full schedule, 8 Newton x 30 CG, against
    the oracle's stored run: every iterate (on the stored sample), every Newton step's residual norm, the final rho
    on Omega and the final display image."""
    from tests.helpers import precision_512_errors
    e = precision_512_errors(torch_cuda, tensor_dft=False)
    assert max(e["per_step_sample"]) < TOL_X, e
    assert e["rho_omega"] < TOL_X and e["image"] < TOL_X, e
    assert max(e["resid_rel"]) < 1e-4, e


def test_autotune_picks_a_candidate_and_keeps_parity(torch_cuda):
    """The autotuner times whole graph replays stage by stage (split, column strip, row blocks, vector blocks x
    dependent launch), keeps one of its candidates, and the reconstruction with the chosen shapes still matches the
    oracle; a second context of the same shape takes the cached choice."""
    torch = torch_cuda
    from paper_1301_1215_gb300.nlinv import Nlinv
    n, J = 128, 4
    s, fr, y = noisy_data(n, J, 16, 1001)
    y = y.astype(np.complex64).astype(np.complex128)
    x0 = synth.initial_guess(n, J)
    ty, tm, tx = _t(torch, y), _t(torch, fr.mask), _t(torch, x0)
    with Nlinv(n, J, newton_steps=3, cg_iters=10) as ctx:
        t = ctx.autotune(ty, tm, tx, reps=2)
        stages = {c["stage"] for c in t["candidates"]}
        assert stages == {0, 1, 2, 3}
        assert {c["split_n1"] for c in t["candidates"] if c["stage"] == 0} == {8, 4}
        assert {c["col_strip"] for c in t["candidates"] if c["stage"] == 1} == {4, 8, 16}
        assert t["ms_per_frame"] > 0 and t["vec_blocks_per_sm"] in (2, 4, 8)
        mine = [c for c in t["candidates"] if all(c[k] == t[k] for k in
                ("split_n1", "col_strip", "row_blocks_per_sm", "vec_blocks_per_sm", "pdl"))]
        assert mine
        xg = ctx.reconstruct(ty, tm, tx).cpu().numpy()
    xo, _ = O.irgnm(s, fr.mask, y, x0, None, 3, 10)
    assert rel(xg, xo) < TOL_X
    with Nlinv(n, J, newton_steps=3, cg_iters=10) as ctx:
        assert ctx.autotune(ty, tm, tx, reps=2) == t


def test_set_shapes_rejects_what_is_not_compiled(torch_cuda):
    from paper_1301_1215_gb300 import _lib
    from paper_1301_1215_gb300.nlinv import Nlinv, NlinvError
    with Nlinv(384, 4, newton_steps=1, cg_iters=2) as ctx:
        for bad in [dict(split_n1=8), dict(split_n1=16, col_strip=6), dict(split_n1=16, row_blocks_per_sm=4),
                    dict(split_n1=16, vec_blocks_per_sm=0)]:
            with pytest.raises(NlinvError) as ei:
                ctx.set_shapes(**bad)
            assert ei.value.status == _lib.EINVAL
        ctx.set_shapes(16, 8)          # the compiled shapes are always accepted
    with Nlinv(512, 2, tensor_dft=True, newton_steps=1, cg_iters=2) as ctx:
        with pytest.raises(NlinvError):
            ctx.set_shapes(16, 4)      # the tensor-core passes keep the compiled strips


@pytest.mark.parametrize("n,split,strip", [(128, 4, 8), (128, 8, 4), (192, 8, 8), (192, 12, 16), (256, 8, 8),
                                           (256, 16, 4), (320, 10, 8), (320, 16, 16), (384, 12, 8), (384, 16, 4),
                                           (384, 16, 16), (512, 16, 4), (512, 16, 16)])
def test_tuning_variants_match_oracle(torch_cuda, n, split, strip):
    """Every transform split and column strip the autotuner may pick: the operators against the oracle (1e-5) and
    a short reconstruction (1e-3), with a ragged field of view as well as the standard one."""
    torch = torch_cuda
    from paper_1301_1215_gb300.nlinv import Nlinv
    J = 3
    for fov in (n // 4, n // 4 - 3):
        so = O.Setup(n, J, fov)
        rng = synth.rng_for(900 + n + split + strip)
        x = synth.random_complex((1 + J, n, n), rng)
        d = synth.random_complex((1 + J, n, n), rng)
        mask = synth.radial_mask(n, 17, 0.3)
        with Nlinv(n, J, fov=fov, newton_steps=2, cg_iters=6) as ctx:
            ctx.set_shapes(split, strip, row_blocks_per_sm=3 if strip == 16 else 2)
            tx, tmk = _t(torch, x), _t(torch, mask)
            f = ctx.forward(tx, tmk).cpu().numpy()
            q = ctx.normal(tx, tmk, _t(torch, d), 0.5).cpu().numpy()
            assert rel(f, O.forward(so, mask, x)) < 1e-5, fov
            assert rel(q, O.normal(so, mask, x, d, 0.5)) < 1e-5, fov
            if fov == n // 4:
                s, fr, y = noisy_data(n, J, 13, 77)
                y = y.astype(np.complex64).astype(np.complex128)
                xg = ctx.reconstruct(_t(torch, y), _t(torch, fr.mask)).cpu().numpy()
                xo, _ = O.irgnm(s, fr.mask, y, synth.initial_guess(n, J), None, 2, 6)
                assert rel(xg, xo) < TOL_X


def test_graph_and_kernel_by_kernel_agree_bitwise(torch_cuda):
    torch = torch_cuda
    from paper_1301_1215_gb300.nlinv import Nlinv
    n, J = 64, 4
    s, fr, y = noisy_data(n, J, 16, 11)
    outs = []
    for g in (True, False, True):
        with Nlinv(n, J, newton_steps=3, cg_iters=8, use_graph=g) as ctx:
            outs.append(ctx.reconstruct(_t(torch, y), _t(torch, fr.mask)).cpu().numpy())
            if g:
                outs.append(ctx.reconstruct(_t(torch, y), _t(torch, fr.mask)).cpu().numpy())
    for o in outs[1:]:
        assert np.array_equal(o, outs[0])


def test_realtime_series_matches_oracle(torch_cuda):
    torch = torch_cuda
    from paper_1301_1215_gb300.nlinv import Nlinv
    n, J, spokes, frames = 64, 4, 9, 3
    datas = [noisy_data(n, J, spokes, 21, frame=k) for k in range(frames)]
    s = datas[0][0]
    ys = [d[2].astype(np.complex64).astype(np.complex128) for d in datas]
    masks = [d[1].mask for d in datas]
    ref = O.realtime_series(s, masks, ys, synth.initial_guess(n, J), 4, 15)
    with Nlinv(n, J, newton_steps=4, cg_iters=15) as ctx:
        x = _t(torch, synth.initial_guess(n, J))
        for k in range(frames):
            ctx.reconstruct_inplace(_t(torch, ys[k]), _t(torch, masks[k]), x)
            assert rel(x.cpu().numpy(), ref[k]) < TOL_X


def test_realtime_series_384_matches_oracle(torch_cuda):
    # the series workload itself: 384 x 384 grid, 10 coils, 13 spokes, 7 Newton x 30 CG, one graph per frame,
    # frame 1 started from and regularised toward frame 0's result
    torch = torch_cuda
    from paper_1301_1215_gb300.nlinv import Nlinv
    n, J, spokes, frames = 384, 10, 13, 2
    datas = [noisy_data(n, J, spokes, 1003, frame=k) for k in range(frames)]
    s = datas[0][0]
    ys = [d[2].astype(np.complex64).astype(np.complex128) for d in datas]
    masks = [d[1].mask for d in datas]
    ref = O.realtime_series(s, masks, ys, synth.initial_guess(n, J), 7, 30)
    with Nlinv(n, J, newton_steps=7, cg_iters=30) as ctx:
        x = _t(torch, synth.initial_guess(n, J))
        for k in range(frames):
            ctx.reconstruct_inplace(_t(torch, ys[k]), _t(torch, masks[k]), x)
            xk = x.cpu().numpy()
            assert rel(xk, ref[k]) < TOL_X
            assert rel(xk[0], ref[k][0]) < TOL_X


def test_host_buffers_give_the_device_result(torch_cuda):
    torch = torch_cuda
    from paper_1301_1215_gb300.nlinv import Nlinv
    n, J = 64, 4
    s, fr, y = noisy_data(n, J, 16, 13)
    x0 = synth.initial_guess(n, J)
    with Nlinv(n, J, newton_steps=3, cg_iters=10) as ctx:
        xd = ctx.reconstruct(_t(torch, y), _t(torch, fr.mask), _t(torch, x0)).cpu().numpy()
        yh = torch.from_numpy(y.astype(np.complex64)).pin_memory()
        mh = torch.from_numpy(fr.mask)
        xh = torch.from_numpy(x0.astype(np.complex64))          # pageable
        _, res = ctx.reconstruct_inplace(yh, mh, xh, resid=True)
        assert np.array_equal(xh.numpy(), xd)
        assert len(res) == 4 and all(np.isfinite(res))


def test_zero_data_at_start_value_stays_put(torch_cuda):
    # y = F(x0) = 0 for chat = 0: the right-hand side vanishes and every CG step is empty
    torch = torch_cuda
    from paper_1301_1215_gb300.nlinv import Nlinv
    n, J = 32, 2
    x0 = synth.initial_guess(n, J)
    with Nlinv(n, J, newton_steps=2, cg_iters=5) as ctx:
        x, res = ctx.reconstruct(_t(torch, np.zeros((J, n, n), complex)), _t(torch, synth.radial_mask(n, 5)),
                                 _t(torch, x0), resid=True)
        ctx.wait(-1)
    assert np.array_equal(x.cpu().numpy(), x0.astype(np.complex64)) and res == [0.0, 0.0, 0.0]


def test_nan_data_reports_breakdown(torch_cuda):
    torch = torch_cuda
    from paper_1301_1215_gb300 import _lib
    from paper_1301_1215_gb300.nlinv import Nlinv, NlinvError
    n, J = 32, 2
    y = np.full((J, n, n), np.nan, complex)
    with Nlinv(n, J, newton_steps=1, cg_iters=2) as ctx:
        with pytest.raises(NlinvError) as ei:
            ctx.reconstruct(_t(torch, y), _t(torch, np.ones((n, n), np.uint8)), resid=True)
        assert ei.value.status == _lib.EBREAKDOWN
        ctx.wait(-1)       # the flag was cleared by the failing call


def test_workspace_allocation_failure_reports_enomem(torch_cuda, monkeypatch):
    """A failed workspace allocation (injected on the host) is ENOMEM with a message, and leaves the device usable."""
    torch = torch_cuda
    from paper_1301_1215_gb300 import _lib
    from paper_1301_1215_gb300.nlinv import Nlinv, NlinvError
    monkeypatch.setenv("NLINV_TEST_FAIL_ALLOC", "1")
    with pytest.raises(NlinvError) as ei:
        Nlinv(64, 4)
    assert ei.value.status == _lib.ENOMEM and "cudaMalloc" in str(ei.value)
    monkeypatch.delenv("NLINV_TEST_FAIL_ALLOC")
    with Nlinv(64, 4, newton_steps=1, cg_iters=1) as ctx:
        n, J = 64, 4
        s, fr, y = noisy_data(n, J, 16, 11)
        assert np.isfinite(ctx.reconstruct(_t(torch, y), _t(torch, fr.mask)).cpu().numpy()).all()


def test_wait_deadline(torch_cuda):
    torch = torch_cuda
    from paper_1301_1215_gb300 import _lib
    from paper_1301_1215_gb300.nlinv import Nlinv, NlinvError
    n, J = 384, 10
    s, fr, y = noisy_data(n, J, 13, 1003)
    with Nlinv(n, J, newton_steps=7, cg_iters=30) as ctx:
        ty, tm = _t(torch, y), _t(torch, fr.mask)
        x = ctx.reconstruct(ty, tm)
        torch.cuda.synchronize()
        for _ in range(3):
            x = ctx.reconstruct(ty, tm)
        with pytest.raises(NlinvError) as ei:
            ctx.wait(0.0)
        assert ei.value.status == _lib.ETIMEOUT
        ctx.wait(-1)
