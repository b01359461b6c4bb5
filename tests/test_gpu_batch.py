"""Batched reconstruction of independent frames of uneven grid side and coil count (nlinv_reconstruct_batch):
each frame against its own single-frame reconstruction on the GPU (same kernels, another block partition of the
FP64 scalar sums: tolerance 1e-5) and one frame against the oracle (1e-3)."""
import numpy as np
import pytest

import oracle.nlinv_oracle as O
from paper_1301_1215_gb300 import synth
from tests.helpers import ensure_built, noisy_data, rel

pytestmark = pytest.mark.gpu
SHAPES = [(64, 4, 12), (128, 6, 15), (64, 5, 9), (96, 3, 11), (128, 4, 20), (64, 4, 16)]   # (n, J, spokes)


@pytest.fixture(scope="module")
def data():
    ensure_built()
    import torch
    frames = [noisy_data(n, J, S, 3000 + i) for i, (n, J, S) in enumerate(SHAPES)]
    return torch, frames


def _t(torch, a, dev):
    if a.dtype == np.uint8:
        return torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    return torch.from_numpy(np.ascontiguousarray(a.astype(np.complex64))).to(dev)


def test_batch_matches_single_frames_and_oracle(data):
    torch, frames = data
    from paper_1301_1215_gb300.nlinv import Nlinv, NlinvBatch
    NS, NC = 3, 10
    dev = torch.device("cuda")
    with NlinvBatch([(n, J) for n, J, _ in SHAPES], newton_steps=NS, cg_iters=NC) as b:
        ys = [_t(torch, y, dev) for _, _, y in frames]
        ms = [_t(torch, fr.mask, dev) for _, fr, _ in frames]
        xs, res = b.reconstruct(ys, ms, resid=True)
        assert b.launch_count > 0
        xs = [x.cpu().numpy() for x in xs]
    for i, ((n, J, _), (s, fr, y)) in enumerate(zip(SHAPES, frames)):
        with Nlinv(n, J, newton_steps=NS, cg_iters=NC) as ctx:
            xg, rg = ctx.reconstruct(_t(torch, y, dev), _t(torch, fr.mask, dev), resid=True)
        assert rel(xs[i], xg.cpu().numpy()) < 1e-5, i
        assert np.allclose(res[i], rg, rtol=1e-5)
    s, fr, y = frames[1]
    xo, _ = O.irgnm(s, fr.mask, y.astype(np.complex64).astype(np.complex128), synth.initial_guess(128, 6), None, NS, NC)
    assert rel(xs[1], xo) < 1e-3


def test_batch_twice_and_host_buffers(data):
    torch, frames = data
    from paper_1301_1215_gb300.nlinv import NlinvBatch
    dev = torch.device("cuda")
    sel = [0, 2, 3]
    with NlinvBatch([SHAPES[i][:2] for i in sel], newton_steps=2, cg_iters=5) as b:
        ys = [_t(torch, frames[i][2], dev) for i in sel]
        ms = [_t(torch, frames[i][1].mask, dev) for i in sel]
        first = [x.cpu().numpy() for x in b.reconstruct(ys, ms)]
        second = [x.cpu().numpy() for x in b.reconstruct(ys, ms)]
        for a, c in zip(first, second):
            assert np.array_equal(a, c)
        xh = []
        for i in sel:
            n, J, _ = SHAPES[i]
            x = torch.zeros((1 + J, n, n), dtype=torch.complex64)
            x[0] = 1.0
            xh.append(x)
        out = b.reconstruct([y.cpu() for y in ys], [m.cpu() for m in ms], xs=xh)
        for a, c in zip(first, out):
            assert np.array_equal(a, c.numpy())


def test_batch_rejects_mismatched_frames(data):
    torch, frames = data
    from paper_1301_1215_gb300.nlinv import NlinvBatch
    with NlinvBatch([(64, 4), (64, 5)], newton_steps=1, cg_iters=1) as b:
        with pytest.raises(ValueError):
            b.reconstruct([torch.zeros((4, 64, 64), dtype=torch.complex64, device="cuda")] * 2,
                          [torch.ones((64, 64), dtype=torch.uint8, device="cuda")] * 2)


# Every grid side of the uneven batch workload (128..384, f = n/4 instantiations, fixed 320-thread row lanes) with
# coil counts up to 16, on a shortened schedule so that the oracle stays within seconds per frame.
WIDE = [(128, 4, 9), (128, 16, 31), (192, 7, 12), (192, 13, 27), (256, 5, 15), (256, 16, 22), (320, 9, 18),
        (320, 12, 31), (384, 10, 13), (384, 16, 29)]


def test_batch_at_workload_sizes_matches_single_frames_and_oracle():
    ensure_built()
    import torch
    from paper_1301_1215_gb300.nlinv import Nlinv, NlinvBatch
    NS, NC = 3, 8
    dev = torch.device("cuda")
    frames = [noisy_data(n, J, S, 7000 + i) for i, (n, J, S) in enumerate(WIDE)]
    ys = [_t(torch, y, dev) for _, _, y in frames]
    ms = [_t(torch, fr.mask, dev) for _, fr, _ in frames]
    with NlinvBatch([(n, J) for n, J, _ in WIDE], newton_steps=NS, cg_iters=NC) as b:
        xs, res = b.reconstruct(ys, ms, resid=True)
        xs = [x.cpu().numpy() for x in xs]
    seen = set()
    for i, ((n, J, _), (s, fr, y)) in enumerate(zip(WIDE, frames)):
        assert np.isfinite(xs[i]).all(), i
        with Nlinv(n, J, newton_steps=NS, cg_iters=NC) as ctx:
            xg, rg = ctx.reconstruct(ys[i], ms[i], resid=True)
        assert rel(xs[i], xg.cpu().numpy()) < 1e-5, (i, n, J)
        assert np.allclose(res[i], rg, rtol=1e-5), (i, n, J)
        if n not in seen:           # one frame per grid side against the oracle
            seen.add(n)
            y64 = y.astype(np.complex64).astype(np.complex128)
            xo, ro = O.irgnm(s, fr.mask, y64, synth.initial_guess(n, J), None, NS, NC)
            assert rel(xs[i], xo) < 1e-3, (i, n, J)
            assert np.allclose(res[i], ro, rtol=1e-4), (i, n, J)
    assert seen == {128, 192, 256, 320, 384}


def test_batch_profile_times_every_cg_kernel(data):
    """nlinv_batch_profile_cg: one positive duration per CG kernel after a batched reconstruction; refused before."""
    torch, frames = data
    from paper_1301_1215_gb300.nlinv import NlinvBatch, NlinvError
    dev = torch.device("cuda")
    with NlinvBatch([SHAPES[i][:2] for i in (0, 1)], newton_steps=2, cg_iters=4) as b:
        with pytest.raises(NlinvError):
            b.profile_cg(reps=2)
        b.reconstruct([_t(torch, frames[i][2], dev) for i in (0, 1)],
                      [_t(torch, frames[i][1].mask, dev) for i in (0, 1)])
        ms = b.profile_cg(reps=2)
    assert len(ms) == 6 and all(v > 0 for v in ms.values())


def test_multi_side_launches_match_per_side_launches(data, monkeypatch):
    # NLINV_BATCH_MULTI=1: one launch per pass for the frames of every grid side in 128..384 together (the block
    # dispatches on its frame's side), instead of one launch per pass and side.  Same pass bodies, same block
    # partition of each frame, so the two forms agree to the FP32 operator tolerance.
    torch, _ = data
    from paper_1301_1215_gb300.nlinv import NlinvBatch
    shapes = [(128, 4, 12), (192, 5, 15), (128, 6, 9), (256, 3, 11)]
    frames = [noisy_data(n, J, S, 3100 + i) for i, (n, J, S) in enumerate(shapes)]
    dev = torch.device("cuda")
    ys = [_t(torch, y, dev) for _, _, y in frames]
    ms = [_t(torch, fr.mask, dev) for _, fr, _ in frames]
    out = {}
    for multi in ("0", "1"):
        monkeypatch.setenv("NLINV_BATCH_MULTI", multi)
        with NlinvBatch([(n, J) for n, J, _ in shapes], newton_steps=3, cg_iters=8) as b:
            out[multi] = [x.cpu().numpy() for x in b.reconstruct(ys, ms)]
    for i, (a, c) in enumerate(zip(out["0"], out["1"])):
        assert np.isfinite(c).all(), i
        assert rel(c, a) < 1e-5, i
