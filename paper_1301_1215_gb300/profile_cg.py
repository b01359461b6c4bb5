"""Profiling driver: one reconstruction of a synthetic frame, then one CG iteration launched kernel by kernel
(nlinv_profile_cg) inside the NVTX range "cgprof", so that a profiler can select exactly those kernels, e.g.

    ncu --set full --clock-control none --nvtx --nvtx-include "cgprof/" -o prof python -m paper_1301_1215_gb300.profile_cg

Defaults: the real-time workload (384 x 384 grid, 10 coils, 13 spokes, 7 Newton steps x 30 CG iterations);
--tensor-dft runs the passes with their radix-16 stages on the tensor cores (n = 256, 512); --batch F profiles the
batched kernels of the uneven workload's first F frames instead (NVTX range "batchprof").
"""
from __future__ import annotations

import argparse
import json

import numpy as np
import torch

from . import synth
from .nlinv import Nlinv


def main(argv=None) -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=384)
    ap.add_argument("--coils", type=int, default=10)
    ap.add_argument("--spokes", type=int, default=13)
    ap.add_argument("--reps", type=int, default=1)
    ap.add_argument("--tensor-dft", action="store_true", help="radix-16 DFT stages on the tensor cores")
    ap.add_argument("--batch", type=int, default=0, metavar="F",
                    help="instead: a batch of the first F frames of the uneven workload (grid 128-384, 4-16 coils), "
                         "one batched reconstruction, then its CG kernels once each inside the NVTX range "
                         "\"batchprof\" (nlinv_batch_profile_cg)")
    args = ap.parse_args(argv)
    if args.batch:
        return batch_main(args.batch)
    fr = synth.make_frame(args.n, args.coils, args.spokes, seed=1003)
    dev = torch.device("cuda")
    with Nlinv(args.n, args.coils, use_graph=False, tensor_dft=args.tensor_dft) as ctx:
        rho = torch.from_numpy(fr.rho.astype(np.complex64)).to(dev)
        coils = torch.from_numpy(fr.coils.astype(np.complex64)).to(dev)
        mask = torch.from_numpy(fr.mask).to(dev)
        y = ctx.simulate(rho, coils, mask)
        ctx.reconstruct(y, mask)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("cgprof")
        ms = ctx.profile_cg(reps=args.reps)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
    print(json.dumps({k: round(v * 1e3, 2) for k, v in ms.items()}))


def batch_main(nframes: int) -> None:
    from .nlinv import NlinvBatch
    dev = torch.device("cuda")
    shapes = synth.uneven_batch_shapes(64)[:nframes]
    ys, ms = [], []
    for i, (n, J, S) in enumerate(shapes):
        fr = synth.make_frame(n, J, S, seed=5000 + i)
        with Nlinv(n, J, use_graph=False) as ctx:
            ys.append(ctx.simulate(torch.from_numpy(fr.rho.astype(np.complex64)).to(dev),
                                   torch.from_numpy(fr.coils.astype(np.complex64)).to(dev),
                                   torch.from_numpy(fr.mask).to(dev)))
        ms.append(torch.from_numpy(fr.mask).to(dev))
    with NlinvBatch([(n, J) for n, J, _ in shapes]) as b:
        b.reconstruct(ys, ms)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("batchprof")
        ms_k = b.profile_cg(reps=1)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
    print(json.dumps({"frames": nframes, "sides": sorted({n for n, _, _ in shapes}),
                      "us": {k: round(v * 1e3, 2) for k, v in ms_k.items()}}))


if __name__ == "__main__":
    main()
