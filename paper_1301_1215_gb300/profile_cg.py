"""Profiling driver: one reconstruction of a synthetic frame, then one CG iteration launched kernel by kernel
(nlinv_profile_cg) inside the NVTX range "cgprof", so that a profiler can select exactly those kernels, e.g.

    ncu --set full --clock-control none --nvtx --nvtx-include "cgprof/" -o prof python -m paper_1301_1215_gb300.profile_cg

Defaults: the real-time workload (384 x 384 grid, 10 coils, 13 spokes, 7 Newton steps x 30 CG iterations);
--tensor-dft runs the passes with their radix-16 stages on the tensor cores (n = 256, 512).
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
    args = ap.parse_args(argv)
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


if __name__ == "__main__":
    main()
