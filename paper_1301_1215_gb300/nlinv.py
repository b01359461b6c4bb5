"""PyTorch-facing binding of libnlinv.so: argument marshalling only.

Every method hands device pointers of complex64 / uint8 tensors to the C interface of include/nlinv.h; the
operators F, DF, DF^H, the normal operator of Eq. 3 and the whole Gauss-Newton reconstruction run in the
library's CUDA kernels.  There is no CPU fallback: without the built library or a GPU the calls raise.

Tensor layouts follow the C interface: a plane is an (n, n) complex64 tensor in natural FFT order; the unknown
x = (rho, chat_1 .. chat_J) has shape (1 + J, n, n); data-space arrays have shape (J, n, n); the sampling pattern
is an (n, n) uint8 tensor.
"""
from __future__ import annotations

import ctypes as C
from typing import Optional, Sequence

import torch

from . import _lib

__all__ = ["Nlinv", "NlinvBatch", "supported_size", "NlinvError"]

NlinvError = _lib.NlinvError


def supported_size(n: int) -> bool:
    """True if the library has a compiled transform for grid side n."""
    return bool(_lib.load().nlinv_supported_size(int(n)))


def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else C.c_void_p(t.data_ptr())


class Nlinv:
    """One NLINV context: grid side ``n``, ``ncoils`` coils and the solver schedule of Eq. 3.

    The context owns a CUDA stream; each call orders itself after the caller's current stream and makes the
    current stream wait for it, so results can be used right away on the current stream.
    """

    def __init__(self, n: int, ncoils: int, *, newton_steps: int = 7, cg_iters: int = 30, alpha0: float = 1.0,
                 alpha_q: float = 0.5, alpha_min: float = 0.0, sobolev_a: float = 220.0, sobolev_l: float = 32.0,
                 fov: Optional[int] = None, use_graph: bool = True, tensor_dft: bool = False, device=None):
        lib = _lib.load()
        if not torch.cuda.is_available():
            raise RuntimeError("Nlinv needs a CUDA device; there is no CPU implementation")
        self.device = torch.device(device if device is not None else "cuda", )
        if self.device.index is None:
            self.device = torch.device("cuda", torch.cuda.current_device())
        p = _lib.Params()
        lib.nlinv_default_params(C.byref(p), int(n), int(ncoils))
        p.newton_steps, p.cg_iters = int(newton_steps), int(cg_iters)
        p.alpha0, p.alpha_q, p.alpha_min = float(alpha0), float(alpha_q), float(alpha_min)
        p.sobolev_a, p.sobolev_l = float(sobolev_a), float(sobolev_l)
        p.fov = int(n // 4 if fov is None else fov)
        p.use_graph = 1 if use_graph else 0
        p.tensor_dft = 1 if tensor_dft else 0
        self.params = p
        self.n, self.ncoils = int(n), int(ncoils)
        self._h = C.c_void_p()
        with torch.cuda.device(self.device):
            self.stream = torch.cuda.Stream(self.device)
            _lib.check(lib.nlinv_create(C.byref(p), C.c_void_p(self.stream.cuda_stream), C.byref(self._h)), None)
        self._lib = lib

    # ------------------------------------------------------------------------------------------ helpers ----
    def close(self) -> None:
        if self._h:
            self._lib.nlinv_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _check(self, status: int) -> None:
        _lib.check(status, self._h)

    def _shape_x(self):
        return (1 + self.ncoils, self.n, self.n)

    def _shape_y(self):
        return (self.ncoils, self.n, self.n)

    def _dev(self, t: torch.Tensor, shape: Sequence[int], dtype, name: str) -> torch.Tensor:
        if not isinstance(t, torch.Tensor):
            raise TypeError(f"{name} must be a torch.Tensor")
        if t.device != self.device:
            raise ValueError(f"{name} must be on {self.device}, got {t.device}")
        if t.dtype != dtype:
            raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
        if tuple(t.shape) != tuple(shape):
            raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
        return t.contiguous()

    def _x(self, t, name="x"):
        return self._dev(t, self._shape_x(), torch.complex64, name)

    def _y(self, t, name="y"):
        return self._dev(t, self._shape_y(), torch.complex64, name)

    def _m(self, t, name="mask"):
        return self._dev(t, (self.n, self.n), torch.uint8, name)

    def _begin(self):
        self.stream.wait_stream(torch.cuda.current_stream(self.device))

    def _end(self):
        torch.cuda.current_stream(self.device).wait_stream(self.stream)

    # ---------------------------------------------------------------------------------------- operators ----
    def forward(self, x: torch.Tensor, mask: torch.Tensor, out: Optional[torch.Tensor] = None) -> torch.Tensor:
        """F x (Eq. 2): P FFT(M rho c_j) with c_j = W^-1 chat_j; shape (J, n, n)."""
        x, mask = self._x(x), self._m(mask)
        out = torch.empty(self._shape_y(), dtype=torch.complex64, device=self.device) if out is None else self._y(out, "out")
        self._begin()
        self._check(self._lib.nlinv_forward(self._h, _ptr(x), _ptr(mask), _ptr(out)))
        self._end()
        return out

    def derivative(self, x, mask, dx, out=None) -> torch.Tensor:
        """DF_x dx: P FFT(M (drho c_j + rho W^-1 dchat_j)); shape (J, n, n)."""
        x, mask, dx = self._x(x), self._m(mask), self._x(dx, "dx")
        out = torch.empty(self._shape_y(), dtype=torch.complex64, device=self.device) if out is None else self._y(out, "out")
        self._begin()
        self._check(self._lib.nlinv_derivative(self._h, _ptr(x), _ptr(mask), _ptr(dx), _ptr(out)))
        self._end()
        return out

    def adjoint(self, x, mask, r, out=None) -> torch.Tensor:
        """DF_x^H r: (sum_j conj(c_j) z_j, w FFT(conj(rho) z_j)) with z_j = M FFT^-1(P r_j); shape (1+J, n, n)."""
        x, mask, r = self._x(x), self._m(mask), self._y(r, "r")
        out = torch.empty(self._shape_x(), dtype=torch.complex64, device=self.device) if out is None else self._x(out, "out")
        self._begin()
        self._check(self._lib.nlinv_adjoint(self._h, _ptr(x), _ptr(mask), _ptr(r), _ptr(out)))
        self._end()
        return out

    def normal(self, x, mask, d, alpha: float, out=None) -> torch.Tensor:
        """(DF_x^H DF_x + alpha I) d, the left-hand side of Eq. 3; shape (1+J, n, n)."""
        x, mask, d = self._x(x), self._m(mask), self._x(d, "d")
        out = torch.empty(self._shape_x(), dtype=torch.complex64, device=self.device) if out is None else self._x(out, "out")
        self._begin()
        self._check(self._lib.nlinv_normal(self._h, _ptr(x), _ptr(mask), _ptr(d), float(alpha), _ptr(out)))
        self._end()
        return out

    def image(self, x, out=None) -> torch.Tensor:
        """Display image rho * sqrt(sum_j |c_j|^2) on Omega, centred; shape (2 fov, 2 fov)."""
        x = self._x(x)
        w = 2 * self.params.fov
        out = torch.empty((w, w), dtype=torch.complex64, device=self.device) if out is None else \
            self._dev(out, (w, w), torch.complex64, "out")
        self._begin()
        self._check(self._lib.nlinv_image(self._h, _ptr(x), _ptr(out)))
        self._end()
        return out

    def simulate(self, rho, coil_img, mask, out=None) -> torch.Tensor:
        """Gridded signal-equation data (Eq. 1) for image-domain coils: P FFT(M rho c_j); shape (J, n, n)."""
        rho = self._dev(rho, (self.n, self.n), torch.complex64, "rho")
        coil_img, mask = self._y(coil_img, "coil_img"), self._m(mask)
        out = torch.empty(self._shape_y(), dtype=torch.complex64, device=self.device) if out is None else self._y(out, "out")
        self._begin()
        self._check(self._lib.nlinv_simulate(self._h, _ptr(rho), _ptr(coil_img), _ptr(mask), _ptr(out)))
        self._end()
        return out

    # ---------------------------------------------------------------------------------- reconstruction ----
    def reconstruct(self, y: torch.Tensor, mask: torch.Tensor, x0: Optional[torch.Tensor] = None,
                    x_ref: Optional[torch.Tensor] = None, resid: bool = False):
        """Gauss-Newton reconstruction (Eq. 3) from x0 (default: rho = 1, chat = 0), regularised toward x_ref
        (default: x0).  Returns x_N, or (x_N, residual norms |y - F x_n| for n = 0..N) when ``resid``."""
        y, mask = self._y(y), self._m(mask)
        if x0 is None:
            x = torch.zeros(self._shape_x(), dtype=torch.complex64, device=self.device)
            x[0] = 1.0
        else:
            x = self._x(x0, "x0").clone()
        xr = None if x_ref is None else self._x(x_ref, "x_ref")
        return self._run(y, mask, xr, x, resid)

    def reconstruct_inplace(self, y, mask, x_inout, x_ref=None, resid: bool = False):
        """As :meth:`reconstruct`, writing x_N over ``x_inout``.  Any argument may be a CPU tensor: host buffers
        are copied through the library's workspace (the call then waits for the result)."""
        return self._run(y, mask, x_ref, x_inout, resid)

    def reconstruct_checkpoints(self, y: torch.Tensor, mask: torch.Tensor, x0: Optional[torch.Tensor] = None,
                                x_ref: Optional[torch.Tensor] = None):
        """Reconstruction that also keeps every Gauss-Newton iterate (nlinv_reconstruct_checkpoints).  Returns
        (x_N, checkpoints) with checkpoints of shape (newton_steps + 1, 1+J, n, n): x_0 .. x_N."""
        y, mask = self._y(y), self._m(mask)
        if x0 is None:
            x = torch.zeros(self._shape_x(), dtype=torch.complex64, device=self.device)
            x[0] = 1.0
        else:
            x = self._x(x0, "x0").clone()
        xr = None if x_ref is None else self._x(x_ref, "x_ref")
        ck = torch.empty((self.params.newton_steps + 1,) + self._shape_x(), dtype=torch.complex64, device=self.device)
        self._begin()
        self._check(self._lib.nlinv_reconstruct_checkpoints(self._h, _ptr(y), _ptr(mask), _ptr(xr), _ptr(x),
                                                            _ptr(ck), None))
        self._end()
        return x, ck

    def reconstruct_vjp(self, y: torch.Tensor, mask: torch.Tensor, checkpoints: torch.Tensor,
                        grad_x: torch.Tensor, want_xref: bool = True, tied: bool = False):
        """Backward pass of the reconstruction (nlinv_reconstruct_vjp) from dL/dx_N over ``checkpoints``.
        Returns (dL/dy, dL/dx_0, dL/dx_ref or None); with ``tied`` (the reconstruction regularised toward its start
        value) the second entry is the gradient with respect to that start value."""
        y, mask, gx = self._y(y), self._m(mask), self._x(grad_x, "grad_x")
        ck = self._dev(checkpoints, (self.params.newton_steps + 1,) + self._shape_x(), torch.complex64,
                       "checkpoints")
        gy = torch.empty(self._shape_y(), dtype=torch.complex64, device=self.device)
        g0 = torch.empty(self._shape_x(), dtype=torch.complex64, device=self.device)
        gr = torch.empty(self._shape_x(), dtype=torch.complex64, device=self.device) if want_xref else None
        self._begin()
        self._check(self._lib.nlinv_reconstruct_vjp(self._h, _ptr(y), _ptr(mask), _ptr(ck), _ptr(gx),
                                                    1 if tied else 0, _ptr(gy), _ptr(g0), _ptr(gr)))
        self._end()
        return gy, g0, gr

    def _run(self, y, mask, xr, x, resid):
        nres = self.params.newton_steps + 1
        buf = (C.c_double * nres)() if resid else None
        self._begin()
        self._check(self._lib.nlinv_reconstruct(self._h, _ptr(y), _ptr(mask), _ptr(xr), _ptr(x),
                                                buf if resid else None))
        self._end()
        if resid:
            return x, [float(v) for v in buf]
        return x

    def wait(self, timeout_s: float = -1.0) -> None:
        """Waits for the context's queued work (raises NlinvError with ETIMEOUT or EBREAKDOWN)."""
        self._check(self._lib.nlinv_wait(self._h, float(timeout_s)))

    CG_KERNELS = ("row p-update/W^-1", "col W^-1/C/FFT", "row PSF", "col FFT^-1/C^H/FFT", "row W^-H+alpha p",
                  "cg step")

    def profile_cg(self, reps: int = 20) -> dict:
        """Steady-state CUDA-event duration (ms) of each kernel of one CG iteration: each is launched ``reps``
        times back to back on the state of the last reconstruction (which it advances), as in a graph replay."""
        ms = (C.c_double * len(self.CG_KERNELS))()
        self._begin()
        self._check(self._lib.nlinv_profile_cg(self._h, int(reps), ms))
        self._end()
        return dict(zip(self.CG_KERNELS, [float(v) for v in ms]))

    def autotune(self, y: torch.Tensor, mask: torch.Tensor, x0: Optional[torch.Tensor] = None,
                 reps: int = 3) -> dict:
        """Picks the transforms' split and column strips and the launch shapes by timing whole graph-replayed
        reconstructions of a representative frame (nlinv_autotune; x0 default: rho = 1, chat = 0), one dimension
        per stage; overwrites the workspace.  Returns the choice and every timed candidate (a dict each)."""
        y, mask = self._y(y), self._m(mask)
        if x0 is None:
            x0 = torch.zeros(self._shape_x(), dtype=torch.complex64, device=self.device)
            x0[0] = 1.0
        x0 = self._x(x0, "x0")
        t = _lib.Tuning()
        table = (_lib.Tuning * _lib.TUNE_TABLE)()
        self._begin()
        self._check(self._lib.nlinv_autotune(self._h, _ptr(y), _ptr(mask), _ptr(x0), int(reps), C.byref(t),
                                             table, _lib.TUNE_TABLE))
        self._end()

        def rec(e):
            return {"split_n1": int(e.split_n1), "col_strip": int(e.col_strip),
                    "row_blocks_per_sm": int(e.row_blocks_per_sm), "vec_blocks_per_sm": int(e.vec_blocks_per_sm),
                    "pdl": bool(e.pdl), "ms_per_frame": round(float(e.ms_per_frame), 4), "stage": int(e.stage)}
        out = rec(t)
        out["candidates"] = [rec(e) for e in table if e.ms_per_frame > 0]
        return out

    def set_shapes(self, split_n1: int, col_strip: int = 8, row_blocks_per_sm: int = 2, vec_blocks_per_sm: int = 4,
                   pdl: bool = True) -> None:
        """Applies explicit tile and launch shapes (nlinv_set_shapes), e.g. a stored nlinv_autotune choice."""
        t = _lib.Tuning()
        t.split_n1, t.col_strip, t.row_blocks_per_sm = int(split_n1), int(col_strip), int(row_blocks_per_sm)
        t.vec_blocks_per_sm, t.pdl = int(vec_blocks_per_sm), 1 if pdl else 0
        self._check(self._lib.nlinv_set_shapes(self._h, C.byref(t)))

    @property
    def last_launch_count(self) -> int:
        """Kernel launches queued by the last call (kernel nodes of the graph when one was replayed)."""
        return int(self._lib.nlinv_last_launch_count(self._h))

    def cg_stops(self) -> list:
        """Per Newton step of the last reconstruction: the CG iteration that reached the rounding floor and
        stopped the solve, or -1 when all CG iterations ran (nlinv_cg_stops; waits for the stream)."""
        nn = int(self.params.newton_steps)
        out = (C.c_int * nn)()
        self._check(self._lib.nlinv_cg_stops(self._h, out, nn))
        return [int(v) for v in out]


class NlinvBatch:
    """Independent frames of uneven grid side and coil count reconstructed together (nlinv_reconstruct_batch):
    every pass is one launch per grid side over all frames of that side, the sides run as parallel graph branches.

    ``shapes`` lists (n, ncoils) per frame; the solver options are those of :class:`Nlinv` (fov = n/4)."""

    def __init__(self, shapes, *, newton_steps: int = 7, cg_iters: int = 30, alpha0: float = 1.0,
                 alpha_q: float = 0.5, alpha_min: float = 0.0, sobolev_a: float = 220.0, sobolev_l: float = 32.0,
                 device=None):
        lib = _lib.load()
        if not torch.cuda.is_available():
            raise RuntimeError("NlinvBatch needs a CUDA device; there is no CPU implementation")
        self.device = torch.device(device if device is not None else "cuda")
        if self.device.index is None:
            self.device = torch.device("cuda", torch.cuda.current_device())
        self.shapes = [(int(n), int(j)) for n, j in shapes]
        p = _lib.Params()
        lib.nlinv_default_params(C.byref(p), self.shapes[0][0], self.shapes[0][1])
        p.newton_steps, p.cg_iters = int(newton_steps), int(cg_iters)
        p.alpha0, p.alpha_q, p.alpha_min = float(alpha0), float(alpha_q), float(alpha_min)
        p.sobolev_a, p.sobolev_l = float(sobolev_a), float(sobolev_l)
        self.params = p
        descs = (_lib.FrameDesc * len(self.shapes))()
        for d, (n, j) in zip(descs, self.shapes):
            d.n, d.ncoils = n, j
        self._h = C.c_void_p()
        with torch.cuda.device(self.device):
            self.stream = torch.cuda.Stream(self.device)
            _lib.check(lib.nlinv_batch_create(C.byref(p), len(self.shapes), descs,
                                              C.c_void_p(self.stream.cuda_stream), C.byref(self._h)), None)
        self._lib = lib

    def close(self) -> None:
        if self._h:
            self._lib.nlinv_batch_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def launch_count(self) -> int:
        return int(self._lib.nlinv_batch_launch_count(self._h))

    def profile_cg(self, reps: int = 10) -> dict:
        """CUDA-event duration (ms) of each batched kernel of one CG iteration, all grid sides, launched ``reps``
        times back to back on the state of the last batched reconstruction (nlinv_batch_profile_cg)."""
        ms = (C.c_double * len(Nlinv.CG_KERNELS))()
        _lib.check(self._lib.nlinv_batch_profile_cg(self._h, int(reps), ms), None)
        return dict(zip(Nlinv.CG_KERNELS, [float(v) for v in ms]))

    def reconstruct(self, ys, masks, xs=None, x_refs=None, resid: bool = False):
        """Reconstructs every frame.  ``xs`` (start values, overwritten with the results; default rho = 1,
        chat = 0) and ``x_refs`` are lists of (1+J, n, n) complex64 tensors; ``ys`` (J, n, n), ``masks`` (n, n)
        uint8.  Tensors may live on the device or on the host.  Returns the list of results (and the residual
        norms per frame when ``resid``)."""
        nf = len(self.shapes)
        if len(ys) != nf or len(masks) != nf:
            raise ValueError("one y and one mask per frame are required")
        if xs is None:
            xs = []
            for n, j in self.shapes:
                x = torch.zeros((1 + j, n, n), dtype=torch.complex64, device=self.device)
                x[0] = 1.0
                xs.append(x)
        descs = (_lib.FrameDesc * nf)()
        bufs = [(C.c_double * (self.params.newton_steps + 1))() for _ in range(nf)] if resid else None
        keep = []
        for i, (n, j) in enumerate(self.shapes):
            y, m, x = ys[i].contiguous(), masks[i].contiguous(), xs[i]
            if tuple(y.shape) != (j, n, n) or tuple(m.shape) != (n, n) or tuple(x.shape) != (1 + j, n, n):
                raise ValueError(f"frame {i}: shapes do not match ({n}, {j})")
            if not x.is_contiguous() or x.dtype != torch.complex64 or y.dtype != torch.complex64 or m.dtype != torch.uint8:
                raise TypeError(f"frame {i}: complex64 y/x (contiguous x) and uint8 mask are required")
            xr = None if x_refs is None or x_refs[i] is None else x_refs[i].contiguous()
            keep += [y, m, xr]
            d = descs[i]
            d.n, d.ncoils = n, j
            d.y, d.mask, d.x_inout = y.data_ptr(), m.data_ptr(), x.data_ptr()
            d.x_ref = None if xr is None else xr.data_ptr()
            d.resid = C.cast(bufs[i], C.POINTER(C.c_double)) if resid else None
        self.stream.wait_stream(torch.cuda.current_stream(self.device))
        _lib.check(self._lib.nlinv_reconstruct_batch(self._h, nf, descs), None)
        torch.cuda.current_stream(self.device).wait_stream(self.stream)
        if resid:
            return xs, [[float(v) for v in b] for b in bufs]
        return xs


class Gridder:
    """Nearest-neighbour gridding of radial spokes onto the n x n grid with averaging (nlinv_gridder_create /
    nlinv_grid): the interpolation that Sec. 3.1 performs before the reconstruction.  ``directions``: (S, 2) array of
    (cos, sin) of the spoke angles.  :meth:`grid` maps samples (J, S, 2n) complex64 on the device to the gridded data
    (J, n, n) and the sampling pattern (n, n) uint8."""

    def __init__(self, n: int, directions, device=None):
        import numpy as np
        self._lib = _lib.load()
        dev = torch.device("cuda") if device is None else torch.device(device)
        if dev.type != "cuda" or not torch.cuda.is_available():
            raise RuntimeError("the NLINV library needs a CUDA device")
        self.device = dev if dev.index is not None else torch.device("cuda", torch.cuda.current_device())
        d = np.ascontiguousarray(np.asarray(directions, dtype=np.float64).reshape(-1, 2))
        self.n, self.nspokes = int(n), int(d.shape[0])
        self.stream = torch.cuda.Stream(device=self.device)
        h = C.c_void_p()
        with torch.cuda.device(self.device):
            _lib.check(self._lib.nlinv_gridder_create(self.n, self.nspokes,
                                                      d.ctypes.data_as(C.POINTER(C.c_double)),
                                                      C.c_void_p(self.stream.cuda_stream), C.byref(h)))
        self._h = h

    def grid(self, samples: torch.Tensor):
        if not isinstance(samples, torch.Tensor) or samples.device != self.device or samples.dtype != torch.complex64:
            raise TypeError(f"samples must be a complex64 tensor on {self.device}")
        if samples.dim() != 3 or tuple(samples.shape[1:]) != (self.nspokes, 2 * self.n):
            raise ValueError(f"samples must have shape (J, {self.nspokes}, {2 * self.n})")
        samples = samples.contiguous()
        J = samples.shape[0]
        y = torch.empty((J, self.n, self.n), dtype=torch.complex64, device=self.device)
        m = torch.empty((self.n, self.n), dtype=torch.uint8, device=self.device)
        self.stream.wait_stream(torch.cuda.current_stream(self.device))
        _lib.check(self._lib.nlinv_grid(self._h, int(J), _ptr(samples), _ptr(y), _ptr(m)))
        torch.cuda.current_stream(self.device).wait_stream(self.stream)
        return y, m

    def close(self) -> None:
        if getattr(self, "_h", None):
            self._lib.nlinv_gridder_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
