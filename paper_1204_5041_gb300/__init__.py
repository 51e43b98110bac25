"""GB300-native full-sky string ISW maps (Eq. 1-2 of arXiv:1204.5041) -- Python binding.

A thin ctypes layer over the C ABI of ``libisw.so`` (include/isw.h): it only marshals
PyTorch CUDA tensors into device pointers and the current CUDA stream; every step of the
computation runs in the library's kernels.  If the library cannot be loaded the calls
raise -- there is no CPU fallback.

Functions carry the names of the C entry points:
  hp_pix2vec_ring, lightcone_intersect, isw_map, isw_map_adjoint, isw_map_batched,
and ``ISWMap`` is the ``torch.autograd.Function`` (forward = isw_map, backward =
isw_map_adjoint).
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

from . import _build

__all__ = [
    "build", "Context", "default_context", "hp_pix2vec_ring", "lightcone_intersect", "isw_map",
    "isw_map_adjoint", "isw_map_batched", "ISWMap", "ISWError", "F64", "F32C", "LINEAR", "BURDEN",
]

OK, EINVAL, ECUDA, EDOMAIN, ENOCONV, ETIMEOUT, ENOMEM = range(7)
F64, F32C = 0, 1
LINEAR, BURDEN = 0, 1
FULLSKY, FLATSKY = 0, 1
SKIP_LIGHTCONE, GRAPH, AUTOTUNE = 1, 2, 4
(PARAM_NEAR_K, PARAM_B_MIN, PARAM_SPLIT, PARAM_VARIANT, PARAM_TIMING, PARAM_D_FAR, PARAM_NUM_VARIANTS,
 PARAM_WAIT_POLLS) = range(8)
_STATUS_NAMES = {0: "ISW_OK", 1: "ISW_EINVAL", 2: "ISW_ECUDA", 3: "ISW_EDOMAIN", 4: "ISW_ENOCONV",
                 5: "ISW_ETIMEOUT", 6: "ISW_ENOMEM"}

_lib = None
_lib_lock = threading.Lock()
_vp, _i64, _i32, _dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double


class ISWError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


def build(force: bool = False) -> str:
    """Compile libisw.so for sm_103a (in-tree)."""
    return _build.build(force=force)


def lib():
    """The loaded libisw.so (built on first use if the toolkit is present)."""
    global _lib
    with _lib_lock:
        if _lib is None:
            path = _build.LIB
            if not _build.up_to_date():
                path = _build.build()
            L = ctypes.CDLL(path)
            sig = {
                "isw_create": (_i32, [ctypes.POINTER(_vp), _i32]),
                "isw_destroy": (_i32, [_vp]),
                "isw_last_error": (ctypes.c_char_p, [_vp]),
                "isw_check_status": (_i32, [_vp, _vp, ctypes.POINTER(_i64)]),
                "isw_fma_rate": (_i32, [_vp, _i32, ctypes.POINTER(_dbl), _vp]),
                "isw_set_param": (_i32, [_vp, _i32, _dbl]),
                "isw_get_param": (_i32, [_vp, _i32, ctypes.POINTER(_dbl)]),
                "isw_get_timing": (_i32, [_vp, ctypes.POINTER(_dbl), ctypes.POINTER(_i64), ctypes.POINTER(_i64),
                                          _i32]),
                "hp_pix2vec_ring": (_i32, [_vp, _i64, _i64, _i64, _vp, _vp, _i64, _vp]),
                "lightcone_intersect": (_i32, [_vp, _i32, _vp, _i64, _i64, _vp, _i64, _i64, _dbl, _vp, _dbl,
                                               _vp, _i64, _vp, _vp, _vp]),
                "isw_map": (_i32, [_vp, _i64, _i64, _i64, _vp, _vp, _i64, _i64, _vp, _dbl, _i32, _i32, _vp,
                                   _vp]),
                "isw_map_adjoint": (_i32, [_vp, _i64, _i64, _i64, _vp, _vp, _i64, _i64, _vp, _dbl, _i32, _vp,
                                           _vp, _i64, _i32, _vp]),
                "isw_map_batched": (_i32, [_vp, _i64, _vp, _i64, _vp, _i64, _vp, _vp, _vp, _i64, _i64, _vp,
                                           _dbl, _dbl, _i32, _i32, _i32, _vp, _vp]),
                "lightcone_adjoint": (_i32, [_vp, _i32, _vp, _i64, _i64, _vp, _i64, _i64, _dbl, _vp, _vp, _vp,
                                             _i64, _i32, _vp, _i64, _vp, _i64, _vp]),
                "hp_vec2pix_ring": (_i32, [_vp, _i64, _vp, _i64, _i64, _vp, _vp]),
                "lightcone_intersect_shells": (_i32, [_vp, _vp, _i64, _vp, _i64, _vp, _vp, _vp, _i64, _i64, _vp,
                                                      _dbl, _vp, _i64, _vp]),
                "box_place": (_i32, [_vp, _vp, _i64, _vp, _i64, _vp, _i64, _vp, _vp, _i64, _vp, _vp]),
                "cone_cut": (_i32, [_vp, _vp, _i64, _vp, _i64, _i64, _vp, _vp, _vp, _vp, _vp, _i64, _vp,
                                    ctypes.POINTER(_i64), _vp]),
                "isw_map_patch": (_i32, [_vp, _vp, _i64, _dbl, _vp, _i64, _i64, _vp, _dbl, _i32, _i32, _i32, _vp,
                                         _vp]),
                "isw_map_cl": (_i32, [_vp, _i64, _vp, _i64, _vp, _vp, _vp]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


class Context:
    """An ``isw_ctx`` bound to one CUDA device (workspace + device status word)."""

    def __init__(self, device: int | None = None):
        if device is None:
            device = torch.cuda.current_device()
        self.device = int(device)
        self._h = _vp()
        r = lib().isw_create(ctypes.byref(self._h), self.device)
        if r != OK:
            raise ISWError(r, f"isw_create(device={self.device}) failed")

    @property
    def handle(self):
        return self._h

    def close(self):
        if self._h:
            lib().isw_destroy(self._h)
            self._h = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def last_error(self) -> str:
        return (lib().isw_last_error(self._h) or b"").decode()

    def check(self, r: int):
        if r != OK:
            raise ISWError(r, self.last_error())

    def set_param(self, key: int, value: float):
        self.check(lib().isw_set_param(self._h, int(key), float(value)))

    def get_param(self, key: int) -> float:
        v = _dbl()
        self.check(lib().isw_get_param(self._h, int(key), ctypes.byref(v)))
        return v.value

    def timing(self, reset: bool = True):
        """(summed device ms of the timed pair-kernel launches, pair-kernel launches, all kernel
        launches) since the last reset; device times need PARAM_TIMING on."""
        ms, n, m = _dbl(), _i64(), _i64()
        self.check(lib().isw_get_timing(self._h, ctypes.byref(ms), ctypes.byref(n), ctypes.byref(m), int(reset)))
        return ms.value, n.value, m.value

    def fma_rate(self, prec="f32c", stream=None) -> float:
        """Measured FMA-pipe throughput of this context's GPU in flop/s (FMA = 2 flops), FP32 or FP64."""
        v = _dbl()
        self.check(lib().isw_fma_rate(self._h, _precision(prec), ctypes.byref(v), _stream(stream, self.device)))
        return v.value

    def check_status(self, stream=None, raise_on_error: bool = False):
        """Synchronise the stream; return (status code, counts dict) and clear the device status."""
        counts = (_i64 * 3)()
        r = lib().isw_check_status(self._h, _stream(stream, self.device), counts)
        if raise_on_error and r != OK:
            raise ISWError(r, self.last_error())
        return r, {"zero_pairs": counts[0], "skipped_samples": counts[1], "near_pairs": counts[2]}


_contexts: dict[int, Context] = {}


def default_context(device: int | None = None) -> Context:
    if device is None:
        device = torch.cuda.current_device()
    if device not in _contexts:
        _contexts[device] = Context(device)
    return _contexts[device]


def _stream(stream, device=None):
    """The stream handle: the given one, else torch's current stream of ``device``."""
    if stream is None:
        return _vp(torch.cuda.current_stream(device).cuda_stream)
    if isinstance(stream, torch.cuda.Stream):
        return _vp(stream.cuda_stream)
    return _vp(int(stream))


def _ptr(t):
    return _vp(t.data_ptr()) if t is not None else _vp(0)


def _dev_tensor(t, dtype, name):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    return t


def _rows(t, nrows, name):
    """A [nrows, n] tensor with unit stride along n and rows that do not overlap -> (n, ld)."""
    if t.dim() != 2 or t.shape[0] != nrows:
        raise ValueError(f"{name} must have shape [{nrows}, n]")
    n = t.shape[1]
    if n > 0 and t.stride(1) != 1:
        raise ValueError(f"{name} must have unit stride along its last axis")
    if nrows == 1 or n == 0:
        return n, max(n, 1)
    if t.stride(0) < n:
        # rows that overlap (an expand() has stride 0): the library would read past the storage
        raise ValueError(f"{name} has row stride {t.stride(0)} < {n}: rows must not overlap")
    return n, t.stride(0)


def _xobs(x_obs):
    x = (0.0, 0.0, 0.0) if x_obs is None else tuple(float(v) for v in x_obs)
    return (_dbl * 3)(*x)


def _ctx(ctx, t=None):
    """The given context, else the default context of the GPU that holds tensor ``t`` (the
    current device when no tensor is given): the kernels must run where the data lives."""
    if ctx is not None:
        return ctx
    if t is not None and getattr(t, "is_cuda", False):
        return default_context(t.device.index if t.device.index is not None else torch.cuda.current_device())
    return default_context()


def _precision(prec) -> int:
    if prec in (F64, "f64", "fp64", torch.float64):
        return F64
    if prec in (F32C, "f32c", "fp32c", torch.float32):
        return F32C
    raise ValueError(f"unknown precision {prec!r}")


def _pixels(nside, pix, pix0, npix):
    if pix is not None:
        pix = _dev_tensor(pix, torch.int64, "pix").contiguous()
        return pix, 0, pix.numel()
    if npix is None:
        npix = 12 * nside * nside - pix0
    return None, int(pix0), int(npix)


def hp_pix2vec_ring(nside: int, pix=None, pix0: int = 0, npix: int | None = None, out=None, ctx=None,
                    stream=None, device=None):
    """RING pixel centres as a float64 CUDA tensor [3, npix]."""
    c = _ctx(ctx, out if out is not None else pix)
    pix, pix0, npix = _pixels(nside, pix, pix0, npix)
    if out is None:
        out = torch.empty((3, npix), dtype=torch.float64, device=device or f"cuda:{c.device}")
    _dev_tensor(out, torch.float64, "out")
    n, ld = _rows(out, 3, "out")
    c.check(lib().hp_pix2vec_ring(c.handle, int(nside), pix0, npix, _ptr(pix), _ptr(out), ld,
                                  _stream(stream, c.device)))
    return out


def lightcone_intersect(mode: int, nodes, loop_params=None, t_box: float = 0.0, x_obs=None, t_obs: float = 1.0,
                        out=None, tau=None, status=None, ctx=None, stream=None):
    """Samples on the observer's past light cone: float64 CUDA tensor [10, n] (and tau, status if given)."""
    c = _ctx(ctx, nodes)
    _dev_tensor(nodes, torch.float64, "nodes")
    n, ld = _rows(nodes, 10, "nodes")
    if out is None:
        out = torch.empty((10, n), dtype=torch.float64, device=nodes.device)
    n2, ld_out = _rows(out, 10, "out")
    if n2 != n:
        raise ValueError("out must have as many columns as nodes")
    P, nloops, ldp = None, 0, 0
    if loop_params is not None:
        _dev_tensor(loop_params, torch.float64, "loop_params")
        nloops, ldp = _rows(loop_params, 17, "loop_params")
        P = loop_params
    if tau is not None:
        _dev_tensor(tau, torch.float64, "tau")
    if status is not None:
        _dev_tensor(status, torch.int32, "status")
    c.check(lib().lightcone_intersect(c.handle, int(mode), _ptr(nodes), n, ld, _ptr(P), nloops, ldp, float(t_box),
                                      _xobs(x_obs), float(t_obs), _ptr(out), ld_out, _ptr(tau), _ptr(status),
                                      _stream(stream, c.device)))
    return out


def isw_map(nside: int, samples, pix=None, pix0: int = 0, npix: int | None = None, x_obs=None, GU: float = 1.0,
            prec="f32c", accumulate: bool = False, out=None, ctx=None, stream=None):
    """Theta of Eq. (1)-(2) at the selected pixels: float64 CUDA tensor [npix]."""
    c = _ctx(ctx, samples)
    _dev_tensor(samples, torch.float64, "samples")
    n, ld = _rows(samples, 10, "samples")
    pix, pix0, npix = _pixels(nside, pix, pix0, npix)
    if out is None:
        out = torch.empty(npix, dtype=torch.float64, device=samples.device)
    _dev_tensor(out, torch.float64, "out")
    if out.numel() != npix or not out.is_contiguous():
        raise ValueError("out must be a contiguous float64 tensor of npix elements")
    c.check(lib().isw_map(c.handle, int(nside), pix0, npix, _ptr(pix), _ptr(samples), n, ld, _xobs(x_obs),
                          float(GU), _precision(prec), int(bool(accumulate)), _ptr(out),
                          _stream(stream, c.device)))
    return out


def isw_map_adjoint(nside: int, samples, dL_dtheta, pix=None, pix0: int = 0, npix: int | None = None, x_obs=None,
                    GU: float = 1.0, prec="f32c", ngrad: int = 6, out=None, ctx=None, stream=None):
    """dL/dX, dL/dXdot (then dL/dX' when ngrad >= 9 and dL/ddsigma when ngrad = 10) per sample:
    float64 CUDA tensor [ngrad, n]."""
    c = _ctx(ctx, samples)
    _dev_tensor(samples, torch.float64, "samples")
    n, ld = _rows(samples, 10, "samples")
    pix, pix0, npix = _pixels(nside, pix, pix0, npix)
    _dev_tensor(dL_dtheta, torch.float64, "dL_dtheta")
    g = dL_dtheta.contiguous()
    if g.numel() != npix:
        raise ValueError("dL_dtheta must have one value per selected pixel")
    if ngrad not in (6, 9, 10):
        raise ValueError("ngrad must be 6, 9 or 10")
    if out is None:
        out = torch.empty((ngrad, n), dtype=torch.float64, device=samples.device)
    _dev_tensor(out, torch.float64, "out")
    _, ld_g = _rows(out, ngrad, "out")
    c.check(lib().isw_map_adjoint(c.handle, int(nside), pix0, npix, _ptr(pix), _ptr(samples), n, ld, _xobs(x_obs),
                                  float(GU), _precision(prec), _ptr(g), _ptr(out), ld_g, int(ngrad),
                                  _stream(stream, c.device)))
    return out


def isw_map_batched(nside: int, nodes, shell_off, t_box, mode, loop_params=None, x_obs=None, t_obs: float = 1.0,
                    GU: float = 1.0, prec="f32c", flags: int = 0, accumulate: bool = False, out=None, ctx=None,
                    stream=None):
    """One full-sky RING map summed over many shells (host shell metadata, device nodes)."""
    import numpy as np

    c = _ctx(ctx, nodes)
    _dev_tensor(nodes, torch.float64, "nodes")
    n, ld = _rows(nodes, 10, "nodes")
    off = np.ascontiguousarray(np.asarray(shell_off, dtype=np.int64))
    tb = np.ascontiguousarray(np.asarray(t_box, dtype=np.float64))
    md = np.ascontiguousarray(np.asarray(mode, dtype=np.int32))
    nshell = len(tb)
    if off.size != nshell + 1 or md.size != nshell or off[-1] != n:
        raise ValueError("shell_off must have nshell + 1 entries ending at n; t_box, mode nshell entries")
    P, nloops, ldp = None, 0, 0
    if loop_params is not None:
        _dev_tensor(loop_params, torch.float64, "loop_params")
        nloops, ldp = _rows(loop_params, 17, "loop_params")
        P = loop_params
    npix = 12 * nside * nside
    if out is None:
        out = torch.empty(npix, dtype=torch.float64, device=nodes.device)
    _dev_tensor(out, torch.float64, "out")
    c.check(lib().isw_map_batched(c.handle, int(nside), _ptr(nodes), ld, off.ctypes.data_as(_vp), nshell,
                                  tb.ctypes.data_as(_vp), md.ctypes.data_as(_vp), _ptr(P), nloops, ldp, _xobs(x_obs),
                                  float(t_obs), float(GU), _precision(prec), int(flags), int(bool(accumulate)),
                                  _ptr(out), _stream(stream, c.device)))
    return out


def lightcone_adjoint(mode: int, nodes, tau, grad_samples, loop_params=None, t_box: float = 0.0, x_obs=None,
                      out=None, out_loops=None, ctx=None, stream=None):
    """Chain dL/d(samples) (rows X, Xdot[, X'[, dsigma]], e.g. from isw_map_adjoint) through the
    light-cone solve.  Returns (grad_nodes [10, n], grad_loops [17, nloops] or None for LINEAR):
    LINEAR gives the box-time node gradients; BURDEN gives node rows 1 (sigma) and 9 (dsigma) and
    the per-loop parameter gradients (the nodes of one loop must be contiguous)."""
    c = _ctx(ctx, nodes)
    _dev_tensor(nodes, torch.float64, "nodes")
    n, ld = _rows(nodes, 10, "nodes")
    _dev_tensor(tau, torch.float64, "tau")
    if tau.numel() != n or not tau.is_contiguous():
        raise ValueError("tau must be a contiguous float64 tensor of n elements")
    _dev_tensor(grad_samples, torch.float64, "grad_samples")
    ngrad = grad_samples.shape[0]
    if ngrad not in (6, 9, 10):
        raise ValueError("grad_samples must have 6, 9 or 10 rows")
    n2, ld_gs = _rows(grad_samples, ngrad, "grad_samples")
    if n2 != n:
        raise ValueError("grad_samples must have as many columns as nodes")
    if out is None:
        out = torch.empty((10, n), dtype=torch.float64, device=nodes.device)
    _dev_tensor(out, torch.float64, "out")
    _, ld_gn = _rows(out, 10, "out")
    P, nloops, ldp, ld_gl = None, 0, 0, 0
    if mode == BURDEN:
        if loop_params is None:
            raise ValueError("BURDEN mode needs loop_params")
        _dev_tensor(loop_params, torch.float64, "loop_params")
        nloops, ldp = _rows(loop_params, 17, "loop_params")
        P = loop_params
        if out_loops is None:
            out_loops = torch.empty((17, nloops), dtype=torch.float64, device=nodes.device)
        _dev_tensor(out_loops, torch.float64, "out_loops")
        _, ld_gl = _rows(out_loops, 17, "out_loops")
    else:
        out_loops = None
    c.check(lib().lightcone_adjoint(c.handle, int(mode), _ptr(nodes), n, ld, _ptr(P), nloops, ldp, float(t_box),
                                    _xobs(x_obs), _ptr(tau), _ptr(grad_samples), ld_gs, int(ngrad), _ptr(out), ld_gn,
                                    _ptr(out_loops), ld_gl, _stream(stream, c.device)))
    return out, out_loops


class ISWMap(torch.autograd.Function):
    """Theta = isw_map(samples); backward returns dL/dsamples with rows X, Xdot, then X' if
    ``ngrad`` >= 9 and dsigma if ``ngrad`` = 10, from isw_map_adjoint (other rows zero)."""

    @staticmethod
    def forward(ctx, samples, nside, pix=None, x_obs=None, GU=1.0, prec="f32c", ngrad=6):
        ctx.save_for_backward(samples, pix)
        ctx.args = (nside, x_obs, GU, prec, ngrad)
        return isw_map(nside, samples.detach(), pix=pix, x_obs=x_obs, GU=GU, prec=prec)

    @staticmethod
    def backward(ctx, grad_theta):
        samples, pix = ctx.saved_tensors
        nside, x_obs, GU, prec, ngrad = ctx.args
        g = isw_map_adjoint(nside, samples.detach(), grad_theta.contiguous().to(torch.float64), pix=pix,
                            x_obs=x_obs, GU=GU, prec=prec, ngrad=ngrad)
        grad = torch.zeros_like(samples)
        grad[:ngrad] = g
        return grad, None, None, None, None, None, None


class ISWLightconeMap(torch.autograd.Function):
    """Theta = isw_map(lightcone_intersect(nodes)) differentiable end to end.

    LINEAR: ``apply(nodes, None, nside, LINEAR, t_box, ...)`` with gradients for the box-time
    nodes (X, Xdot, X', dsigma).  BURDEN: ``apply(nodes, loop_params, nside, BURDEN, ...)`` with
    gradients for node rows sigma and dsigma and for the loop parameters.  Backward runs
    isw_map_adjoint (all 10 sample rows) and lightcone_adjoint on the GPU."""

    @staticmethod
    def forward(ctx, nodes, loop_params, nside, mode, t_box=0.0, pix=None, x_obs=None, t_obs=1.0, GU=1.0,
                prec="f32c"):
        n = nodes.shape[1]
        tau = torch.empty(n, dtype=torch.float64, device=nodes.device)
        P = loop_params.detach() if loop_params is not None else None
        samples = lightcone_intersect(mode, nodes.detach(), P, t_box=t_box, x_obs=x_obs, t_obs=t_obs, tau=tau)
        ctx.save_for_backward(nodes, P, samples, tau, pix)
        ctx.args = (nside, mode, t_box, x_obs, GU, prec, loop_params is not None)
        return isw_map(nside, samples, pix=pix, x_obs=x_obs, GU=GU, prec=prec)

    @staticmethod
    def backward(ctx, grad_theta):
        nodes, P, samples, tau, pix = ctx.saved_tensors
        nside, mode, t_box, x_obs, GU, prec, has_loops = ctx.args
        gs = isw_map_adjoint(nside, samples, grad_theta.contiguous().to(torch.float64), pix=pix, x_obs=x_obs, GU=GU,
                             prec=prec, ngrad=10)
        gn, gl = lightcone_adjoint(mode, nodes.detach(), tau, gs, loop_params=P, t_box=t_box, x_obs=x_obs)
        return gn, (gl if has_loops else None), None, None, None, None, None, None, None, None


def hp_vec2pix_ring(nside: int, vec, out=None, ctx=None, stream=None):
    """RING pixel of each direction (columns of a float64 CUDA tensor [3, n]): int64 tensor [n]."""
    c = _ctx(ctx, vec)
    _dev_tensor(vec, torch.float64, "vec")
    n, ld = _rows(vec, 3, "vec")
    if out is None:
        out = torch.empty(n, dtype=torch.int64, device=vec.device)
    _dev_tensor(out, torch.int64, "out")
    c.check(lib().hp_vec2pix_ring(c.handle, int(nside), _ptr(vec), n, ld, _ptr(out),
                                  _stream(stream, c.device)))
    return out


def _host_i64(a):
    import numpy as np

    return np.ascontiguousarray(np.asarray(a, dtype=np.int64))


def lightcone_intersect_shells(nodes, shell_off, t_box, mode, loop_params=None, x_obs=None, t_obs: float = 1.0,
                               out=None, ctx=None, stream=None):
    """Light-cone samples of many shells in one launch: float64 CUDA tensor [10, n]."""
    import numpy as np

    c = _ctx(ctx, nodes)
    _dev_tensor(nodes, torch.float64, "nodes")
    n, ld = _rows(nodes, 10, "nodes")
    off = _host_i64(shell_off)
    tb = np.ascontiguousarray(np.asarray(t_box, dtype=np.float64))
    md = np.ascontiguousarray(np.asarray(mode, dtype=np.int32))
    if off.size != tb.size + 1 or md.size != tb.size or off[-1] != n:
        raise ValueError("shell_off must have nshell + 1 entries ending at n; t_box, mode nshell entries")
    P, nloops, ldp = None, 0, 0
    if loop_params is not None:
        _dev_tensor(loop_params, torch.float64, "loop_params")
        nloops, ldp = _rows(loop_params, 17, "loop_params")
        P = loop_params
    if out is None:
        out = torch.empty((10, n), dtype=torch.float64, device=nodes.device)
    _, ld_out = _rows(out, 10, "out")
    c.check(lib().lightcone_intersect_shells(c.handle, _ptr(nodes), ld, off.ctypes.data_as(_vp), tb.size,
                                             tb.ctypes.data_as(_vp), md.ctypes.data_as(_vp), _ptr(P), nloops, ldp,
                                             _xobs(x_obs), float(t_obs), _ptr(out), ld_out,
                                             _stream(stream, c.device)))
    return out


def box_place(nodes_box, box_off, shell_box, place, out=None, ctx=None, stream=None):
    """Nodes of every shell placed from its box: returns (nodes [10, n_out] CUDA tensor,
    shell_off_out host int64 array)."""
    import numpy as np

    c = _ctx(ctx, nodes_box)
    _dev_tensor(nodes_box, torch.float64, "nodes_box")
    _, ldb = _rows(nodes_box, 10, "nodes_box")
    boff, sbox = _host_i64(box_off), _host_i64(shell_box)
    _dev_tensor(place, torch.float64, "place")
    if place.numel() != 12 * sbox.size or not place.is_contiguous():
        raise ValueError("place must be a contiguous float64 CUDA tensor [nshell, 12]")
    n_out = int(sum(boff[b + 1] - boff[b] for b in sbox if 0 <= b < boff.size - 1))   # bad ids: the call rejects
    if out is None:
        out = torch.empty((10, max(n_out, 1)), dtype=torch.float64, device=nodes_box.device)
    _, ld_out = _rows(out, 10, "out")
    off = np.zeros(sbox.size + 1, dtype=np.int64)
    c.check(lib().box_place(c.handle, _ptr(nodes_box), ldb, boff.ctypes.data_as(_vp), boff.size - 1,
                            sbox.ctypes.data_as(_vp), sbox.size, _ptr(place), _ptr(out), ld_out,
                            off.ctypes.data_as(_vp), _stream(stream, c.device)))
    return out[:, :n_out], off


def cone_cut(samples, shell_off, nside_hz: int, cone_pix, r_lo, r_hi, x_obs=None, out=None, ctx=None, stream=None):
    """Samples inside each shell's HEALPix cone and radius range, compacted in input order:
    returns (kept [10, m] CUDA tensor view, shell offsets int64 CUDA tensor [nshell + 1]).
    Synchronises the stream to read m."""
    c = _ctx(ctx, samples)
    _dev_tensor(samples, torch.float64, "samples")
    n, ld = _rows(samples, 10, "samples")
    off = _host_i64(shell_off)
    nshell = off.size - 1
    if off[-1] != n:
        raise ValueError("shell_off must end at the sample count")
    for t, dt, name in ((cone_pix, torch.int64, "cone_pix"), (r_lo, torch.float64, "r_lo"),
                        (r_hi, torch.float64, "r_hi")):
        _dev_tensor(t, dt, name)
        if t.numel() != nshell or not t.is_contiguous():
            raise ValueError(f"{name} must be a contiguous CUDA tensor of nshell entries")
    if out is None:
        out = torch.empty((10, max(n, 1)), dtype=torch.float64, device=samples.device)
    _, ld_out = _rows(out, 10, "out")
    off_out = torch.empty(nshell + 1, dtype=torch.int64, device=samples.device)
    cnt = _i64(0)
    c.check(lib().cone_cut(c.handle, _ptr(samples), ld, off.ctypes.data_as(_vp), nshell, int(nside_hz),
                           _ptr(cone_pix), _ptr(r_lo), _ptr(r_hi), _xobs(x_obs), _ptr(out), ld_out, _ptr(off_out),
                           ctypes.byref(cnt), _stream(stream, c.device)))
    return out[:, :cnt.value], off_out


def isw_map_stacked(nside: int, nodes_box, box_off, shell_box, place, t_box, nside_hz: int, cone_pix, r_lo, r_hi,
                    x_obs=None, t_obs: float = 1.0, GU: float = 1.0, prec="f32c", out=None, ctx=None, stream=None):
    """Full-sky map of boxes stacked into HEALPix cones (Sec. III.B): box_place ->
    lightcone_intersect_shells (LINEAR) -> cone_cut -> isw_map.  Returns (theta, kept samples)."""
    import numpy as np

    placed, off = box_place(nodes_box, box_off, shell_box, place, ctx=ctx, stream=stream)
    mode = np.zeros(len(off) - 1, dtype=np.int32)
    samples = lightcone_intersect_shells(placed, off, t_box, mode, x_obs=x_obs, t_obs=t_obs, ctx=ctx, stream=stream)
    kept, _ = cone_cut(samples, off, nside_hz, cone_pix, r_lo, r_hi, x_obs=x_obs, ctx=ctx, stream=stream)
    theta = isw_map(nside, kept, x_obs=x_obs, GU=GU, prec=prec, out=out, ctx=ctx, stream=stream)
    return theta, kept


def isw_map_patch(frame, M: int, width: float, samples, approx: int = FULLSKY, x_obs=None, GU: float = 1.0,
                  prec="f32c", accumulate: bool = False, out=None, ctx=None, stream=None):
    """Theta on an M x M gnomonic patch (frame rows e1, e2, e3 with e3 the centre; gnomonic
    coordinate width ``width``), full sky or flat sky: float64 CUDA tensor [M, M] (row j = eta)."""
    import numpy as np

    c = _ctx(ctx, samples)
    fr = np.ascontiguousarray(np.asarray(frame, dtype=np.float64).reshape(9))
    _dev_tensor(samples, torch.float64, "samples")
    n, ld = _rows(samples, 10, "samples")
    if out is None:
        out = torch.empty((M, M), dtype=torch.float64, device=samples.device)
    _dev_tensor(out, torch.float64, "out")
    if out.numel() != M * M or not out.is_contiguous():
        raise ValueError("out must be a contiguous float64 tensor of M*M elements")
    c.check(lib().isw_map_patch(c.handle, fr.ctypes.data_as(_vp), int(M), float(width), _ptr(samples), n, ld,
                                _xobs(x_obs), float(GU), _precision(prec), int(approx), int(bool(accumulate)),
                                _ptr(out), _stream(stream, c.device)))
    return out


def isw_map_cl(nside: int, theta, lmax: int, with_alm: bool = False, ctx=None, stream=None):
    """Angular power spectrum of a full-sky RING map (float64 CUDA tensor [12 nside^2]): returns
    cl [lmax + 1], or (alm complex [lmax + 1 (m), lmax + 1 (l)], cl) with ``with_alm``."""
    c = _ctx(ctx, theta)
    _dev_tensor(theta, torch.float64, "theta")
    if theta.numel() != 12 * nside * nside or not theta.is_contiguous():
        raise ValueError("theta must be a contiguous full-sky RING map")
    cl = torch.empty(lmax + 1, dtype=torch.float64, device=theta.device)
    alm = torch.empty((2, lmax + 1, lmax + 1), dtype=torch.float64, device=theta.device) if with_alm else None
    c.check(lib().isw_map_cl(c.handle, int(nside), _ptr(theta), int(lmax), _ptr(alm), _ptr(cl),
                             _stream(stream, c.device)))
    if with_alm:
        return torch.complex(alm[0], alm[1]), cl
    return cl
