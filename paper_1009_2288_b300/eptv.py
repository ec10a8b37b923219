"""Python binding of libeptv.so (include/eptv.h): argument marshalling only.

Every function has the name of the C entry point it calls and takes torch CUDA tensors
(float32, contiguous) for device buffers; all arithmetic runs in the library's sm_103a
kernels.  There is no CPU fallback: if the library is missing or no GPU is present the
calls raise.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

from . import build as _build
from .inputs import EptvParams, FanGeometry

EPTV_OK = 0
ERRORS = {-1: "EPTV_ERR_ARG", -2: "EPTV_ERR_CUDA", -3: "EPTV_ERR_NONFINITE",
          -4: "EPTV_ERR_TIMEOUT", -5: "EPTV_ERR_NOMEM"}

EXPORTED = [
    "eptv_default_params", "eptv_create_geometry", "eptv_destroy_geometry", "eptv_project",
    "eptv_project_t", "eptv_transpose", "eptv_backproject", "eptv_cgls", "eptv_sigma",
    "eptv_tv_gradient", "eptv_tv_step", "eptv_reconstruct", "eptv_report_energy",
    "eptv_select_kth", "eptv_reconstruct_batched", "eptv_last_error", "eptv_version",
    "eptv_get_log", "eptv_select_kth_noalloc", "eptv_set_tuning", "eptv_set_tv_kernel", "eptv_debug_set_p2_wait", "eptv_autotune",
    "eptv_autotune_batched", "eptv_unet_conv3x3", "eptv_unet_conv3x3_wgrad",
    "eptv_unet_weights_to_bf16", "eptv_unet_set_conv_kernel", "eptv_unet_tc_status", "eptv_unet_maxpool2", "eptv_unet_maxpool2_bwd",
    "eptv_unet_upsample2", "eptv_unet_upsample2_bwd", "eptv_unet_relu_bwd", "eptv_unet_head",
    "eptv_unet_adam", "eptv_unet_pack_input", "eptv_set_operator", "eptv_autotune_operator", "eptv_matrix_info",
    "eptv_copy_matrix", "eptv_backproject_eq11", "eptv_quality_metrics",
    "eptv3_create_geometry", "eptv3_destroy_geometry", "eptv3_set_tuning", "eptv3_set_backprojector_stack", "eptv3_project",
    "eptv3_backproject", "eptv3_cgls", "eptv3_tv_step", "eptv3_reconstruct", "eptv3_report_energy",
]


class EptvError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class GeometryDesc(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("dx", ctypes.c_double),
                ("dy", ctypes.c_double), ("n_views", ctypes.c_int),
                ("angles", ctypes.POINTER(ctypes.c_double)), ("n_bins", ctypes.c_int),
                ("dbeta", ctypes.c_double), ("bin_offset", ctypes.c_double),
                ("sid", ctypes.c_double), ("sdd", ctypes.c_double), ("detector", ctypes.c_int)]


class Params(ctypes.Structure):
    _fields_ = [("n_outer", ctypes.c_int), ("cgls_iters", ctypes.c_int), ("n_gd", ctypes.c_int),
                ("lam", ctypes.c_double), ("mu", ctypes.c_double), ("sigma_q", ctypes.c_double),
                ("sigma_floor", ctypes.c_double), ("eps", ctypes.c_double),
                ("step_rule", ctypes.c_int), ("t_fixed", ctypes.c_double),
                ("armijo_c", ctypes.c_double), ("armijo_shrink", ctypes.c_double),
                ("armijo_grow", ctypes.c_double), ("max_trials", ctypes.c_int),
                ("t_max", ctypes.c_double), ("t_init", ctypes.c_double),
                ("weights_mode", ctypes.c_int), ("prior_iters", ctypes.c_int)]


class Stats(ctypes.Structure):
    _fields_ = [("sigma", ctypes.c_double), ("energy_first", ctypes.c_double),
                ("energy_last", ctypes.c_double), ("t_prev", ctypes.c_double),
                ("n_accepted", ctypes.c_int), ("n_fail", ctypes.c_int), ("status", ctypes.c_int)]


class GeometryDesc3(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("dx", ctypes.c_double), ("dy", ctypes.c_double), ("dz", ctypes.c_double),
                ("n_views", ctypes.c_int), ("angles", ctypes.POINTER(ctypes.c_double)),
                ("nu", ctypes.c_int), ("nv", ctypes.c_int), ("du", ctypes.c_double), ("dv", ctypes.c_double),
                ("u_off", ctypes.c_double), ("v_off", ctypes.c_double), ("sid", ctypes.c_double),
                ("sdd", ctypes.c_double)]


class Quality(ctypes.Structure):
    _fields_ = [("rel_error", ctypes.c_double), ("ecc", ctypes.c_double), ("edges", ctypes.c_longlong),
                ("edges_ref", ctypes.c_longlong), ("edges_both", ctypes.c_longlong),
                ("snr_db", ctypes.c_double)]


class Report(ctypes.Structure):
    _fields_ = [("n_outer", ctypes.c_int), ("sigma_last", ctypes.c_double),
                ("t_prev", ctypes.c_double), ("n_fail", ctypes.c_int), ("status", ctypes.c_int),
                ("n_launches", ctypes.c_longlong)]


_lib = None


def lib_path() -> str:
    return _build.LIB


def load():
    """Load libeptv.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_1009_2288_b300.build.build()")
    L = ctypes.CDLL(path)
    vp, c_int, c_long, dbl = ctypes.c_void_p, ctypes.c_int, ctypes.c_long, ctypes.c_double
    sig = {
        "eptv_default_params": (None, [ctypes.POINTER(Params)]),
        "eptv_create_geometry": (c_int, [ctypes.POINTER(GeometryDesc), ctypes.POINTER(vp)]),
        "eptv_destroy_geometry": (None, [vp]),
        "eptv_project": (c_int, [vp, vp, vp, vp]),
        "eptv_project_t": (c_int, [vp, vp, vp, vp, vp]),
        "eptv_transpose": (c_int, [vp, vp, vp, vp]),
        "eptv_backproject": (c_int, [vp, vp, vp, vp]),
        "eptv_cgls": (c_int, [vp, c_int, vp, vp, vp]),
        "eptv_sigma": (c_int, [vp, ctypes.POINTER(Params), vp, ctypes.POINTER(dbl), vp]),
        "eptv_tv_gradient": (c_int, [vp, ctypes.POINTER(Params), dbl, vp, vp, vp,
                                     ctypes.POINTER(dbl), vp]),
        "eptv_tv_step": (c_int, [vp, ctypes.POINTER(Params), vp, vp, ctypes.POINTER(dbl), vp,
                                 ctypes.POINTER(Stats), vp]),
        "eptv_reconstruct": (c_int, [vp, ctypes.POINTER(Params), vp, vp, vp,
                                     ctypes.POINTER(Report), vp]),
        "eptv_report_energy": (c_int, [vp, ctypes.POINTER(Params), dbl, vp, vp,
                                       ctypes.POINTER(dbl), vp]),
        "eptv_select_kth": (c_int, [vp, vp, c_long, c_long, vp, vp]),
        "eptv_select_kth_noalloc": (c_int, [vp, c_long, c_long, vp, vp]),
        "eptv_reconstruct_batched": (c_int, [c_int, ctypes.POINTER(vp), ctypes.POINTER(Params),
                                             ctypes.POINTER(vp), ctypes.POINTER(vp),
                                             ctypes.POINTER(Report), vp]),
        "eptv_get_log": (c_int, [vp, ctypes.POINTER(dbl), c_int, ctypes.POINTER(dbl), c_int,
                                 ctypes.POINTER(c_int), ctypes.POINTER(c_int)]),
        "eptv_set_tuning": (c_int, [vp, c_int, c_int]),
        "eptv_set_tv_kernel": (c_int, [vp, c_int]),
        "eptv_debug_set_p2_wait": (c_int, [vp, c_int, ctypes.c_longlong]),
        "eptv_autotune": (c_int, [vp, ctypes.POINTER(c_int), ctypes.POINTER(c_int)]),
        "eptv_autotune_batched": (c_int, [c_int, ctypes.POINTER(vp), ctypes.POINTER(c_int),
                                          ctypes.POINTER(c_int)]),
        "eptv_unet_conv3x3": (c_int, [vp, c_int, c_int, c_int, c_int, c_int, c_int, vp, vp, c_int,
                                      vp, c_int, c_int, c_int, vp]),
        "eptv_unet_conv3x3_wgrad": (c_int, [vp, c_int, c_int, c_int, c_int, c_int, c_int, vp, c_int,
                                            c_int, c_int, vp, vp, vp]),
        "eptv_unet_weights_to_bf16": (c_int, [vp, c_int, c_int, vp, vp, vp]),
        "eptv_unet_set_conv_kernel": (c_int, [c_int]),
        "eptv_unet_tc_status": (c_int, []),
        "eptv_unet_maxpool2": (c_int, [vp, c_int, c_int, c_int, c_int, c_int, c_int, vp, c_int, c_int, vp]),
        "eptv_unet_maxpool2_bwd": (c_int, [vp, c_int, c_int, c_int, c_int, c_int, c_int, vp, c_int,
                                           c_int, vp, c_int, c_int, c_int, vp]),
        "eptv_unet_upsample2": (c_int, [vp, c_int, c_int, c_int, c_int, c_int, c_int, vp, c_int, c_int, vp]),
        "eptv_unet_upsample2_bwd": (c_int, [vp, c_int, c_int, c_int, c_int, c_int, c_int, vp, c_int,
                                            c_int, vp]),
        "eptv_unet_relu_bwd": (c_int, [vp, c_int, c_int, vp, c_int, c_int, vp, c_int, c_int,
                                       ctypes.c_longlong, c_int, vp]),
        "eptv_unet_head": (c_int, [vp, c_int, c_int, ctypes.c_longlong, vp, vp, vp, vp, vp, ctypes.c_float,
                                   vp, vp, vp, c_int, c_int, vp, vp, vp, vp]),
        "eptv_unet_pack_input": (c_int, [vp, ctypes.c_float, vp, ctypes.c_float, ctypes.c_longlong, vp, vp]),
        "eptv_set_operator": (c_int, [vp, c_int, ctypes.POINTER(ctypes.c_longlong)]),
        "eptv_autotune_operator": (c_int, [vp, ctypes.c_longlong, ctypes.POINTER(c_int)]),
        "eptv_backproject_eq11": (c_int, [vp, vp, vp, vp]),
        "eptv3_create_geometry": (c_int, [ctypes.POINTER(GeometryDesc3), ctypes.POINTER(vp)]),
        "eptv3_destroy_geometry": (None, [vp]),
        "eptv3_set_tuning": (c_int, [vp, c_int]),
        "eptv3_set_backprojector_stack": (c_int, [vp, c_int]),
        "eptv3_project": (c_int, [vp, vp, vp, vp]),
        "eptv3_backproject": (c_int, [vp, vp, vp, vp]),
        "eptv3_cgls": (c_int, [vp, c_int, vp, vp, vp]),
        "eptv3_tv_step": (c_int, [vp, ctypes.POINTER(Params), vp, vp, ctypes.POINTER(dbl), ctypes.POINTER(Stats), vp]),
        "eptv3_reconstruct": (c_int, [vp, ctypes.POINTER(Params), vp, vp, ctypes.POINTER(Report), vp]),
        "eptv3_report_energy": (c_int, [vp, ctypes.POINTER(Params), dbl, vp, vp, ctypes.POINTER(dbl), vp]),
        "eptv_quality_metrics": (c_int, [vp, vp, vp, ctypes.POINTER(c_int), ctypes.c_double, vp, vp,
                                         ctypes.POINTER(Quality), vp]),
        "eptv_matrix_info": (c_int, [vp, c_int, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong),
                                     ctypes.POINTER(ctypes.c_longlong)]),
        "eptv_copy_matrix": (c_int, [vp, c_int, vp, vp, vp, vp]),
        "eptv_unet_adam": (c_int, [vp, vp, vp, vp, ctypes.c_longlong, ctypes.c_float, ctypes.c_float,
                                   ctypes.c_float, ctypes.c_float, c_int, vp]),
        "eptv_last_error": (ctypes.c_char_p, []),
        "eptv_version": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def _check(rc: int):
    if rc != EPTV_OK and rc < 0:
        raise EptvError(rc, load().eptv_last_error().decode())
    return rc


def _stream(stream) -> Optional[int]:
    import torch
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    return getattr(stream, "cuda_stream", stream)


def _ptr(t, numel: Optional[int] = None, name: str = "tensor"):
    import torch
    if t is None:
        return None
    if not (t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
        raise ValueError(f"{name} must be a contiguous float32 CUDA tensor")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{name} has {t.numel()} elements, expected {numel}")
    return t.data_ptr()


def params(p: Optional[EptvParams] = None) -> Params:
    """ctypes copy of a parameter record (library defaults where p is None)."""
    out = Params()
    load().eptv_default_params(ctypes.byref(out))
    if p is None:
        return out
    for f, _ in Params._fields_:
        setattr(out, f, getattr(p, f))
    return out


class Geometry:
    """Owner of one eptv_geometry handle (ray tables + workspace on the current device)."""

    def __init__(self, g: FanGeometry):
        L = load()
        self.g = g
        self._angles = None
        d = GeometryDesc(g.nx, g.ny, g.dx, g.dy, g.n_views, None, g.n_bins, g.dbeta,
                         g.bin_offset, g.sid, g.sdd, g.detector)
        if g.angles is not None:
            arr = (ctypes.c_double * g.n_views)(*[float(a) for a in g.angles])
            self._angles = arr
            d.angles = ctypes.cast(arr, ctypes.POINTER(ctypes.c_double))
        h = ctypes.c_void_p()
        _check(L.eptv_create_geometry(ctypes.byref(d), ctypes.byref(h)))
        self.handle = h

    def close(self):
        if getattr(self, "handle", None):
            load().eptv_destroy_geometry(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def n_pix(self):
        return self.g.nx * self.g.ny

    @property
    def n_rays(self):
        return self.g.n_views * self.g.n_bins


def eptv_project(geom: Geometry, f, y, stream=None):
    _check(load().eptv_project(geom.handle, _ptr(f, geom.n_pix, "f"), _ptr(y, geom.n_rays, "y"),
                               _stream(stream)))
    return y


def eptv_project_t(geom: Geometry, f, fT, y, stream=None):
    _check(load().eptv_project_t(geom.handle, _ptr(f, geom.n_pix, "f"),
                                 _ptr(fT, geom.n_pix, "fT"), _ptr(y, geom.n_rays, "y"),
                                 _stream(stream)))
    return y


def eptv_transpose(geom: Geometry, f, fT, stream=None):
    _check(load().eptv_transpose(geom.handle, _ptr(f, geom.n_pix, "f"),
                                 _ptr(fT, geom.n_pix, "fT"), _stream(stream)))
    return fT


def eptv_backproject(geom: Geometry, y, f, stream=None):
    _check(load().eptv_backproject(geom.handle, _ptr(y, geom.n_rays, "y"),
                                   _ptr(f, geom.n_pix, "f"), _stream(stream)))
    return f


def eptv_cgls(geom: Geometry, M: int, y, u, stream=None):
    _check(load().eptv_cgls(geom.handle, int(M), _ptr(y, geom.n_rays, "y"),
                            _ptr(u, geom.n_pix, "u"), _stream(stream)))
    return u


def eptv_sigma(geom: Geometry, p: EptvParams, v, stream=None) -> float:
    out = ctypes.c_double()
    pp = params(p)
    _check(load().eptv_sigma(geom.handle, ctypes.byref(pp), _ptr(v, geom.n_pix, "v"),
                             ctypes.byref(out), _stream(stream)))
    return out.value


def eptv_tv_gradient(geom: Geometry, p: EptvParams, sigma: float, f, v, g, stream=None):
    """Returns the (P2) energy at f (the gradient is written to g)."""
    out = ctypes.c_double()
    pp = params(p)
    _check(load().eptv_tv_gradient(geom.handle, ctypes.byref(pp), float(sigma),
                                   _ptr(f, geom.n_pix, "f"), _ptr(v, geom.n_pix, "v"),
                                   _ptr(g, geom.n_pix, "g"), ctypes.byref(out), _stream(stream)))
    return out.value


def eptv_tv_step(geom: Geometry, p: EptvParams, v, f, t_prev: Optional[float] = None,
                 weights=None, stream=None):
    """One (P2) solve + clamp; returns (Stats, t_prev after the solve)."""
    pp = params(p)
    st = Stats()
    tp = ctypes.c_double(t_prev if t_prev is not None else p.t_init_eff)
    nw = 2 * (geom.g.nx + 1) * (geom.g.ny + 1)
    _check(load().eptv_tv_step(geom.handle, ctypes.byref(pp), _ptr(v, geom.n_pix, "v"),
                               _ptr(f, geom.n_pix, "f"), ctypes.byref(tp),
                               _ptr(weights, nw, "weights"), ctypes.byref(st), _stream(stream)))
    return st, tp.value


def eptv_reconstruct(geom: Geometry, p: EptvParams, y, f, wprior=None, report: bool = True,
                     stream=None):
    pp = params(p)
    rep = Report()
    _check(load().eptv_reconstruct(geom.handle, ctypes.byref(pp), _ptr(y, geom.n_rays, "y"),
                                   _ptr(f, geom.n_pix, "f"), _ptr(wprior, geom.n_pix, "wprior"),
                                   ctypes.byref(rep) if report else None, _stream(stream)))
    return rep if report else None


def eptv_report_energy(geom: Geometry, p: EptvParams, sigma_ref: float, f, y, stream=None):
    out = ctypes.c_double()
    pp = params(p)
    _check(load().eptv_report_energy(geom.handle, ctypes.byref(pp), float(sigma_ref),
                                     _ptr(f, geom.n_pix, "f"), _ptr(y, geom.n_rays, "y"),
                                     ctypes.byref(out), _stream(stream)))
    return out.value


def eptv_select_kth(geom: Geometry, vals, k: int, out, stream=None):
    _check(load().eptv_select_kth(geom.handle, _ptr(vals, None, "vals"), vals.numel(), int(k),
                                  _ptr(out, 1, "out"), _stream(stream)))
    return out


def eptv_select_kth_noalloc(vals, k: int, out, stream=None):
    """k-th smallest of vals without a geometry handle and without any device
    allocation (working memory compiled into the library); see eptv.h.  Runs on the
    device that holds vals; out must be on the same device."""
    import torch
    if out.device != vals.device:
        raise EptvError(-1, "out must be on the device of vals")
    with torch.cuda.device(vals.device):
        _check(load().eptv_select_kth_noalloc(_ptr(vals, None, "vals"), vals.numel(), int(k),
                                              _ptr(out, 1, "out"), _stream(stream)))
    return out


def eptv_reconstruct_batched(geoms: Sequence[Geometry], p: EptvParams, ys, fs,
                             report: bool = True, stream=None):
    n = len(geoms)
    H = (ctypes.c_void_p * n)(*[g.handle.value for g in geoms])
    Y = (ctypes.c_void_p * n)(*[_ptr(y, g.n_rays, "y") for g, y in zip(geoms, ys)])
    F = (ctypes.c_void_p * n)(*[_ptr(f, g.n_pix, "f") for g, f in zip(geoms, fs)])
    reps = (Report * n)() if report else None
    pp = params(p)
    _check(load().eptv_reconstruct_batched(n, H, ctypes.byref(pp), Y, F, reps, _stream(stream)))
    return list(reps) if report else None


def eptv_get_log(geom: Geometry):
    """(steps [n_outer][n_gd], sigmas [n_outer]) of the last eptv_reconstruct on geom."""
    import numpy as np
    no, ng = ctypes.c_int(), ctypes.c_int()
    L = load()
    _check(L.eptv_get_log(geom.handle, None, 0, None, 0, ctypes.byref(no), ctypes.byref(ng)))
    steps = np.zeros(no.value * ng.value)
    sig = np.zeros(no.value)
    _check(L.eptv_get_log(geom.handle, steps.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                          steps.size, sig.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                          sig.size, None, None))
    return steps.reshape(no.value, ng.value), sig


OPERATOR_ON_THE_FLY, OPERATOR_STORED, OPERATOR_EQ11, OPERATOR_STORED_PT = 0, 1, 2, 3


def eptv_backproject_eq11(geom: Geometry, y, f, stream=None):
    """The paper's interpolating back projector, Eq. (11) (see eptv.h)."""
    _check(load().eptv_backproject_eq11(geom.handle, _ptr(y, geom.n_rays, "y"), _ptr(f, geom.n_pix, "f"),
                                        _stream(stream)))
    return f


def eptv_set_operator(geom: Geometry, mode: int) -> int:
    """Select the on-the-fly kernels or the stored CSR matrices for P and P^T of geom
    (building the matrices on the first switch to stored); returns the stored entries of P."""
    nnz = ctypes.c_longlong(0)
    _check(load().eptv_set_operator(geom.handle, int(mode), ctypes.byref(nnz)))
    return nnz.value


def eptv_autotune_operator(geom: Geometry, max_matrix_bytes: int) -> int:
    """P^T of geom from the kernel or from the stored matrix, whichever is faster (within
    the memory bound); returns the operator mode kept."""
    mode = ctypes.c_int(0)
    _check(load().eptv_autotune_operator(geom.handle, int(max_matrix_bytes), ctypes.byref(mode)))
    return mode.value


def eptv_matrix_info(geom: Geometry, which: int):
    """(rows, CSR entries incl. padding, SELL-32 entries) of the built P (which = 0) or P^T (1)."""
    rows, nnz, sell = ctypes.c_longlong(), ctypes.c_longlong(), ctypes.c_longlong()
    _check(load().eptv_matrix_info(geom.handle, int(which), ctypes.byref(rows), ctypes.byref(nnz),
                                   ctypes.byref(sell)))
    return rows.value, nnz.value, sell.value


def eptv_matrix(geom: Geometry, which: int):
    """(ptr, col, val) device tensors: a copy of the stored P (which = 0) or P^T (1)."""
    import torch
    rows, nnz, _ = eptv_matrix_info(geom, which)
    rows, nnz = ctypes.c_longlong(rows), ctypes.c_longlong(nnz)
    ptr = torch.empty(rows.value + 1, dtype=torch.int32, device="cuda")
    col = torch.empty(max(nnz.value, 1), dtype=torch.int32, device="cuda")
    val = torch.empty(max(nnz.value, 1), dtype=torch.float32, device="cuda")
    _check(load().eptv_copy_matrix(geom.handle, int(which), ptr.data_ptr(), col.data_ptr(), val.data_ptr(),
                                   _stream(None)))
    return ptr, col[:nnz.value], val[:nnz.value]


def eptv_quality_metrics(geom: Geometry, f, ref=None, roi=None, edge_scale: float = 2.0, edges=None,
                         edges_ref=None, stream=None) -> Quality:
    """Relative error (Eq. 12), edge correlation (Eq. 13) and ROI SNR (Eq. 14) of f (see
    eptv.h); roi = (x0, y0, w, h); edges / edges_ref: optional uint8 CUDA tensors [ny*nx]."""
    q = Quality()
    r = (ctypes.c_int * 4)(*roi) if roi is not None else None
    for t in (edges, edges_ref):
        if t is not None and (t.dtype.itemsize != 1 or t.numel() != geom.n_pix or not t.is_cuda):
            raise ValueError("edge maps must be uint8 CUDA tensors of n_pix elements")
    _check(load().eptv_quality_metrics(geom.handle, _ptr(f, geom.n_pix, "f"), _ptr(ref, geom.n_pix, "ref"),
                                       r, float(edge_scale), edges.data_ptr() if edges is not None else None,
                                       edges_ref.data_ptr() if edges_ref is not None else None,
                                       ctypes.byref(q), _stream(stream)))
    return q


def eptv_set_tuning(geom: Geometry, k1_seg: int, k2_vg: int):
    _check(load().eptv_set_tuning(geom.handle, int(k1_seg), int(k2_vg)))


TV_AUTO, TV_PER_ITERATION = 0, 1


def eptv_set_tv_kernel(geom: Geometry, mode: int):
    """(P2) kernel of geom's solves: TV_AUTO (one persistent launch per (P2) solve when it
    fits) or TV_PER_ITERATION (one launch per GD iteration); results are bit-identical."""
    _check(load().eptv_set_tv_kernel(geom.handle, int(mode)))


def eptv_debug_set_p2_wait(geom: Geometry, extra_blocks: int, wait_cycles: int):
    """Test hook: the persistent (P2) kernel's barrier waits for extra_blocks phantom blocks
    and gives up after wait_cycles SM cycles (EPTV_ERR_TIMEOUT)."""
    _check(load().eptv_debug_set_p2_wait(geom.handle, int(extra_blocks), int(wait_cycles)))


def eptv_autotune(geom: Geometry):
    """Times the projector / back-projector launch shapes on geom; returns (k1_seg, k2_vg)."""
    a, b = ctypes.c_int(), ctypes.c_int()
    _check(load().eptv_autotune(geom.handle, ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def eptv_autotune_batched(geoms: Sequence[Geometry]):
    n = len(geoms)
    H = (ctypes.c_void_p * n)(*[g.handle.value for g in geoms])
    a, b = ctypes.c_int(), ctypes.c_int()
    _check(load().eptv_autotune_batched(n, H, ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


# ------------------------------------------------------------------ U-Net layer kernels
# Activations are torch bfloat16 tensors [n, H, W, C] (C = channel stride); a call reads or
# writes channels [off, off + c) of such a tensor.

def _p(t):
    return None if t is None else t.data_ptr()


def eptv_unet_conv3x3(x, x_off, cin, wt, bias, cout, y, y_off, relu, stream=None):
    n, h, w, xs = x.shape
    _check(load().eptv_unet_conv3x3(_p(x), n, h, w, cin, xs, x_off, _p(wt), _p(bias), cout, _p(y),
                                    y.shape[3], y_off, int(relu), _stream(stream)))


def eptv_unet_conv3x3_wgrad(x, x_off, cin, dy, dy_off, cout, dw, db, stream=None):
    n, h, w, xs = x.shape
    _check(load().eptv_unet_conv3x3_wgrad(_p(x), n, h, w, cin, xs, x_off, _p(dy), dy.shape[3], dy_off,
                                          cout, _p(dw), _p(db), _stream(stream)))


def eptv_unet_weights_to_bf16(w, cout, cin, wf, wb, stream=None):
    _check(load().eptv_unet_weights_to_bf16(_p(w), cout, cin, _p(wf), _p(wb), _stream(stream)))


def eptv_unet_maxpool2(x, x_off, c, y, y_off, stream=None):
    n, h, w, xs = x.shape
    _check(load().eptv_unet_maxpool2(_p(x), n, h, w, xs, x_off, c, _p(y), y.shape[3], y_off, _stream(stream)))


def eptv_unet_maxpool2_bwd(x, x_off, c, dy, dy_off, dx, dx_off, accumulate, stream=None):
    n, h, w, xs = x.shape
    _check(load().eptv_unet_maxpool2_bwd(_p(x), n, h, w, xs, x_off, c, _p(dy), dy.shape[3], dy_off,
                                         _p(dx), dx.shape[3], dx_off, int(accumulate), _stream(stream)))


def eptv_unet_upsample2(x, x_off, c, y, y_off, stream=None):
    n, h, w, xs = x.shape
    _check(load().eptv_unet_upsample2(_p(x), n, h, w, xs, x_off, c, _p(y), y.shape[3], y_off, _stream(stream)))


def eptv_unet_upsample2_bwd(dy, dy_off, c, dx, dx_off, stream=None):
    n, h, w, dys = dy.shape
    _check(load().eptv_unet_upsample2_bwd(_p(dy), n, h, w, dys, dy_off, c, _p(dx), dx.shape[3], dx_off,
                                          _stream(stream)))


def eptv_unet_relu_bwd(a, a_off, dy, dy_off, dz, dz_off, c, stream=None):
    n, h, w, as_ = a.shape
    _check(load().eptv_unet_relu_bwd(_p(a), as_, a_off, _p(dy), dy.shape[3], dy_off, _p(dz), dz.shape[3],
                                     dz_off, n * h * w, c, _stream(stream)))


def eptv_unet_head(x, hw, hb, f0=None, w=None, base=None, f_scale=1.0, ft=None, wt=None, dx=None,
                   dhw=None, dhb=None, loss=None, stream=None):
    n, h, ww, xs = x.shape
    _check(load().eptv_unet_head(_p(x), xs, 0, n * h * ww, _p(hw), _p(hb), _p(f0), _p(w), _p(base),
                                 float(f_scale), _p(ft), _p(wt), _p(dx),
                                 dx.shape[3] if dx is not None else 0, 0, _p(dhw), _p(dhb), _p(loss),
                                 _stream(stream)))


def eptv_unet_pack_input(a, scale_a, b, scale_b, x, stream=None):
    """a, b: FP32 [npix] (b may be None); x: BF16 [..., 16] with npix rows."""
    npix = a.numel()
    if x.numel() != 16 * npix or (b is not None and b.numel() != npix):
        raise ValueError("pack_input: size mismatch")
    _check(load().eptv_unet_pack_input(_p(a), float(scale_a), _p(b), float(scale_b), npix, _p(x),
                                       _stream(stream)))


def eptv_unet_adam(p, g, m, v, lr, beta1, beta2, eps, step, stream=None):
    _check(load().eptv_unet_adam(_p(p), _p(g), _p(m), _p(v), p.numel(), lr, beta1, beta2, eps, int(step),
                                 _stream(stream)))


def version() -> str:
    return load().eptv_version().decode()


# ------------------------------------------------------------------ 3-D cone beam

class Geometry3:
    """Owner of one eptv3_geometry handle (cone-beam ray tables + workspace)."""

    def __init__(self, g):
        L = load()
        self.g = g
        self._angles = None
        d = GeometryDesc3(g.nx, g.ny, g.nz, g.dx, g.dy, g.dz, g.n_views, None, g.nu, g.nv, g.du, g.dv,
                          g.u_off, g.v_off, g.sid, g.sdd)
        if g.angles is not None:
            arr = (ctypes.c_double * g.n_views)(*[float(a) for a in g.angles])
            self._angles = arr
            d.angles = ctypes.cast(arr, ctypes.POINTER(ctypes.c_double))
        h = ctypes.c_void_p()
        _check(L.eptv3_create_geometry(ctypes.byref(d), ctypes.byref(h)))
        self.handle = h

    def close(self):
        if getattr(self, "handle", None):
            load().eptv3_destroy_geometry(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def n_vox(self):
        return self.g.n_vox

    @property
    def n_rays(self):
        return self.g.n_rays


def eptv3_set_tuning(geom: Geometry3, seg: int):
    _check(load().eptv3_set_tuning(geom.handle, int(seg)))


def eptv3_set_backprojector_stack(geom: Geometry3, zp: int):
    _check(load().eptv3_set_backprojector_stack(geom.handle, int(zp)))


def eptv3_project(geom: Geometry3, f, y, stream=None):
    _check(load().eptv3_project(geom.handle, _ptr(f, geom.n_vox, "f"), _ptr(y, geom.n_rays, "y"), _stream(stream)))
    return y


def eptv3_backproject(geom: Geometry3, y, f, stream=None):
    _check(load().eptv3_backproject(geom.handle, _ptr(y, geom.n_rays, "y"), _ptr(f, geom.n_vox, "f"),
                                    _stream(stream)))
    return f


def eptv3_cgls(geom: Geometry3, M: int, y, u, stream=None):
    _check(load().eptv3_cgls(geom.handle, int(M), _ptr(y, geom.n_rays, "y"), _ptr(u, geom.n_vox, "u"),
                             _stream(stream)))
    return u


def eptv3_tv_step(geom: Geometry3, p: EptvParams, v, f, t_prev: Optional[float] = None, stream=None):
    pp = params(p)
    st = Stats()
    tp = ctypes.c_double(t_prev if t_prev is not None else 0.0)
    _check(load().eptv3_tv_step(geom.handle, ctypes.byref(pp), _ptr(v, geom.n_vox, "v"), _ptr(f, geom.n_vox, "f"),
                                ctypes.byref(tp), ctypes.byref(st), _stream(stream)))
    return st, tp.value


def eptv3_reconstruct(geom: Geometry3, p: EptvParams, y, f, report: bool = True, stream=None):
    pp = params(p)
    rep = Report()
    _check(load().eptv3_reconstruct(geom.handle, ctypes.byref(pp), _ptr(y, geom.n_rays, "y"),
                                    _ptr(f, geom.n_vox, "f"), ctypes.byref(rep) if report else None,
                                    _stream(stream)))
    return rep if report else None


def eptv3_report_energy(geom: Geometry3, p: EptvParams, sigma_ref: float, f, y, stream=None) -> float:
    out = ctypes.c_double()
    pp = params(p)
    _check(load().eptv3_report_energy(geom.handle, ctypes.byref(pp), float(sigma_ref), _ptr(f, geom.n_vox, "f"),
                                      _ptr(y, geom.n_rays, "y"), ctypes.byref(out), _stream(stream)))
    return out.value


CONV_TENSOR_MEMORY, CONV_MMA_SYNC, CONV_TENSOR_MEMORY_ALL = 0, 1, 2


def eptv_unet_set_conv_kernel(mode: int):
    """Kernel of the 3x3 convs: CONV_TENSOR_MEMORY (tcgen05 for the shapes where it is not
    slower), CONV_MMA_SYNC, or CONV_TENSOR_MEMORY_ALL (tcgen05 wherever it tiles the
    image); see eptv.h."""
    _check(load().eptv_unet_set_conv_kernel(int(mode)))


def eptv_unet_tc_status():
    """Raises EptvError(EPTV_ERR_TIMEOUT) if a bounded wait of the tensor-memory conv ran out."""
    _check(load().eptv_unet_tc_status())
