"""Python binding of libtagi (ctypes).

Argument marshalling only: every function here passes device pointers, sizes
and the current CUDA stream to the C ABI declared in ``include/tagi.h`` and
raises ``TagiError`` on a non-zero status.  No arithmetic of the method runs
in Python.  PyTorch provides the device memory and the stream.

The shared library must have been built in-tree (``__graft_entry__.build()``
or ``python paper_2003_01833_gb300/build.py``); importing a function whose
library is missing raises immediately -- there is no fallback.
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtagi.so")

TAGI_OK = 0
TAGI_ERR_INVALID_ARG = 1
TAGI_ERR_CUDA = 2
TAGI_ERR_OOM = 3
TAGI_ERR_TIMEOUT = 4
TAGI_ERR_STATE = 5
TAGI_FP64 = 0
TAGI_FP32C = 1


class TagiError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"tagi status {status}: {msg}")
        self.status = status


class tagi_params(ctypes.Structure):
    _fields_ = [("theta", ctypes.c_double), ("degree", ctypes.c_int), ("leaf_size", ctypes.c_int),
                ("batch_size", ctypes.c_int), ("prec", ctypes.c_int), ("ss", ctypes.c_int),
                ("alpha", ctypes.c_double), ("segment", ctypes.c_int)]


class tagi_tree_stats(ctypes.Structure):
    _fields_ = [("n_points", ctypes.c_int64), ("n_clusters", ctypes.c_int32), ("n_leaves", ctypes.c_int32),
                ("depth", ctypes.c_int32), ("n_far_clusters", ctypes.c_int32),
                ("n_list_entries", ctypes.c_int64), ("n_items", ctypes.c_int64),
                ("near_pairs", ctypes.c_int64), ("far_pairs", ctypes.c_int64), ("degree", ctypes.c_int32),
                ("n_proxies", ctypes.c_int32), ("near_pairs_nogauss", ctypes.c_int64),
                ("far_pairs_nogauss", ctypes.c_int64), ("ant_points", ctypes.c_int64)]


class tagi_gi_params(ctypes.Structure):
    _fields_ = [("tol_gi", ctypes.c_double), ("max_iter", ctypes.c_int), ("beta", ctypes.c_double),
                ("history", ctypes.c_int), ("mix_tol", ctypes.c_double), ("store_output", ctypes.c_int)]


class tagi_gi_stats(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_int), ("n_converged", ctypes.c_int), ("field_steps", ctypes.c_int64)]


class tagi_scf_params(ctypes.Structure):
    _fields_ = [("n_electrons", ctypes.c_double), ("kT", ctypes.c_double), ("e_zz", ctypes.c_double),
                ("beta", ctypes.c_double), ("history", ctypes.c_int), ("tol_gi_first", ctypes.c_double),
                ("tol_gi_final", ctypes.c_double), ("tol_gi_ramp", ctypes.c_int), ("gi_max_iter", ctypes.c_int),
                ("gi_beta", ctypes.c_double), ("gi_history", ctypes.c_int), ("gi_mix_tol_first", ctypes.c_double),
                ("gi_store_output", ctypes.c_int)]


class tagi_scf_report(ctypes.Structure):
    _fields_ = [("step", ctypes.c_int), ("tol_gi", ctypes.c_double), ("mu", ctypes.c_double),
                ("residual", ctypes.c_double), ("e_band", ctypes.c_double), ("e_hartree", ctypes.c_double),
                ("e_xc", ctypes.c_double), ("e_vxc", ctypes.c_double), ("e_zz", ctypes.c_double),
                ("e_total", ctypes.c_double), ("gi", tagi_gi_stats)]


_lib = None
_vp = ctypes.c_void_p
_D = ctypes.POINTER(ctypes.c_double)
_I32 = ctypes.POINTER(ctypes.c_int32)
_I64 = ctypes.POINTER(ctypes.c_int64)


class tagi_adam_params(ctypes.Structure):
    _fields_ = [("lr", ctypes.c_double), ("beta1", ctypes.c_double), ("beta2", ctypes.c_double),
                ("eps", ctypes.c_double)]


def lib():
    """Load libtagi.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        L.tagi_tree_build.argtypes = [_vp, _vp, ctypes.c_int64, ctypes.POINTER(tagi_params), _vp,
                                      ctypes.POINTER(_vp)]
        L.tagi_tree_destroy.argtypes = [_vp]
        L.tagi_tree_info.argtypes = [_vp, ctypes.POINTER(tagi_tree_stats)]
        L.tagi_tree_export.argtypes = [_vp, _I32, _I32, _I32, _D, _D, _I32, _I32, _I32]
        L.tagi_tree_lists.argtypes = [_vp, ctypes.c_int64, _I32, _I32, _I32, _I64]
        L.tagi_anterpolate.argtypes = [_vp, _vp, ctypes.c_int, _vp, _vp]
        L.tagi_yukawa_conv.argtypes = [_vp, _vp, _D, ctypes.c_int, _vp, _vp]
        L.tagi_coulomb_conv.argtypes = [_vp, _vp, _vp, _vp]
        L.tagi_fields_conv.argtypes = [_vp, _vp, _D, ctypes.c_int, _vp, _vp, _vp, _vp]
        L.tagi_green_step.argtypes = [_vp, _vp, ctypes.c_double, _vp, _D, ctypes.c_int, _vp, _vp, _D, _D, _vp]
        L.tagi_kernel_launches.restype = ctypes.c_int64
        L.tagi_green_iterate.argtypes = [_vp, _vp, ctypes.c_double, _vp, _D, ctypes.c_int,
                                         ctypes.POINTER(tagi_gi_params), _D, _I32, ctypes.POINTER(tagi_gi_stats),
                                         _vp]
        L.tagi_scf_create.argtypes = [_vp, ctypes.POINTER(tagi_scf_params), ctypes.POINTER(_vp)]
        L.tagi_scf_step.argtypes = [_vp, _vp, ctypes.c_double, _vp, _vp, _D, ctypes.c_int, _D, _vp,
                                    ctypes.POINTER(tagi_scf_report), _vp]
        L.tagi_scf_destroy.argtypes = [_vp]
        L.tagi_profile_enable.argtypes = [ctypes.c_int]
        L.tagi_fp32_bias.argtypes = [_D, _D, _vp]
        L.tagi_green_graph_create.argtypes = [_vp, _vp, ctypes.c_double, _vp, _vp, ctypes.c_int, _vp, _vp, _vp, _vp,
                                              _vp, ctypes.POINTER(_vp)]
        L.tagi_green_graph_launch.argtypes = [_vp, _vp]
        L.tagi_green_graph_check.argtypes = [_vp, _vp]
        L.tagi_green_graph_destroy.argtypes = [_vp]
        L.tagi_trim_cache.argtypes = []
        for name in ("tagi_green_graph_create", "tagi_green_graph_launch", "tagi_green_graph_check",
                     "tagi_green_graph_destroy", "tagi_trim_cache"):
            getattr(L, name).restype = ctypes.c_int
        L.tagi_yukawa_direct_noalloc.argtypes = [_vp, _vp, _vp, _D, ctypes.c_int, ctypes.c_int64, _vp, _vp]
        L.tagi_yukawa_direct_noalloc.restype = ctypes.c_int
        L.tagi_unit_rates.argtypes = [_D, ctypes.c_int, _vp]
        L.tagi_unit_rates.restype = ctypes.c_int
        L.tagi_tree_batches.argtypes = [_vp, _I32, _I64]
        L.tagi_fields_conv_batches.argtypes = [_vp, _vp, _D, ctypes.c_int, _vp, _vp, _vp, _I32, ctypes.c_int, _vp]
        L.tagi_green_conv_batches.argtypes = [_vp, _vp, ctypes.c_double, _vp, _D, ctypes.c_int, _vp, _vp, _vp,
                                              _I32, ctypes.c_int, _vp]
        L.tagi_green_reduce.argtypes = [_vp, _vp, ctypes.c_double, _vp, _D, ctypes.c_int, _vp, _vp, _vp, _D, _D,
                                        _vp]
        for name in ("tagi_tree_batches", "tagi_fields_conv_batches", "tagi_green_conv_batches",
                     "tagi_green_reduce"):
            getattr(L, name).restype = ctypes.c_int
        L.tagi_mlp_create.argtypes = [ctypes.c_int, ctypes.c_int, _D, ctypes.c_int64, ctypes.POINTER(_vp)]
        L.tagi_mlp_get_params.argtypes = [_vp, _D, ctypes.c_int64, _vp]
        L.tagi_mlp_features.argtypes = [_vp, ctypes.c_int64, _D, ctypes.c_int, _vp, _vp]
        L.tagi_mlp_features_ordered.argtypes = [_vp, ctypes.c_int64, _D, _vp, _vp]
        L.tagi_mlp_features_ordered.restype = ctypes.c_int
        L.tagi_mlp_features_scaled.argtypes = [_vp, ctypes.c_int64, _D, _D, ctypes.c_int, ctypes.c_int, _vp, _vp]
        L.tagi_mlp_features_scaled.restype = ctypes.c_int
        L.tagi_mlp_forward.argtypes = [_vp, _vp, ctypes.c_int64, _vp, _vp]
        L.tagi_mlp_gradient.argtypes = [_vp, _vp, _vp, _vp, ctypes.c_int64, _D, _D, _vp]
        L.tagi_mlp_train_step.argtypes = [_vp, _vp, _vp, _vp, ctypes.c_int64, ctypes.POINTER(tagi_adam_params),
                                          _D, _vp]
        L.tagi_mlp_warm_start.argtypes = [_vp, _vp, _vp, _vp, ctypes.c_int64, _vp, _vp]
        L.tagi_mlp_destroy.argtypes = [_vp]
        for name in ("tagi_mlp_create", "tagi_mlp_get_params", "tagi_mlp_features", "tagi_mlp_forward",
                     "tagi_mlp_gradient", "tagi_mlp_train_step", "tagi_mlp_warm_start", "tagi_mlp_destroy"):
            getattr(L, name).restype = ctypes.c_int
        L.tagi_profile_read.argtypes = [ctypes.c_int, _D, _I64]
        L.tagi_last_error.restype = ctypes.c_char_p
        L.tagi_version.restype = ctypes.c_char_p
        for name in ("tagi_tree_build", "tagi_tree_destroy", "tagi_tree_info", "tagi_tree_export",
                     "tagi_tree_lists", "tagi_anterpolate", "tagi_yukawa_conv", "tagi_coulomb_conv",
                     "tagi_green_step", "tagi_profile_enable", "tagi_profile_read", "tagi_fp32_bias"):
            getattr(L, name).restype = ctypes.c_int
        _lib = L
    return _lib


def _check(status):
    if status != TAGI_OK:
        raise TagiError(status, lib().tagi_last_error().decode())


def _stream(stream):
    if stream is not None:
        return ctypes.c_void_p(stream)
    import torch

    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _dptr(t, name, numel=None):
    """Device pointer of a contiguous float64 CUDA tensor (None -> NULL)."""
    if t is None:
        return None
    import torch

    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise TypeError(f"{name} must be a contiguous float64 CUDA tensor")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{name} must have {numel} elements, has {t.numel()}")
    return ctypes.c_void_p(t.data_ptr())


def _hd(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(_D)


def make_params(theta=0.7, degree=8, leaf_size=2000, prec=TAGI_FP32C, ss=True, alpha=1.0, segment=0):
    return tagi_params(float(theta), int(degree), int(leaf_size), int(leaf_size), int(prec), int(bool(ss)),
                       float(alpha), int(segment))


# ----------------------------------------------------------------- C ABI names
def tagi_tree_build(xyz, w, params, stream=None):
    """xyz: (3, n) float64 CUDA tensor, w: (n,) float64 CUDA tensor."""
    n = w.numel()
    h = ctypes.c_void_p()
    _check(lib().tagi_tree_build(_dptr(xyz, "xyz", 3 * n), _dptr(w, "w", n), n, ctypes.byref(params),
                                 _stream(stream), ctypes.byref(h)))
    _SIZES[h.value] = tagi_tree_info(h)
    return h


_SIZES: dict = {}  # handle -> sizes, so the size checks below need no device sync


def _sizes(tree):
    key = tree.value if isinstance(tree, ctypes.c_void_p) else tree
    if key not in _SIZES:
        _SIZES[key] = tagi_tree_info(tree)
    return _SIZES[key]


def _tree_n(tree):
    return _sizes(tree)["n_points"]


def tagi_tree_destroy(tree):
    key = tree.value if isinstance(tree, ctypes.c_void_p) else tree
    _SIZES.pop(key, None)
    _check(lib().tagi_tree_destroy(tree))


def tagi_tree_info(tree):
    st = tagi_tree_stats()
    _check(lib().tagi_tree_info(tree, ctypes.byref(st)))
    return {k: getattr(st, k) for k, _ in tagi_tree_stats._fields_}


def tagi_tree_export(tree):
    info = tagi_tree_info(tree)
    n, nc = info["n_points"], info["n_clusters"]
    perm = np.empty(n, np.int32)
    begin = np.empty(nc, np.int32)
    end = np.empty(nc, np.int32)
    lo = np.empty((nc, 3))
    hi = np.empty((nc, 3))
    parent = np.empty(nc, np.int32)
    nchild = np.empty(nc, np.int32)
    child = np.empty((nc, 8), np.int32)
    p32 = lambda a: a.ctypes.data_as(_I32)
    _check(lib().tagi_tree_export(tree, p32(perm), p32(begin), p32(end), lo.ctypes.data_as(_D),
                                  hi.ctypes.data_as(_D), p32(parent), p32(nchild), p32(child)))
    return dict(perm=perm, begin=begin, end=end, lo=lo, hi=hi, parent=parent, nchild=nchild, child=child)


def tagi_tree_lists(tree):
    cnt = ctypes.c_int64()
    _check(lib().tagi_tree_lists(tree, 0, None, None, None, ctypes.byref(cnt)))
    m = cnt.value
    b, c, k = np.empty(m, np.int32), np.empty(m, np.int32), np.empty(m, np.int32)
    p32 = lambda a: a.ctypes.data_as(_I32)
    _check(lib().tagi_tree_lists(tree, m, p32(b), p32(c), p32(k), ctypes.byref(cnt)))
    return b, c, k


def tagi_anterpolate(tree, q, qh, stream=None):
    """q: (nq, n) float64 CUDA; qh: (n_clusters, nq, P) float64 CUDA (output)."""
    nq = q.shape[0] if q.dim() == 2 else 1
    info = _sizes(tree)
    if q.numel() != nq * info["n_points"]:
        raise ValueError("q must have nq * n elements")
    if qh.numel() != info["n_clusters"] * nq * info["n_proxies"]:
        raise ValueError("qh must have n_clusters * nq * (degree+1)^3 elements")
    _check(lib().tagi_anterpolate(tree, _dptr(q, "q"), nq, _dptr(qh, "qh"), _stream(stream)))


def tagi_yukawa_conv(tree, f, k, u, stream=None):
    """f, u: (nf, n) float64 CUDA tensors; k: nf host floats."""
    nf = f.shape[0] if f.dim() == 2 else 1
    if f.numel() != nf * _tree_n(tree):
        raise ValueError("f must have nf * n elements")
    ka, kp = _hd(np.atleast_1d(k))
    if ka.size != nf:
        raise ValueError("one k per field")
    _check(lib().tagi_yukawa_conv(tree, _dptr(f, "f"), kp, nf, _dptr(u, "u", f.numel()), _stream(stream)))


def tagi_coulomb_conv(tree, rho, vh, stream=None):
    if rho.numel() != _tree_n(tree):
        raise ValueError("rho must have n elements")
    _check(lib().tagi_coulomb_conv(tree, _dptr(rho, "rho"), _dptr(vh, "vh", rho.numel()), _stream(stream)))


def tagi_fields_conv(tree, f, k, u, rho=None, vh=None, stream=None):
    """Yukawa fields f (nf_y, n) with decay rates k into u, and the Coulomb
    field of rho into vh, in one pass (float64 CUDA tensors; f and u may be
    None when only rho is given)."""
    n = _tree_n(tree)
    nf_y = 0 if f is None else (f.shape[0] if f.dim() == 2 else 1)
    if (f is not None and (f.numel() != nf_y * n or u is None or u.numel() != nf_y * n)) or (
            rho is not None and (rho.numel() != n or vh is None or vh.numel() != n)):
        raise ValueError("f and u must be (nf_y, n); rho and vh must have n elements")
    ka = np.ascontiguousarray(np.atleast_1d(k if k is not None else []), dtype=np.float64)
    if ka.size != nf_y:
        raise ValueError("one decay rate per Yukawa field")
    _check(lib().tagi_fields_conv(tree, _dptr(f, "f"), ka.ctypes.data_as(_D), nf_y, _dptr(rho, "rho"),
                                  _dptr(u, "u"), _dptr(vh, "vh"), _stream(stream)))


def tagi_tree_batches(tree):
    """Per batch (the tree's batch order): (targets, interactions per field)
    as NumPy int arrays."""
    nb = tagi_tree_info(tree)["n_leaves"]
    size = np.zeros(nb, dtype=np.int32)
    cost = np.zeros(nb, dtype=np.int64)
    _check(lib().tagi_tree_batches(tree, size.ctypes.data_as(_I32), cost.ctypes.data_as(_I64)))
    return size, cost


def _batch_list(batches):
    b = np.ascontiguousarray(np.atleast_1d(np.asarray(batches, dtype=np.int64)), dtype=np.int32)
    return b, (b.ctypes.data_as(_I32) if b.size else None)


def tagi_fields_conv_batches(tree, f, k, u, batches, rho=None, vh=None, stream=None):
    """tagi_fields_conv for the targets of the listed batches only."""
    n = _tree_n(tree)
    nf_y = 0 if f is None else (f.shape[0] if f.dim() == 2 else 1)
    if (f is not None and (f.numel() != nf_y * n or u is None or u.numel() != nf_y * n)) or (
            rho is not None and (rho.numel() != n or vh is None or vh.numel() != n)):
        raise ValueError("f and u must be (nf_y, n); rho and vh must have n elements")
    ka = np.ascontiguousarray(np.atleast_1d(k if k is not None else []), dtype=np.float64)
    if ka.size != nf_y:
        raise ValueError("one decay rate per Yukawa field")
    b, bp = _batch_list(batches)
    _check(lib().tagi_fields_conv_batches(tree, _dptr(f, "f"), ka.ctypes.data_as(_D), nf_y, _dptr(rho, "rho"),
                                          _dptr(u, "u"), _dptr(vh, "vh"), bp, int(b.size), _stream(stream)))


def tagi_green_conv_batches(tree, veff, vshift, psi, eps, u, batches, rho=None, vh=None, stream=None):
    """The convolutions of a Green step for the targets of the listed batches:
    u (nw, n) <- Yukawa_k[(veff + vshift) psi], vh <- Hartree[rho] there."""
    nw = psi.shape[0] if psi.dim() == 2 else 1
    n = _tree_n(tree)
    if psi.numel() != nw * n or u.numel() != nw * n or veff.numel() != n or (
            rho is not None and (rho.numel() != n or vh is None or vh.numel() != n)):
        raise ValueError("psi and u must be (nw, n); veff, rho and vh must have n elements")
    ea, ep = _hd(np.atleast_1d(eps).copy())
    if ea.size != nw:
        raise ValueError("one eigenvalue per orbital")
    b, bp = _batch_list(batches)
    _check(lib().tagi_green_conv_batches(tree, _dptr(veff, "veff"), float(vshift), _dptr(psi, "psi"), ep, nw,
                                         _dptr(rho, "rho"), _dptr(u, "u"), _dptr(vh, "vh"), bp, int(b.size),
                                         _stream(stream)))


def tagi_green_reduce(tree, veff, vshift, psi, eps, u, rho=None, vh=None, stream=None):
    """Algorithm 2 lines 4-6 given the full convolution results u; psi is
    updated in place.  Returns (eps_new, resid, eh) like tagi_green_step."""
    nw = psi.shape[0] if psi.dim() == 2 else 1
    n = _tree_n(tree)
    if psi.numel() != nw * n or u.numel() != nw * n or veff.numel() != n or (
            rho is not None and (rho.numel() != n or vh is None or vh.numel() != n)):
        raise ValueError("psi and u must be (nw, n); veff, rho and vh must have n elements")
    ea, ep = _hd(np.atleast_1d(eps).copy())
    if ea.size != nw:
        raise ValueError("one eigenvalue per orbital")
    res = np.zeros(nw)
    eh = np.zeros(1)
    _check(lib().tagi_green_reduce(tree, _dptr(veff, "veff"), float(vshift), _dptr(psi, "psi"), ep, nw,
                                   _dptr(u, "u"), _dptr(rho, "rho"), _dptr(vh, "vh"), res.ctypes.data_as(_D),
                                   eh.ctypes.data_as(_D) if rho is not None else None, _stream(stream)))
    return ea, res, (float(eh[0]) if rho is not None else None)


def tagi_green_step(tree, veff, vshift, psi, eps, rho=None, vh=None, stream=None):
    """psi: (nw, n) float64 CUDA, updated in place; eps: nw host floats.

    Returns (eps_new, resid, eh) as NumPy values (eh is None without rho)."""
    nw = psi.shape[0] if psi.dim() == 2 else 1
    n = _tree_n(tree)
    if psi.numel() != nw * n or veff.numel() != n or (rho is not None and (rho.numel() != n or vh is None
                                                                           or vh.numel() != n)):
        raise ValueError("psi must be (nw, n); veff, rho and vh must have n elements")
    ea, ep = _hd(np.atleast_1d(eps).copy())
    if ea.size != nw:
        raise ValueError("one eigenvalue per orbital")
    res = np.zeros(nw)
    eh = np.zeros(1)
    _check(lib().tagi_green_step(tree, _dptr(veff, "veff"), float(vshift), _dptr(psi, "psi"), ep, nw,
                                 _dptr(rho, "rho"), _dptr(vh, "vh"), res.ctypes.data_as(_D),
                                 eh.ctypes.data_as(_D) if rho is not None else None, _stream(stream)))
    return ea, res, (float(eh[0]) if rho is not None else None)


def tagi_green_iterate(tree, veff, vshift, psi, eps, tol_gi, max_iter, beta=0.5, history=5, mix_tol=math.inf,
                       stream=None, store_output=False):
    """Green Iteration with Anderson mixing of eigenpairs until every orbital's
    residual is below tol_gi (or max_iter steps).  psi: (nw, n) float64 CUDA,
    updated in place; eps: nw host floats.

    Returns a dict: eps, resid, iters (step of convergence, -1 if none),
    steps, n_converged, field_steps."""
    nw = psi.shape[0] if psi.dim() == 2 else 1
    n = _tree_n(tree)
    if psi.numel() != nw * n or veff.numel() != n:
        raise ValueError("psi must be (nw, n) and veff must have n elements")
    ea, ep = _hd(np.atleast_1d(eps).copy())
    if ea.size != nw:
        raise ValueError("one eigenvalue per orbital")
    res = np.full(nw, np.nan)
    its = np.full(nw, -1, dtype=np.int32)
    gp = tagi_gi_params(float(tol_gi), int(max_iter), float(beta), int(history), float(mix_tol),
                        int(bool(store_output)))
    st = tagi_gi_stats()
    _check(lib().tagi_green_iterate(tree, _dptr(veff, "veff"), float(vshift), _dptr(psi, "psi"), ep, nw,
                                    ctypes.byref(gp), res.ctypes.data_as(_D), its.ctypes.data_as(_I32),
                                    ctypes.byref(st), _stream(stream)))
    return {"eps": ea, "resid": res, "iters": its, "steps": st.steps, "n_converged": st.n_converged,
            "field_steps": st.field_steps}


class Scf:
    """SCF iteration state on one tree (tagi_scf_*): density-mixing history
    and the tol_gi schedule.  Use as a context manager or call close()."""

    def __init__(self, tree, n_electrons, kT=6.3336e-4, e_zz=0.0, beta=0.5, history=5, tol_gi_first=3e-3,
                 tol_gi_final=1e-5, tol_gi_ramp=4, gi_max_iter=100, gi_beta=0.5, gi_history=5,
                 gi_mix_tol_first=math.inf, gi_store_output=False):
        self.tree = tree
        p = tagi_scf_params(float(n_electrons), float(kT), float(e_zz), float(beta), int(history),
                            float(tol_gi_first), float(tol_gi_final), int(tol_gi_ramp), int(gi_max_iter),
                            float(gi_beta), int(gi_history), float(gi_mix_tol_first), int(bool(gi_store_output)))
        h = _vp()
        _check(lib().tagi_scf_create(tree, ctypes.byref(p), ctypes.byref(h)))
        self.handle = h

    def step(self, vext, vshift, rho, psi, eps, rho_out=None, stream=None):
        """One SCF iteration: rho (n,) CUDA in: rho_in, out: the mixed next
        input; psi (nw, n) CUDA in/out; eps nw host floats.  Returns a dict of
        the report fields plus eps and occ (NumPy)."""
        nw = psi.shape[0] if psi.dim() == 2 else 1
        n = _tree_n(self.tree)
        if psi.numel() != nw * n or vext.numel() != n or rho.numel() != n or (
                rho_out is not None and rho_out.numel() != n):
            raise ValueError("psi must be (nw, n); vext, rho and rho_out must have n elements")
        ea, ep = _hd(np.atleast_1d(eps).copy())
        if ea.size != nw:
            raise ValueError("one eigenvalue per orbital")
        occ = np.zeros(nw)
        rep = tagi_scf_report()
        _check(lib().tagi_scf_step(self.handle, _dptr(vext, "vext"), float(vshift), _dptr(rho, "rho"),
                                   _dptr(psi, "psi"), ep, nw, occ.ctypes.data_as(_D), _dptr(rho_out, "rho_out"),
                                   ctypes.byref(rep), _stream(stream)))
        out = {f: getattr(rep, f) for f, _ in tagi_scf_report._fields_ if f != "gi"}
        out["gi"] = {"steps": rep.gi.steps, "n_converged": rep.gi.n_converged, "field_steps": rep.gi.field_steps}
        out["eps"] = ea
        out["occ"] = occ
        return out

    def close(self):
        if self.handle is not None:
            _check(lib().tagi_scf_destroy(self.handle))
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


PROFILE_GROUPS = {"build": 0, "anterp": 1, "interact": 2, "epilogue": 3, "reduce": 4}


def tagi_kernel_launches():
    return int(lib().tagi_kernel_launches())


def tagi_profile_enable(on=True):
    _check(lib().tagi_profile_enable(int(bool(on))))


def tagi_profile_read(group):
    ms = ctypes.c_double()
    cnt = ctypes.c_int64()
    g = PROFILE_GROUPS[group] if isinstance(group, str) else int(group)
    _check(lib().tagi_profile_read(g, ctypes.byref(ms), ctypes.byref(cnt)))
    return ms.value, cnt.value


def tagi_fp32_bias(stream=None):
    a, b = ctypes.c_double(), ctypes.c_double()
    _check(lib().tagi_fp32_bias(ctypes.byref(a), ctypes.byref(b), _stream(stream)))
    return a.value, b.value


UNIT_RATE_NAMES = ("ffma", "ffma_packed", "ex2", "rsqrt", "dfma")


def tagi_unit_rates(stream=None):
    """Measured thread operations per SM per SM clock of the units that bound
    the near/far kernel: FP32 FMA (scalar, packed f32x2), ex2.approx,
    rsqrt.approx, FP64 FMA (see include/tagi.h)."""
    out = np.zeros(5)
    _check(lib().tagi_unit_rates(out.ctypes.data_as(_D), 5, _stream(stream)))
    return dict(zip(UNIT_RATE_NAMES, (float(x) for x in out)))


def tagi_yukawa_direct_noalloc(xyz, w, f, k, u, stream=None):
    """Direct-sum Yukawa convolution without any device allocation (see
    include/tagi.h).  xyz (3, n), w (n,), f and u (nf, n): float64 CUDA
    tensors; k: nf host floats."""
    n = w.numel()
    nf = f.shape[0] if f.dim() == 2 else 1
    ka, kp = _hd(np.atleast_1d(k))
    if ka.size != nf:
        raise ValueError("one k per field")
    _check(lib().tagi_yukawa_direct_noalloc(_dptr(xyz, "xyz", 3 * n), _dptr(w, "w", n), _dptr(f, "f", nf * n), kp,
                                            nf, n, _dptr(u, "u", nf * n), _stream(stream)))


def tagi_green_graph_create(tree, veff, vshift, psi, eps, resid, rho=None, vh=None, eh=None, stream=None):
    """Capture one Green iteration as a CUDA graph.  psi (nw, n), eps (nw,),
    resid (nw,), veff/rho/vh (n,), eh (1,): float64 CUDA tensors, all kept
    by the graph (replays update psi and eps in place)."""
    nw = psi.shape[0] if psi.dim() == 2 else 1
    n = _tree_n(tree)
    if psi.numel() != nw * n or eps.numel() != nw or resid.numel() != nw or veff.numel() != n:
        raise ValueError("psi (nw, n), eps (nw,), resid (nw,), veff (n,)")
    if rho is not None and (rho.numel() != n or vh is None or vh.numel() != n or eh is None or eh.numel() < 1):
        raise ValueError("rho and vh (n,) and eh (1,) go together")
    h = ctypes.c_void_p()
    _check(lib().tagi_green_graph_create(tree, _dptr(veff, "veff"), float(vshift), _dptr(psi, "psi"), _dptr(eps, "eps"),
                                         nw, _dptr(rho, "rho"), _dptr(vh, "vh"), _dptr(resid, "resid"),
                                         _dptr(eh, "eh"), _stream(stream), ctypes.byref(h)))
    return h


def tagi_green_graph_launch(graph, stream=None):
    _check(lib().tagi_green_graph_launch(graph, _stream(stream)))


def tagi_green_graph_check(graph, stream=None):
    _check(lib().tagi_green_graph_check(graph, _stream(stream)))


def tagi_green_graph_destroy(graph):
    _check(lib().tagi_green_graph_destroy(graph))


def tagi_trim_cache():
    _check(lib().tagi_trim_cache())


def tagi_last_error():
    return lib().tagi_last_error().decode()


def tagi_version():
    return lib().tagi_version().decode()


class Tree:
    """Owning wrapper of a tagi_tree handle."""

    def __init__(self, xyz, w, **params):
        self.params = make_params(**params)
        self.handle = tagi_tree_build(xyz, w, self.params)
        self.n = w.numel()

    def close(self):
        if getattr(self, "handle", None):
            tagi_tree_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def info(self):
        return tagi_tree_info(self.handle)


# ------------------------------------------------------------ learned warm start
MLP_FEATURES = 8
MLP_HIDDEN = 32
MLP_PARAMS = 1377


def mlp_params(hidden: int) -> int:
    """Parameter count of the warm-start network with `hidden` units."""
    F, H = MLP_FEATURES, hidden
    return H * F + H + H * H + H + H + 1


def _tptr(t, name, dtype, numel):
    """Device pointer of a contiguous CUDA tensor of the given dtype."""
    import torch

    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == dtype and t.is_contiguous()):
        raise TypeError(f"{name} must be a contiguous {dtype} CUDA tensor")
    if t.numel() != numel:
        raise ValueError(f"{name} must have {numel} elements, has {t.numel()}")
    return ctypes.c_void_p(t.data_ptr())


def tagi_mlp_features(xyz, nuclei, feat=None, stream=None, ordered=False, scale=None):
    """xyz (3, n) float64 CUDA; nuclei (m, 3) host positions.  Returns the
    (n, 8) bfloat16 encodings as an int16 CUDA tensor (feat if given).
    ordered: two nuclei in list order (tagi_mlp_features_ordered); scale:
    m decay rates of the first two features (tagi_mlp_features_scaled)."""
    import torch

    n = xyz.numel() // 3
    nu = np.ascontiguousarray(np.asarray(nuclei, dtype=np.float64).reshape(-1, 3))
    if feat is None:
        feat = torch.empty((n, MLP_FEATURES), dtype=torch.int16, device=xyz.device)
    fp = _tptr(feat, "feat", torch.int16, n * MLP_FEATURES)
    if scale is not None:
        zs = np.ascontiguousarray(np.asarray(scale, dtype=np.float64).ravel())
        if zs.size != nu.shape[0]:
            raise ValueError("one decay rate per nucleus")
        _check(lib().tagi_mlp_features_scaled(_dptr(xyz, "xyz", 3 * n), n, nu.ctypes.data_as(_D),
                                              zs.ctypes.data_as(_D), nu.shape[0], int(bool(ordered)), fp,
                                              _stream(stream)))
    elif ordered:
        if nu.shape[0] != 2:
            raise ValueError("list order needs exactly two nuclei")
        _check(lib().tagi_mlp_features_ordered(_dptr(xyz, "xyz", 3 * n), n, nu.ctypes.data_as(_D), fp,
                                               _stream(stream)))
    else:
        _check(lib().tagi_mlp_features(_dptr(xyz, "xyz", 3 * n), n, nu.ctypes.data_as(_D), nu.shape[0], fp,
                                       _stream(stream)))
    return feat


class Mlp:
    """Warm-start MLP on the device (tagi_mlp_*).  Use as a context manager
    or call close()."""

    def __init__(self, params, hidden=MLP_HIDDEN):
        p = np.ascontiguousarray(np.asarray(params, dtype=np.float64))
        h = _vp()
        _check(lib().tagi_mlp_create(MLP_FEATURES, int(hidden), p.ctypes.data_as(_D), p.size, ctypes.byref(h)))
        self.handle = h
        self.hidden = int(hidden)
        self.n_params = mlp_params(self.hidden)

    def params(self, stream=None):
        out = np.empty(self.n_params)
        _check(lib().tagi_mlp_get_params(self.handle, out.ctypes.data_as(_D), self.n_params, _stream(stream)))
        return out

    def _data(self, feat, target=None, wt=None):
        import torch

        n = feat.shape[0]
        args = [_tptr(feat, "feat", torch.int16, n * MLP_FEATURES)]
        if target is not None:
            args += [_tptr(target, "target", torch.float32, n), _tptr(wt, "wt", torch.float32, n)]
        return n, args

    def forward(self, feat, y=None, stream=None):
        import torch

        n, (fp,) = self._data(feat)
        if y is None:
            y = torch.empty(n, dtype=torch.float32, device=feat.device)
        _check(lib().tagi_mlp_forward(self.handle, fp, n, _tptr(y, "y", torch.float32, n), _stream(stream)))
        return y

    def gradient(self, feat, target, wt, stream=None):
        """(loss, gradient) of the current master weights."""
        n, (fp, tp, wp) = self._data(feat, target, wt)
        g = np.empty(self.n_params)
        loss = np.zeros(1)
        _check(lib().tagi_mlp_gradient(self.handle, fp, tp, wp, n, g.ctypes.data_as(_D), loss.ctypes.data_as(_D),
                                       _stream(stream)))
        return float(loss[0]), g

    def train_step(self, feat, target, wt, lr, beta1=0.9, beta2=0.999, eps=1e-8, want_loss=False, stream=None):
        n, (fp, tp, wp) = self._data(feat, target, wt)
        a = tagi_adam_params(float(lr), float(beta1), float(beta2), float(eps))
        loss = np.zeros(1)
        _check(lib().tagi_mlp_train_step(self.handle, fp, tp, wp, n, ctypes.byref(a),
                                         loss.ctypes.data_as(_D) if want_loss else None, _stream(stream)))
        return float(loss[0]) if want_loss else None

    def warm_start(self, feat, s, w, psi=None, stream=None):
        import torch

        n, (fp,) = self._data(feat)
        if psi is None:
            psi = torch.empty(n, dtype=torch.float64, device=feat.device)
        _check(lib().tagi_mlp_warm_start(self.handle, fp, _dptr(s, "s", n), _dptr(w, "w", n), n,
                                         _dptr(psi, "psi", n), _stream(stream)))
        return psi

    def close(self):
        if getattr(self, "handle", None):
            lib().tagi_mlp_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
