"""Thin ctypes binding of ``include/hgmm.h``, ``include/hgmm_proposal.h`` and
``include/hgmm_flat.h``.

Argument marshalling only: every function below forwards to the entry point
of the same name in ``_lib/libhgmm.so``, passing raw device pointers taken
from PyTorch tensors (PyTorch owns the caller's device memory and streams) or
host pointers from numpy arrays.  There is no fallback: if the compiled
library is missing, importing this module raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "_lib", "libhgmm.so")

HGMM_OK = 0
HGMM_EINVAL = -1
HGMM_ENOMEM = -2
HGMM_ECUDA = -3
HGMM_ETIMEOUT = -4
HGMM_EDEGENERATE = -5
HGMM_ENONFINITE = -6
HGMM_ECAPACITY = -7
HGMM_J = 8
HGMM_MAX_DEPTH = 5
HGMM_NODE_DOUBLES = 16
HGMM_MLP_IN = 1280
HGMM_MLP_HIDDEN = 256
HGMM_MLP_OUT = 9
HGMM_MLP_PARAMS = 396041
HGMM_FEAT_PER_CLOUD = 640
HGMM_FRAME_DOUBLES = 16
HGMM_LABEL_FLOATS = 12


class HgmmError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {strerror(code)} ({code})")


class hgmm_params(ctypes.Structure):
    _fields_ = [("em_iters", ctypes.c_int32), ("n_min", ctypes.c_float),
                ("lam_c", ctypes.c_float), ("eps_rel", ctypes.c_float),
                ("precision", ctypes.c_int32), ("debug_stop_level", ctypes.c_int32),
                ("debug_stop_iters", ctypes.c_int32), ("flags", ctypes.c_int32)]


HGMM_DESCENT_ML_LOCAL = 0
HGMM_DESCENT_ML_GLOBAL = 1
HGMM_DESCENT_MULTIPATH = 2


class hgmm_descent(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("tau", ctypes.c_float), ("lam_c", ctypes.c_float),
                ("full_eq7", ctypes.c_int32)]


def _load():
    if not os.path.exists(_LIB_PATH):
        raise ImportError(
            f"{_LIB_PATH} is missing: build it with "
            "`python -c 'import __graft_entry__ as g; g.build()'` (needs nvcc)")
    lib = ctypes.CDLL(_LIB_PATH)
    vp, i32, i64, f32 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_float
    P = ctypes.POINTER
    sig = {
        "hgmm_params_default": (None, [P(hgmm_params)]),
        "hgmm_tree_create": (ctypes.c_int, [i64, i32, P(vp)]),
        "hgmm_tree_destroy": (None, [vp]),
        "hgmm_build": (ctypes.c_int, [vp, vp, i64, i32, i32, P(hgmm_params), vp]),
        "hgmm_register": (ctypes.c_int, [vp, vp, i64, vp, i32, f32, vp, vp, vp]),
        "hgmm_sync": (ctypes.c_int, [vp, vp]),
        "hgmm_register_pair_host": (ctypes.c_int, [vp, vp, i64, vp, i64, i32, P(hgmm_params),
                                                   vp, i32, vp, vp]),
        "hgmm_tree_export": (ctypes.c_int, [vp, i32, vp, i64]),
        "hgmm_debug_labels": (ctypes.c_int, [vp, i32, vp, i64]),
        "hgmm_debug_root": (ctypes.c_int, [vp, vp]),
        "hgmm_debug_posteriors": (ctypes.c_int, [vp, i32, vp, i64]),
        "hgmm_propose": (ctypes.c_int, [vp, vp, vp, vp, vp]),
        "hgmm_debug_reg_moments": (ctypes.c_int, [vp, vp, i64]),
        "hgmm_node_count": (i64, [i32]),
        "hgmm_profile": (ctypes.c_int, [vp, i32]),
        "hgmm_debug_barrier_timeout": (ctypes.c_int, [vp, i64, vp]),
        "hgmm_trace": (ctypes.c_int, [vp, i32]),
        "hgmm_fit_level0_noalloc": (ctypes.c_int, [vp, i64, P(hgmm_params), vp, vp]),
        "hgmm_batch_create": (ctypes.c_int, [i64, i32, i32, P(vp)]),
        "hgmm_batch_destroy": (None, [vp]),
        "hgmm_batch_plan": (ctypes.c_int, [vp, i32, vp, vp, vp]),
        "hgmm_batch_plan_ranges": (ctypes.c_int, [vp, i32, vp, vp, vp]),
        "hgmm_batch_set_shape": (ctypes.c_int, [vp, i32]),
        "hgmm_batch_get_shape": (ctypes.c_int, [vp, P(i32), P(i32)]),
        "hgmm_batch_register": (ctypes.c_int, [vp, vp, P(hgmm_params), vp, i32, vp, vp, vp, vp]),
        "hgmm_batch_debug_tree": (ctypes.c_int, [vp, i32, i32, vp, i64]),
        "hgmm_batch_set_build_shape": (ctypes.c_int, [vp, i32, i32, i32, i32]),
        "hgmm_batch_get_build_shape": (ctypes.c_int, [vp, vp, vp]),
        "hgmm_batch_pair_ns": (ctypes.c_int, [vp, vp, i64]),
        "hgmm_batch_debug_root": (ctypes.c_int, [vp, i32, vp]),
        "hgmm_batch_autotune": (ctypes.c_int, [vp, vp, P(hgmm_params), vp, i32, vp, vp, vp]),
        "hgmm_trace_read": (ctypes.c_int, [vp, vp, i64, P(i32), P(i32)]),
        "hgmm_profile_read": (ctypes.c_int, [vp, i32, P(ctypes.c_char_p), P(ctypes.c_double),
                                             P(ctypes.c_int64)]),
        "hgmm_strerror": (ctypes.c_char_p, [ctypes.c_int]),
        "hgmm_register_objective": (ctypes.c_int, [vp, vp, vp]),
        "hgmm_register_descent": (ctypes.c_int, [vp, vp, i64, vp, i32, P(hgmm_descent), vp, vp, vp]),
        "hgmm_batch_objective": (ctypes.c_int, [vp, vp, vp]),
        "hgmm_batch_features": (ctypes.c_int, [vp, vp, P(hgmm_params), vp, vp, vp]),
        "hgmm_mlp_create": (ctypes.c_int, [i32, P(vp)]),
        "hgmm_mlp_destroy": (None, [vp]),
        "hgmm_mlp_set_params": (ctypes.c_int, [vp, vp, i64]),
        "hgmm_mlp_get_params": (ctypes.c_int, [vp, vp, i64]),
        "hgmm_mlp_read_grads": (ctypes.c_int, [vp, vp, i64]),
        "hgmm_mlp_forward": (ctypes.c_int, [vp, vp, i32, vp, vp]),
        "hgmm_mlp_gradients": (ctypes.c_int, [vp, vp, vp, vp, i32, i32, f32, vp, vp]),
        "hgmm_mlp_adam": (ctypes.c_int, [vp, f32, vp]),
        "hgmm_mlp_train_step": (ctypes.c_int, [vp, vp, vp, vp, i32, i32, f32, f32, vp, vp]),
        "hgmm_mlp_sync": (ctypes.c_int, [vp, vp]),
        "hgmm_tree_features": (ctypes.c_int, [vp, vp, vp, vp]),
        "hgmm_pose_decode": (ctypes.c_int, [vp, vp, i32, vp, vp]),
        "hgmm_pose_encode": (ctypes.c_int, [vp, vp, i32, vp, vp]),
        "hgmm_pose_select": (ctypes.c_int, [i32, vp, vp, vp, vp, vp, vp, vp, vp]),
        "hgmm_pose_compose": (ctypes.c_int, [i32, vp, vp, vp, vp]),
        "hgmm_debug_gemm": (ctypes.c_int, [vp, i64, i64, vp, i64, i64, i32, i32, i32, vp, vp]),
        "hgmm_flat_create": (ctypes.c_int, [i64, i32, P(vp)]),
        "hgmm_flat_destroy": (None, [vp]),
        "hgmm_flat_from_tree": (ctypes.c_int, [vp, vp, i32, vp]),
        "hgmm_flat_fit": (ctypes.c_int, [vp, vp, i64, i32, f32, vp]),
        "hgmm_flat_register": (ctypes.c_int, [vp, vp, i64, vp, i32, vp, vp, vp]),
        "hgmm_flat_objective": (ctypes.c_int, [vp, vp, vp]),
        "hgmm_flat_export": (ctypes.c_int, [vp, vp, i64, P(i32), vp]),
        "hgmm_flat_debug_moments": (ctypes.c_int, [vp, vp, i64, P(i32)]),
        "hgmm_flat_sync": (ctypes.c_int, [vp, vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = _load()
LIB_PATH = _LIB_PATH


def strerror(code: int) -> str:
    return _lib.hgmm_strerror(int(code)).decode()


def _check(rc: int, where: str):
    if rc != HGMM_OK:
        raise HgmmError(rc, where)


HGMM_FLAG_EM_COOPERATIVE = 1


def params(em_iters=8, n_min=8.0, lam_c=0.01, eps_rel=1e-3, precision=0,
           debug_stop_level=0, debug_stop_iters=0, flags=0) -> hgmm_params:
    p = hgmm_params()
    _lib.hgmm_params_default(ctypes.byref(p))
    p.em_iters, p.n_min, p.lam_c, p.eps_rel, p.precision = em_iters, n_min, lam_c, eps_rel, precision
    p.debug_stop_level, p.debug_stop_iters, p.flags = debug_stop_level, debug_stop_iters, flags
    return p


def _stream_ptr(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _dev_points(x, name):
    if x.dtype != __import__("torch").float32 or x.dim() != 2 or x.shape[1] != 4:
        raise ValueError(f"{name}: expected an (N, 4) float32 tensor")
    if not x.is_cuda or not x.is_contiguous():
        raise ValueError(f"{name}: expected a contiguous CUDA tensor")
    return ctypes.c_void_p(x.data_ptr())


def _dptr(x):
    return ctypes.c_void_p(0 if x is None else x.data_ptr())


# ---------------------------------------------------------------- entry points
def hgmm_node_count(depth: int) -> int:
    return int(_lib.hgmm_node_count(int(depth)))


def hgmm_tree_create(max_points: int, max_depth: int) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check(_lib.hgmm_tree_create(int(max_points), int(max_depth), ctypes.byref(h)),
           "hgmm_tree_create")
    return h


def hgmm_tree_destroy(h) -> None:
    _lib.hgmm_tree_destroy(h)


def hgmm_build(h, points, depth: int, J: int = HGMM_J, prm: hgmm_params | None = None,
               stream=None) -> None:
    _check(_lib.hgmm_build(h, _dev_points(points, "points"), points.shape[0], int(depth),
                           int(J), None if prm is None else ctypes.byref(prm),
                           _stream_ptr(stream)), "hgmm_build")


def hgmm_register(h, src, T_init=None, iters: int = 30, lam_c: float = -1.0, stream=None,
                  T_out=None, T_hist=None):
    """Returns the device tensor T_out (4x4 float64)."""
    import torch
    if T_out is None:
        T_out = torch.empty((4, 4), dtype=torch.float64, device=src.device)
    for name, x in (("T_init", T_init), ("T_out", T_out), ("T_hist", T_hist)):
        if x is not None and (x.dtype != torch.float64 or not x.is_cuda or not x.is_contiguous()):
            raise ValueError(f"{name}: expected a contiguous float64 CUDA tensor")
    _check(_lib.hgmm_register(h, _dev_points(src, "src"), src.shape[0], _dptr(T_init),
                              int(iters), float(lam_c), _stream_ptr(stream), _dptr(T_out),
                              _dptr(T_hist)), "hgmm_register")
    return T_out


def hgmm_register_descent(h, src, mode: int, tau: float = 0.0, T_init=None, iters: int = 30,
                          lam_c: float = -1.0, stream=None, T_out=None, T_hist=None, full_eq7: bool = False):
    """hgmm_register with a descent variant (HGMM_DESCENT_*) and optionally the
    full Eq. 7 M-step; returns T_out."""
    import torch
    if T_out is None:
        T_out = torch.empty((4, 4), dtype=torch.float64, device=src.device)
    for name, x in (("T_init", T_init), ("T_out", T_out), ("T_hist", T_hist)):
        if x is not None and (x.dtype != torch.float64 or not x.is_cuda or not x.is_contiguous()):
            raise ValueError(f"{name}: expected a contiguous float64 CUDA tensor")
    d = hgmm_descent(int(mode), float(tau), float(lam_c), int(bool(full_eq7)))
    _check(_lib.hgmm_register_descent(h, _dev_points(src, "src"), src.shape[0], _dptr(T_init), int(iters),
                                      ctypes.byref(d), _stream_ptr(stream), _dptr(T_out), _dptr(T_hist)),
           "hgmm_register_descent")
    return T_out


def hgmm_sync(h, stream=None) -> None:
    _check(_lib.hgmm_sync(h, _stream_ptr(stream)), "hgmm_sync")


def _host_points(x, name):
    if hasattr(x, "data_ptr"):  # torch CPU tensor (possibly pinned)
        if x.dtype != __import__("torch").float32 or x.dim() != 2 or x.shape[1] != 4 \
                or x.is_cuda or not x.is_contiguous():
            raise ValueError(f"{name}: expected a contiguous (N, 4) float32 host tensor")
        return ctypes.c_void_p(x.data_ptr()), x.shape[0]
    a = np.ascontiguousarray(x, dtype=np.float32)
    if a.ndim != 2 or a.shape[1] != 4:
        raise ValueError(f"{name}: expected (N, 4) float32")
    return ctypes.c_void_p(a.ctypes.data), a.shape[0], a


def hgmm_register_pair_host(h, tgt, src, depth: int, prm: hgmm_params | None = None,
                            T_init=None, iters: int = 30, stream=None) -> np.ndarray:
    t_ptr, n_t, *keep_t = _host_points(tgt, "tgt")
    s_ptr, n_s, *keep_s = _host_points(src, "src")
    Ti = None if T_init is None else np.ascontiguousarray(T_init, dtype=np.float64)
    out = np.empty((4, 4), dtype=np.float64)
    _check(_lib.hgmm_register_pair_host(
        h, t_ptr, n_t, s_ptr, n_s, int(depth), None if prm is None else ctypes.byref(prm),
        None if Ti is None else ctypes.c_void_p(Ti.ctypes.data), int(iters),
        _stream_ptr(stream), ctypes.c_void_p(out.ctypes.data)), "hgmm_register_pair_host")
    del keep_t, keep_s
    return out


def hgmm_tree_export(h, level: int, n_nodes: int) -> np.ndarray:
    out = np.empty((n_nodes, HGMM_NODE_DOUBLES), dtype=np.float64)
    _check(_lib.hgmm_tree_export(h, int(level), ctypes.c_void_p(out.ctypes.data), out.size),
           "hgmm_tree_export")
    return out


def hgmm_debug_labels(h, level: int, n: int) -> np.ndarray:
    out = np.empty(n, dtype=np.int32)
    _check(_lib.hgmm_debug_labels(h, int(level), ctypes.c_void_p(out.ctypes.data), n),
           "hgmm_debug_labels")
    return out


def hgmm_debug_posteriors(h, level: int, n: int) -> np.ndarray:
    """(n, 8) float32 Eq. 3 posteriors of each input point over its parent's
    children at ``level`` (synchronous)."""
    out = np.zeros((n, 8), np.float32)
    _check(_lib.hgmm_debug_posteriors(h, int(level), ctypes.c_void_p(out.ctypes.data), out.size),
           "hgmm_debug_posteriors")
    return out


def hgmm_debug_root(h) -> np.ndarray:
    out = np.empty(12, dtype=np.float64)
    _check(_lib.hgmm_debug_root(h, ctypes.c_void_p(out.ctypes.data)), "hgmm_debug_root")
    return out


def hgmm_debug_reg_moments(h, n_nodes: int) -> np.ndarray:
    out = np.empty((n_nodes, 4), dtype=np.float64)
    _check(_lib.hgmm_debug_reg_moments(h, ctypes.c_void_p(out.ctypes.data), out.size),
           "hgmm_debug_reg_moments")
    return out


HGMM_PROF_KERNELS = 16


def hgmm_debug_barrier_timeout(h, spin_limit: int, stream=None) -> None:
    _check(_lib.hgmm_debug_barrier_timeout(h, int(spin_limit), _stream_ptr(stream)),
           "hgmm_debug_barrier_timeout")


def hgmm_fit_level0_noalloc(points, prm: hgmm_params | None = None, stream=None, out=None):
    """Allocation-free level-0 GMM fit; `out` is a caller-owned (129,) float64
    CUDA tensor (8 node records of 16 + a status word), returned.  The call is
    asynchronous: once the stream has run, out[128] holds 0 or an HGMM_E*
    code (non-finite input, a wait that timed out, a degenerate covariance)
    that the caller must check before using the nodes."""
    import torch
    if out is None:
        raise ValueError("out: a (129,) float64 CUDA tensor owned by the caller is required")
    if out.dtype != torch.float64 or not out.is_cuda or not out.is_contiguous() or out.numel() < 129:
        raise ValueError("out: expected a contiguous float64 CUDA tensor of 129 elements")
    _check(_lib.hgmm_fit_level0_noalloc(_dev_points(points, "points"), points.shape[0],
                                        None if prm is None else ctypes.byref(prm),
                                        _stream_ptr(stream), ctypes.c_void_p(out.data_ptr())),
           "hgmm_fit_level0_noalloc")
    return out


def _node_dict(a: np.ndarray) -> dict:
    """(m, 16) exported node records -> named fields (Sigma as (m, 3, 3))."""
    m = a.shape[0]
    S = np.empty((m, 3, 3))
    iu = [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]
    for k, (i, j) in enumerate(iu):
        S[:, i, j] = a[:, 4 + k]
        S[:, j, i] = a[:, 4 + k]
    return {"pi": a[:, 0], "mu": a[:, 1:4], "Sigma": S, "live": a[:, 10] > 0.5,
            "count": a[:, 11].astype(np.int64), "complexity": a[:, 12], "lam": a[:, 13:16]}


def _root_dict(r: np.ndarray) -> dict:
    S = np.array([[r[4], r[5], r[6]], [r[5], r[7], r[8]], [r[6], r[8], r[9]]])
    return {"n": r[0], "mu": r[1:4], "Sigma": S, "extent": r[10], "eps": r[11]}


def hgmm_batch_create(max_points: int, max_depth: int, max_pairs: int):
    h = ctypes.c_void_p()
    _check(_lib.hgmm_batch_create(int(max_points), int(max_depth), int(max_pairs), ctypes.byref(h)),
           "hgmm_batch_create")
    return h


def hgmm_batch_destroy(h) -> None:
    _lib.hgmm_batch_destroy(h)


def hgmm_batch_plan(h, tgt_off, src_off, depth) -> None:
    t = np.ascontiguousarray(tgt_off, dtype=np.int64)
    s_ = np.ascontiguousarray(src_off, dtype=np.int64)
    d = np.ascontiguousarray(depth, dtype=np.int32)
    _check(_lib.hgmm_batch_plan(h, d.shape[0], ctypes.c_void_p(t.ctypes.data),
                                ctypes.c_void_p(s_.ctypes.data), ctypes.c_void_p(d.ctypes.data)),
           "hgmm_batch_plan")


def hgmm_batch_plan_ranges(h, tgt_rng, src_rng, depth) -> None:
    """tgt_rng / src_rng: (n_pairs, 2) int64 [start, end) point ranges."""
    t = np.ascontiguousarray(tgt_rng, dtype=np.int64).reshape(-1)
    s_ = np.ascontiguousarray(src_rng, dtype=np.int64).reshape(-1)
    d = np.ascontiguousarray(depth, dtype=np.int32)
    if t.shape[0] != 2 * d.shape[0] or s_.shape[0] != 2 * d.shape[0]:
        raise ValueError("ranges: expected (n_pairs, 2) arrays matching depth")
    _check(_lib.hgmm_batch_plan_ranges(h, d.shape[0], ctypes.c_void_p(t.ctypes.data),
                                       ctypes.c_void_p(s_.ctypes.data), ctypes.c_void_p(d.ctypes.data)),
           "hgmm_batch_plan_ranges")


def hgmm_batch_set_shape(h, cluster_ctas: int) -> None:
    _check(_lib.hgmm_batch_set_shape(h, int(cluster_ctas)), "hgmm_batch_set_shape")


def hgmm_batch_get_shape(h):
    c = ctypes.c_int32()
    n = ctypes.c_int32()
    _check(_lib.hgmm_batch_get_shape(h, ctypes.byref(c), ctypes.byref(n)), "hgmm_batch_get_shape")
    return c.value, n.value


def hgmm_batch_register(h, points, T_out, prm: hgmm_params | None = None, T_init=None,
                        iters: int = 30, stream=None, pair_status=None, T_hist=None):
    """T_hist (optional): n_pairs x iters x 16 float64 CUDA tensor, the pose
    of every pair after every round."""
    _check(_lib.hgmm_batch_register(h, _dev_points(points, "points"),
                                    None if prm is None else ctypes.byref(prm), _dptr(T_init),
                                    int(iters), _stream_ptr(stream), _dptr(T_out),
                                    _dptr(pair_status), _dptr(T_hist)), "hgmm_batch_register")
    return T_out


def hgmm_batch_pair_ns(h, n_pairs: int) -> np.ndarray:
    """Each pair's device run time (ns) in the last batched launch."""
    out = np.zeros(n_pairs, np.uint64)
    _check(_lib.hgmm_batch_pair_ns(h, ctypes.c_void_p(out.ctypes.data), int(n_pairs)), "hgmm_batch_pair_ns")
    return out


def hgmm_batch_debug_tree(h, pair: int, level: int) -> dict:
    """Level ``level`` of the tree the last launch built for ``pair`` (the
    hgmm_tree_export fields), while its workspace still holds it."""
    m = 8 ** (level + 1)
    buf = np.zeros((m, HGMM_NODE_DOUBLES), np.float64)
    _check(_lib.hgmm_batch_debug_tree(h, int(pair), int(level), ctypes.c_void_p(buf.ctypes.data),
                                      buf.size), "hgmm_batch_debug_tree")
    return _node_dict(buf)


def hgmm_batch_debug_root(h, pair: int) -> dict:
    r = np.zeros(12, np.float64)
    _check(_lib.hgmm_batch_debug_root(h, int(pair), ctypes.c_void_p(r.ctypes.data)),
           "hgmm_batch_debug_root")
    return _root_dict(r)


def hgmm_batch_autotune(h, points, T_out, prm: hgmm_params | None = None, T_init=None,
                        iters: int = 30, stream=None) -> list:
    ms = (ctypes.c_float * 4)()
    _check(_lib.hgmm_batch_autotune(h, _dev_points(points, "points"),
                                    None if prm is None else ctypes.byref(prm), _dptr(T_init),
                                    int(iters), _stream_ptr(stream), _dptr(T_out), ms),
           "hgmm_batch_autotune")
    return list(ms)


HGMM_BATCH_BUCKETS = 3


def hgmm_batch_set_build_shape(h, bucket: int, warp_item_parents: int, mstep_cta_runs: int,
                               offsets_cta_items: int) -> None:
    _check(_lib.hgmm_batch_set_build_shape(h, int(bucket), int(warp_item_parents), int(mstep_cta_runs),
                                           int(offsets_cta_items)), "hgmm_batch_set_build_shape")


def hgmm_batch_get_build_shape(h):
    """((3, 3) int32 build shape per size bucket, [default ms, tuned ms] of the
    last autotune)."""
    sh = np.zeros(9, np.int32)
    ms = np.zeros(2, np.float32)
    _check(_lib.hgmm_batch_get_build_shape(h, ctypes.c_void_p(sh.ctypes.data), ctypes.c_void_p(ms.ctypes.data)),
           "hgmm_batch_get_build_shape")
    return sh.reshape(3, 3), [float(ms[0]), float(ms[1])]


def hgmm_batch_objective(h, out, stream=None):
    """Per pair of the last hgmm_batch_register: Eq. 11 objective of its last
    round into ``out`` (n_pairs float64, CUDA)."""
    _check(_lib.hgmm_batch_objective(h, _dptr(out), _stream_ptr(stream)), "hgmm_batch_objective")
    return out


def hgmm_batch_features(h, points, feat, frame, prm: hgmm_params | None = None, stream=None):
    """Features (n_pairs x 640 bfloat16) and frames (n_pairs x 16 float64) of
    every planned pair's target cloud."""
    _check(_lib.hgmm_batch_features(h, _dev_points(points, "points"),
                                    None if prm is None else ctypes.byref(prm), _dptr(feat),
                                    _dptr(frame), _stream_ptr(stream)), "hgmm_batch_features")
    return feat, frame


class Batch:
    """Owns one hgmm_batch: planned pairs over one concatenated point buffer."""

    def __init__(self, max_points: int, max_depth: int, max_pairs: int):
        self.handle = hgmm_batch_create(max_points, max_depth, max_pairs)

    def close(self):
        if getattr(self, "handle", None):
            hgmm_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def hgmm_trace(h, enable: bool) -> None:
    _check(_lib.hgmm_trace(h, 1 if enable else 0), "hgmm_trace")


def hgmm_trace_read(h, max_iters: int = 64, max_ctas: int = 4096) -> np.ndarray:
    """(iters, ctas, 6) int64 globaltimer stamps of the last traced registration."""
    buf = np.zeros(max_iters * max_ctas * 6, dtype=np.int64)
    it = ctypes.c_int32()
    nc = ctypes.c_int32()
    _check(_lib.hgmm_trace_read(h, ctypes.c_void_p(buf.ctypes.data), buf.size,
                                ctypes.byref(it), ctypes.byref(nc)), "hgmm_trace_read")
    return buf[: it.value * nc.value * 6].reshape(it.value, nc.value, 6)


def hgmm_profile(h, enable: bool) -> None:
    _check(_lib.hgmm_profile(h, 1 if enable else 0), "hgmm_profile")


def hgmm_profile_read(h) -> dict:
    """{kernel name: (total ms, launches)} of the launches recorded since
    hgmm_profile(h, True)."""
    out = {}
    for k in range(HGMM_PROF_KERNELS):
        name = ctypes.c_char_p()
        ms = ctypes.c_double()
        cnt = ctypes.c_int64()
        _check(_lib.hgmm_profile_read(h, k, ctypes.byref(name), ctypes.byref(ms),
                                      ctypes.byref(cnt)), "hgmm_profile_read")
        out[name.value.decode()] = (ms.value, cnt.value)
    return out


def hgmm_register_objective(h, out, stream=None):
    _check(_lib.hgmm_register_objective(h, _dptr(out), _stream_ptr(stream)),
           "hgmm_register_objective")
    return out


# ---------------------------------------------------------------- proposal
def _need(x, dtype, numel, name):
    import torch
    if x is None or x.dtype != dtype or not x.is_cuda or not x.is_contiguous() or x.numel() < numel:
        raise ValueError(f"{name}: expected a contiguous CUDA {dtype} tensor of >= {numel} elements")
    return ctypes.c_void_p(x.data_ptr())


def hgmm_mlp_create(max_batch: int):
    h = ctypes.c_void_p()
    _check(_lib.hgmm_mlp_create(int(max_batch), ctypes.byref(h)), "hgmm_mlp_create")
    return h


def hgmm_mlp_destroy(h) -> None:
    _lib.hgmm_mlp_destroy(h)


def hgmm_mlp_set_params(h, params) -> None:
    p = np.ascontiguousarray(params, dtype=np.float32)
    _check(_lib.hgmm_mlp_set_params(h, ctypes.c_void_p(p.ctypes.data), p.size), "hgmm_mlp_set_params")


def hgmm_mlp_get_params(h) -> np.ndarray:
    p = np.empty(HGMM_MLP_PARAMS, dtype=np.float32)
    _check(_lib.hgmm_mlp_get_params(h, ctypes.c_void_p(p.ctypes.data), p.size), "hgmm_mlp_get_params")
    return p


def hgmm_mlp_read_grads(h) -> np.ndarray:
    g = np.empty(HGMM_MLP_PARAMS, dtype=np.float32)
    _check(_lib.hgmm_mlp_read_grads(h, ctypes.c_void_p(g.ctypes.data), g.size), "hgmm_mlp_read_grads")
    return g


def hgmm_mlp_forward(h, x, y, stream=None):
    """x: (B, 1280) bfloat16 CUDA tensor; y: (B, 9) float32 CUDA tensor."""
    import torch
    B = int(x.shape[0])
    _check(_lib.hgmm_mlp_forward(h, _need(x, torch.bfloat16, B * HGMM_MLP_IN, "x"), B,
                                 _need(y, torch.float32, B * HGMM_MLP_OUT, "y"), _stream_ptr(stream)),
           "hgmm_mlp_forward")
    return y


def hgmm_mlp_gradients(h, x, labels, batch: int, index=None, w_t: float = 1.0, loss=None,
                       stream=None):
    import torch
    n_rows = int(x.shape[0])
    _check(_lib.hgmm_mlp_gradients(h, _need(x, torch.bfloat16, HGMM_MLP_IN, "x"),
                                   _need(labels, torch.float32, HGMM_LABEL_FLOATS, "labels"),
                                   None if index is None else _need(index, torch.int32, batch, "index"),
                                   int(batch), n_rows, float(w_t), _dptr(loss), _stream_ptr(stream)),
           "hgmm_mlp_gradients")


def hgmm_mlp_adam(h, lr: float, stream=None) -> None:
    _check(_lib.hgmm_mlp_adam(h, float(lr), _stream_ptr(stream)), "hgmm_mlp_adam")


def hgmm_mlp_train_step(h, x, labels, batch: int, index=None, w_t: float = 1.0, lr: float = 1e-3,
                        loss=None, stream=None):
    import torch
    n_rows = int(x.shape[0])
    _check(_lib.hgmm_mlp_train_step(h, _need(x, torch.bfloat16, HGMM_MLP_IN, "x"),
                                    _need(labels, torch.float32, HGMM_LABEL_FLOATS, "labels"),
                                    None if index is None else _need(index, torch.int32, batch, "index"),
                                    int(batch), n_rows, float(w_t), float(lr), _dptr(loss),
                                    _stream_ptr(stream)), "hgmm_mlp_train_step")


def hgmm_mlp_sync(h, stream=None) -> None:
    _check(_lib.hgmm_mlp_sync(h, _stream_ptr(stream)), "hgmm_mlp_sync")


def hgmm_tree_features(h, feat, frame, stream=None):
    import torch
    _check(_lib.hgmm_tree_features(h, _need(feat, torch.bfloat16, HGMM_FEAT_PER_CLOUD, "feat"),
                                   _need(frame, torch.float64, HGMM_FRAME_DOUBLES, "frame"),
                                   _stream_ptr(stream)), "hgmm_tree_features")
    return feat, frame


def hgmm_propose(tgt_tree, src_tree, mlp, T_out, stream=None):
    """The network's initial pose for one pair (16 float64 CUDA tensor) in
    one library call: features of both trees, forward, decode."""
    _check(_lib.hgmm_propose(tgt_tree, src_tree, mlp, _stream_ptr(stream), _dptr(T_out)), "hgmm_propose")
    return T_out


def hgmm_pose_decode(y, frames, T, stream=None):
    import torch
    n = int(y.shape[0])
    _check(_lib.hgmm_pose_decode(_need(y, torch.float32, 9 * n, "y"), _need(frames, torch.float64, 32 * n, "frames"),
                                 n, _need(T, torch.float64, 16 * n, "T"), _stream_ptr(stream)),
           "hgmm_pose_decode")
    return T


def hgmm_pose_encode(T, frames, labels, stream=None):
    import torch
    n = int(T.shape[0])
    _check(_lib.hgmm_pose_encode(_need(T, torch.float64, 16 * n, "T"), _need(frames, torch.float64, 32 * n, "frames"),
                                 n, _need(labels, torch.float32, 12 * n, "labels"), _stream_ptr(stream)),
           "hgmm_pose_encode")
    return labels


def hgmm_pose_select(T_a, obj_a, T_b, obj_b, T_out, choice=None, stream=None, obj_out=None):
    import torch
    n = int(T_a.shape[0])
    _check(_lib.hgmm_pose_select(n, _need(T_a, torch.float64, 16 * n, "T_a"),
                                 _need(obj_a, torch.float64, n, "obj_a"),
                                 _need(T_b, torch.float64, 16 * n, "T_b"),
                                 _need(obj_b, torch.float64, n, "obj_b"),
                                 _need(T_out, torch.float64, 16 * n, "T_out"),
                                 None if choice is None else _need(choice, torch.int32, n, "choice"),
                                 None if obj_out is None else _need(obj_out, torch.float64, n, "obj_out"),
                                 _stream_ptr(stream)), "hgmm_pose_select")
    return T_out


def hgmm_pose_compose(A, Bm, out, stream=None):
    """out[i] = A[i] @ B[i] for (n, 16) (or (n, 4, 4)) float64 CUDA tensors."""
    import torch
    n = int(A.shape[0])
    _check(_lib.hgmm_pose_compose(n, _need(A, torch.float64, 16 * n, "A"), _need(Bm, torch.float64, 16 * n, "B"),
                                  _need(out, torch.float64, 16 * n, "out"), _stream_ptr(stream)),
           "hgmm_pose_compose")
    return out


def hgmm_debug_gemm(A, a_m: int, a_k: int, B, b_n: int, b_k: int, M: int, N: int, K: int, out,
                    stream=None):
    """out[m, n] = sum_k A[m][k] B[n][k] on the tensor cores; A and B are
    bfloat16 CUDA tensors addressed by element strides."""
    import torch
    _check(_lib.hgmm_debug_gemm(_need(A, torch.bfloat16, 1, "A"), int(a_m), int(a_k),
                                _need(B, torch.bfloat16, 1, "B"), int(b_n), int(b_k), int(M), int(N),
                                int(K), _need(out, torch.float32, M * N, "out"), _stream_ptr(stream)),
           "hgmm_debug_gemm")
    return out


class Mlp:
    """Owns one hgmm_mlp (the proposal network and its training state)."""

    def __init__(self, max_batch: int):
        self.handle = hgmm_mlp_create(max_batch)
        self.max_batch = max_batch

    def close(self):
        if getattr(self, "handle", None):
            hgmm_mlp_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------ flat GMM J=n variant
def hgmm_flat_create(max_points: int, max_components: int) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check(_lib.hgmm_flat_create(int(max_points), int(max_components), ctypes.byref(h)), "hgmm_flat_create")
    return h


def hgmm_flat_destroy(h) -> None:
    _lib.hgmm_flat_destroy(h)


def hgmm_flat_from_tree(h, tree_handle, level: int = -1, stream=None) -> None:
    _check(_lib.hgmm_flat_from_tree(h, tree_handle, int(level), _stream_ptr(stream)), "hgmm_flat_from_tree")


def hgmm_flat_fit(h, points, em_iters: int, n_min: float = 8.0, stream=None) -> None:
    _check(_lib.hgmm_flat_fit(h, _dev_points(points, "points"), points.shape[0], int(em_iters), float(n_min),
                              _stream_ptr(stream)), "hgmm_flat_fit")


def hgmm_flat_register(h, src, T_init=None, iters: int = 30, stream=None, T_out=None, T_hist=None):
    """Returns the device tensor T_out (4x4 float64)."""
    import torch
    if T_out is None:
        T_out = torch.empty((4, 4), dtype=torch.float64, device=src.device)
    for name, x in (("T_init", T_init), ("T_out", T_out), ("T_hist", T_hist)):
        if x is not None and (x.dtype != torch.float64 or not x.is_cuda or not x.is_contiguous()):
            raise ValueError(f"{name}: expected a contiguous float64 CUDA tensor")
    _check(_lib.hgmm_flat_register(h, _dev_points(src, "src"), src.shape[0], _dptr(T_init), int(iters),
                                   _stream_ptr(stream), _dptr(T_out), _dptr(T_hist)), "hgmm_flat_register")
    return T_out


def hgmm_flat_objective(h, out, stream=None):
    _check(_lib.hgmm_flat_objective(h, _dptr(out), _stream_ptr(stream)), "hgmm_flat_objective")
    return out


def hgmm_flat_export(h, cap: int):
    """(J, components (min(J, cap), 10) float64, nodes (min(J, cap), 2) int32)."""
    out = np.zeros((max(cap, 1), 10), np.float64)
    node = np.zeros((max(cap, 1), 2), np.int32)
    J = ctypes.c_int32()
    _check(_lib.hgmm_flat_export(h, out.ctypes.data_as(ctypes.c_void_p), int(cap), ctypes.byref(J),
                                 node.ctypes.data_as(ctypes.c_void_p)), "hgmm_flat_export")
    m = min(J.value, cap)
    return J.value, out[:m], node[:m]


def hgmm_flat_debug_moments(h, cap: int) -> np.ndarray:
    """(min(J, cap), 4) float64: M0, M1 of every component (last round)."""
    out = np.zeros((max(cap, 1), 4), np.float64)
    J = ctypes.c_int32()
    _check(_lib.hgmm_flat_debug_moments(h, out.ctypes.data_as(ctypes.c_void_p), int(cap), ctypes.byref(J)),
           "hgmm_flat_debug_moments")
    return out[:min(J.value, cap)]


def hgmm_flat_sync(h, stream=None) -> None:
    _check(_lib.hgmm_flat_sync(h, _stream_ptr(stream)), "hgmm_flat_sync")


class Flat:
    """Owns one hgmm_flat: the single-level "GMM J=n" model of Sec. 5."""

    def __init__(self, max_points: int, max_components: int):
        self.handle = hgmm_flat_create(max_points, max_components)
        self.max_components = max_components

    def close(self):
        if getattr(self, "handle", None):
            hgmm_flat_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def from_tree(self, tree, level: int = -1, stream=None):
        hgmm_flat_from_tree(self.handle, tree.handle, level, stream)
        return self

    def fit(self, points, em_iters: int, n_min: float = 8.0, stream=None):
        hgmm_flat_fit(self.handle, points, em_iters, n_min, stream)
        return self

    def register(self, src, T_init=None, iters: int = 30, stream=None, T_out=None, T_hist=None):
        return hgmm_flat_register(self.handle, src, T_init, iters, stream, T_out, T_hist)

    def sync(self, stream=None):
        hgmm_flat_sync(self.handle, stream)

    def export(self) -> dict:
        J, a, node = hgmm_flat_export(self.handle, self.max_components)
        S = np.empty((a.shape[0], 3, 3))
        iu = [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]
        for k, (i, j) in enumerate(iu):
            S[:, i, j] = a[:, 4 + k]
            S[:, j, i] = a[:, 4 + k]
        return {"J": J, "pi": a[:, 0], "mu": a[:, 1:4], "Sigma": S, "node": node}

    def moments(self) -> np.ndarray:
        return hgmm_flat_debug_moments(self.handle, self.max_components)


# ---------------------------------------------------------------- convenience
class Tree:
    """Owns one hgmm_tree (device memory sized for max_points / max_depth)."""

    def __init__(self, max_points: int, max_depth: int = 4):
        self.handle = hgmm_tree_create(max_points, max_depth)
        self.max_points = max_points
        self.max_depth = max_depth
        self.n = 0
        self.depth = 0

    def close(self):
        if getattr(self, "handle", None):
            hgmm_tree_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def build(self, points, depth: int, prm: hgmm_params | None = None, stream=None):
        hgmm_build(self.handle, points, depth, HGMM_J, prm, stream)
        self.n, self.depth = int(points.shape[0]), int(depth)
        return self

    def register(self, src, T_init=None, iters: int = 30, lam_c: float = -1.0, stream=None,
                 T_out=None, T_hist=None):
        return hgmm_register(self.handle, src, T_init, iters, lam_c, stream, T_out, T_hist)

    def register_descent(self, src, mode: int, tau: float = 0.0, T_init=None, iters: int = 30,
                         lam_c: float = -1.0, stream=None, T_out=None, T_hist=None, full_eq7: bool = False):
        return hgmm_register_descent(self.handle, src, mode, tau, T_init, iters, lam_c, stream, T_out, T_hist,
                                     full_eq7)

    def sync(self, stream=None):
        hgmm_sync(self.handle, stream)

    def export(self, level: int) -> dict:
        return _node_dict(hgmm_tree_export(self.handle, level, 8 ** (level + 1)))

    def labels(self, level: int) -> np.ndarray:
        return hgmm_debug_labels(self.handle, level, self.n)

    def posteriors(self, level: int) -> np.ndarray:
        return hgmm_debug_posteriors(self.handle, level, self.n)

    def root(self) -> dict:
        return _root_dict(hgmm_debug_root(self.handle))

    def profile(self, enable: bool):
        hgmm_profile(self.handle, enable)

    def profile_read(self) -> dict:
        return hgmm_profile_read(self.handle)

    def reg_moments(self) -> np.ndarray:
        return hgmm_debug_reg_moments(self.handle, hgmm_node_count(self.depth))
