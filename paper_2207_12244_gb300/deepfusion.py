"""Thin ctypes binding of libdeepfusion (include/deepfusion.h).

Argument marshalling only: every step of the solve runs in the CUDA library.
Functions keep the C names. Buffers may be torch tensors (CUDA or CPU,
contiguous) or numpy arrays (host); device-ness is read from the tensor. The
stream defaults to torch's current stream on the tensor's device.

If the compiled library is missing, every call raises: there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import re
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdeepfusion.so")

DF_OK, DF_EINVAL, DF_ENOMEM, DF_EBUDGET, DF_ECUDA, DF_ETIMEOUT, DF_ESTATE, DF_ENOTSUP = range(8)
DF_F32, DF_BF16, DF_F16 = 0, 1, 2
DF_TERM_SEMI, DF_TERM_NET, DF_TERM_GRAD = 1, 2, 4
DF_TERMS_ALL = 7
DF_LOSS_HUBER, DF_LOSS_TUKEY = 0, 1
DF_SOLVER_AUTO, DF_SOLVER_LAUNCHES, DF_SOLVER_FUSED = 0, 1, 2
DF_SCALE_FIXED, DF_SCALE_ALTERNATE, DF_SCALE_JOINT = 0, 1, 2


class df_keyframe_desc(C.Structure):
    _fields_ = [("width", C.c_int32), ("height", C.c_int32), ("cnn_dtype", C.c_int32)]


class df_solve_params(C.Structure):
    _fields_ = [("n_gn", C.c_int32), ("n_pcg", C.c_int32), ("delta", C.c_float),
                ("loss", C.c_int32), ("terms", C.c_int32), ("scale_step", C.c_int32),
                ("solver", C.c_int32), ("tol", C.c_double), ("warm_gn", C.c_int32),
                ("warm_delta", C.c_float)]


class df_solve_report(C.Structure):
    _fields_ = [("scale_log", C.c_double), ("res_norm", C.c_double),
                ("iters_done", C.c_int32), ("flags", C.c_int32)]


class df_tuning(C.Structure):
    _fields_ = [("mode", C.c_int32), ("vec", C.c_int32), ("tile_rows", C.c_int32),
                ("max_ctas", C.c_int32), ("gn_per_launch", C.c_int32),
                ("debug_skip_cta", C.c_int32), ("assembly", C.c_int32)]


DF_MODE_AUTO, DF_MODE_STREAMING, DF_MODE_RESIDENT = 0, 1, 2


class df_server_config(C.Structure):
    _fields_ = [("memory_budget", C.c_size_t), ("max_batch", C.c_int32),
                ("max_inflight", C.c_int32), ("batching", C.c_int32), ("pad", C.c_int32),
                ("params", df_solve_params)]


class df_completion(C.Structure):
    _fields_ = [("tag", C.c_uint64), ("stream_id", C.c_int32), ("status", C.c_int32),
                ("t_submit_ns", C.c_int64), ("t_launch_ns", C.c_int64), ("t_done_ns", C.c_int64),
                ("batch_size", C.c_int32), ("pad", C.c_int32)]


class df_camera(C.Structure):
    _fields_ = [(n, C.c_float) for n in ("fx", "fy", "cx", "cy")]


class df_pose(C.Structure):
    _fields_ = [("R", C.c_float * 9), ("t", C.c_float * 3)]


class df_mvs_params(C.Structure):
    _fields_ = [(n, C.c_float) for n in ("grad_min", "d_min", "d_max", "sigma_range", "ssd_max",
                                         "photo_var")] + [("max_steps", C.c_int32)]


DF_MVS_OK, DF_MVS_FLAT, DF_MVS_INTERVAL, DF_MVS_LINE, DF_MVS_NOSTEP, DF_MVS_SSD, \
    DF_MVS_NEIGHBOUR = range(7)


class DFError(RuntimeError):
    def __init__(self, status: int, where: str, message: str):
        self.status = status
        super().__init__(f"{where}: {_STATUS.get(status, status)}: {message}")


_STATUS = {0: "DF_OK", 1: "DF_EINVAL", 2: "DF_ENOMEM", 3: "DF_EBUDGET", 4: "DF_ECUDA",
           5: "DF_ETIMEOUT", 6: "DF_ESTATE", 7: "DF_ENOTSUP"}

_lib = None


def load(path: Optional[str] = None) -> C.CDLL:
    """Load the compiled library (raises if it has not been built)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"libdeepfusion.so not found at {p}: build it with "
                           "paper_2207_12244_gb300._build.build() (CUDA toolkit required)")
    L = C.CDLL(p)
    vp, i32, st = C.c_void_p, C.c_int32, C.c_int
    L.df_default_params.argtypes = [C.POINTER(df_solve_params)]
    L.df_default_params.restype = None
    L.df_keyframe_create.argtypes = [C.POINTER(df_keyframe_desc)] + [vp] * 6 + [C.c_int, vp,
                                                                              C.POINTER(vp)]
    L.df_keyframe_reset.argtypes = [vp] * 7 + [C.c_int, vp]
    L.df_frame_update.argtypes = [vp, vp, vp, C.c_int, vp]
    L.df_optimise.argtypes = [vp, C.POINTER(df_solve_params), vp, C.POINTER(df_solve_report)]
    L.df_optimise_batch.argtypes = [C.POINTER(vp), i32, C.POINTER(df_solve_params), vp,
                                     C.POINTER(df_solve_report)]
    L.df_fetch_depth.argtypes = [vp, vp, C.c_int, C.c_int, vp]
    L.df_keyframe_get_state.argtypes = [vp, vp, vp, C.c_int, vp]
    L.df_keyframe_set_state.argtypes = [vp, vp, C.c_double, C.c_int, vp]
    L.df_cost.argtypes = [vp, C.POINTER(df_solve_params), vp, C.POINTER(C.c_double)]
    L.df_keyframe_check.argtypes = [vp, vp]
    L.df_scale_fit_ls.argtypes = [vp, vp]
    L.df_depth_accuracy.argtypes = [vp, vp, C.c_int, C.c_double, vp, C.POINTER(C.c_int64),
                                    C.POINTER(C.c_int64)]
    L.df_scale_fit_ls.restype = C.c_int
    L.df_keyframe_info.argtypes = [vp, C.POINTER(df_keyframe_desc), C.POINTER(C.c_size_t)]
    L.df_keyframe_destroy.argtypes = [vp]
    L.df_keyframe_destroy.restype = None
    L.df_keyframe_bytes.argtypes = [i32, i32, i32]
    L.df_keyframe_bytes.restype = C.c_size_t
    L.df_set_memory_budget.argtypes = [C.c_size_t]
    L.df_memory_in_use.argtypes = []
    L.df_memory_in_use.restype = C.c_size_t
    L.df_semi_to_log.argtypes = [vp, vp, vp, vp, C.c_int64, C.c_int, vp]
    L.df_optimise_noalloc.argtypes = [C.c_int32, C.c_int32] + [vp] * 10 + [
        C.POINTER(df_solve_params), vp]
    L.df_optimise_noalloc.restype = C.c_int
    L.df_batch_prepare.argtypes = [C.POINTER(vp), i32, vp]
    L.df_keyframe_reset_batch.argtypes = [C.POINTER(vp), i32, C.POINTER(vp), C.c_int, vp]
    L.df_frame_update_batch.argtypes = [C.POINTER(vp), i32, C.POINTER(vp), C.POINTER(vp),
                                        C.c_int, vp]
    L.df_fetch_depth_batch.argtypes = [C.POINTER(vp), i32, C.POINTER(vp), C.c_int, C.c_int, vp]
    L.df_batch_release.argtypes = [C.POINTER(vp), i32]
    L.df_mvs_default_params.argtypes = [C.POINTER(df_mvs_params)]
    L.df_mvs_default_params.restype = None
    L.df_mvs_create.argtypes = [i32, i32, C.POINTER(vp)]
    L.df_mvs_destroy.argtypes = [vp]
    L.df_mvs_destroy.restype = None
    L.df_mvs_last_steps.argtypes = [vp, vp, C.POINTER(C.c_uint64)]
    L.df_mvs_update.argtypes = [vp, vp, vp, C.POINTER(df_camera), C.POINTER(df_pose),
                                C.POINTER(df_mvs_params), vp, vp, vp, vp, vp]
    L.df_server_create.argtypes = [C.POINTER(df_server_config), C.POINTER(vp)]
    L.df_server_destroy.argtypes = [vp]
    L.df_server_destroy.restype = None
    L.df_server_open_stream.argtypes = [vp, C.POINTER(df_keyframe_desc)] + [vp] * 6 + [
        C.c_int, C.POINTER(C.c_int32)]
    L.df_server_close_stream.argtypes = [vp, C.c_int32]
    L.df_server_submit.argtypes = [vp, C.c_int32, vp, vp, C.c_int, C.c_uint64]
    L.df_server_progress.argtypes = [vp, C.POINTER(df_completion), C.c_int32,
                                     C.POINTER(C.c_int32)]
    L.df_server_pending.argtypes = [vp]
    L.df_server_pending.restype = C.c_int32
    L.df_server_fetch_depth.argtypes = [vp, C.c_int32, vp, C.c_int, C.c_int]
    L.df_server_get_state.argtypes = [vp, C.c_int32, vp, C.POINTER(C.c_double), C.c_int]
    for name in ("df_server_create", "df_server_open_stream", "df_server_close_stream",
                 "df_server_submit", "df_server_progress", "df_server_fetch_depth",
                 "df_server_get_state"):
        getattr(L, name).restype = C.c_int
    L.df_autotune.argtypes = [C.POINTER(vp), C.c_int32, C.POINTER(df_solve_params), vp,
                              C.POINTER(df_tuning), C.POINTER(C.c_float)]
    L.df_autotune.restype = C.c_int
    L.df_set_tuning.argtypes = [C.POINTER(df_tuning)]
    L.df_get_tuning.argtypes = [C.POINTER(df_tuning)]
    L.df_set_spin_limit_ns.argtypes = [C.c_uint64]
    for name in ("df_set_tuning", "df_get_tuning", "df_set_spin_limit_ns"):
        getattr(L, name).restype = C.c_int
    L.df_kernel_launches.argtypes = []
    L.df_kernel_launches.restype = C.c_uint64
    L.df_status_str.argtypes = [st]
    L.df_status_str.restype = C.c_char_p
    L.df_last_error.argtypes = []
    L.df_last_error.restype = C.c_char_p
    for name in ("df_keyframe_create", "df_keyframe_reset", "df_frame_update", "df_optimise",
                 "df_optimise_batch", "df_fetch_depth", "df_keyframe_get_state",
                 "df_keyframe_set_state", "df_cost", "df_keyframe_check", "df_keyframe_info",
                 "df_set_memory_budget", "df_semi_to_log", "df_keyframe_reset_batch",
                 "df_frame_update_batch", "df_fetch_depth_batch"):
        getattr(L, name).restype = st
    if path is None:
        _lib = L
    return L


def header_functions(header: Optional[str] = None) -> list:
    """Names of the functions declared in include/deepfusion.h."""
    h = header or os.path.join(os.path.dirname(_HERE), "include", "deepfusion.h")
    text = open(h).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(df_[a-z0-9_]+)\s*\(", text)))


def _check(status: int, where: str):
    if status != DF_OK:
        msg = load().df_last_error().decode(errors="replace")
        raise DFError(status, where, msg)


# ---- buffer marshalling ---------------------------------------------------

def _is_torch(a) -> bool:
    return type(a).__module__.startswith("torch")


def _ptr(a, want_device: Optional[bool] = None):
    """(pointer, on_device) of a contiguous tensor / array."""
    if a is None:
        return None, False
    if _is_torch(a):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr(), bool(a.is_cuda)
    if isinstance(a, np.ndarray):
        if not a.flags.c_contiguous:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data, False
    raise TypeError(f"unsupported buffer type {type(a)}")


def _stream(stream, like=None):
    """The cudaStream_t to pass: the given one, else torch's current stream
    (on the tensor's device if one is given), else the legacy default."""
    if stream is not None:
        if isinstance(stream, int):
            return stream
        return int(getattr(stream, "cuda_stream", stream))
    try:
        import torch
    except ImportError:
        return 0
    if like is not None and _is_torch(like) and like.is_cuda:
        return torch.cuda.current_stream(like.device).cuda_stream
    if torch.cuda.is_available() and torch.cuda.is_initialized():
        return torch.cuda.current_stream().cuda_stream
    return 0


def _same_side(bufs: Sequence, where: str) -> int:
    sides = {_ptr(b)[1] for b in bufs if b is not None}
    if len(sides) > 1:
        raise ValueError(f"{where}: mix of host and device buffers")
    return int(sides.pop()) if sides else 0


def _dtype_code(a) -> int:
    if _is_torch(a):
        import torch
        return {torch.float32: DF_F32, torch.bfloat16: DF_BF16, torch.float16: DF_F16}[a.dtype]
    if a.dtype == np.float32:
        return DF_F32
    if a.dtype == np.float16:
        return DF_F16
    raise ValueError("numpy network planes must be float32 or float16 "
                     "(pass bf16 as a torch.bfloat16 tensor or set cnn_dtype explicitly)")


# ---- entry points ---------------------------------------------------------

def df_default_params(**overrides) -> df_solve_params:
    p = df_solve_params()
    load().df_default_params(C.byref(p))
    for k, v in overrides.items():
        if not hasattr(p, k):
            raise AttributeError(k)
        setattr(p, k, v)
    return p


def df_keyframe_create(width: int, height: int, mu_net, var_net, gx, var_gx, gy, var_gy,
                       cnn_dtype: Optional[int] = None, stream=None) -> C.c_void_p:
    planes = [mu_net, var_net, gx, var_gx, gy, var_gy]
    on_dev = _same_side(planes, "df_keyframe_create")
    for p in planes:
        if _numel(p) != width * height:
            raise ValueError("network plane size != width*height")
    dt = _dtype_code(mu_net) if cnn_dtype is None else cnn_dtype
    desc = df_keyframe_desc(width, height, dt)
    out = C.c_void_p()
    _check(load().df_keyframe_create(C.byref(desc), *[_ptr(p)[0] for p in planes], on_dev,
                                     _stream(stream, mu_net), C.byref(out)), "df_keyframe_create")
    return out


def df_keyframe_reset(kf, mu_net, var_net, gx, var_gx, gy, var_gy, stream=None):
    planes = [mu_net, var_net, gx, var_gx, gy, var_gy]
    on_dev = _same_side(planes, "df_keyframe_reset")
    _check(load().df_keyframe_reset(kf, *[_ptr(p)[0] for p in planes], on_dev,
                                    _stream(stream, mu_net)), "df_keyframe_reset")


def df_frame_update(kf, mu_semi, var_semi, stream=None):
    """The frame's semi-dense log-depth and variance (H x W float32), both on
    the host or both on the device. Host buffers must already hold the data
    (they may be read before the stream reaches the call) and stay unchanged
    until the stream has passed it."""
    on_dev = _same_side([mu_semi, var_semi], "df_frame_update")
    _check(load().df_frame_update(kf, _ptr(mu_semi)[0], _ptr(var_semi)[0], on_dev,
                                  _stream(stream, mu_semi)), "df_frame_update")


def df_optimise(kf, params: Optional[df_solve_params] = None, stream=None,
                report: bool = False) -> Optional[df_solve_report]:
    rep = df_solve_report() if report else None
    _check(load().df_optimise(kf, C.byref(params) if params is not None else None,
                              _stream(stream), C.byref(rep) if report else None), "df_optimise")
    return rep


def df_optimise_batch(kfs: Sequence, params: Optional[df_solve_params] = None, stream=None,
                      report: bool = False):
    n = len(kfs)
    arr = (C.c_void_p * max(n, 1))(*[k.value if isinstance(k, C.c_void_p) else k for k in kfs])
    reps = (df_solve_report * max(n, 1))() if report else None
    _check(load().df_optimise_batch(arr, n, C.byref(params) if params is not None else None,
                                    _stream(stream), reps), "df_optimise_batch")
    return list(reps)[:n] if report else None


def _kf_array(kfs):
    n = len(kfs)
    return (C.c_void_p * max(n, 1))(*[k.value if isinstance(k, C.c_void_p) else k for k in kfs]), n


def df_batch_prepare(kfs: Sequence, stream=None):
    """Keep the launch plans of this keyframe list (for repeated batched
    solves and CUDA graph capture)."""
    arr, n = _kf_array(kfs)
    _check(load().df_batch_prepare(arr, n, _stream(stream)), "df_batch_prepare")


def df_batch_release(kfs: Sequence):
    arr, n = _kf_array(kfs)
    _check(load().df_batch_release(arr, n), "df_batch_release")


def _batch_buffers(kfs, lists, where: str, per_kf_dtype: bool):
    """Check that every buffer of a batched call has its keyframe's W*H
    elements (and, for torch tensors, the element type the call reads), all
    on one side; returns (keyframe array, n, pointer array, on_device)."""
    arr, n = _kf_array(kfs)
    flat = []
    for j, k in enumerate(kfs):
        W, H, dt, _ = df_keyframe_info(k)
        want = {DF_F32: 4, DF_BF16: 2, DF_F16: 2}[dt] if per_kf_dtype else 4
        for b in lists[j]:
            if b is None:
                raise ValueError(f"{where}: buffer of keyframe {j} is None")
            if _numel(b) != W * H:
                raise ValueError(f"{where}: buffer of keyframe {j} has {_numel(b)} elements, "
                                 f"not {W} x {H}")
            size = b.element_size() if _is_torch(b) else b.itemsize
            if size != want:
                raise ValueError(f"{where}: buffer of keyframe {j} has {size}-byte elements, "
                                 f"the keyframe needs {want}")
            flat.append(b)
    on_dev = _same_side(flat, where)
    ptrs = (C.c_void_p * max(len(flat), 1))(*[_ptr(b)[0] for b in flat])
    return arr, n, ptrs, on_dev, flat


def df_keyframe_reset_batch(kfs: Sequence, planes: Sequence[Sequence], stream=None):
    """df_keyframe_reset of every keyframe in one or two device passes per 24
    keyframes: planes[j] = the six network planes of keyframe j."""
    arr, n, ptrs, on_dev, flat = _batch_buffers(kfs, planes, "df_keyframe_reset_batch", True)
    _check(load().df_keyframe_reset_batch(arr, n, ptrs, on_dev,
                                          _stream(stream, flat[0] if flat else None)),
           "df_keyframe_reset_batch")


def df_frame_update_batch(kfs: Sequence, mu_semi: Sequence, var_semi: Sequence, stream=None):
    """df_frame_update of every keyframe in one device pass per 24 keyframes."""
    arr, n, ptrs, on_dev, flat = _batch_buffers(
        kfs, [[m, v] for m, v in zip(mu_semi, var_semi)], "df_frame_update_batch", False)
    if len(mu_semi) != n or len(var_semi) != n:
        raise ValueError("df_frame_update_batch: one mu_semi and one var_semi per keyframe")
    mu = (C.c_void_p * max(n, 1))(*[ptrs[2 * j] for j in range(n)])
    var = (C.c_void_p * max(n, 1))(*[ptrs[2 * j + 1] for j in range(n)])
    _check(load().df_frame_update_batch(arr, n, mu, var, on_dev,
                                        _stream(stream, flat[0] if flat else None)),
           "df_frame_update_batch")


def df_fetch_depth_batch(kfs: Sequence, outs: Sequence, log_space: bool = False, stream=None):
    """df_fetch_depth of every keyframe in one device pass per 24 keyframes."""
    arr, n, ptrs, on_dev, flat = _batch_buffers(kfs, [[o] for o in outs], "df_fetch_depth_batch",
                                                False)
    if len(outs) != n:
        raise ValueError("df_fetch_depth_batch: one output per keyframe")
    _check(load().df_fetch_depth_batch(arr, n, ptrs, int(log_space), on_dev,
                                       _stream(stream, flat[0] if flat else None)),
           "df_fetch_depth_batch")
    return outs


def df_fetch_depth(kf, out, log_space: bool = False, stream=None):
    p, dev = _ptr(out)
    _check(load().df_fetch_depth(kf, p, int(log_space), int(dev), _stream(stream, out)),
           "df_fetch_depth")
    return out


def df_keyframe_get_state(kf, x_out=None, stream=None) -> float:
    p, dev = _ptr(x_out)
    t = C.c_double(0.0)
    _check(load().df_keyframe_get_state(kf, p, C.addressof(t), 0, _stream(stream, x_out)),
           "df_keyframe_get_state")
    return t.value


def df_keyframe_set_state(kf, x=None, t: float = 0.0, stream=None):
    p, dev = _ptr(x)
    _check(load().df_keyframe_set_state(kf, p, float(t), int(dev), _stream(stream, x)),
           "df_keyframe_set_state")


def df_cost(kf, params: Optional[df_solve_params] = None, stream=None) -> float:
    c = C.c_double(0.0)
    _check(load().df_cost(kf, C.byref(params) if params is not None else None, _stream(stream),
                          C.byref(c)), "df_cost")
    return c.value


def df_scale_fit_ls(kf, stream=None):
    _check(load().df_scale_fit_ls(kf, _stream(stream)), "df_scale_fit_ls")


def df_depth_accuracy(kf, depth_true, rel_tol: float = 0.1, stream=None):
    """(n_within, n_valid): pixels whose depth is within rel_tol of the truth
    (Section III-B's accuracy measure) and pixels with a valid truth."""
    p, dev = _ptr(depth_true)
    a, b = C.c_int64(0), C.c_int64(0)
    _check(load().df_depth_accuracy(kf, p, int(dev), float(rel_tol), _stream(stream, depth_true),
                                    C.byref(a), C.byref(b)), "df_depth_accuracy")
    return a.value, b.value


def df_keyframe_check(kf, stream=None):
    _check(load().df_keyframe_check(kf, _stream(stream)), "df_keyframe_check")


def df_keyframe_info(kf):
    d = df_keyframe_desc()
    n = C.c_size_t(0)
    _check(load().df_keyframe_info(kf, C.byref(d), C.byref(n)), "df_keyframe_info")
    return d.width, d.height, d.cnn_dtype, n.value


def df_keyframe_destroy(kf):
    load().df_keyframe_destroy(kf)


def df_keyframe_bytes(width: int, height: int, cnn_dtype: int = DF_F32) -> int:
    return int(load().df_keyframe_bytes(width, height, cnn_dtype))


def df_set_memory_budget(nbytes: int):
    _check(load().df_set_memory_budget(int(nbytes)), "df_set_memory_budget")


def df_memory_in_use() -> int:
    return int(load().df_memory_in_use())


def df_semi_to_log(depth, var_depth, mu_out, var_out, stream=None):
    on_dev = _same_side([depth, var_depth, mu_out, var_out], "df_semi_to_log")
    _check(load().df_semi_to_log(_ptr(depth)[0], _ptr(var_depth)[0], _ptr(mu_out)[0],
                                 _ptr(var_out)[0], _numel(depth), on_dev, _stream(stream, depth)),
           "df_semi_to_log")


DF_NOALLOC_MAX_PIXELS = 196608


def df_server_create(memory_budget: int = 0, max_batch: int = 64, max_inflight: int = 2,
                     batching: bool = True, params: Optional[df_solve_params] = None):
    cfg = df_server_config(int(memory_budget), int(max_batch), int(max_inflight),
                           1 if batching else 0, 0, params or df_default_params())
    out = C.c_void_p()
    _check(load().df_server_create(C.byref(cfg), C.byref(out)), "df_server_create")
    return out


def df_server_destroy(srv):
    load().df_server_destroy(srv)


def df_server_open_stream(srv, width, height, mu_net, var_net, gx, var_gx, gy, var_gy,
                          cnn_dtype: Optional[int] = None) -> int:
    planes = [mu_net, var_net, gx, var_gx, gy, var_gy]
    on_dev = _same_side(planes, "df_server_open_stream")
    dt = _dtype_code(mu_net) if cnn_dtype is None else cnn_dtype
    desc = df_keyframe_desc(width, height, dt)
    sid = C.c_int32(-1)
    _check(load().df_server_open_stream(srv, C.byref(desc), *[_ptr(p)[0] for p in planes],
                                        on_dev, C.byref(sid)), "df_server_open_stream")
    return sid.value


def df_server_close_stream(srv, sid: int):
    _check(load().df_server_close_stream(srv, int(sid)), "df_server_close_stream")


def df_server_submit(srv, sid: int, mu_semi, var_semi, tag: int):
    on_dev = _same_side([mu_semi, var_semi], "df_server_submit")
    _check(load().df_server_submit(srv, int(sid), _ptr(mu_semi)[0], _ptr(var_semi)[0], on_dev,
                                   int(tag)), "df_server_submit")


def df_server_progress(srv, cap: int = 256):
    buf = (df_completion * cap)()
    n = C.c_int32(0)
    _check(load().df_server_progress(srv, buf, cap, C.byref(n)), "df_server_progress")
    return [buf[i] for i in range(n.value)]


def df_server_pending(srv) -> int:
    return int(load().df_server_pending(srv))


def df_server_fetch_depth(srv, sid: int, out, log_space: bool = False):
    p, dev = _ptr(out)
    _check(load().df_server_fetch_depth(srv, int(sid), p, int(log_space), int(dev)),
           "df_server_fetch_depth")
    return out


def df_server_get_state(srv, sid: int, x_out=None) -> float:
    """The stream's log scale t; its log-depth x goes to x_out if given
    (host or device, H x W float32)."""
    p, dev = _ptr(x_out)
    t = C.c_double(0.0)
    _check(load().df_server_get_state(srv, int(sid), p, C.byref(t), int(dev)),
           "df_server_get_state")
    return t.value


_NOALLOC_PLANES = ("mu_net", "var_net", "gx", "var_gx", "gy", "var_gy", "mu_semi", "var_semi",
                   "x_inout")


def _noalloc_check(width: int, height: int, bufs) -> None:
    """Refuse buffers df_optimise_noalloc would read or write out of bounds:
    the nine planes float32 with at least width*height elements, the scale a
    float64 tensor with at least one element, every buffer a contiguous CUDA
    tensor, all on one device. Metadata only: nothing is launched."""
    import torch

    n = int(width) * int(height)
    planes, scale = bufs[:9], bufs[9]
    if any(b is None for b in planes[:6]) or planes[8] is None or scale is None:
        raise ValueError("df_optimise_noalloc: the network planes, x_inout and scale_log_inout "
                         "are required")
    if (planes[6] is None) != (planes[7] is None):
        raise ValueError("df_optimise_noalloc: mu_semi and var_semi go together")
    named = [(nm, b) for nm, b in zip(_NOALLOC_PLANES, planes) if b is not None]
    for nm, b in named + [("scale_log_inout", scale)]:
        if not isinstance(b, torch.Tensor):
            raise TypeError(f"df_optimise_noalloc: {nm} must be a torch tensor")
        if not b.is_contiguous():
            raise ValueError(f"df_optimise_noalloc: {nm} must be contiguous")
    for nm, b in named:
        if b.dtype != torch.float32:
            raise ValueError(f"df_optimise_noalloc: {nm} must be float32, not {b.dtype}")
        if b.numel() < n:
            raise ValueError(f"df_optimise_noalloc: {nm} holds {b.numel()} elements, "
                             f"fewer than {width} x {height}")
    if scale.dtype != torch.float64 or scale.numel() < 1:
        raise ValueError("df_optimise_noalloc: scale_log_inout must be a float64 tensor with "
                         "at least one element")
    devs = {b.device for _, b in named} | {scale.device}
    if any(d.type != "cuda" for d in devs):
        raise ValueError("df_optimise_noalloc takes device buffers only")
    if len(devs) != 1:
        raise ValueError("df_optimise_noalloc: every buffer must be on one device")


def df_optimise_noalloc(width: int, height: int, mu_net, var_net, gx, var_gx, gy, var_gy,
                        mu_semi, var_semi, x_inout, scale_log_inout,
                        params: Optional[df_solve_params] = None, stream=None):
    """The solve without device allocation: every buffer is the caller's
    (contiguous CUDA tensors on one device: nine float32 planes of at least
    width*height elements, scale_log_inout a float64 tensor of one element).
    The call runs with that device current, on its current stream unless
    'stream' is given."""
    import torch

    bufs = [mu_net, var_net, gx, var_gx, gy, var_gy, mu_semi, var_semi, x_inout, scale_log_inout]
    _noalloc_check(width, height, bufs)
    ptrs = [None if b is None else b.data_ptr() for b in bufs]
    with torch.cuda.device(x_inout.device):
        _check(load().df_optimise_noalloc(int(width), int(height), *ptrs,
                                          C.byref(params) if params is not None else None,
                                          _stream(stream, x_inout)), "df_optimise_noalloc")


def df_set_tuning(mode: int = 0, vec: int = 0, tile_rows: int = 0, max_ctas: int = 0,
                  debug_skip_cta: int = -1, gn_per_launch: int = 0, assembly: int = 0):
    t = df_tuning(mode, vec, tile_rows, max_ctas, gn_per_launch, debug_skip_cta, assembly)
    _check(load().df_set_tuning(C.byref(t)), "df_set_tuning")


def df_autotune(kfs: Sequence, params: Optional[df_solve_params] = None, stream=None):
    """Time the fused solver's launch shapes on these keyframes; the fastest
    becomes current. Returns (df_tuning, ms per solve)."""
    n = len(kfs)
    arr = (C.c_void_p * max(n, 1))(*[k.value if isinstance(k, C.c_void_p) else k for k in kfs])
    best = df_tuning()
    ms = C.c_float(0.0)
    _check(load().df_autotune(arr, n, C.byref(params) if params is not None else None,
                              _stream(stream), C.byref(best), C.byref(ms)), "df_autotune")
    return best, ms.value


def df_get_tuning() -> df_tuning:
    t = df_tuning()
    _check(load().df_get_tuning(C.byref(t)), "df_get_tuning")
    return t


def df_set_spin_limit_ns(ns: int):
    _check(load().df_set_spin_limit_ns(int(ns)), "df_set_spin_limit_ns")


def df_kernel_launches() -> int:
    return int(load().df_kernel_launches())


def df_status_str(s: int) -> str:
    return load().df_status_str(s).decode()


def df_last_error() -> str:
    return load().df_last_error().decode(errors="replace")


def _numel(a) -> int:
    return int(a.numel()) if _is_torch(a) else int(a.size)


def df_mvs_default_params(**overrides) -> df_mvs_params:
    p = df_mvs_params()
    load().df_mvs_default_params(C.byref(p))
    for k, v in overrides.items():
        if not hasattr(p, k):
            raise AttributeError(k)
        setattr(p, k, v)
    return p


def df_mvs_create(width: int, height: int) -> C.c_void_p:
    out = C.c_void_p()
    _check(load().df_mvs_create(int(width), int(height), C.byref(out)), "df_mvs_create")
    return out


def df_mvs_destroy(m):
    load().df_mvs_destroy(m)


def df_mvs_update(m, img_key, img_ref, cam, R, t, depth, var, status=None, best_step=None,
                  params: Optional[df_mvs_params] = None, stream=None):
    """One stereo update (Section II-B) of depth / var in place; all planes
    are contiguous H x W device tensors (status / best_step int32, optional)."""
    c = df_camera(*[float(v) for v in cam])
    pose = df_pose((C.c_float * 9)(*[float(v) for v in np.asarray(R, np.float64).ravel()]),
                   (C.c_float * 3)(*[float(v) for v in np.asarray(t, np.float64).ravel()]))
    ptrs = []
    for a in (img_key, img_ref, depth, var, status, best_step):
        p, dev = _ptr(a)
        if a is not None and not dev:
            raise ValueError("df_mvs_update takes device buffers")
        ptrs.append(p)
    _check(load().df_mvs_update(m, ptrs[0], ptrs[1], C.byref(c), C.byref(pose),
                                C.byref(params) if params is not None else None, ptrs[2],
                                ptrs[3], ptrs[4], ptrs[5], _stream(stream, depth)),
           "df_mvs_update")


def df_mvs_last_steps(m, stream=None) -> int:
    n = C.c_uint64(0)
    _check(load().df_mvs_last_steps(m, _stream(stream), C.byref(n)), "df_mvs_last_steps")
    return n.value


class SemiDense:
    """Owner of a df_mvs work space for images of one size."""

    def __init__(self, width: int, height: int):
        self.width, self.height = width, height
        self.handle = df_mvs_create(width, height)

    def update(self, img_key, img_ref, cam, R, t, depth, var, status=None, best_step=None,
               params=None, stream=None):
        df_mvs_update(self.handle, img_key, img_ref, cam, R, t, depth, var, status, best_step,
                      params, stream)

    def last_steps(self, stream=None) -> int:
        return df_mvs_last_steps(self.handle, stream)

    def close(self):
        if self.handle is not None and self.handle.value:
            df_mvs_destroy(self.handle)
        self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Keyframe:
    """Owning handle around a df_keyframe (calls the entry points above)."""

    def __init__(self, width, height, mu_net, var_net, gx, var_gx, gy, var_gy,
                 cnn_dtype=None, stream=None):
        self.width, self.height = width, height
        self.handle = df_keyframe_create(width, height, mu_net, var_net, gx, var_gx, gy, var_gy,
                                         cnn_dtype, stream)

    def reset(self, *planes, stream=None):
        df_keyframe_reset(self.handle, *planes, stream=stream)

    def frame_update(self, mu_semi, var_semi, stream=None):
        df_frame_update(self.handle, mu_semi, var_semi, stream)

    def optimise(self, params=None, stream=None, report=False):
        return df_optimise(self.handle, params, stream, report)

    def fetch_depth(self, out, log_space=False, stream=None):
        return df_fetch_depth(self.handle, out, log_space, stream)

    def get_state(self, x_out=None, stream=None):
        return df_keyframe_get_state(self.handle, x_out, stream)

    def set_state(self, x=None, t=0.0, stream=None):
        df_keyframe_set_state(self.handle, x, t, stream)

    def cost(self, params=None, stream=None):
        return df_cost(self.handle, params, stream)

    def check(self, stream=None):
        df_keyframe_check(self.handle, stream)

    def scale_fit_ls(self, stream=None):
        df_scale_fit_ls(self.handle, stream)

    def depth_accuracy(self, depth_true, rel_tol=0.1, stream=None):
        return df_depth_accuracy(self.handle, depth_true, rel_tol, stream)

    def close(self):
        if self.handle is not None and self.handle.value:
            df_keyframe_destroy(self.handle)
        self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
