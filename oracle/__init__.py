"""FP64 CPU oracle for DeepFusion's keyframe optimisation -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline /
reference leg may import this package. The product path (the CUDA library and
its Python binding) never loads it and shares no code with it.

The arithmetic lives in ``df_oracle.c`` (plain C, FP64, single thread,
compiled without FMA contraction). This wrapper only compiles it with gcc,
loads it with ctypes and converts numpy arrays to float64.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from dataclasses import dataclass
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "df_oracle.c")
_SRCS = [_SRC, os.path.join(_HERE, "df_mvs.c")]
_BUILD = os.path.join(_HERE, "_build")
_LOCK = threading.Lock()

TERM_SEMI, TERM_NET, TERM_GRAD = 1, 2, 4
TERMS_ALL = TERM_SEMI | TERM_NET | TERM_GRAD
LOSS_HUBER, LOSS_TUKEY = 0, 1
SCALE_FIXED, SCALE_ALTERNATE, SCALE_JOINT = 0, 1, 2
HUBER_DELTA = 1.345


class _Problem(C.Structure):
    _fields_ = [("width", C.c_int32), ("height", C.c_int32)] + [
        (n, C.POINTER(C.c_double))
        for n in ("mu_n", "var_n", "gx", "var_gx", "gy", "var_gy", "mu_s", "var_s")
    ]


class _Camera(C.Structure):
    _fields_ = [(n, C.c_double) for n in ("fx", "fy", "cx", "cy")]


class _Pose(C.Structure):
    _fields_ = [("R", C.c_double * 9), ("t", C.c_double * 3)]


class _MvsParams(C.Structure):
    _fields_ = [(n, C.c_double) for n in ("grad_min", "d_min", "d_max", "sigma_range",
                                           "ssd_max", "photo_var")] + [("max_steps", C.c_int32)]


MVS_DEFAULTS = dict(grad_min=20.0, d_min=0.3, d_max=10.0, sigma_range=2.0, ssd_max=5 * 20.0 ** 2,
                    photo_var=1.0, max_steps=512)
MVS_OK, MVS_FLAT, MVS_INTERVAL, MVS_LINE, MVS_NOSTEP, MVS_SSD, MVS_NEIGHBOUR = range(7)


class _Params(C.Structure):
    _fields_ = [("n_gn", C.c_int32), ("n_pcg", C.c_int32), ("delta", C.c_double),
                ("tol", C.c_double), ("terms", C.c_int32), ("loss", C.c_int32),
                ("scale_step", C.c_int32), ("warm_gn", C.c_int32), ("warm_delta", C.c_double)]


class _Report(C.Structure):
    _fields_ = [("scale_log", C.c_double), ("res_norm", C.c_double),
                ("iters_done", C.c_int32)]


@dataclass
class Report:
    scale_log: float
    res_norm: float
    iters_done: int


def build(mutant: int = 0, force: bool = False) -> str:
    """Compile the oracle (or a planted-mistake variant) and return the .so path."""
    os.makedirs(_BUILD, exist_ok=True)
    name = "liboracle.so" if mutant == 0 else f"liboracle_m{mutant}.so"
    out = os.path.join(_BUILD, name)
    with _LOCK:
        newest = max(os.path.getmtime(p) for p in _SRCS)
        if force or not os.path.exists(out) or os.path.getmtime(out) < newest:
            tmp = out + f".{os.getpid()}.tmp"
            cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                   f"-DORC_MUTANT={int(mutant)}", *_SRCS, "-o", tmp, "-lm"]
            subprocess.run(cmd, check=True)
            os.replace(tmp, out)
    return out


def _dp(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64)).ravel()


class Oracle:
    """ctypes front end of one compiled oracle library."""

    def __init__(self, path: Optional[str] = None):
        self.path = path or build()
        L = C.CDLL(self.path)
        P, D, I = C.POINTER(_Problem), C.POINTER(C.c_double), C.c_int32
        L.orc_rho.restype = C.c_double
        L.orc_rho.argtypes = [C.c_double, C.c_double, I]
        L.orc_omega.restype = C.c_double
        L.orc_omega.argtypes = [C.c_double, C.c_double, I]
        L.orc_cost.restype = C.c_double
        L.orc_cost.argtypes = [P, D, C.c_double, C.c_double, I, I]
        L.orc_scale_step.restype = C.c_double
        L.orc_scale_step.argtypes = [P, D, C.c_double, C.c_double, I]
        L.orc_assemble.restype = None
        L.orc_assemble.argtypes = [P, D, C.c_double, C.c_double, I, I, D, D, D, D]
        L.orc_apply.restype = None
        L.orc_apply.argtypes = [I, I, D, D, D, D, D]
        L.orc_pcg.restype = I
        L.orc_pcg.argtypes = [I, I, D, D, D, D, D, I, C.c_double, D]
        L.orc_optimise.restype = I
        L.orc_optimise.argtypes = [P, D, D, C.POINTER(_Params), C.POINTER(_Report), D]
        L.orc_depth.restype = None
        L.orc_depth.argtypes = [C.c_int64, D, D]
        L.orc_semi_to_log.restype = None
        L.orc_semi_to_log.argtypes = [C.c_int64, D, D, D, D]
        L.orc_ls_scale_fit.restype = None
        L.orc_ls_scale_fit.argtypes = [P, D, D]
        L.orc_semi_dense.restype = C.c_int64
        L.orc_semi_dense.argtypes = [I, I, C.POINTER(C.c_float), C.POINTER(C.c_float),
                                     C.POINTER(_Camera), C.POINTER(_Pose), C.POINTER(_MvsParams),
                                     D, D, C.POINTER(C.c_int32), C.POINTER(C.c_int32), D]
        L.orc_within.restype = None
        L.orc_within.argtypes = [C.c_int64, D, D, C.c_double, C.POINTER(C.c_int64),
                                 C.POINTER(C.c_int64)]
        self.lib = L

    # -- problem marshalling ------------------------------------------------
    def _problem(self, kf, semi: bool = True):
        W, H = int(kf.width), int(kf.height)
        keep = [_f64(getattr(kf, n)) for n in ("mu_n", "var_n", "gx", "var_gx", "gy", "var_gy")]
        ms = getattr(kf, "mu_s", None) if semi else None
        vs = getattr(kf, "var_s", None) if semi else None
        if ms is not None and vs is not None:
            keep += [_f64(ms), _f64(vs)]
        for a in keep:
            if a.size != W * H:
                raise ValueError("plane size does not match width*height")
        ptrs = [_dp(a) for a in keep] + [None] * (8 - len(keep))
        prob = _Problem(W, H, *ptrs)
        return prob, keep

    # -- elementary pieces ---------------------------------------------------
    def rho(self, u: float, delta: float, loss: int = LOSS_HUBER) -> float:
        return self.lib.orc_rho(float(u), float(delta), int(loss))

    def omega(self, u: float, delta: float, loss: int = LOSS_HUBER) -> float:
        return self.lib.orc_omega(float(u), float(delta), int(loss))

    def cost(self, kf, x, t: float, delta: float = HUBER_DELTA, terms: int = TERMS_ALL,
             loss: int = LOSS_HUBER) -> float:
        prob, keep = self._problem(kf)
        xx = _f64(x)
        return self.lib.orc_cost(C.byref(prob), _dp(xx), float(t), float(delta), int(terms), int(loss))

    def scale_step(self, kf, x, t: float, delta: float = HUBER_DELTA, loss: int = LOSS_HUBER) -> float:
        prob, keep = self._problem(kf)
        xx = _f64(x)
        return self.lib.orc_scale_step(C.byref(prob), _dp(xx), float(t), float(delta), int(loss))

    def assemble(self, kf, x, t: float, delta: float = HUBER_DELTA, terms: int = TERMS_ALL,
                 loss: int = LOSS_HUBER):
        prob, keep = self._problem(kf)
        N = kf.width * kf.height
        xx = _f64(x)
        out = [np.zeros(N) for _ in range(4)]
        self.lib.orc_assemble(C.byref(prob), _dp(xx), float(t), float(delta), int(terms),
                              int(loss), *[_dp(a) for a in out])
        return tuple(out)  # diag, wx, wy, b

    def apply(self, W: int, H: int, diag, wx, wy, p) -> np.ndarray:
        d, a, b_, pp = _f64(diag), _f64(wx), _f64(wy), _f64(p)
        q = np.zeros(W * H)
        self.lib.orc_apply(W, H, _dp(d), _dp(a), _dp(b_), _dp(pp), _dp(q))
        return q

    def pcg(self, W: int, H: int, diag, wx, wy, b, x0, n_pcg: int, tol: float = 0.0):
        d, a, c, bb = _f64(diag), _f64(wx), _f64(wy), _f64(b)
        x = _f64(x0).copy()
        rn = C.c_double(0.0)
        it = self.lib.orc_pcg(W, H, _dp(d), _dp(a), _dp(c), _dp(bb), _dp(x), int(n_pcg),
                              float(tol), C.byref(rn))
        return x, int(it), rn.value

    # -- the per-frame solve -------------------------------------------------
    def optimise(self, kf, x0=None, t0: float = 0.0, n_gn: int = 10, n_pcg: int = 3,
                 delta: float = HUBER_DELTA, tol: float = 0.0, terms: int = TERMS_ALL,
                 loss: int = LOSS_HUBER, scale_step: int = SCALE_ALTERNATE, trace: bool = False,
                 warm_gn: int = 0, warm_delta: float = HUBER_DELTA):
        """Run the schedule from (x0, t0); x0 defaults to mu_n (keyframe init).

        scale_step: SCALE_FIXED (t kept), SCALE_ALTERNATE (scale half, then
        depth half, per GN iteration) or SCALE_JOINT (bordered PCG in (x, t));
        True / False mean SCALE_ALTERNATE / SCALE_FIXED.
        warm_gn: the first warm_gn GN iterations use the Huber loss with
        threshold warm_delta, the others ``loss`` with ``delta``. The cost
        trace is always the cost of ``loss`` with ``delta``.

        Returns (x [H, W] float64, t, Report[, cost trace of 2*n_gn+1 values]).
        """
        prob, keep = self._problem(kf)
        x = _f64(kf.mu_n if x0 is None else x0).copy()
        t = C.c_double(float(t0))
        prm = _Params(int(n_gn), int(n_pcg), float(delta), float(tol), int(terms),
                      int(loss), int(scale_step), int(warm_gn), float(warm_delta))
        rep = _Report()
        tr = np.zeros(2 * int(n_gn) + 1) if trace else None
        self.lib.orc_optimise(C.byref(prob), _dp(x), C.byref(t), C.byref(prm), C.byref(rep),
                              _dp(tr) if trace else None)
        out = (x.reshape(kf.height, kf.width), t.value,
               Report(rep.scale_log, rep.res_norm, rep.iters_done))
        return out + (tr,) if trace else out

    def optimise_sequence(self, kf, mu_s_frames, var_s_frames, n_gn: int = 10, n_pcg: int = 5,
                          delta: float = HUBER_DELTA, frames=None,
                          scale_step: int = SCALE_ALTERNATE):
        """Warm-started per-frame re-optimisation (Section II, every new frame).

        Returns the (x, t) after the last processed frame.
        """
        class _KF:  # a view with the frame's semi-dense planes swapped in
            pass
        v = _KF()
        for n in ("width", "height", "mu_n", "var_n", "gx", "var_gx", "gy", "var_gy"):
            setattr(v, n, getattr(kf, n))
        x = _f64(kf.mu_n).copy()
        t = 0.0
        idx = range(len(mu_s_frames)) if frames is None else frames
        for f in idx:
            v.mu_s, v.var_s = mu_s_frames[f], var_s_frames[f]
            x, t, _ = self.optimise(v, x0=x, t0=t, n_gn=n_gn, n_pcg=n_pcg, delta=delta,
                                    scale_step=scale_step)
            x = x.ravel()
        return x.reshape(kf.height, kf.width), t

    def semi_dense(self, img_key, img_ref, cam, R, t, depth=None, var=None, **params):
        """One stereo update (Section II-B). Returns (depth, var, status,
        best_step, margin, n_measured); depth / var start from the given
        estimate (None: no estimate anywhere)."""
        H, W = np.shape(img_key)
        ik = np.ascontiguousarray(img_key, dtype=np.float32)
        ir = np.ascontiguousarray(img_ref, dtype=np.float32)
        d = np.zeros(H * W) if depth is None else _f64(depth).copy()
        vv = np.zeros(H * W) if var is None else _f64(var).copy()
        st = np.zeros(H * W, np.int32)
        bs = np.zeros(H * W, np.int32)
        mg = np.zeros(H * W)
        p = dict(MVS_DEFAULTS)
        p.update(params)
        prm = _MvsParams(*[float(p[k]) for k in ("grad_min", "d_min", "d_max", "sigma_range",
                                                 "ssd_max", "photo_var")], int(p["max_steps"]))
        camc = _Camera(*[float(c) for c in cam])
        pose = _Pose((C.c_double * 9)(*np.asarray(R, np.float64).ravel()),
                     (C.c_double * 3)(*np.asarray(t, np.float64).ravel()))
        fp = C.POINTER(C.c_float)
        ip = C.POINTER(C.c_int32)
        n = self.lib.orc_semi_dense(W, H, ik.ctypes.data_as(fp), ir.ctypes.data_as(fp),
                                    C.byref(camc), C.byref(pose), C.byref(prm), _dp(d), _dp(vv),
                                    st.ctypes.data_as(ip), bs.ctypes.data_as(ip), _dp(mg))
        sh = (H, W)
        return d.reshape(sh), vv.reshape(sh), st.reshape(sh), bs.reshape(sh), mg.reshape(sh), int(n)

    def within(self, x, d_true, rel_tol: float = 0.1):
        """(n_within, n_valid) of Section III-B's accuracy measure."""
        xx, dd = _f64(x).ravel(), _f64(d_true).ravel()
        a, b = C.c_int64(0), C.c_int64(0)
        self.lib.orc_within(xx.size, _dp(xx), _dp(dd), float(rel_tol), C.byref(a), C.byref(b))
        return a.value, b.value

    def depth(self, x) -> np.ndarray:
        xx = _f64(x)
        d = np.zeros_like(xx)
        self.lib.orc_depth(xx.size, _dp(xx), _dp(d))
        return d.reshape(np.shape(x))

    def semi_to_log(self, d, var_d):
        dd, vv = _f64(d), _f64(var_d)
        mu, var = np.zeros_like(dd), np.zeros_like(dd)
        self.lib.orc_semi_to_log(dd.size, _dp(dd), _dp(vv), _dp(mu), _dp(var))
        return mu.reshape(np.shape(d)), var.reshape(np.shape(d))

    def ls_scale_fit(self, kf, x, t: float = 0.0):
        prob, keep = self._problem(kf)
        xx = _f64(x).copy()
        tt = C.c_double(float(t))
        self.lib.orc_ls_scale_fit(C.byref(prob), _dp(xx), C.byref(tt))
        return xx.reshape(kf.height, kf.width), tt.value


_DEFAULT: Optional[Oracle] = None


def get() -> Oracle:
    """The (lazily built) unmutated oracle."""
    global _DEFAULT
    if _DEFAULT is None:
        _DEFAULT = Oracle()
    return _DEFAULT
