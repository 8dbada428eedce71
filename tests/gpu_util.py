"""Helpers shared by the GPU tests: run the CUDA path through the C ABI and
compare with the FP64 oracle."""
from __future__ import annotations

import types

import numpy as np

from paper_2207_12244_gb300 import deepfusion as dfl

# Parity bar for FP32 solves: max relative depth error (|d_gpu - d_oracle| /
# d_oracle, d = exp(x)) at equal iteration count.
DEPTH_RTOL = 1e-4
# Log scale t: absolute error (the relative error of s = exp(t)).
SCALE_ATOL = 1e-4


def torch_cuda():
    import torch

    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return torch


def to_dev(a, dtype=None):
    torch = torch_cuda()
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def create(kf, on_device=True, cnn_dtype=None):
    """Create a keyframe on the GPU from a synth.Keyframe-like object."""
    planes = [np.ascontiguousarray(p) for p in kf.cnn_planes]
    if on_device:
        if cnn_dtype is None or cnn_dtype == dfl.DF_F32:
            planes = [to_dev(p) for p in planes]
        else:
            torch = torch_cuda()
            td = torch.bfloat16 if cnn_dtype == dfl.DF_BF16 else torch.float16
            planes = [to_dev(p).to(td) for p in planes]
    return dfl.Keyframe(kf.width, kf.height, *planes, cnn_dtype=cnn_dtype)


def params(**kw):
    base = dict(n_gn=10, n_pcg=3, solver=dfl.DF_SOLVER_LAUNCHES)
    base.update(kw)
    return dfl.df_default_params(**base)


def solve(kf, prm, semi=True, on_device=True, cnn_dtype=None, x0=None, t0=0.0):
    """One keyframe, one frame: returns (x float64 [H, W], t, report)."""
    torch = torch_cuda()
    k = create(kf, on_device, cnn_dtype)
    try:
        if semi and kf.mu_s is not None:
            if on_device:
                k.frame_update(to_dev(kf.mu_s), to_dev(kf.var_s))
            else:
                k.frame_update(np.ascontiguousarray(kf.mu_s), np.ascontiguousarray(kf.var_s))
        if x0 is not None or t0 != 0.0:
            k.set_state(None if x0 is None else to_dev(np.asarray(x0, np.float32).reshape(
                kf.height, kf.width)), t0)
        rep = k.optimise(prm, report=True)
        out = torch.empty((kf.height, kf.width), dtype=torch.float32, device="cuda")
        k.fetch_depth(out, log_space=True)
        torch.cuda.synchronize()
        x = out.double().cpu().numpy()
        return x, rep.scale_log, rep
    finally:
        k.close()


def oracle_solve(o, kf, prm, semi=True, x0=None, t0=0.0):
    view = kf
    if not semi:
        view = types.SimpleNamespace(**{n: getattr(kf, n) for n in (
            "width", "height", "mu_n", "var_n", "gx", "var_gx", "gy", "var_gy")})
        view.mu_s = None
        view.var_s = None
    return o.optimise(view, x0=x0, t0=t0, n_gn=prm.n_gn, n_pcg=prm.n_pcg, delta=prm.delta,
                      tol=prm.tol, terms=prm.terms, loss=prm.loss,
                      scale_step=int(prm.scale_step), warm_gn=prm.warm_gn,
                      warm_delta=prm.warm_delta)


def depth_rel_err(x_gpu, x_orc):
    return np.abs(np.expm1(np.asarray(x_gpu, np.float64) - np.asarray(x_orc, np.float64)))


def assert_parity(x_gpu, t_gpu, x_orc, t_orc, rtol=DEPTH_RTOL, atol_t=SCALE_ATOL, what=""):
    e = depth_rel_err(x_gpu, x_orc)
    assert e.max() <= rtol, f"{what}: max rel depth err {e.max():.3g} at {np.unravel_index(e.argmax(), e.shape)}"
    assert abs(t_gpu - t_orc) <= atol_t, f"{what}: t {t_gpu} vs {t_orc}"
    return float(e.max())
