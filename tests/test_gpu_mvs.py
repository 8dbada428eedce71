"""Semi-dense two-view depth (Section II-B) on the GPU through the C ABI,
against the FP64 oracle.

The method takes integer decisions in floating point (texture and SSD
thresholds, the argmin over steps, the neighbour choice, the step count,
image-border tests). The oracle reports, per pixel, how far its decisions
were from flipping; where that margin is clear the GPU must take the same
decisions and give the same depth and variance, elsewhere a GPU
measurement must only be a valid one."""
import numpy as np
import pytest

import oracle as orc
from gpu_util import create, params, to_dev, torch_cuda
from paper_2207_12244_gb300 import deepfusion as dfl
from paper_2207_12244_gb300 import synth

pytestmark = pytest.mark.gpu

CLEAR = 1e-3     # oracle decision margin above which decisions must agree
# Tolerances of the continuous results, from the FP32 arithmetic: sample
# positions carry ~3e-5 px of rounding, i.e. an error eps ~ 1e-3 intensity
# units on each photometric error e. The linearised fit moves its fraction
# by eps / |de|, and sigma = |dd| / |de| (Eq. 4 with photo_var = 1), so the
# depth moves by about eps * sigma, and sigma^2 by a relative 2 eps / |de|
# ~ 2 eps * (disparity) * sigma / d. Hence: depth within 1e-4 d + 0.02 sigma,
# variance within 2e-3 + 0.1 sigma / d (relative).
DEPTH_RTOL = 1e-4
DEPTH_SIGMA_TOL = 0.02
VAR_RTOL = 2e-3
VAR_SIGMA_TOL = 0.1


@pytest.fixture(scope="module")
def o():
    return orc.get()


def _f32_geometry(cam, R, t):
    """The geometry exactly as the GPU receives it (FP32)."""
    return (tuple(float(np.float32(c)) for c in cam), np.asarray(R, np.float32).astype(np.float64),
            np.asarray(t, np.float32).astype(np.float64))


def _gpu(ik, ir, cam, R, t, depth=None, var=None, **kw):
    torch = torch_cuda()
    H, W = ik.shape
    d = to_dev(np.zeros((H, W), np.float32) if depth is None else depth.astype(np.float32))
    v = to_dev(np.zeros((H, W), np.float32) if var is None else var.astype(np.float32))
    st = torch.full((H, W), -7, dtype=torch.int32, device="cuda")
    bs = torch.full((H, W), -7, dtype=torch.int32, device="cuda")
    m = dfl.SemiDense(W, H)
    try:
        m.update(to_dev(ik), to_dev(ir), cam, R, t, d, v, st, bs,
                 params=dfl.df_mvs_default_params(**kw) if kw else None)
        torch.cuda.synchronize()
    finally:
        m.close()
    return (d.double().cpu().numpy(), v.double().cpu().numpy(), st.cpu().numpy(),
            bs.cpu().numpy())


def _compare(gpu, orc_out, what, max_unclear=0.02):
    d, v, st, bs = gpu
    od, ov, ost, obs, mg, n = orc_out
    assert np.all(st >= 0) and np.all(st <= 6), what  # every pixel got a status
    clear = mg > CLEAR
    assert (~clear).mean() <= max_unclear, (what, (~clear).mean())
    bad = clear & (st != ost)
    assert not bad.any(), (what, "status", np.argwhere(bad)[:5], st[bad][:5], ost[bad][:5])
    both = clear & (ost == orc.MVS_OK)
    assert np.array_equal(bs[both], obs[both]), what
    sig = np.sqrt(ov[both])
    err_d = np.abs(d[both] - od[both])
    tol_d = DEPTH_RTOL * od[both] + DEPTH_SIGMA_TOL * sig
    assert np.all(err_d <= tol_d), (what, (err_d / tol_d).max())
    rel_v = np.abs(v[both] / ov[both] - 1.0)
    tol_v = VAR_RTOL + VAR_SIGMA_TOL * sig / od[both]
    assert np.all(rel_v <= tol_v), (what, (rel_v / tol_v).max())
    # most pixels are well conditioned and meet the plain relative bound
    if both.sum() >= 100:
        assert np.mean(err_d <= DEPTH_RTOL * od[both]) > 0.99, what
    # near a decision edge: a GPU measurement must be a valid one
    g = ~clear & (st == orc.MVS_OK)
    assert np.all(np.isfinite(d[g]) & (d[g] > 0) & np.isfinite(v[g]) & (v[g] > 0)), what
    return int(both.sum())


@pytest.mark.parametrize("W,H,seed", [(640, 480, 1), (320, 240, 2), (333, 177, 3)])
def test_first_update_matches_oracle(o, W, H, seed):
    sp = synth.make_stereo_pair(W, H, seed)
    cam, R, t = _f32_geometry(sp.cam, sp.R, sp.t)
    want = o.semi_dense(sp.img_key, sp.img_ref, cam, R, t)
    got = _gpu(sp.img_key, sp.img_ref, cam, R, t)
    n = _compare(got, want, f"{W}x{H}")
    assert n > 0.1 * W * H


def test_update_with_an_estimate_matches_oracle(o):
    """Second view: the search runs in d +- 2 sigma of the first estimate and
    the measurement is fused with it."""
    sp = synth.make_stereo_pair(320, 240, 4)
    cam, R, t = _f32_geometry(sp.cam, sp.R, sp.t)
    d0, v0, *_ = o.semi_dense(sp.img_key, sp.img_ref, cam, R, t)
    d0, v0 = d0.astype(np.float32), v0.astype(np.float32)
    sp2 = synth.make_stereo_pair(320, 240, 4, baseline=0.06, rot_deg=0.8)
    cam2, R2, t2 = _f32_geometry(sp2.cam, sp2.R, sp2.t)
    want = o.semi_dense(sp2.img_key, sp2.img_ref, cam2, R2, t2, depth=d0, var=v0)
    got = _gpu(sp2.img_key, sp2.img_ref, cam2, R2, t2, depth=d0, var=v0)
    _compare(got, want, "with estimate")
    assert np.sum(want[2] == orc.MVS_OK) > 1000


def test_rectified_closed_form():
    """Ramp images, sideways baseline: the depth the GPU fits between steps is
    the closed form of the linearised fit (the oracle's pin, on the GPU)."""
    fx, tx, W, H = 50.0, 0.25, 64, 32  # fx * tx = 12.5: exact in FP32
    u = np.arange(W, dtype=np.float64)[None, :]
    v = np.arange(H, dtype=np.float64)[:, None]
    ik = ((3.0 * u + 0.5 * v + 10.0) * np.ones((H, W))).astype(np.float32)
    dstar = 8.25
    ir = (ik - 3.0 * dstar).astype(np.float32)
    cam = (fx, fx, W / 2.0, H / 2.0)
    d, var, st, bs = _gpu(ik, ir, cam, np.eye(3), np.array([tx, 0.0, 0.0]), grad_min=1.0,
                          d_min=0.5, d_max=10.0, ssd_max=1e9)
    B = fx * tx
    da, db = B / 8.0, B / 9.0
    ea, eb = 3.0 * (8.0 - dstar), 3.0 * (9.0 - dstar)
    s = -ea / (eb - ea)
    want_d = da + s * (db - da)
    want_v = (db - da) ** 2 / (5.0 * (eb - ea) ** 2)
    for yy, xx in ((16, 20), (10, 30), (20, 35)):
        assert st[yy, xx] == dfl.DF_MVS_OK
        assert abs(d[yy, xx] / want_d - 1) < 1e-5, (d[yy, xx], want_d)
        assert abs(var[yy, xx] / want_v - 1) < 1e-4, (var[yy, xx], want_v)
    assert np.all(st[0, :] == dfl.DF_MVS_FLAT) and np.all(st[:, -1] == dfl.DF_MVS_FLAT)


@pytest.mark.parametrize("W,H", [(3, 3), (2, 9), (9, 2), (1, 1), (40, 3)])
def test_tiny_images(o, W, H):
    rng = np.random.default_rng(W * 31 + H)
    ik = (rng.random((H, W)) * 255).astype(np.float32)
    ir = (rng.random((H, W)) * 255).astype(np.float32)
    cam = (0.9 * W, 0.9 * W, W / 2.0, H / 2.0)
    R, t = np.eye(3), np.array([0.05, 0.01, 0.0])
    want = o.semi_dense(ik, ir, cam, R, t)
    got = _gpu(ik, ir, cam, R, t)
    _compare(got, want, f"tiny {W}x{H}", max_unclear=1.0)


def test_invalid_arguments():
    torch = torch_cuda()
    z = torch.zeros((8, 8), device="cuda")
    m = dfl.SemiDense(8, 8)
    try:
        with pytest.raises(dfl.DFError) as e:
            m.update(z, z, (8, 8, 4, 4), np.eye(3), np.zeros(3), z, z,
                     params=dfl.df_mvs_default_params(d_min=0.0))
        assert e.value.status == dfl.DF_EINVAL
        with pytest.raises(dfl.DFError) as e:
            m.update(z, z, (0, 8, 4, 4), np.eye(3), np.zeros(3), z, z)
        assert e.value.status == dfl.DF_EINVAL
    finally:
        m.close()


def test_stereo_feeds_the_solve(o):
    """The whole frame on the GPU: stereo depth -> log space -> semi-dense term
    of the solve. Fusing it lifts the share of depths within 10 % of the
    truth above the network prior's."""
    torch = torch_cuda()
    W, H, seed = 320, 240, 6
    sp = synth.make_stereo_pair(W, H, seed)
    kf = synth.make_keyframe(W, H, seed)
    assert np.allclose(sp.depth_true, np.exp(kf.log_depth_true))  # one scene
    cam, R, t = _f32_geometry(sp.cam, sp.R, sp.t)
    d = torch.zeros((H, W), device="cuda")
    v = torch.zeros((H, W), device="cuda")
    m = dfl.SemiDense(W, H)
    k = create(kf)
    try:
        m.update(to_dev(sp.img_key), to_dev(sp.img_ref), cam, R, t, d, v)
        mu = torch.empty_like(d)
        vs = torch.empty_like(d)
        dfl.df_semi_to_log(d, v, mu, vs)
        truth = to_dev(sp.depth_true.astype(np.float32))
        n0, nv = k.depth_accuracy(truth)
        k.frame_update(mu, vs)
        k.optimise(params(n_gn=10, n_pcg=5))
        n1, _ = k.depth_accuracy(truth)
    finally:
        k.close()
        m.close()
    assert n1 / nv > n0 / nv + 0.1, (n0 / nv, n1 / nv)
