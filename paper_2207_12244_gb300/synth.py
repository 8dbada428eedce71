"""Seeded synthetic inputs shaped like DeepFusion's workloads.

This module only *simulates the inputs* of the per-frame keyframe optimisation
(Section II-C): a piecewise-planar scene seen by a pinhole camera, the CNN's
log-depth / log-depth-gradient predictions with their variances (Section II-A,
Eq. 1 gives the variance meaning), and the semi-dense multiview-stereo
log-depths with their variances (Section II-B). It contains none of the
optimisation's arithmetic: both the FP64 oracle and the CUDA path consume the
arrays produced here, so neither depends on the other's random numbers.

Recipe (all draws from ``numpy.random.default_rng(seed)``):

* Scene: 3 planes, labelled by a Voronoi partition of 3 random seed pixels.
  Each plane n.X = dist seen through K (fx = fy = 0.9 W, cx = W/2, cy = H/2)
  has affine inverse depth 1/D = n.K^-1 [u, v, 1]^T / dist; normals and
  distances are rejection-sampled until D lies in [0.5, 5] m on the plane's
  region (fronto-parallel fallback).
* CNN: mu_n = ln D + N(0, 0.1^2); reported sigma_n ~ U(0.05, 0.3) per pixel,
  var_n = sigma_n^2. gx, gy = forward differences of ln D (jumps at plane
  boundaries included) + N(0, sigma_g^2), sigma_g ~ U(0.01, 0.1) per pixel
  and direction, var_g = sigma_g^2. gx in the last column and gy in the last
  row have no partner pixel; they are set to 0 with variance 1 and are ignored
  by the method.
* Semi-dense: candidates = pixels within 2 px of a label boundary, plus 8x8
  "texture" blocks kept with p = 0.3. The mask is round(f N) pixels drawn from
  the candidates (topped up from the rest). Depth noise sigma_d = k D^2 with
  k = 0.01 / m, i.e. sigma = k D in log-depth; mu_s = ln D - ln s_true + noise
  with s_true ~ U(0.5, 2) per keyframe (the scale the method must recover).
  Invalid pixels carry var_s = 0 and mu_s = 0.
* Sequence: a nested mask that grows linearly from 5 % to 40 % of the pixels
  over the frames; every masked pixel receives one new observation per frame,
  fused into its running estimate by the Gaussian product (the semi-dense
  system's own filtering, outside the optimisation).

All planes are float32, row-major H x W.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Tuple

import numpy as np

K_SEMI = 0.01  # depth noise sigma_d = K_SEMI * D^2  (metres)


@dataclass
class Keyframe:
    """One keyframe's inputs (float32 planes, H x W) plus the scene's truth."""

    width: int
    height: int
    mu_n: np.ndarray
    var_n: np.ndarray
    gx: np.ndarray
    var_gx: np.ndarray
    gy: np.ndarray
    var_gy: np.ndarray
    mu_s: np.ndarray
    var_s: np.ndarray
    log_depth_true: np.ndarray  # float64, ln D
    scale_log_true: float  # ln s_true
    labels: np.ndarray = field(repr=False, default=None)

    @property
    def cnn_planes(self) -> Tuple[np.ndarray, ...]:
        return (self.mu_n, self.var_n, self.gx, self.var_gx, self.gy, self.var_gy)

    @property
    def n_pixels(self) -> int:
        return self.width * self.height


def _intrinsics(W: int, H: int):
    f = 0.9 * W
    return f, f, W / 2.0, H / 2.0


def make_scene(W: int, H: int, rng: np.random.Generator, n_planes: int = 3):
    """Return (ln D float64 [H, W], labels int32 [H, W])."""
    log_d, labels, _ = _scene_planes(W, H, rng, n_planes)
    return log_d, labels


def _scene_planes(W: int, H: int, rng: np.random.Generator, n_planes: int = 3):
    """The scene of make_scene plus each plane as (n, dist) with n.X = dist in
    the keyframe's camera coordinates (a fronto-parallel fallback plane has
    n = (0, 0, 1))."""
    fx, fy, cx, cy = _intrinsics(W, H)
    planes = [(np.array([0.0, 0.0, 1.0]), 1.0)] * n_planes
    u = np.arange(W, dtype=np.float64)[None, :]
    v = np.arange(H, dtype=np.float64)[:, None]
    su = rng.integers(0, W, size=n_planes)
    sv = rng.integers(0, H, size=n_planes)
    d2 = (u[None] - su[:, None, None]) ** 2 + (v[None] - sv[:, None, None]) ** 2
    labels = np.argmin(d2, axis=0).astype(np.int32)
    ray_x = (u - cx) / fx  # K^-1 [u, v, 1]^T, z component 1
    ray_y = (v - cy) / fy
    inv_d = np.empty((H, W), dtype=np.float64)
    for k in range(n_planes):
        region = labels == k
        if not region.any():
            continue
        ok = False
        for _ in range(200):
            d0 = rng.uniform(0.8, 4.0)
            n = rng.normal(size=3)
            n[2] = abs(n[2]) + 0.6  # roughly facing the camera
            n /= np.linalg.norm(n)
            seed_ray = np.array([(su[k] - cx) / fx, (sv[k] - cy) / fy, 1.0])
            dist = d0 * float(n @ seed_ray)
            if dist <= 0:
                continue
            cand = (n[0] * ray_x + n[1] * ray_y + n[2]) / dist
            vals = cand[region] if cand.shape == region.shape else np.broadcast_to(cand, region.shape)[region]
            if np.all(vals > 0) and np.all(1.0 / vals >= 0.5) and np.all(1.0 / vals <= 5.0):
                inv_d[region] = np.broadcast_to(cand, (H, W))[region]
                planes[k] = (n.copy(), dist)
                ok = True
                break
        if not ok:  # fronto-parallel plane at a valid depth
            dfp = rng.uniform(0.8, 4.0)
            inv_d[region] = 1.0 / dfp
            planes[k] = (np.array([0.0, 0.0, 1.0]), dfp)
    return np.log(1.0 / inv_d), labels, planes


def _candidates(labels: np.ndarray, rng: np.random.Generator) -> np.ndarray:
    H, W = labels.shape
    edge = np.zeros((H, W), dtype=bool)
    dx = labels[:, 1:] != labels[:, :-1]
    dy = labels[1:, :] != labels[:-1, :]
    edge[:, 1:] |= dx
    edge[:, :-1] |= dx
    edge[1:, :] |= dy
    edge[:-1, :] |= dy
    dil = edge.copy()
    for s in (1, 2):  # Chebyshev dilation by 2 px
        for a, b in ((s, 0), (-s, 0), (0, s), (0, -s), (s, s), (s, -s), (-s, s), (-s, -s)):
            sh = np.zeros_like(edge)
            ys = slice(max(a, 0), H + min(a, 0))
            yd = slice(max(-a, 0), H + min(-a, 0))
            xs = slice(max(b, 0), W + min(b, 0))
            xd = slice(max(-b, 0), W + min(-b, 0))
            sh[yd, xd] = edge[ys, xs]
            dil |= sh
    bh, bw = (H + 7) // 8, (W + 7) // 8
    blocks = rng.random((bh, bw)) < 0.3
    tex = np.repeat(np.repeat(blocks, 8, axis=0), 8, axis=1)[:H, :W]
    return dil | tex


def _mask_order(labels: np.ndarray, rng: np.random.Generator) -> np.ndarray:
    """Flat pixel indices: candidates (shuffled) first, then the rest (shuffled)."""
    cand = _candidates(labels, rng).ravel()
    idx = np.arange(cand.size)
    c = rng.permutation(idx[cand])
    o = rng.permutation(idx[~cand])
    return np.concatenate([c, o])


def make_keyframe(W: int, H: int, seed: int, semi_fraction: float = 0.2,
                  noise: bool = True) -> Keyframe:
    """One keyframe with one frame of semi-dense measurements (config-1 recipe)."""
    rng = np.random.default_rng(seed)
    L, labels = make_scene(W, H, rng)
    shape = (H, W)
    D = np.exp(L)
    mu_n = L + (rng.normal(0.0, 0.1, shape) if noise else 0.0)
    var_n = rng.uniform(0.05, 0.3, shape) ** 2
    sgx = rng.uniform(0.01, 0.1, shape)
    sgy = rng.uniform(0.01, 0.1, shape)
    gx = np.zeros(shape)
    gy = np.zeros(shape)
    gx[:, :-1] = L[:, 1:] - L[:, :-1]
    gy[:-1, :] = L[1:, :] - L[:-1, :]
    if noise:
        gx += rng.normal(0.0, 1.0, shape) * sgx
        gy += rng.normal(0.0, 1.0, shape) * sgy
    var_gx = sgx ** 2
    var_gy = sgy ** 2
    gx[:, -1] = 0.0
    var_gx[:, -1] = 1.0
    gy[-1, :] = 0.0
    var_gy[-1, :] = 1.0
    s_true = rng.uniform(0.5, 2.0)
    order = _mask_order(labels, rng)
    n_mask = int(round(semi_fraction * W * H))
    sel = order[:n_mask]
    sig = K_SEMI * D.ravel()[sel]
    mu_s = np.zeros(W * H)
    var_s = np.zeros(W * H)
    obs = L.ravel()[sel] - np.log(s_true)
    if noise:
        obs = obs + rng.normal(0.0, 1.0, sel.size) * sig
    mu_s[sel] = obs
    var_s[sel] = sig ** 2
    f32 = lambda a: np.ascontiguousarray(a, dtype=np.float32).reshape(shape)
    return Keyframe(W, H, f32(mu_n), f32(var_n), f32(gx), f32(var_gx), f32(gy),
                    f32(var_gy), f32(mu_s), f32(var_s), L, float(np.log(s_true)),
                    labels)


def make_sequence(W: int, H: int, seed: int, n_frames: int = 100,
                  frac0: float = 0.05, frac1: float = 0.40):
    """Keyframe + per-frame semi-dense maps (config-2 recipe).

    Returns (keyframe, mu_s [F, H, W] float32, var_s [F, H, W] float32). The
    keyframe's own mu_s/var_s are frame 0's.
    """
    kf = make_keyframe(W, H, seed, semi_fraction=frac0)
    rng = np.random.default_rng(seed + 7919)
    N = W * H
    order = _mask_order(kf.labels, rng)
    D = np.exp(kf.log_depth_true).ravel()
    target = kf.log_depth_true.ravel() - kf.scale_log_true
    vo_all = (K_SEMI * D) ** 2
    mu = np.zeros(N)
    var = np.zeros(N)
    seen = np.zeros(N, dtype=bool)
    mus = np.empty((n_frames, H, W), dtype=np.float32)
    vars_ = np.empty((n_frames, H, W), dtype=np.float32)
    for f in range(n_frames):
        frac = frac0 + (frac1 - frac0) * (f / max(n_frames - 1, 1))
        sel = order[: int(round(frac * N))]
        vo = vo_all[sel]
        o = target[sel] + rng.normal(0.0, 1.0, sel.size) * np.sqrt(vo)
        new = ~seen[sel]
        m0, v0 = mu[sel], var[sel]
        fused_v = v0 * vo / np.where(new, 1.0, v0 + vo)
        fused_m = (m0 * vo + o * v0) / np.where(new, 1.0, v0 + vo)
        mu[sel] = np.where(new, o, fused_m)
        var[sel] = np.where(new, vo, fused_v)
        seen[sel] = True
        mus[f] = mu.reshape(H, W)
        vars_[f] = var.reshape(H, W)
    kf.mu_s = mus[0].copy()
    kf.var_s = vars_[0].copy()
    return kf, mus, vars_


BATCH_SIZES = ((320, 240), (512, 384), (640, 480), (1280, 960))


def batch_shapes(n: int, seed: int, choices=BATCH_SIZES) -> List[Tuple[int, int]]:
    """Uneven keyframe sizes (config-3 recipe): n draws from ``choices``."""
    rng = np.random.default_rng(seed)
    return [tuple(choices[i]) for i in rng.integers(0, len(choices), size=n)]


def to_bf16(a: np.ndarray) -> np.ndarray:
    """Round float32 -> bfloat16 (round to nearest even); returns the 16-bit codes."""
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    rounding = 0x7FFF + ((u >> 16) & 1)
    return ((u + rounding) >> 16).astype(np.uint16)


def bf16_to_f32(codes: np.ndarray) -> np.ndarray:
    return (codes.astype(np.uint32) << 16).view(np.float32)


def to_f16(a: np.ndarray) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float32).astype(np.float16).view(np.uint16)


def f16_to_f32(codes: np.ndarray) -> np.ndarray:
    return codes.view(np.float16).astype(np.float32)


# ---- two views of a textured piecewise-planar scene (semi-dense input) -----
#
# The semi-dense stereo step (Section II-B) needs images: a keyframe image
# and a reference image of the same scene from a known relative pose. The
# planes of _scene_planes carry an aperiodic texture fixed to the surface
# (value noise over plane coordinates, two octaves), so both views see the
# same surface pattern. The reference view is ray-cast: a ray meets plane k
# where that point falls inside plane k's region of the keyframe image; the
# nearest such hit is seen, else a far background plane.

@dataclass
class StereoPair:
    width: int
    height: int
    img_key: np.ndarray   # float32 [H, W], intensities in [0, 255]
    img_ref: np.ndarray   # float32 [H, W]
    cam: Tuple[float, float, float, float]  # fx, fy, cx, cy (both views)
    R: np.ndarray         # float64 3 x 3: X_ref = R X_key + t
    t: np.ndarray         # float64 3
    depth_true: np.ndarray  # float64 [H, W], keyframe depth (metres)
    labels: np.ndarray = field(repr=False, default=None)


def _hash01(i: np.ndarray, j: np.ndarray, salt: int) -> np.ndarray:
    """Deterministic pseudo-random values in [0, 1) per integer lattice point."""
    h = (i.astype(np.int64) * 73856093) ^ (j.astype(np.int64) * 19349663) ^ (salt * 83492791)
    h = (h ^ (h >> 13)) * 1274126177
    h = h ^ (h >> 16)
    return (h & 0xFFFFFF).astype(np.float64) / float(1 << 24)


def _value_noise(a: np.ndarray, b: np.ndarray, cell: float, salt: int) -> np.ndarray:
    x, y = a / cell, b / cell
    i, j = np.floor(x), np.floor(y)
    fx, fy = x - i, y - j
    wx, wy = fx * fx * (3 - 2 * fx), fy * fy * (3 - 2 * fy)  # smoothstep
    v00, v10 = _hash01(i, j, salt), _hash01(i + 1, j, salt)
    v01, v11 = _hash01(i, j + 1, salt), _hash01(i + 1, j + 1, salt)
    return (v00 * (1 - wx) + v10 * wx) * (1 - wy) + (v01 * (1 - wx) + v11 * wx) * wy


def _texture(X: np.ndarray, n: np.ndarray, salt: int, cell: float) -> np.ndarray:
    """Intensity of surface points X (..., 3) on a plane with normal n."""
    helper = np.array([1.0, 0.0, 0.0]) if abs(n[0]) < 0.9 else np.array([0.0, 1.0, 0.0])
    e1 = np.cross(n, helper)
    e1 /= np.linalg.norm(e1)
    e2 = np.cross(n, e1)
    a, b = X @ e1, X @ e2
    v = 0.65 * _value_noise(a, b, cell, salt) + 0.35 * _value_noise(a, b, cell * 0.5, salt + 7)
    return 255.0 * v


def _rotation(axis: np.ndarray, angle: float) -> np.ndarray:
    axis = axis / np.linalg.norm(axis)
    K = np.array([[0, -axis[2], axis[1]], [axis[2], 0, -axis[0]], [-axis[1], axis[0], 0]])
    return np.eye(3) + np.sin(angle) * K + (1 - np.cos(angle)) * (K @ K)


def make_stereo_pair(W: int, H: int, seed: int, baseline: float = 0.04, rot_deg: float = 0.5,
                     cell: float = 0.025, noise: float = 0.0, view: int = 0) -> StereoPair:
    """Keyframe and reference images of one seeded scene (the scene of
    make_keyframe(W, H, seed)) from a relative pose with the given baseline
    (metres, mostly sideways) and a small rotation; optional Gaussian image
    noise (intensity units). 'view' draws another reference pose of the same
    keyframe (the keyframe image does not depend on it)."""
    rng = np.random.default_rng(seed)
    log_d, labels, planes = _scene_planes(W, H, rng)
    fx, fy, cx, cy = _intrinsics(W, H)
    prng = np.random.default_rng([seed, 104729] + ([view] if view else []))
    R = _rotation(prng.normal(size=3), np.deg2rad(rot_deg))
    d = prng.normal(size=3)
    d[2] *= 0.2  # mostly sideways motion
    t = baseline * d / np.linalg.norm(d)
    D = np.exp(log_d)
    u = np.arange(W, dtype=np.float64)[None, :]
    v = np.arange(H, dtype=np.float64)[:, None]
    rays = np.stack(np.broadcast_arrays((u - cx) / fx, (v - cy) / fy, np.ones((H, W))), axis=-1)
    Xk = rays * D[..., None]
    img_key = np.zeros((H, W))
    for k, (n, dist) in enumerate(planes):
        m = labels == k
        img_key[m] = _texture(Xk[m], n, 1000 * seed + k, cell)
    # reference view: X_key = R^T (X_ref - t) along reference rays X_ref = lam r
    Rt = R.T
    dir_k = rays @ R  # (R^T r) for every reference ray r
    orig_k = -Rt @ t
    best = np.full((H, W), np.inf)
    img_ref = np.zeros((H, W))
    for k, (n, dist) in enumerate(planes):
        den = dir_k @ n
        with np.errstate(divide="ignore", invalid="ignore"):
            lam = (dist - orig_k @ n) / den
        X = orig_k + lam[..., None] * dir_k
        with np.errstate(divide="ignore", invalid="ignore"):
            u0 = fx * X[..., 0] / X[..., 2] + cx
            v0 = fy * X[..., 1] / X[..., 2] + cy
        ok = (lam > 0) & (X[..., 2] > 0) & np.isfinite(u0) & np.isfinite(v0)
        iu = np.clip(np.rint(np.where(ok, u0, 0)), 0, W - 1).astype(int)
        iv = np.clip(np.rint(np.where(ok, v0, 0)), 0, H - 1).astype(int)
        ok &= (u0 > -0.5) & (u0 < W - 0.5) & (v0 > -0.5) & (v0 < H - 0.5)
        ok &= labels[iv, iu] == k
        take = ok & (lam < best)
        best[take] = lam[take]
        img_ref[take] = _texture(X[take], n, 1000 * seed + k, cell)
    bg = ~np.isfinite(best)
    if bg.any():  # far fronto-parallel background in the keyframe frame
        nb = np.array([0.0, 0.0, 1.0])
        lam = (10.0 - orig_k @ nb) / (dir_k[bg] @ nb)
        img_ref[bg] = _texture(orig_k + lam[:, None] * dir_k[bg], nb, 1000 * seed + 99, cell)
    if noise > 0:
        nrng = np.random.default_rng([seed, 7919, view])
        img_key = img_key + nrng.normal(0, noise, img_key.shape)
        img_ref = img_ref + nrng.normal(0, noise, img_ref.shape)
    return StereoPair(W, H, img_key.astype(np.float32), img_ref.astype(np.float32),
                      (fx, fy, cx, cy), R, t, D, labels)
