"""Write the golden fixtures of this folder from the FP64 oracle.

Each fixture is one small keyframe solve (Section II-C: the cost of Eqs. 5-8,
n_gn Gauss-Newton iterations of a scale step then a Jacobi-PCG depth step)
stored as text: the float32 input planes and the oracle's float64 result,
every number as an exact hexadecimal float. The inputs come from the seeded
scene generator; the expected values come from ``oracle/`` alone.

The fixtures freeze the oracle's output, so that

* a later change to the oracle's arithmetic shows up as a changed fixture
  (the change then names the passage of the paper that justifies it), and
* the oracle built on another host (the GPU machine is an Arm machine) can be
  checked to give the same bits as the one that wrote them.

A stereo case stores one semi-dense update (Section II-B) the same way:
the two images and the relative pose, and the oracle's depth, variance,
decision margin, status and best step per pixel.

Run from the repository root:  python tests/golden/make_golden.py
"""
from __future__ import annotations

import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2207_12244_gb300 import synth  # noqa: E402

PLANES = ("mu_n", "var_n", "gx", "var_gx", "gy", "var_gy", "mu_s", "var_s")
LOSS_NAMES = {oracle.LOSS_HUBER: "huber", oracle.LOSS_TUKEY: "tukey"}
SCALE_NAMES = {oracle.SCALE_FIXED: "fixed", oracle.SCALE_ALTERNATE: "alternate",
               oracle.SCALE_JOINT: "joint"}

# name, W, H, seed, n_gn, n_pcg, delta, loss, scale_step, terms, what it covers
CASES = [
    ("huber_alternate_9x7", 9, 7, 11, 10, 3, oracle.HUBER_DELTA, oracle.LOSS_HUBER,
     oracle.SCALE_ALTERNATE, oracle.TERMS_ALL,
     "the paper's schedule: Huber loss (Section II-C, last paragraph), scale and depth "
     "alternating, 10 GN x 3 PCG"),
    ("least_squares_alternate_8x6", 8, 6, 12, 6, 5, 0.0, oracle.LOSS_HUBER,
     oracle.SCALE_ALTERNATE, oracle.TERMS_ALL,
     "pure least squares (Eqs. 5-8 without the robust loss), 6 GN x 5 PCG"),
    ("tukey_alternate_7x9", 7, 9, 13, 8, 3, 4.685, oracle.LOSS_TUKEY,
     oracle.SCALE_ALTERNATE, oracle.TERMS_ALL,
     "Tukey's biweight, the robust loss Section IV names, 8 GN x 3 PCG"),
    ("huber_joint_8x5", 8, 5, 14, 10, 4, oracle.HUBER_DELTA, oracle.LOSS_HUBER,
     oracle.SCALE_JOINT, oracle.TERMS_ALL,
     "the joint (x, t) variant: one PCG on the bordered normal equations, 10 GN x 4 PCG"),
    ("no_pairwise_fixed_6x4", 6, 4, 15, 3, 2, oracle.HUBER_DELTA, oracle.LOSS_HUBER,
     oracle.SCALE_FIXED, oracle.TERM_SEMI | oracle.TERM_NET,
     "Table III's variant without the gradient term, scale held at t0 = 0"),
]


def _hex32(a) -> str:
    return " ".join(float(v).hex() for v in np.asarray(a, np.float32).ravel())


def _hex64(a) -> str:
    return " ".join(float(v).hex() for v in np.asarray(a, np.float64).ravel())


def write_case(o, case) -> str:
    name, W, H, seed, n_gn, n_pcg, delta, loss, scale_step, terms, what = case
    kf = synth.make_keyframe(W, H, seed)
    delta = float(np.float32(delta))  # the C ABI takes the threshold as a float32
    x, t, rep = o.optimise(kf, n_gn=n_gn, n_pcg=n_pcg, delta=delta, terms=terms, loss=loss,
                           scale_step=scale_step)
    lines = [
        f"# golden case {name}: {what}.",
        "# Cost of Eqs. 5-8 (Section II-C): semi-dense, network and gradient terms, each",
        "# whitened by its variance; x = log-depth from x0 = mu_n (keyframe initialisation),",
        "# t = log-scale from t0 = 0. Written by tests/golden/make_golden.py from oracle/;",
        f"# inputs from synth.make_keyframe({W}, {H}, seed={seed}). Numbers are hex floats:",
        "# planes as float32 row-major H x W, the result x as float64.",
        f"W {W}",
        f"H {H}",
        f"n_gn {n_gn}",
        f"n_pcg {n_pcg}",
        f"delta {float(delta).hex()}",
        f"loss {LOSS_NAMES[loss]}",
        f"scale_step {SCALE_NAMES[scale_step]}",
        f"terms {terms}",
    ]
    for p in PLANES:
        lines.append(f"plane {p} {_hex32(getattr(kf, p))}")
    lines.append(f"expect_t {float(t).hex()}")
    lines.append(f"expect_iters {rep.iters_done}")
    lines.append(f"expect_x {_hex64(x)}")
    path = os.path.join(HERE, name + ".txt")
    with open(path, "w") as f:
        f.write("\n".join(lines) + "\n")
    return path


# name, W, H, seed, baseline (m), what it covers
STEREO_CASES = [
    ("stereo_40x30", 40, 30, 5, 0.08,
     "one semi-dense update (Section II-B, Eqs. 2-4): epipolar 5-point SSD search, sub-pixel "
     "fit and variance, every rejection status"),
]


def _f32_list(a) -> str:
    return " ".join(float(v).hex() for v in np.asarray(a, np.float32).astype(np.float64).ravel())


def write_stereo_case(o, case) -> str:
    name, W, H, seed, baseline, what = case
    sp = synth.make_stereo_pair(W, H, seed, baseline=baseline)
    # the geometry exactly as the C ABI takes it (float32)
    cam = [float(np.float32(c)) for c in sp.cam]
    R = np.asarray(sp.R, np.float32).astype(np.float64)
    t = np.asarray(sp.t, np.float32).astype(np.float64)
    d, v, st, bs, mg, n = o.semi_dense(sp.img_key, sp.img_ref, cam, R, t)
    lines = [
        f"# golden case {name}: {what}.",
        "# Written by tests/golden/make_golden.py from oracle/ (default stereo parameters);",
        f"# images from synth.make_stereo_pair({W}, {H}, seed={seed}, baseline={baseline}).",
        "# Hex floats: images and geometry as float32 values, depth / variance as float64,",
        "# the decision margin as float32; status and best step as integers.",
        "kind stereo",
        f"W {W}",
        f"H {H}",
        f"cam {_f32_list(cam)}",
        f"R {_f32_list(R)}",
        f"t {_f32_list(t)}",
        f"image img_key {_hex32(sp.img_key)}",
        f"image img_ref {_hex32(sp.img_ref)}",
        f"expect_depth {_hex64(d)}",
        f"expect_var {_hex64(v)}",
        f"expect_margin {_f32_list(mg)}",
        "expect_status " + " ".join(str(int(x)) for x in st.ravel()),
        "expect_best " + " ".join(str(int(x)) for x in bs.ravel()),
        f"expect_measured {n}",
    ]
    path = os.path.join(HERE, name + ".txt")
    with open(path, "w") as f:
        f.write("\n".join(lines) + "\n")
    return path


def main():
    o = oracle.get()
    for case in CASES:
        print(write_case(o, case))
    for case in STEREO_CASES:
        print(write_stereo_case(o, case))


if __name__ == "__main__":
    main()
