"""Reader of the golden fixtures (written by make_golden.py from the FP64 oracle)."""
from __future__ import annotations

import glob
import os
import types

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))

LOSSES = {"huber": 0, "tukey": 1}
SCALE_STEPS = {"fixed": 0, "alternate": 1, "joint": 2}


def paths(kind="solve"):
    """The fixtures of one kind: "solve" (keyframe solves) or "stereo"."""
    out = []
    for p in sorted(glob.glob(os.path.join(HERE, "*.txt"))):
        with open(p) as f:
            is_stereo = any(line.strip() == "kind stereo" for line in f)
        if is_stereo == (kind == "stereo"):
            out.append(p)
    return out


def load(path):
    """One fixture as a namespace: the keyframe planes (float32 [H, W]), the
    solve's parameters and the expected x (float64 [H, W]), t and iterations."""
    g = types.SimpleNamespace(name=os.path.basename(path)[:-4])
    planes = {}
    with open(path) as f:
        for line in f:
            if not line.strip() or line.startswith("#"):
                continue
            key, _, rest = line.strip().partition(" ")
            if key == "plane":
                pname, _, vals = rest.partition(" ")
                planes[pname] = [float.fromhex(v) for v in vals.split()]
            elif key == "expect_x":
                g.x = np.array([float.fromhex(v) for v in rest.split()], np.float64)
            elif key == "kind":
                g.kind = rest
            elif key in ("cam", "R", "t", "expect_depth", "expect_var", "expect_margin"):
                setattr(g, key, np.array([float.fromhex(v) for v in rest.split()], np.float64))
            elif key == "image":
                pname, _, vals = rest.partition(" ")
                planes[pname] = [float.fromhex(v) for v in vals.split()]
            elif key in ("expect_status", "expect_best"):
                setattr(g, key, np.array([int(v) for v in rest.split()], np.int32))
            elif key == "expect_measured":
                g.expect_measured = int(rest)
            elif key in ("W", "H", "n_gn", "n_pcg", "terms", "expect_iters"):
                setattr(g, key, int(rest))
            elif key in ("delta", "expect_t"):
                setattr(g, key, float.fromhex(rest))
            elif key == "loss":
                g.loss = LOSSES[rest]
            elif key == "scale_step":
                g.scale_step = SCALE_STEPS[rest]
            else:
                raise ValueError(f"{path}: unknown key {key}")
    g.width, g.height = g.W, g.H
    for n, v in planes.items():
        a = np.array(v, np.float32).reshape(g.H, g.W)
        setattr(g, n, a)
    if getattr(g, "kind", "solve") == "stereo":
        g.R = g.R.reshape(3, 3)
        for n in ("expect_depth", "expect_var", "expect_margin", "expect_status", "expect_best"):
            setattr(g, n, getattr(g, n).reshape(g.H, g.W))
        return g
    g.x = g.x.reshape(g.H, g.W)
    g.cnn_planes = tuple(getattr(g, n) for n in ("mu_n", "var_n", "gx", "var_gx", "gy", "var_gy"))
    return g
