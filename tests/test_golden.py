"""Golden fixtures (tests/golden/*.txt, written from the FP64 oracle).

CPU: the oracle built on this host reproduces every fixture bit for bit
(plain C, FP64, no FMA contraction, so x86 and Arm agree), which freezes its
arithmetic between changes.
GPU: the CUDA path, through the C ABI, meets its parity bar against the
stored results without running the oracle (the FP32 bar for the solves; for
the stereo update the decision-margin rule of tests/test_gpu_mvs.py).
"""
import numpy as np
import pytest

import golden
import oracle

CASES = golden.paths()
STEREO = golden.paths("stereo")


def test_fixtures_present():
    assert len(CASES) >= 5 and len(STEREO) >= 1


@pytest.mark.parametrize("path", CASES, ids=lambda p: p.rsplit("/", 1)[-1][:-4])
def test_oracle_reproduces_golden_bitwise(path):
    g = golden.load(path)
    x, t, rep = oracle.get().optimise(g, n_gn=g.n_gn, n_pcg=g.n_pcg, delta=g.delta,
                                      terms=g.terms, loss=g.loss, scale_step=g.scale_step)
    assert rep.iters_done == g.expect_iters
    assert float(t).hex() == g.expect_t.hex()
    bad = np.flatnonzero(x.ravel() != g.x.ravel())
    assert bad.size == 0, f"{bad.size} pixels differ, first {bad[0]}: {x.ravel()[bad[0]]!r} vs {g.x.ravel()[bad[0]]!r}"


@pytest.mark.gpu
@pytest.mark.parametrize("path", CASES, ids=lambda p: p.rsplit("/", 1)[-1][:-4])
@pytest.mark.parametrize("solver", ["launches", "fused"])
def test_cuda_path_meets_golden(path, solver):
    from gpu_util import assert_parity, params, solve
    from paper_2207_12244_gb300 import deepfusion as dfl

    g = golden.load(path)
    sv = dfl.DF_SOLVER_LAUNCHES if solver == "launches" else dfl.DF_SOLVER_FUSED
    prm = params(n_gn=g.n_gn, n_pcg=g.n_pcg, delta=g.delta, terms=g.terms, loss=g.loss,
                 scale_step=g.scale_step, solver=sv)
    x, t, _ = solve(g, prm)
    assert_parity(x, t, g.x, g.expect_t, what=g.name)


@pytest.mark.parametrize("path", STEREO, ids=lambda p: p.rsplit("/", 1)[-1][:-4])
def test_stereo_oracle_reproduces_golden_bitwise(path):
    g = golden.load(path)
    d, v, st, bs, mg, n = oracle.get().semi_dense(g.img_key, g.img_ref, tuple(g.cam), g.R, g.t)
    assert n == g.expect_measured
    assert np.array_equal(st, g.expect_status) and np.array_equal(bs, g.expect_best)
    assert np.array_equal(d, g.expect_depth) and np.array_equal(v, g.expect_var)
    assert np.array_equal(mg.astype(np.float32).astype(np.float64), g.expect_margin)


@pytest.mark.gpu
@pytest.mark.parametrize("path", STEREO, ids=lambda p: p.rsplit("/", 1)[-1][:-4])
def test_cuda_stereo_meets_golden(path):
    from test_gpu_mvs import _compare, _gpu

    g = golden.load(path)
    got = _gpu(g.img_key, g.img_ref, tuple(g.cam), g.R, g.t)
    want = (g.expect_depth, g.expect_var, g.expect_status, g.expect_best, g.expect_margin,
            g.expect_measured)
    n = _compare(got, want, g.name)
    assert n > 0.2 * g.expect_measured
