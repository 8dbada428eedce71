"""Golden fixtures (tests/golden/*.txt, written from the FP64 oracle).

CPU: the oracle built on this host reproduces every fixture bit for bit
(plain C, FP64, no FMA contraction, so x86 and Arm agree), which freezes its
arithmetic between changes.
GPU: the CUDA path, through the C ABI, meets the FP32 parity bar against the
stored results without running the oracle.
"""
import numpy as np
import pytest

import golden
import oracle

CASES = golden.paths()


def test_fixtures_present():
    assert len(CASES) >= 5


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
