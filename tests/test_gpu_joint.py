"""Joint (x, t) variant of the GN iteration (bordered Jacobi-PCG) and the
accuracy measure of Section III-B, on the GPU through the C ABI, against the
FP64 oracle."""
import numpy as np
import pytest

import oracle as orc
from gpu_util import (DEPTH_RTOL, SCALE_ATOL, assert_parity, create, oracle_solve, params,
                      solve, to_dev, torch_cuda)
from paper_2207_12244_gb300 import deepfusion as dfl
from paper_2207_12244_gb300 import synth

pytestmark = pytest.mark.gpu

JOINT = dfl.DF_SCALE_JOINT


@pytest.fixture(scope="module")
def o():
    return orc.get()


# (solver, fused kernel mode, pixels per lane): the launch solver, the
# resident kernel, and the streaming kernel with 4 pixels per lane
SOLVERS = [(dfl.DF_SOLVER_LAUNCHES, dfl.DF_MODE_AUTO, 0),
           (dfl.DF_SOLVER_FUSED, dfl.DF_MODE_RESIDENT, 0),
           (dfl.DF_SOLVER_FUSED, dfl.DF_MODE_STREAMING, 4)]


@pytest.fixture(params=SOLVERS, ids=["launches", "resident", "streaming"])
def solver(request):
    sv, mode, vec = request.param
    dfl.df_set_tuning(mode=mode, vec=vec)
    yield sv
    dfl.df_set_tuning()


@pytest.mark.parametrize("W,H", [(256, 192), (37, 23), (1, 1), (129, 3), (3, 130), (300, 41)])
@pytest.mark.parametrize("delta", [1.345, float("inf")], ids=["huber", "l2"])
def test_joint_matches_oracle(o, W, H, delta, solver):
    kf = synth.make_keyframe(W, H, 300 + W + H)
    prm = params(n_gn=10, n_pcg=3, delta=delta, scale_step=JOINT, solver=solver)
    x, t, rep = solve(kf, prm)
    xo, to, ro = oracle_solve(o, kf, prm)
    assert rep.iters_done == ro.iters_done
    assert_parity(x, t, xo, to, what=f"joint {W}x{H}")
    if W * H > 1:
        assert abs(t) > 1e-3  # the border moved t


def test_joint_on_the_streaming_kernel_at_1920x1440(o):
    """A keyframe beyond the on-chip capacity: the joint solve runs on the
    streaming kernel (4 pixels per lane, the automatic launch shape) with
    DF_SOLVER_FUSED and matches the oracle at every pixel."""
    kf = synth.make_keyframe(1920, 1440, 33)
    prm = params(n_gn=10, n_pcg=3, scale_step=JOINT, solver=dfl.DF_SOLVER_FUSED)
    x, t, rep = solve(kf, prm)
    xo, to, ro = oracle_solve(o, kf, prm)
    assert rep.iters_done == ro.iters_done == 30
    assert_parity(x, t, xo, to, what="joint 1920x1440 streaming")
    assert abs(t) > 1e-3


def test_joint_routing(o):
    """AUTO runs the joint solve on the resident kernel, or on the launch
    solver where the launch shape streams one pixel per lane or a tolerance
    is set; FUSED is refused in those cases."""
    kf = synth.make_keyframe(96, 72, 7)
    want = oracle_solve(o, kf, params(n_gn=5, n_pcg=4, scale_step=JOINT))
    x, t, _ = solve(kf, params(n_gn=5, n_pcg=4, scale_step=JOINT, solver=dfl.DF_SOLVER_AUTO))
    assert_parity(x, t, want[0], want[1], what="joint auto")
    dfl.df_set_tuning(mode=dfl.DF_MODE_STREAMING, vec=1)
    try:
        x, t, _ = solve(kf, params(n_gn=5, n_pcg=4, scale_step=JOINT, solver=dfl.DF_SOLVER_AUTO))
        assert_parity(x, t, want[0], want[1], what="joint auto, streaming shape")
        with pytest.raises(dfl.DFError) as e:
            solve(kf, params(scale_step=JOINT, solver=dfl.DF_SOLVER_FUSED))
        assert e.value.status == dfl.DF_ENOTSUP
    finally:
        dfl.df_set_tuning()
    with pytest.raises(dfl.DFError) as e:
        solve(kf, params(scale_step=JOINT, solver=dfl.DF_SOLVER_FUSED, tol=1e-3))
    assert e.value.status == dfl.DF_ENOTSUP
    with pytest.raises(dfl.DFError) as e:
        solve(kf, params(scale_step=3))
    assert e.value.status == dfl.DF_EINVAL


def test_joint_without_semi_keeps_t(o):
    kf = synth.make_keyframe(64, 48, 9)
    xj, tj, _ = solve(kf, params(n_gn=4, n_pcg=5, scale_step=JOINT), semi=False, t0=0.3)
    xf, tf, _ = solve(kf, params(n_gn=4, n_pcg=5, scale_step=dfl.DF_SCALE_FIXED), semi=False,
                      t0=0.3)
    assert tj == 0.3 and tf == 0.3
    assert np.array_equal(xj, xf)


def test_long_runs_of_both_variants(o):
    """Long runs (many GN iterations, converged PCG) of each variant match the
    oracle's run of the same schedule; that the two variants share one
    minimiser is shown in FP64 by the oracle's pins. The joint variant gets
    there in far fewer GN iterations than the alternation."""
    kf = synth.make_keyframe(48, 36, 11)
    pj = params(n_gn=40, n_pcg=30, scale_step=JOINT)
    xj, tj, _ = solve(kf, pj)
    xo, to, _ = oracle_solve(o, kf, pj)
    assert_parity(xj, tj, xo, to, rtol=2e-4, atol_t=2e-4, what="joint long")
    pa = params(n_gn=40, n_pcg=30)
    xa, ta, _ = solve(kf, pa)
    xao, tao, _ = oracle_solve(o, kf, pa)
    assert_parity(xa, ta, xao, tao, rtol=2e-4, atol_t=2e-4, what="alternation long")
    xstar, tstar, _ = o.optimise(kf, n_gn=200, n_pcg=300, scale_step=orc.SCALE_JOINT)
    assert abs(tj - tstar) < 0.1 * abs(ta - tstar)


def test_joint_warm_started_sequence(o, solver):
    torch = torch_cuda()
    kf, mus, vs = synth.make_sequence(128, 96, 23, n_frames=30)
    prm = params(n_gn=10, n_pcg=5, scale_step=JOINT, solver=solver)
    k = create(kf)
    try:
        dmu, dvs = to_dev(mus), to_dev(vs)
        for f in range(mus.shape[0]):
            k.frame_update(dmu[f], dvs[f])
            k.optimise(prm)
        out = torch.empty((kf.height, kf.width), dtype=torch.float32, device="cuda")
        k.fetch_depth(out, log_space=True)
        t = k.get_state()
        x = out.double().cpu().numpy()
    finally:
        k.close()
    xo, to = o.optimise_sequence(kf, mus, vs, n_gn=10, n_pcg=5, delta=prm.delta,
                                 scale_step=orc.SCALE_JOINT)
    assert_parity(x, t, xo, to, what="joint sequence")


@pytest.mark.parametrize("on_device", [True, False], ids=["device", "host"])
def test_accuracy_counts_equal_oracle(o, on_device):
    """Counts are integers: bit-exact against the oracle on the same x."""
    torch = torch_cuda()
    kf = synth.make_keyframe(333, 177, 13)
    truth = np.exp(kf.log_depth_true).astype(np.float32)
    truth[5, 7] = 0.0        # invalid truths are not counted
    truth[9, 300] = np.nan
    truth[100, 0] = -2.0
    k = create(kf)
    fracs = []
    try:
        k.frame_update(to_dev(kf.mu_s), to_dev(kf.var_s))
        for stage in range(3):
            if stage:
                k.optimise(params(n_gn=stage * 3, n_pcg=3))
            out = torch.empty((kf.height, kf.width), dtype=torch.float32, device="cuda")
            k.fetch_depth(out, log_space=True)
            x = out.double().cpu().numpy()
            g = np.ascontiguousarray(truth)
            for tol in (0.1, 0.05, 0.25):
                got = k.depth_accuracy(to_dev(g) if on_device else g, tol)
                assert got == o.within(x, g.astype(np.float64), tol), (stage, tol)
            assert got[1] == kf.width * kf.height - 3
            fracs.append(got[0] / got[1])
        assert fracs[2] > fracs[0]  # fusing the semi-dense depth beats the network prior
    finally:
        k.close()
