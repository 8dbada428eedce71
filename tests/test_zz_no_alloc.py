"""df_optimise_noalloc: the solve for callers that cannot allocate device
memory, such as a real-time loop that forbids cudaMalloc after start-up, or
a plugin whose host program owns the device memory through its own
allocator. It works in a static scratch array of the library instead of
allocating. Its result must match the FP64 oracle at the FP32 bar, and the
keyframe entry points' (which allocate at df_keyframe_create) on the same
inputs.

This file is collected last so that a failure here comes after every other
test has run; it also passes alone in a fresh process.
"""
import numpy as np
import pytest

import oracle
from gpu_util import (DEPTH_RTOL, SCALE_ATOL, assert_parity, create, oracle_solve, params, to_dev,
                      torch_cuda)
from paper_2207_12244_gb300 import deepfusion as dfl
from paper_2207_12244_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def o():
    return oracle.get()


def _via_keyframe(kf, prm):
    """The allocating entry points (create, frame update, optimise)."""
    torch = torch_cuda()
    k = create(kf)
    try:
        k.frame_update(to_dev(kf.mu_s), to_dev(kf.var_s))
        rep = k.optimise(prm, report=True)
        out = torch.empty((kf.height, kf.width), dtype=torch.float32, device="cuda")
        k.fetch_depth(out, log_space=True)
        torch.cuda.synchronize()
        return out.double().cpu().numpy(), rep.scale_log
    finally:
        k.close()


def _inputs(kf, semi=True):
    torch = torch_cuda()
    planes = [to_dev(p) for p in kf.cnn_planes]
    semi_planes = [to_dev(kf.mu_s), to_dev(kf.var_s)] if semi else [None, None]
    x = to_dev(kf.mu_n.copy())  # keyframe initialisation: x = mu_n, t = 0
    t = torch.zeros(1, dtype=torch.float64, device="cuda")
    return planes, semi_planes, x, t


def _via_noalloc(kf, prm, semi=True):
    torch = torch_cuda()
    planes, semi_planes, x, t = _inputs(kf, semi)
    dfl.df_optimise_noalloc(kf.width, kf.height, *planes, *semi_planes, x, t, prm)
    torch.cuda.synchronize()
    return x.double().cpu().numpy(), float(t.item())


def test_noalloc_matches_the_oracle_twice_in_a_row(o):
    """10 GN x 3 PCG, Huber, against the FP64 oracle: the paper's 256 x 192
    and an odd size, back to back, so the second call runs on the scratch
    the first one left behind."""
    prm = params(n_gn=10, n_pcg=3, solver=dfl.DF_SOLVER_LAUNCHES)
    for seed, (W, H) in ((41, (256, 192)), (42, (173, 97))):
        kf = synth.make_keyframe(W, H, seed)
        x, t = _via_noalloc(kf, prm)
        xo, to, _ = oracle_solve(o, kf, prm)
        assert_parity(x, t, xo, to, what=f"noalloc vs oracle {W}x{H}")


def test_noalloc_matches_allocating_entry_points_twice_in_a_row():
    prm = params(n_gn=10, n_pcg=3, solver=dfl.DF_SOLVER_LAUNCHES)
    # different keyframes back to back, the last one at the size limit
    # (512 x 384, where the last scratch plane ends at the end of the array)
    for seed, (W, H) in ((31, (256, 192)), (32, (173, 97)), (33, (512, 384))):
        kf = synth.make_keyframe(W, H, seed)
        x_ref, t_ref = _via_keyframe(kf, prm)
        x, t = _via_noalloc(kf, prm)
        assert_parity(x, t, x_ref, t_ref, rtol=DEPTH_RTOL, atol_t=SCALE_ATOL,
                      what=f"noalloc {W}x{H}")


def test_noalloc_allocates_nothing():
    """After a first call (which also loads the kernels), a second call on
    the same device leaves the device's free memory and the library's
    accounted memory unchanged."""
    torch = torch_cuda()
    prm = params(n_gn=4, n_pcg=3, solver=dfl.DF_SOLVER_LAUNCHES)
    kf = synth.make_keyframe(320, 240, 43)
    planes, semi_planes, x, t = _inputs(kf)
    dfl.df_optimise_noalloc(kf.width, kf.height, *planes, *semi_planes, x, t, prm)
    torch.cuda.synchronize()
    free0, used0 = torch.cuda.mem_get_info()[0], dfl.df_memory_in_use()
    dfl.df_optimise_noalloc(kf.width, kf.height, *planes, *semi_planes, x, t, prm)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert dfl.df_memory_in_use() == used0


def test_noalloc_rejects_sizes_beyond_its_limit():
    torch = torch_cuda()
    W, H = 512, 385  # one row more than the 512 x 384 limit
    assert W * H > dfl.DF_NOALLOC_MAX_PIXELS
    z = torch.ones((H, W), device="cuda")
    t = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(dfl.DFError) as e:
        dfl.df_optimise_noalloc(W, H, z, z, z, z, z, z, None, None, z, t, params())
    assert e.value.status == dfl.DF_EINVAL
    assert "no-allocation limit" in str(e.value)


def test_noalloc_joint_variant(o):
    """With the semi-dense term, the joint (x, t) solve needs a scratch plane
    the array does not hold, and the call is refused before anything runs.
    Without it, the joint system's border row is empty: t stays, and the
    result is the oracle's joint solve."""
    torch = torch_cuda()
    z = torch.ones((8, 8), device="cuda")
    t = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(dfl.DFError) as e:
        dfl.df_optimise_noalloc(8, 8, z, z, z, z, z, z, z, z, z, t,
                                params(scale_step=dfl.DF_SCALE_JOINT))
    assert e.value.status == dfl.DF_ENOTSUP
    kf = synth.make_keyframe(96, 72, 44)
    prm = params(n_gn=5, n_pcg=4, scale_step=dfl.DF_SCALE_JOINT)
    x, tj = _via_noalloc(kf, prm, semi=False)
    xo, to, _ = oracle_solve(o, kf, prm, semi=False)
    assert tj == 0.0
    assert_parity(x, tj, xo, to, what="noalloc joint without semi-dense planes")
