"""df_optimise_noalloc: the solve for callers that cannot allocate device
memory (for example code running under someone else's CUDA graph capture, or
a real-time loop that forbids cudaMalloc). It works in a static scratch array
of the library instead of allocating; its result must match the keyframe
entry points' (which allocate at df_keyframe_create) on the same inputs.

This file is collected last so that a failure here comes after every other
test has run; it also passes alone in a fresh process.
"""
import numpy as np
import pytest

from gpu_util import DEPTH_RTOL, SCALE_ATOL, assert_parity, create, params, to_dev, torch_cuda
from paper_2207_12244_gb300 import deepfusion as dfl
from paper_2207_12244_gb300 import synth

pytestmark = pytest.mark.gpu


def _via_keyframe(kf, prm):
    """Reference: the allocating entry points (create, frame update, optimise)."""
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


def _via_noalloc(kf, prm):
    torch = torch_cuda()
    planes = [to_dev(p) for p in kf.cnn_planes]
    x = to_dev(kf.mu_n.copy())  # keyframe initialisation: x = mu_n, t = 0
    t = torch.zeros(1, dtype=torch.float64, device="cuda")
    dfl.df_optimise_noalloc(kf.width, kf.height, *planes, to_dev(kf.mu_s), to_dev(kf.var_s),
                            x, t, prm)
    torch.cuda.synchronize()
    return x.double().cpu().numpy(), float(t.item())


def test_noalloc_matches_allocating_entry_points_twice_in_a_row():
    prm = params(n_gn=10, n_pcg=3, solver=dfl.DF_SOLVER_LAUNCHES)
    # two different keyframes back to back: the second call reuses the
    # scratch the first one left behind
    for seed, (W, H) in ((31, (256, 192)), (32, (173, 97))):
        kf = synth.make_keyframe(W, H, seed)
        x_ref, t_ref = _via_keyframe(kf, prm)
        x, t = _via_noalloc(kf, prm)
        assert_parity(x, t, x_ref, t_ref, rtol=DEPTH_RTOL, atol_t=SCALE_ATOL,
                      what=f"noalloc {W}x{H}")


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


def test_noalloc_refuses_the_joint_variant():
    """Its scratch has no plane for the semi-dense weights the joint (x, t)
    solve keeps; the call is refused before anything runs."""
    torch = torch_cuda()
    z = torch.ones((8, 8), device="cuda")
    t = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(dfl.DFError) as e:
        dfl.df_optimise_noalloc(8, 8, z, z, z, z, z, z, z, z, z, t,
                                params(scale_step=dfl.DF_SCALE_JOINT))
    assert e.value.status == dfl.DF_ENOTSUP
