"""Batched uneven keyframes and reduced-precision network planes vs the oracle.

* Batches: several keyframes of different sizes solved by one fused launch
  (df_optimise_batch) match the oracle keyframe by keyframe, and each
  result is the one df_optimise gives that keyframe alone (same bar).
* BF16 / FP16 network planes: against the oracle run on the same rounded
  inputs the bar is the FP32 one (the arithmetic is identical); against the
  oracle on the original FP32 inputs the error is the rounding's, stated and
  bounded.
"""
import numpy as np
import pytest

import oracle
from gpu_util import assert_parity, create, depth_rel_err, oracle_solve, params, solve, to_dev, \
    torch_cuda
from paper_2207_12244_gb300 import deepfusion as dfl
from paper_2207_12244_gb300 import synth

pytestmark = pytest.mark.gpu

MODES = [dfl.DF_MODE_STREAMING, dfl.DF_MODE_RESIDENT, dfl.DF_MODE_AUTO]
MODE_IDS = ["streaming", "resident", "auto"]


@pytest.fixture(scope="module")
def o():
    return oracle.get()


@pytest.fixture(params=MODES, ids=MODE_IDS)
def mode(request):
    dfl.df_set_tuning(mode=request.param)
    yield request.param
    dfl.df_set_tuning()


def _fetch(k, kf):
    torch = torch_cuda()
    out = torch.empty((kf.height, kf.width), dtype=torch.float32, device="cuda")
    k.fetch_depth(out, log_space=True)
    t = k.get_state()
    return out.double().cpu().numpy(), t


def _batch(kfs, prm):
    ks = [create(kf) for kf in kfs]
    try:
        for k, kf in zip(ks, kfs):
            k.frame_update(to_dev(kf.mu_s), to_dev(kf.var_s))
        reps = dfl.df_optimise_batch([k.handle for k in ks], prm, report=True)
        return [_fetch(k, kf) for k, kf in zip(ks, kfs)], reps
    finally:
        for k in ks:
            k.close()


SHAPES = [(64, 48), (37, 29), (100, 70), (16, 16), (128, 96), (1, 40), (200, 3)]


def test_batch_uneven_matches_oracle_and_alone(o, mode):
    kfs = [synth.make_keyframe(W, H, 500 + i) for i, (W, H) in enumerate(SHAPES)]
    prm = params(n_gn=6, n_pcg=4, solver=dfl.DF_SOLVER_FUSED)
    res, reps = _batch(kfs, prm)
    for i, (kf, (x, t), rep) in enumerate(zip(kfs, res, reps)):
        xo, to, ro = oracle_solve(o, kf, prm)
        assert_parity(x, t, xo, to, what=f"batch item {i} {kf.width}x{kf.height}")
        assert rep.iters_done == ro.iters_done
        xa, ta, _ = solve(kf, prm)  # the same keyframe alone
        assert_parity(x, t, xa, ta, what=f"alone vs batch {i}")


def test_many_small_keyframes_share_ctas(o):
    """More keyframes than a CTA's segment capacity: the streaming plan
    splits or caps segments, every result still matches."""
    rng = np.random.default_rng(9)
    kfs = [synth.make_keyframe(int(rng.integers(8, 40)), int(rng.integers(4, 30)), 700 + i)
           for i in range(40)]
    prm = params(n_gn=3, n_pcg=3, solver=dfl.DF_SOLVER_FUSED)
    try:
        # (mode, grid cap, pixels per lane, assembly placement): the 4-wide
        # streaming kernel with its assembly in a kernel of its own and in a
        # pass of the persistent kernel
        for m, cap, vec, asm in ((dfl.DF_MODE_STREAMING, 4, 0, 0), (dfl.DF_MODE_STREAMING, 0, 0, 0),
                                 (dfl.DF_MODE_STREAMING, 0, 4, 2), (dfl.DF_MODE_STREAMING, 6, 4, 2),
                                 (dfl.DF_MODE_STREAMING, 0, 4, 1), (dfl.DF_MODE_RESIDENT, 0, 0, 0)):
            dfl.df_set_tuning(mode=m, max_ctas=cap, vec=vec, assembly=asm)
            res, _ = _batch(kfs, prm)
            for i, (kf, (x, t)) in enumerate(zip(kfs, res)):
                xo, to, _ = oracle_solve(o, kf, prm)
                assert_parity(x, t, xo, to, what=f"mode {m} cap {cap} vec {vec} asm {asm} item {i}")
    finally:
        dfl.df_set_tuning()


def test_batch_with_launch_schedule_and_bad_lists(o):
    kfs = [synth.make_keyframe(W, H, 800 + i) for i, (W, H) in enumerate(SHAPES[:3])]
    prm = params(n_gn=4, n_pcg=3, solver=dfl.DF_SOLVER_LAUNCHES)
    res, _ = _batch(kfs, prm)
    for kf, (x, t) in zip(kfs, res):
        xo, to, _ = oracle_solve(o, kf, prm)
        assert_parity(x, t, xo, to, what="launch batch")
    k = create(kfs[0])
    try:
        with pytest.raises(dfl.DFError) as e:
            dfl.df_optimise_batch([k.handle, k.handle], prm)
        assert e.value.status == dfl.DF_EINVAL
        assert dfl.df_optimise_batch([], prm) is None
    finally:
        k.close()


@pytest.mark.parametrize("mode", [dfl.DF_MODE_STREAMING, dfl.DF_MODE_RESIDENT],
                         ids=["streaming", "resident"])
def test_prepared_batch_captured_in_a_cuda_graph(o, mode):
    """A batched solve of uneven keyframes, prepared once and captured in a
    CUDA graph, replays to the eager result bitwise; capturing an unprepared
    batch is refused without touching the capture."""
    torch = torch_cuda()
    kfs = [synth.make_keyframe(W, H, 900 + i) for i, (W, H) in enumerate(SHAPES[:5])]
    prm = params(n_gn=4, n_pcg=3, solver=dfl.DF_SOLVER_FUSED)
    dfl.df_set_tuning(mode=mode)
    ks = [create(kf) for kf in kfs]
    try:
        semi = [(to_dev(kf.mu_s), to_dev(kf.var_s)) for kf in kfs]
        handles = [k.handle for k in ks]

        def frame():
            for k, (m, v) in zip(ks, semi):
                k.frame_update(m, v)
            dfl.df_optimise_batch(handles, prm)

        frame()
        eager = [_fetch(k, kf) for k, kf in zip(ks, kfs)]
        for k, kf in zip(ks, kfs):
            k.set_state(to_dev(kf.mu_n), 0.0)
        torch.cuda.synchronize()
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        g0 = torch.cuda.CUDAGraph()
        refused = None
        with torch.cuda.stream(s):
            with torch.cuda.graph(g0, stream=s):
                try:
                    dfl.df_optimise_batch(handles, prm)
                except dfl.DFError as e:
                    refused = e.status
        assert refused == dfl.DF_ENOTSUP
        dfl.df_batch_prepare(handles)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.stream(s):
            with torch.cuda.graph(g, stream=s):
                frame()
        torch.cuda.current_stream().wait_stream(s)
        g.replay()
        torch.cuda.synchronize()
        got = [_fetch(k, kf) for k, kf in zip(ks, kfs)]
        for i, ((xe, te), (xg, tg)) in enumerate(zip(eager, got)):
            assert np.array_equal(xe, xg) and te == tg, f"item {i}"
            xo, to, _ = oracle_solve(o, kfs[i], prm)
            assert_parity(xg, tg, xo, to, what=f"graph item {i}")
        dfl.df_batch_release(handles)
    finally:
        for k in ks:
            k.close()
        dfl.df_set_tuning()


def _rounded(kf, torch_dtype):
    """The network planes rounded to torch_dtype on the CPU (round to nearest
    even) and a copy of the keyframe whose planes are those values in FP32."""
    import copy

    torch = torch_cuda()
    planes = [torch.from_numpy(np.ascontiguousarray(p)).to(torch_dtype) for p in kf.cnn_planes]
    kr = copy.copy(kf)
    names = ("mu_n", "var_n", "gx", "var_gx", "gy", "var_gy")
    for n, p in zip(names, planes):
        setattr(kr, n, p.float().numpy())
    return planes, kr


@pytest.mark.parametrize("dt", [dfl.DF_BF16, dfl.DF_F16], ids=["bf16", "fp16"])
@pytest.mark.parametrize("sv", [(dfl.DF_SOLVER_LAUNCHES, 0), (dfl.DF_SOLVER_FUSED, 1),
                                (dfl.DF_SOLVER_FUSED, 2)], ids=["launches", "streaming", "resident"])
def test_reduced_precision_network_planes(o, dt, sv):
    torch = torch_cuda()
    solver, m = sv
    kf = synth.make_keyframe(160, 120, 901)
    td = torch.bfloat16 if dt == dfl.DF_BF16 else torch.float16
    planes, kr = _rounded(kf, td)
    prm = params(n_gn=10, n_pcg=3, solver=solver)
    dfl.df_set_tuning(mode=m)
    try:
        k = dfl.Keyframe(kf.width, kf.height, *[p.cuda() for p in planes], cnn_dtype=dt)
        try:
            k.frame_update(to_dev(kf.mu_s), to_dev(kf.var_s))
            k.optimise(prm)
            x, t = _fetch(k, kf)
        finally:
            k.close()
    finally:
        dfl.df_set_tuning()
    # same rounded inputs: the FP32 bar
    xr, tr, _ = oracle_solve(o, kr, prm)
    assert_parity(x, t, xr, tr, what="rounded inputs")
    # original FP32 inputs: the rounding's own error, stated
    xo, to, _ = oracle_solve(o, kf, prm)
    e = depth_rel_err(x, xo)
    bound = 2e-2 if dt == dfl.DF_BF16 else 3e-3
    print(f"{'bf16' if dt == dfl.DF_BF16 else 'fp16'}: vs FP32-input oracle max {e.max():.3g} "
          f"mean {e.mean():.3g}, |dt| {abs(t - to):.3g}")
    assert e.max() < bound and abs(t - to) < bound


def test_reduced_precision_host_pointers():
    """BF16 codes from the host go through the same host-side checks."""
    torch = torch_cuda()
    kf = synth.make_keyframe(48, 32, 902)
    planes = [torch.from_numpy(np.ascontiguousarray(p)).to(torch.bfloat16) for p in kf.cnn_planes]
    xd = solve(kf, params(), cnn_dtype=dfl.DF_BF16)  # device pointers
    k = dfl.Keyframe(kf.width, kf.height, *planes, cnn_dtype=dfl.DF_BF16)  # host pointers
    try:
        k.frame_update(np.ascontiguousarray(kf.mu_s), np.ascontiguousarray(kf.var_s))
        k.optimise(params())
        x, t = _fetch(k, kf)
    finally:
        k.close()
    assert np.array_equal(x, xd[0])
    bad = [p.clone() for p in planes]
    bad[1][0, 0] = -1.0
    with pytest.raises(dfl.DFError) as e:
        dfl.Keyframe(kf.width, kf.height, *bad, cnn_dtype=dfl.DF_BF16)
    assert e.value.status == dfl.DF_EINVAL


@pytest.mark.parametrize("mode", [dfl.DF_MODE_STREAMING, dfl.DF_MODE_RESIDENT],
                         ids=["streaming", "resident"])
def test_batch_of_mixed_network_precisions(o, mode):
    """One fused launch over keyframes whose network planes are stored in
    FP32, BF16 and FP16: each keyframe meets the FP32 bar against the oracle
    on its own (rounded) inputs."""
    torch = torch_cuda()
    shapes = [(96, 72), (50, 37), (128, 40), (33, 90)]
    dts = [dfl.DF_F32, dfl.DF_BF16, dfl.DF_F16, dfl.DF_BF16]
    kfs = [synth.make_keyframe(W, H, 1100 + i) for i, (W, H) in enumerate(shapes)]
    prm = params(n_gn=6, n_pcg=4, solver=dfl.DF_SOLVER_FUSED)
    dfl.df_set_tuning(mode=mode)
    ks, refs = [], []
    try:
        for kf, dt in zip(kfs, dts):
            if dt == dfl.DF_F32:
                ks.append(create(kf))
                refs.append(kf)
            else:
                td = torch.bfloat16 if dt == dfl.DF_BF16 else torch.float16
                planes, kr = _rounded(kf, td)
                ks.append(dfl.Keyframe(kf.width, kf.height, *[p.cuda() for p in planes],
                                       cnn_dtype=dt))
                refs.append(kr)
        for k, kf in zip(ks, kfs):
            k.frame_update(to_dev(kf.mu_s), to_dev(kf.var_s))
        dfl.df_optimise_batch([k.handle for k in ks], prm)
        for i, (k, kf, kr) in enumerate(zip(ks, kfs, refs)):
            x, t = _fetch(k, kf)
            xo, to, _ = oracle_solve(o, kr, prm)
            assert_parity(x, t, xo, to, what=f"mixed batch item {i} dtype {dts[i]}")
    finally:
        for k in ks:
            k.close()
        dfl.df_set_tuning()
