"""Batched per-frame bookkeeping (df_keyframe_reset_batch, df_frame_update_batch,
df_fetch_depth_batch) against the single-keyframe calls and the oracle.

The batched calls do the same work as one df_keyframe_reset /
df_frame_update / df_fetch_depth per keyframe, so every result must be
bitwise the same: the copied planes, the initial state, the device-side
input check and the depth output. Covered: uneven sizes (widths that take
the 16-byte vector path and widths that do not), more keyframes than one
launch holds, FP32 / BF16 / FP16 network planes in one list, host buffers,
CUDA-graph capture, and the refusals.
"""
import types

import numpy as np
import pytest

import oracle
from gpu_util import assert_parity, oracle_solve, params, to_dev, torch_cuda
from paper_2207_12244_gb300 import deepfusion as dfl
from paper_2207_12244_gb300 import synth

pytestmark = pytest.mark.gpu

# 30 keyframes (two launches of the batched copies): widths divisible by 8
# (vector path for every dtype), by 4 only (vector path for f32 only) and odd
SHAPES = [(64, 48), (37, 23), (100, 20), (33, 9), (128, 96), (17, 13)] * 5
DTYPES = [dfl.DF_F32, dfl.DF_BF16, dfl.DF_F16]


@pytest.fixture(scope="module")
def o():
    return oracle.get()


def _planes(kf, dt, dev=True):
    torch = torch_cuda()
    td = {dfl.DF_F32: torch.float32, dfl.DF_BF16: torch.bfloat16, dfl.DF_F16: torch.float16}[dt]
    ps = [torch.from_numpy(np.ascontiguousarray(p)).to(td) for p in kf.cnn_planes]
    return [p.cuda() for p in ps] if dev else ps


def _make(n=len(SHAPES), seed=500):
    kfs = [synth.make_keyframe(W, H, seed + i) for i, (W, H) in enumerate(SHAPES[:n])]
    dts = [DTYPES[i % 3] for i in range(n)]
    return kfs, dts


def _keyframes(kfs, dts):
    # created from different planes (so that a reset really changes them)
    return [dfl.Keyframe(kf.width, kf.height, *_planes(synth.make_keyframe(kf.width, kf.height, 7),
                                                        dt), cnn_dtype=dt)
            for kf, dt in zip(kfs, dts)]


def _state(ks, kfs):
    torch = torch_cuda()
    out = []
    for k, kf in zip(ks, kfs):
        x = torch.empty((kf.height, kf.width), dtype=torch.float32, device="cuda")
        t = k.get_state(x)
        out.append((x.cpu().numpy(), t))
    return out


def test_batched_calls_equal_the_single_keyframe_calls(o):
    torch = torch_cuda()
    kfs, dts = _make()
    planes = [_planes(kf, dt) for kf, dt in zip(kfs, dts)]
    semi = [(to_dev(kf.mu_s), to_dev(kf.var_s)) for kf in kfs]
    prm = params(n_gn=3, n_pcg=3, solver=dfl.DF_SOLVER_FUSED)
    a, b = _keyframes(kfs, dts), _keyframes(kfs, dts)
    try:
        # reset: x = mu_n and t = 0, bitwise as the single call
        dfl.df_keyframe_reset_batch([k.handle for k in a], planes)
        for k, p in zip(b, planes):
            k.reset(*p)
        sa, sb = _state(a, kfs), _state(b, kfs)
        for i, ((xa, ta), (xb, tb)) in enumerate(zip(sa, sb)):
            assert np.array_equal(xa, xb) and ta == tb == 0.0, i
            want = planes[i][0].float().cpu().numpy()
            assert np.array_equal(xa, want), i
        # frame update, solve, fetch
        dfl.df_frame_update_batch([k.handle for k in a], [m for m, _ in semi], [v for _, v in semi])
        for k, (m, v) in zip(b, semi):
            k.frame_update(m, v)
        dfl.df_optimise_batch([k.handle for k in a], prm)
        dfl.df_optimise_batch([k.handle for k in b], prm)
        for log_space in (False, True):
            outs = [torch.empty((kf.height, kf.width), device="cuda") for kf in kfs]
            dfl.df_fetch_depth_batch([k.handle for k in a], outs, log_space=log_space)
            for i, (k, kf, o_) in enumerate(zip(b, kfs, outs)):
                ref = torch.empty_like(o_)
                k.fetch_depth(ref, log_space=log_space)
                assert torch.equal(o_, ref), (i, log_space)
        for i, ((xa, ta), (xb, tb)) in enumerate(zip(_state(a, kfs), _state(b, kfs))):
            assert np.array_equal(xa, xb) and ta == tb, i
        # and against the oracle on the planes as stored (rounded for 16-bit)
        for i in (0, 1, 2, 4, 5):
            kf = kfs[i]
            view = types.SimpleNamespace(**vars(kf))
            rounded = [p.float().cpu().numpy() for p in planes[i]]
            for n_, p in zip(("mu_n", "var_n", "gx", "var_gx", "gy", "var_gy"), rounded):
                setattr(view, n_, p)
            xo, to, _ = oracle_solve(o, view, prm)
            xa, ta = _state(a[i:i + 1], kfs[i:i + 1])[0]
            assert_parity(xa.astype(np.float64), ta, xo, to, what=f"batched io {i}")
    finally:
        for k in a + b:
            k.close()


def test_batched_reset_checks_inputs_like_the_single_call():
    """Invalid network values flag exactly the keyframes the single-keyframe
    reset flags; values the method never reads (gx in the last column, gy in
    the last row) are ignored."""
    kfs, dts = _make(6, seed=620)
    cases = []
    for i, (kf, dt) in enumerate(zip(kfs, dts)):
        p = [q.clone() for q in _planes(kf, dt)]
        H, W = kf.height, kf.width
        if i == 0:
            p[1][H // 2, W // 3] = -1.0          # a negative network variance
        elif i == 1:
            p[2][H - 1, W - 1] = float("nan")    # gx in the last column: not read
            p[5][H - 1, 0] = 0.0                 # var_gy in the last row: not read
        elif i == 2:
            p[4][0, W - 1] = float("inf")        # gy in row 0: read
        elif i == 3:
            p[0][H - 1, W - 1] = float("nan")    # mu_n
        cases.append(p)
    a, b = _keyframes(kfs, dts), _keyframes(kfs, dts)
    try:
        dfl.df_keyframe_reset_batch([k.handle for k in a], cases)
        for k, p in zip(b, cases):
            k.reset(*p)
        for i, (ka, kb) in enumerate(zip(a, b)):
            st = []
            for k in (ka, kb):
                try:
                    k.check()
                    st.append(dfl.DF_OK)
                except dfl.DFError as e:
                    st.append(e.status)
            assert st[0] == st[1], (i, st)
            assert (st[0] != dfl.DF_OK) == (i in (0, 2, 3)), (i, st)
    finally:
        for k in a + b:
            k.close()


def test_batched_calls_from_host_buffers_equal_device_buffers():
    torch = torch_cuda()
    kfs, dts = _make(8, seed=640)
    a, b = _keyframes(kfs, dts), _keyframes(kfs, dts)
    try:
        dfl.df_keyframe_reset_batch([k.handle for k in a], [_planes(kf, dt) for kf, dt in zip(kfs, dts)])
        host = []
        for kf, dt in zip(kfs, dts):
            ps = _planes(kf, dt, dev=False)
            host.append([p.numpy() if p.dtype != torch.bfloat16 else p.view(torch.int16).numpy()
                         for p in ps])
        dfl.df_keyframe_reset_batch([k.handle for k in b], host)
        dfl.df_frame_update_batch([k.handle for k in a], [to_dev(kf.mu_s) for kf in kfs],
                                  [to_dev(kf.var_s) for kf in kfs])
        dfl.df_frame_update_batch([k.handle for k in b], [np.ascontiguousarray(kf.mu_s) for kf in kfs],
                                  [np.ascontiguousarray(kf.var_s) for kf in kfs])
        prm = params(n_gn=2, n_pcg=2, solver=dfl.DF_SOLVER_FUSED)
        dfl.df_optimise_batch([k.handle for k in a], prm)
        dfl.df_optimise_batch([k.handle for k in b], prm)
        dev_out = [torch.empty((kf.height, kf.width), device="cuda") for kf in kfs]
        host_out = [np.empty((kf.height, kf.width), np.float32) for kf in kfs]
        dfl.df_fetch_depth_batch([k.handle for k in a], dev_out)
        dfl.df_fetch_depth_batch([k.handle for k in b], host_out)
        torch.cuda.synchronize()
        for i, (d, h) in enumerate(zip(dev_out, host_out)):
            assert np.array_equal(d.cpu().numpy(), h), i
    finally:
        for k in a + b:
            k.close()


def test_batched_frame_captured_in_a_cuda_graph():
    """Reset, frame update, batched solve and depth output of a prepared list
    captured once in a CUDA graph replay to the eager result bitwise."""
    torch = torch_cuda()
    kfs, dts = _make(26, seed=660)
    planes = [_planes(kf, dt) for kf, dt in zip(kfs, dts)]
    mu = [to_dev(kf.mu_s) for kf in kfs]
    var = [to_dev(kf.var_s) for kf in kfs]
    outs = [torch.empty((kf.height, kf.width), device="cuda") for kf in kfs]
    prm = params(n_gn=3, n_pcg=2, solver=dfl.DF_SOLVER_FUSED)
    ks = _keyframes(kfs, dts)
    h = [k.handle for k in ks]
    try:
        def frame():
            dfl.df_keyframe_reset_batch(h, planes)
            dfl.df_frame_update_batch(h, mu, var)
            dfl.df_optimise_batch(h, prm)
            dfl.df_fetch_depth_batch(h, outs)

        frame()
        torch.cuda.synchronize()
        eager = [o_.clone() for o_ in outs]
        for o_ in outs:
            o_.zero_()
        dfl.df_batch_prepare(h)
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        g = torch.cuda.CUDAGraph()
        with torch.cuda.stream(s):
            with torch.cuda.graph(g, stream=s):
                frame()
        torch.cuda.current_stream().wait_stream(s)
        g.replay()
        torch.cuda.synchronize()
        for i, (e, o_) in enumerate(zip(eager, outs)):
            assert torch.equal(e, o_), i
        dfl.df_batch_release(h)
    finally:
        for k in ks:
            k.close()


def test_batched_calls_refuse_bad_lists():
    torch = torch_cuda()
    kfs, dts = _make(2, seed=680)
    ks = _keyframes(kfs, dts)
    try:
        h = [k.handle for k in ks]
        planes = [_planes(kf, dt) for kf, dt in zip(kfs, dts)]
        for bad in ([h[0], h[0]], [h[0], None]):  # a repeated or a missing keyframe
            with pytest.raises(dfl.DFError) as e:
                dfl.df_keyframe_reset_batch(bad, [planes[0], planes[0]])
            assert e.value.status == dfl.DF_EINVAL
        assert dfl.load().df_fetch_depth_batch(None, 2, None, 0, 1, None) == dfl.DF_EINVAL
        with pytest.raises(ValueError):  # a plane of the wrong size
            dfl.df_keyframe_reset_batch(h, [planes[0], planes[0]])
        with pytest.raises(ValueError):
            dfl.df_fetch_depth_batch(h, [torch.empty(3, device="cuda")] * 2)
    finally:
        for k in ks:
            k.close()


def test_pinned_host_buffers_are_read_and_written_directly():
    """Pinned host buffers take the kernels' direct path: the same bits as
    device buffers for the reset, the frame update and the depth output;
    an invalid network value flags its keyframe on the device (the call
    itself succeeds, as with device buffers)."""
    torch = torch_cuda()
    kfs, dts = _make(10, seed=700)
    a, b = _keyframes(kfs, dts), _keyframes(kfs, dts)
    try:
        dev = [_planes(kf, dt) for kf, dt in zip(kfs, dts)]
        pin = [[p.cpu().pin_memory() for p in ps] for ps in dev]
        pin[3][1][2, 5] = -1.0  # a negative network variance in pinned memory
        dev[3][1][2, 5] = -1.0
        dfl.df_keyframe_reset_batch([k.handle for k in a], dev)
        dfl.df_keyframe_reset_batch([k.handle for k in b], pin)
        mu_p = [torch.from_numpy(np.ascontiguousarray(kf.mu_s)).pin_memory() for kf in kfs]
        var_p = [torch.from_numpy(np.ascontiguousarray(kf.var_s)).pin_memory() for kf in kfs]
        dfl.df_frame_update_batch([k.handle for k in a], [to_dev(kf.mu_s) for kf in kfs],
                                  [to_dev(kf.var_s) for kf in kfs])
        dfl.df_frame_update_batch([k.handle for k in b], mu_p, var_p)
        prm = params(n_gn=2, n_pcg=2, solver=dfl.DF_SOLVER_FUSED)
        dfl.df_optimise_batch([k.handle for k in a], prm)
        dfl.df_optimise_batch([k.handle for k in b], prm)
        dev_out = [torch.empty((kf.height, kf.width), device="cuda") for kf in kfs]
        pin_out = [torch.empty((kf.height, kf.width)).pin_memory() for kf in kfs]
        dfl.df_fetch_depth_batch([k.handle for k in a], dev_out)
        dfl.df_fetch_depth_batch([k.handle for k in b], pin_out)
        torch.cuda.synchronize()
        for i, (d, h) in enumerate(zip(dev_out, pin_out)):
            assert torch.equal(d.cpu(), h), i
        for i, (ka, kb) in enumerate(zip(a, b)):
            for k in (ka, kb):
                if i == 3:
                    with pytest.raises(dfl.DFError) as e:
                        k.check()
                    assert e.value.status == dfl.DF_EINVAL
                else:
                    k.check()
    finally:
        for k in a + b:
            k.close()


def test_pinned_host_step_captured_in_a_cuda_graph():
    """The whole per-frame step from pinned host buffers (reset, frame
    update, batched solve, depth output) captured once and replayed: the
    replay reads the host inputs and writes the host outputs again, equal
    to the eager step bitwise."""
    torch = torch_cuda()
    kfs, dts = _make(12, seed=720)
    pin = [[p.cpu().pin_memory() for p in _planes(kf, dt)] for kf, dt in zip(kfs, dts)]
    mu_p = [torch.from_numpy(np.ascontiguousarray(kf.mu_s)).pin_memory() for kf in kfs]
    var_p = [torch.from_numpy(np.ascontiguousarray(kf.var_s)).pin_memory() for kf in kfs]
    outs = [torch.empty((kf.height, kf.width)).pin_memory() for kf in kfs]
    prm = params(n_gn=3, n_pcg=2, solver=dfl.DF_SOLVER_FUSED)
    ks = _keyframes(kfs, dts)
    h = [k.handle for k in ks]
    try:
        s = torch.cuda.Stream()

        def frame():
            dfl.df_keyframe_reset_batch(h, pin, stream=s)
            dfl.df_frame_update_batch(h, mu_p, var_p, stream=s)
            dfl.df_optimise_batch(h, prm, stream=s)
            dfl.df_fetch_depth_batch(h, outs, stream=s)

        with torch.cuda.stream(s):
            frame()
        torch.cuda.synchronize()
        eager = [o.clone() for o in outs]
        dfl.df_batch_prepare(h)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.stream(s):
            with torch.cuda.graph(g, stream=s):
                frame()
        for o in outs:
            o.zero_()
        with torch.cuda.stream(s):
            g.replay()
        torch.cuda.synchronize()
        for i, (e, o) in enumerate(zip(eager, outs)):
            assert torch.equal(e, o), i
        dfl.df_batch_release(h)
    finally:
        for k in ks:
            k.close()
