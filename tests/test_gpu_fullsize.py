"""Parity at the benchmarks' full sizes, in the launch configuration bench.py
times (one batched solve of all keyframes per frame, automatic kernel choice;
for the 64-keyframe batch the autotuned launch shape replayed from a CUDA
graph).

* One 1920 x 1440 keyframe, 10 GN x 3 PCG, with FP32, BF16 and FP16 network
  planes: every pixel against the FP64 oracle on the same (rounded) inputs.
* 64 keyframes of uneven sizes, 10 x 3: every pixel of a sample of
  keyframes that covers each size class (the oracle solves one keyframe at a
  time, ~0.5 s for 1280 x 960), and the depth of every keyframe finite and
  positive.
"""
import numpy as np
import pytest

import oracle
from gpu_util import assert_parity, torch_cuda
from paper_2207_12244_gb300 import deepfusion as dfl
from paper_2207_12244_gb300 import replicas
from paper_2207_12244_gb300 import synth

pytestmark = pytest.mark.gpu

SEED = 1  # bench.py's default seed (rank 0)


@pytest.fixture(scope="module")
def o():
    return oracle.get()


def _solve_batch(kfs, cnn_dtype, graph=False, autotune=False):
    """The bench's path: keyframes created from device planes, one frame of
    semi-dense data each, one df_optimise_batch; log-depth and t returned."""
    torch = torch_cuda()
    tdt = {dfl.DF_F32: torch.float32, dfl.DF_BF16: torch.bfloat16,
           dfl.DF_F16: torch.float16}[cnn_dtype]
    prm = dfl.df_default_params(n_gn=10, n_pcg=3)
    ks = []
    try:
        for kf in kfs:
            planes = [torch.from_numpy(p).to(tdt).cuda() for p in kf.cnn_planes]
            k = dfl.Keyframe(kf.width, kf.height, *planes, cnn_dtype=cnn_dtype)
            ks.append(k)
            k.frame_update(torch.from_numpy(kf.mu_s).cuda(), torch.from_numpy(kf.var_s).cuda())
        handles = [k.handle for k in ks]
        if autotune:
            dfl.df_autotune(handles, prm)
            for k, kf in zip(ks, kfs):  # the autotuner leaves the state as it found it
                k.frame_update(torch.from_numpy(kf.mu_s).cuda(),
                               torch.from_numpy(kf.var_s).cuda())
        if graph:
            stream = torch.cuda.Stream()
            dfl.df_batch_prepare(handles, stream=stream.cuda_stream)
            torch.cuda.synchronize()
            g = torch.cuda.CUDAGraph()
            with torch.cuda.stream(stream):
                with torch.cuda.graph(g, stream=stream):
                    dfl.df_optimise_batch(handles, prm, stream=stream.cuda_stream)
            torch.cuda.synchronize()
            g.replay()
        else:
            dfl.df_optimise_batch(handles, prm)
        out = []
        for k, kf in zip(ks, kfs):
            d = torch.empty((kf.height, kf.width), dtype=torch.float32, device="cuda")
            k.fetch_depth(d, log_space=True)
            out.append((d, k))
        torch.cuda.synchronize()
        return [(d.double().cpu().numpy(), k.get_state()) for d, k in out]
    finally:
        for k in ks:
            k.close()
        dfl.df_set_tuning()


def _rounded_view(kf, cnn_dtype):
    """The keyframe with its network planes rounded to the storage type (the
    values the GPU reads), in float32."""
    import copy

    if cnn_dtype == dfl.DF_F32:
        return kf
    torch = torch_cuda()
    tdt = torch.bfloat16 if cnn_dtype == dfl.DF_BF16 else torch.float16
    kr = copy.copy(kf)
    for n in ("mu_n", "var_n", "gx", "var_gx", "gy", "var_gy"):
        setattr(kr, n, torch.from_numpy(np.ascontiguousarray(getattr(kf, n))).to(tdt).float().numpy())
    return kr


@pytest.mark.parametrize("cnn_dtype", [dfl.DF_F32, dfl.DF_BF16, dfl.DF_F16],
                         ids=["f32", "bf16", "f16"])
def test_1920x1440_every_pixel(o, cnn_dtype):
    kf = synth.make_keyframe(1920, 1440, replicas.rank_seed(SEED, 0))
    (x, t), = _solve_batch([kf], cnn_dtype)
    xo, to, _ = o.optimise(_rounded_view(kf, cnn_dtype), n_gn=10, n_pcg=3)
    assert_parity(x, t, xo, to, what=f"1920x1440 dtype {cnn_dtype}")


def test_batch64_sampled_keyframes(o):
    base = replicas.rank_seed(SEED, 0)
    shapes = synth.batch_shapes(64, base)
    kfs = [synth.make_keyframe(W, H, base + 17 * i) for i, (W, H) in enumerate(shapes)]
    res = _solve_batch(kfs, dfl.DF_F32, graph=True, autotune=True)
    for (x, t), kf in zip(res, kfs):
        assert np.all(np.isfinite(x)), (kf.width, kf.height)
    # the first keyframe of each size class, and the last keyframe
    sample = sorted({shapes.index(s) for s in set(shapes)} | {len(kfs) - 1})
    for i in sample:
        xo, to, _ = o.optimise(kfs[i], n_gn=10, n_pcg=3)
        assert_parity(res[i][0], res[i][1], xo, to, what=f"keyframe {i} {shapes[i]}")
