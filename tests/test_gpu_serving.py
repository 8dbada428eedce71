"""Serving layer on the GPU: continuous batching gives each stream the result
(log-depth and scale) it gets alone, and the oracle's; admission follows the
memory budget; every frame completes exactly once."""
import numpy as np
import pytest

import oracle
from gpu_util import DEPTH_RTOL, SCALE_ATOL, assert_parity, create, params, to_dev, torch_cuda
from paper_2207_12244_gb300 import deepfusion as dfl
from paper_2207_12244_gb300 import serving, synth

pytestmark = pytest.mark.gpu

SIZES = [(64, 48), (96, 72), (40, 30), (128, 96), (64, 48), (80, 60)]


@pytest.fixture(scope="module")
def o():
    return oracle.get()

NF = 4


def _streams():
    seqs = [synth.make_sequence(W, H, 40 + i, n_frames=NF) for i, (W, H) in enumerate(SIZES)]
    frames = [[(to_dev(mus[f]), to_dev(vs[f])) for f in range(NF)] for _, mus, vs in seqs]
    return seqs, frames


def _alone(kf, frames, prm):
    """Reference: one keyframe, its frames in order, one df_optimise each."""
    torch = torch_cuda()
    k = create(kf)
    try:
        for mu, var in frames:
            k.frame_update(mu, var)
            k.optimise(prm)
        out = torch.empty((kf.height, kf.width), dtype=torch.float32, device="cuda")
        k.fetch_depth(out, log_space=True)
        t = k.get_state()
        return out.double().cpu().numpy(), t
    finally:
        k.close()


@pytest.mark.parametrize("batching", [True, False], ids=["batched", "plain"])
def test_each_result_is_the_same_alone_and_in_the_mix(o, batching):
    torch = torch_cuda()
    prm = params(n_gn=10, n_pcg=5, solver=dfl.DF_SOLVER_AUTO)
    seqs, frames = _streams()
    srv = dfl.df_server_create(max_batch=8, max_inflight=2, batching=batching, params=prm)
    try:
        sids = [dfl.df_server_open_stream(srv, kf.width, kf.height,
                                          *[to_dev(p) for p in kf.cnn_planes])
                for kf, _, _ in seqs]
        # every stream gets all its frames, interleaved at random Poisson times
        t, _ = serving.poisson_schedule(len(SIZES) * NF, 3000.0, len(SIZES), seed=5)
        order = np.random.default_rng(6).permutation(np.repeat(np.arange(len(SIZES)), NF))
        st = serving.run(srv, sids, frames, t, order)
        assert st.n == len(SIZES) * NF
        if batching:
            assert st.mean_batch > 1.0  # frames really were solved together
        mode = "batched" if batching else "plain"
        for i, (kf, _, _) in enumerate(seqs):
            out = torch.empty((kf.height, kf.width), dtype=torch.float32, device="cuda")
            dfl.df_server_fetch_depth(srv, sids[i], out, log_space=True)
            x = out.double().cpu().numpy()
            xs = torch.empty_like(out)
            t = dfl.df_server_get_state(srv, sids[i], xs)
            assert torch.equal(xs, out)  # the state's x is the fetched log-depth
            xa, ta = _alone(kf, frames[i], prm)
            assert t != 0.0  # the scale step moved t
            assert_parity(x, t, xa, ta, rtol=DEPTH_RTOL, atol_t=SCALE_ATOL,
                          what=f"stream {i} {mode}")
        # one stream against the FP64 oracle over the same frames in order
        i = 3
        kf, mus, vs = seqs[i]
        x = torch.empty((kf.height, kf.width), dtype=torch.float32, device="cuda")
        t = dfl.df_server_get_state(srv, sids[i], x)
        xo, to = o.optimise_sequence(kf, mus, vs, n_gn=prm.n_gn, n_pcg=prm.n_pcg)
        assert_parity(x.double().cpu().numpy(), t, xo, to, what=f"stream {i} {mode} vs oracle")
    finally:
        dfl.df_server_destroy(srv)


def test_admission_follows_the_memory_budget():
    kf = synth.make_keyframe(64, 48, 77)
    need = dfl.df_keyframe_bytes(64, 48)
    srv = dfl.df_server_create(memory_budget=2 * need + need // 2, params=params())
    try:
        planes = [to_dev(p) for p in kf.cnn_planes]
        a = dfl.df_server_open_stream(srv, 64, 48, *planes)
        b = dfl.df_server_open_stream(srv, 64, 48, *planes)
        with pytest.raises(dfl.DFError) as e:
            dfl.df_server_open_stream(srv, 64, 48, *planes)
        assert e.value.status == dfl.DF_EBUDGET
        # a frame queued on a stream that then closes is finished first
        dfl.df_server_submit(srv, a, to_dev(kf.mu_s), to_dev(kf.var_s), 1)
        dfl.df_server_close_stream(srv, a)
        c = dfl.df_server_open_stream(srv, 64, 48, *planes)  # memory came back
        assert c == a  # the slot is reused
        got = []
        while dfl.df_server_pending(srv) > 0:
            got += dfl.df_server_progress(srv)
        assert [g.tag for g in got] == [1]
        assert b != c
    finally:
        dfl.df_server_destroy(srv)


def test_every_frame_completes_exactly_once():
    seqs, frames = _streams()
    srv = dfl.df_server_create(max_batch=3, max_inflight=3, params=params(n_gn=2, n_pcg=2))
    try:
        sids = [dfl.df_server_open_stream(srv, kf.width, kf.height,
                                          *[to_dev(p) for p in kf.cnn_planes])
                for kf, _, _ in seqs]
        tags = []
        for r in range(3):
            for i, sid in enumerate(sids):
                mu, var = frames[i][r]
                tag = 100 * r + i
                dfl.df_server_submit(srv, sid, mu, var, tag)
                tags.append(tag)
        done = []
        while dfl.df_server_pending(srv) > 0:
            done += dfl.df_server_progress(srv, cap=2)
        assert sorted(c.tag for c in done) == sorted(tags)
        assert all(1 <= c.batch_size <= 3 for c in done)
        assert all(c.t_submit_ns <= c.t_launch_ns <= c.t_done_ns for c in done)
    finally:
        dfl.df_server_destroy(srv)
