"""CUDA path vs the FP64 oracle, element by element, through the C ABI.

Bar (FP32 storage and arithmetic, FP64 reductions): max relative depth error
<= 1e-4 and |t_gpu - t_oracle| <= 1e-4 at equal iteration count.
"""
import numpy as np
import pytest

import oracle
from gpu_util import (DEPTH_RTOL, assert_parity, create, oracle_solve, params, solve,
                      to_dev, torch_cuda)
from paper_2207_12244_gb300 import deepfusion as dfl
from paper_2207_12244_gb300 import synth

pytestmark = pytest.mark.gpu

# (solver, fused kernel mode, assembly placement): the per-phase launches,
# the streaming fused kernel (assembly in a kernel of its own, the default,
# or in a pass of the persistent kernel) and the shared-memory-resident
# fused kernel
SOLVERS = [(dfl.DF_SOLVER_LAUNCHES, dfl.DF_MODE_AUTO, 0),
           (dfl.DF_SOLVER_FUSED, dfl.DF_MODE_STREAMING, 0),
           (dfl.DF_SOLVER_FUSED, dfl.DF_MODE_STREAMING, 1),
           (dfl.DF_SOLVER_FUSED, dfl.DF_MODE_RESIDENT, 0)]
SOLVER_IDS = ["launches", "streaming", "streaming-inkernel-assembly", "resident"]


@pytest.fixture(scope="module")
def o():
    return oracle.get()


@pytest.fixture(params=SOLVERS, ids=SOLVER_IDS)
def solver(request):
    sv, mode, assembly = request.param
    dfl.df_set_tuning(mode=mode, assembly=assembly)
    yield sv
    dfl.df_set_tuning()


# The workload of the paper's network resolution: 256 x 192, 10 GN x 3 PCG.
def test_config1_256x192(o, solver):
    kf = synth.make_keyframe(256, 192, 0)
    prm = params(n_gn=10, n_pcg=3, solver=solver)
    x, t, rep = solve(kf, prm)
    xo, to, ro = oracle_solve(o, kf, prm)
    assert_parity(x, t, xo, to, what="256x192")
    assert rep.iters_done == ro.iters_done == 30
    assert rep.flags == 0
    assert np.isclose(rep.res_norm, ro.res_norm, rtol=1e-2)


@pytest.mark.parametrize("W,H", [(1, 1), (2, 2), (1, 17), (23, 1), (17, 13), (33, 9),
                                  (100, 37), (129, 65), (31, 200)])
def test_edge_sizes(o, solver, W, H):
    kf = synth.make_keyframe(W, H, 100 + W * 7 + H)
    prm = params(n_gn=4, n_pcg=4, solver=solver)
    x, t, rep = solve(kf, prm)
    xo, to, ro = oracle_solve(o, kf, prm)
    assert_parity(x, t, xo, to, what=f"{W}x{H}")
    assert rep.iters_done == ro.iters_done


@pytest.mark.parametrize("mode", ["l2", "huber", "tukey", "huber-then-tukey", "semi+net",
                                  "net+grad", "semi+grad", "no-scale-step"])
def test_modes(o, solver, mode):
    kf = synth.make_keyframe(96, 72, 7)
    kw = dict(n_gn=6, n_pcg=5, solver=solver)
    if mode == "l2":
        kw["delta"] = float("inf")
    elif mode == "tukey":
        kw.update(loss=dfl.DF_LOSS_TUKEY, delta=4.685)
    elif mode == "huber-then-tukey":  # 2 Huber GN iterations, then 4 Tukey
        kw.update(loss=dfl.DF_LOSS_TUKEY, delta=4.685, warm_gn=2, warm_delta=1.345)
    elif mode == "semi+net":
        kw["terms"] = dfl.DF_TERM_SEMI | dfl.DF_TERM_NET
    elif mode == "net+grad":
        kw["terms"] = dfl.DF_TERM_NET | dfl.DF_TERM_GRAD
    elif mode == "semi+grad":
        kw.update(terms=dfl.DF_TERM_SEMI | dfl.DF_TERM_GRAD, scale_step=0)
    elif mode == "no-scale-step":
        kw["scale_step"] = 0
    prm = params(**kw)
    x, t, rep = solve(kf, prm)
    xo, to, ro = oracle_solve(o, kf, prm)
    assert_parity(x, t, xo, to, what=mode)
    if mode == "semi+net":
        # diagonal system: Jacobi-PCG is exact after one iteration; later
        # iterations run on rounding residue (1e-80 in FP64, exact zeros in
        # FP32 stop earlier), so only the depth is comparable
        assert 6 <= rep.iters_done <= ro.iters_done
    else:
        assert rep.iters_done == ro.iters_done


@pytest.mark.parametrize("n_pcg", [0, 1, 2])
def test_short_depth_steps(o, solver, n_pcg):
    """Depth steps of no, one and two CG iterations over three Gauss-Newton
    iterations: the fused kernels' pass sequences without CG iteration
    passes (the first CG pass straight into the last x update) or without
    any depth pass (assembly after assembly, each with the scale step
    before it), against the oracle."""
    kf = synth.make_keyframe(100, 70, 61 + n_pcg)
    prm = params(n_gn=3, n_pcg=n_pcg, solver=solver)
    x, t, rep = solve(kf, prm)
    xo, to, ro = oracle_solve(o, kf, prm)
    assert_parity(x, t, xo, to, what=f"n_pcg={n_pcg}")
    assert rep.iters_done == ro.iters_done


def test_prior_only_returns_cnn_depth_bitwise(o, solver):
    kf = synth.make_keyframe(64, 48, 9)
    prm = params(terms=dfl.DF_TERM_NET, solver=solver)
    x, t, rep = solve(kf, prm)
    assert np.array_equal(x.astype(np.float32), kf.mu_n)
    assert t == 0.0 and rep.iters_done == 0
    # from a perturbed start one Jacobi-PCG iteration lands on mu_n
    rng = np.random.default_rng(0)
    x0 = kf.mu_n + rng.normal(0, 0.3, kf.mu_n.shape).astype(np.float32)
    x, t, rep = solve(kf, params(terms=dfl.DF_TERM_NET, n_gn=1, n_pcg=1, solver=solver), x0=x0)
    assert np.abs(x - kf.mu_n).max() < 1e-6


def test_no_semi_frame(o, solver):
    kf = synth.make_keyframe(80, 60, 11)
    prm = params(solver=solver)
    x, t, rep = solve(kf, prm, semi=False)
    xo, to, _ = oracle_solve(o, kf, prm, semi=False)
    assert t == 0.0 and to == 0.0
    assert_parity(x, t, xo, to, what="no semi")


def test_invalid_semi_pixels_are_missing(o, solver):
    kf = synth.make_keyframe(70, 50, 12)
    rng = np.random.default_rng(4)
    idx = rng.choice(kf.n_pixels, 400, replace=False)
    ms, vs = kf.mu_s.ravel().copy(), kf.var_s.ravel().copy()
    ms[idx[:100]] = np.nan
    vs[idx[100:200]] = np.inf
    vs[idx[200:300]] = -1.0
    ms[idx[300:]] = np.inf
    vs[idx[300:]] = 1e-3
    kf.mu_s, kf.var_s = ms.reshape(kf.mu_s.shape), vs.reshape(kf.var_s.shape)
    prm = params(solver=solver)
    x, t, _ = solve(kf, prm)
    xo, to, _ = oracle_solve(o, kf, prm)
    assert_parity(x, t, xo, to, what="invalid semi")


def test_host_and_device_pointers_agree(solver):
    kf = synth.make_keyframe(120, 90, 13)
    prm = params(solver=solver)
    xd, td, _ = solve(kf, prm, on_device=True)
    xh, th, _ = solve(kf, prm, on_device=False)
    assert np.array_equal(xd, xh) and td == th


def test_host_frame_updates_overlap_and_agree(solver):
    """Frame updates from host buffers (pageable arrays and pinned tensors)
    are uploaded on the keyframe's copy stream while the previous frame is
    solved; a warm-started sequence issued without any synchronisation
    between frames gives bitwise the device-pointer result."""
    torch = torch_cuda()
    kf, mus, vs = synth.make_sequence(96, 64, 21, n_frames=6)
    prm = params(n_gn=4, n_pcg=3, solver=solver)

    def run(kind):
        # every buffer stays alive until the stream has passed its call
        if kind == "device":
            src = [(to_dev(m), to_dev(v)) for m, v in zip(mus, vs)]
        elif kind == "pinned":
            src = [(torch.from_numpy(m).pin_memory(), torch.from_numpy(v).pin_memory())
                   for m, v in zip(mus, vs)]
        else:
            src = [(np.ascontiguousarray(m), np.ascontiguousarray(v)) for m, v in zip(mus, vs)]
        k = create(kf)
        try:
            outs = []
            for f in range(len(mus)):
                k.frame_update(*src[f])
                k.optimise(prm)
                out = torch.empty((kf.height, kf.width), dtype=torch.float32, device="cuda")
                k.fetch_depth(out, log_space=True)
                outs.append(out)
            torch.cuda.synchronize()
            return [o.cpu().numpy() for o in outs], k.get_state()
        finally:
            k.close()

    xd, td = run("device")
    for kind in ("pinned", "pageable"):
        xh, th = run(kind)
        assert all(np.array_equal(a, b) for a, b in zip(xd, xh)) and td == th, kind


def test_deterministic(solver):
    kf = synth.make_keyframe(200, 150, 14)
    prm = params(n_gn=5, n_pcg=5, solver=solver)
    a = solve(kf, prm)
    b = solve(kf, prm)
    assert np.array_equal(a[0], b[0]) and a[1] == b[1]


def test_tolerance_mode(o, solver):
    kf = synth.make_keyframe(64, 64, 15)
    prm = params(n_gn=5, n_pcg=200, tol=1e-3, solver=solver)
    x, t, rep = solve(kf, prm)
    xo, to, ro = oracle_solve(o, kf, prm)
    assert rep.iters_done < 5 * 200
    assert abs(rep.iters_done - ro.iters_done) <= 2
    assert_parity(x, t, xo, to, rtol=5e-4, atol_t=5e-4, what="tol")


def test_warm_started_sequence(o, solver):
    """Config-2 recipe at reduced size: 100 frames, mask 5% -> 40%, 10 x 5."""
    torch = torch_cuda()
    kf, mus, vs = synth.make_sequence(128, 96, 21, n_frames=100)
    prm = params(n_gn=10, n_pcg=5, solver=solver)
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
    xo, to = o.optimise_sequence(kf, mus, vs, n_gn=10, n_pcg=5, delta=prm.delta)
    assert_parity(x, t, xo, to, what="sequence")


def test_full_size_640x480_first_frames(o, solver):
    """The benchmark's keyframe size (640 x 480) and schedule (10 x 5), first
    frames of the sequence, every pixel compared."""
    torch = torch_cuda()
    kf, mus, vs = synth.make_sequence(640, 480, 1, n_frames=100)
    prm = params(n_gn=10, n_pcg=5, solver=solver)
    k = create(kf)
    nf = 3
    try:
        for f in range(nf):
            k.frame_update(to_dev(mus[f]), to_dev(vs[f]))
            k.optimise(prm)
        out = torch.empty((480, 640), dtype=torch.float32, device="cuda")
        k.fetch_depth(out, log_space=True)
        t = k.get_state()
        x = out.double().cpu().numpy()
    finally:
        k.close()
    xo, to = o.optimise_sequence(kf, mus, vs, n_gn=10, n_pcg=5, delta=prm.delta,
                                 frames=range(nf))
    assert_parity(x, t, xo, to, what="640x480")


def test_cost_matches_oracle(o):
    kf = synth.make_keyframe(90, 70, 16)
    k = create(kf)
    try:
        k.frame_update(to_dev(kf.mu_s), to_dev(kf.var_s))
        rng = np.random.default_rng(1)
        x0 = (kf.mu_n + rng.normal(0, 0.05, kf.mu_n.shape)).astype(np.float32)
        k.set_state(to_dev(x0), 0.3)
        for delta, loss in ((1.345, 0), (float("inf"), 0), (4.685, 1)):
            c = k.cost(params(delta=delta, loss=loss))
            co = o.cost(kf, x0, 0.3, delta, loss=loss)
            assert np.isclose(c, co, rtol=1e-5), (delta, loss, c, co)
    finally:
        k.close()


def test_state_roundtrip_and_fetch_depth():
    torch = torch_cuda()
    kf = synth.make_keyframe(50, 40, 17)
    k = create(kf)
    try:
        x = np.random.default_rng(2).normal(0, 1, (40, 50)).astype(np.float32)
        k.set_state(x, -0.25)
        xb = np.empty_like(x)
        t = k.get_state(xb)
        assert np.array_equal(xb, x) and t == -0.25
        d = np.empty_like(x)
        k.fetch_depth(d)  # host output
        assert np.allclose(d, np.exp(x.astype(np.float64)), rtol=2e-7)
        dd = torch.empty((40, 50), dtype=torch.float32, device="cuda")
        k.fetch_depth(dd)
        assert np.array_equal(dd.cpu().numpy(), d)
    finally:
        k.close()


def test_semi_to_log_matches_oracle(o):
    torch = torch_cuda()
    rng = np.random.default_rng(5)
    n = 100003
    d = rng.uniform(0.3, 6.0, n).astype(np.float32)
    vd = (0.01 * d ** 2) ** 2
    vd = vd.astype(np.float32)
    d[:50] = -1.0
    vd[50:100] = 0.0
    d[100] = np.nan
    mu_o, var_o = o.semi_to_log(d, vd)
    mu = torch.empty(n, device="cuda")
    var = torch.empty(n, device="cuda")
    dfl.df_semi_to_log(to_dev(d), to_dev(vd), mu, var)
    assert np.allclose(mu.cpu().numpy(), mu_o, rtol=0, atol=2e-7)
    assert np.allclose(var.cpu().numpy(), var_o, rtol=2e-6, atol=0)
    mh, vh = np.empty(n, np.float32), np.empty(n, np.float32)
    dfl.df_semi_to_log(d, vd, mh, vh)
    assert np.array_equal(mh, mu.cpu().numpy()) and np.array_equal(vh, var.cpu().numpy())


def test_device_input_check_marks_keyframe():
    kf = synth.make_keyframe(40, 30, 18)
    planes = [p.copy() for p in kf.cnn_planes]
    planes[1][3, 4] = -0.5  # a negative network variance
    k = dfl.Keyframe(40, 30, *[to_dev(p) for p in planes])
    try:
        with pytest.raises(dfl.DFError) as e:
            k.check()
        assert e.value.status == dfl.DF_EINVAL
        with pytest.raises(dfl.DFError) as e:
            k.optimise(params(), report=True)
        assert e.value.status == dfl.DF_ESTATE
        x = np.empty((30, 40), np.float32)
        k.get_state(x)
        assert np.array_equal(x, planes[0])  # solve left the state untouched
    finally:
        k.close()


def test_budget_accounting_with_gpu():
    kf = synth.make_keyframe(64, 48, 19)
    need = dfl.df_keyframe_bytes(64, 48)
    base = dfl.df_memory_in_use()
    dfl.df_set_memory_budget(base + need + need // 2)
    try:
        a = create(kf)
        assert dfl.df_memory_in_use() == base + need
        with pytest.raises(dfl.DFError) as e:
            create(kf)
        assert e.value.status == dfl.DF_EBUDGET
        a.close()
        assert dfl.df_memory_in_use() == base
        b = create(kf)
        b.close()
    finally:
        dfl.df_set_memory_budget(0)


@pytest.mark.parametrize("mode", [dfl.DF_MODE_STREAMING, dfl.DF_MODE_RESIDENT],
                         ids=["streaming", "resident"])
def test_streaming_tile_shapes(o, mode):
    """Every tile shape of the streaming kernel (and grid caps for both
    kernels) gives the same answer."""
    kf = synth.make_keyframe(300, 140, 22)
    prm = params(n_gn=3, n_pcg=4, solver=dfl.DF_SOLVER_FUSED)
    xo, to, _ = oracle_solve(o, kf, prm)
    shapes = ([(1, 1, 0), (1, 5, 0), (4, 3, 0), (4, 16, 0), (4, 64, 7), (1, 2, 1)]
              if mode == dfl.DF_MODE_STREAMING else [(0, 0, 0), (0, 0, 40), (0, 0, 9)])
    try:
        for vec, th, cap in shapes:
            dfl.df_set_tuning(mode=mode, vec=vec, tile_rows=th, max_ctas=cap)
            x, t, rep = solve(kf, prm)
            assert_parity(x, t, xo, to, what=f"mode {mode} vec {vec} th {th} cap {cap}")
        if mode == dfl.DF_MODE_RESIDENT:
            # one CTA's shared memory cannot hold a 300 x 140 keyframe
            dfl.df_set_tuning(mode=mode, max_ctas=1)
            with pytest.raises(dfl.DFError) as e:
                solve(kf, prm)
            assert e.value.status == dfl.DF_ENOTSUP
    finally:
        dfl.df_set_tuning()


@pytest.mark.parametrize("scale", ["alternate", "fixed"])
@pytest.mark.parametrize("mode", [dfl.DF_MODE_STREAMING, dfl.DF_MODE_RESIDENT],
                         ids=["streaming", "resident"])
def test_barrier_wait_times_out_cleanly(mode, scale):
    """One CTA leaves without arriving at its first exchange (test switch):
    the others' bounded waits run out, the solve reports DF_ETIMEOUT, and
    the next solve on the same context is correct. With the scale fixed the
    resident kernel's first synchronisation is the assembly's edge hand-off,
    where the CTA also withholds its flag: its neighbours' flag waits run
    out."""
    kf = synth.make_keyframe(160, 120, 23)
    extra = {} if scale == "alternate" else dict(scale_step=dfl.DF_SCALE_FIXED)
    prm = params(n_gn=2, n_pcg=3, solver=dfl.DF_SOLVER_FUSED, **extra)
    ref = solve(kf, prm)
    try:
        dfl.df_set_spin_limit_ns(50_000_000)
        dfl.df_set_tuning(mode=mode, debug_skip_cta=1, max_ctas=4)
        k = create(kf)
        try:
            k.frame_update(to_dev(kf.mu_s), to_dev(kf.var_s))
            with pytest.raises(dfl.DFError) as e:
                k.optimise(prm, report=True)
            assert e.value.status == dfl.DF_ETIMEOUT
            with pytest.raises(dfl.DFError) as e:
                k.check()
            assert e.value.status == dfl.DF_ETIMEOUT
        finally:
            k.close()
    finally:
        dfl.df_set_tuning()
        dfl.df_set_spin_limit_ns(2_000_000_000)
    again = solve(kf, prm)
    assert np.array_equal(again[0], ref[0]) and again[1] == ref[1]


def test_huber_warm_start_is_two_chained_solves(o, solver):
    """The Huber-then-Tukey schedule in one call equals, bit for bit, a Huber
    solve of warm_gn iterations continued by a Tukey solve of the rest, and
    its report counts the PCG iterations of both; warm_gn >= n_gn is the
    Huber solve."""
    torch = torch_cuda()
    kf = synth.make_keyframe(100, 70, 27)
    tk = dict(loss=dfl.DF_LOSS_TUKEY, delta=4.685, n_pcg=4, solver=solver)

    def run(prms):
        k = create(kf)
        try:
            k.frame_update(to_dev(kf.mu_s), to_dev(kf.var_s))
            iters = 0
            for prm in prms:
                iters += k.optimise(prm, report=True).iters_done
            out = torch.empty((kf.height, kf.width), dtype=torch.float32, device="cuda")
            k.fetch_depth(out, log_space=True)
            return out.cpu().numpy(), k.get_state(), iters
        finally:
            k.close()

    x1, t1, i1 = run([params(n_gn=7, warm_gn=3, warm_delta=1.345, **tk)])
    x2, t2, i2 = run([params(n_gn=3, n_pcg=4, solver=solver), params(n_gn=4, **tk)])
    assert np.array_equal(x1, x2) and t1 == t2 and i1 == i2 == 28
    xh, th, _ = run([params(n_gn=5, n_pcg=4, solver=solver)])
    xw, tw, _ = run([params(n_gn=5, warm_gn=9, warm_delta=1.345, **tk)])
    assert np.array_equal(xh, xw) and th == tw
    xo, to, _ = oracle_solve(o, kf, params(n_gn=7, warm_gn=3, warm_delta=1.345, **tk))
    assert_parity(x1.astype(np.float64), t1, xo, to, what="huber then tukey")


def test_table2_scale_ambiguous_solve_then_ls_fit(o, solver):
    """Table II variant: semi + gradient terms with t fixed, then the
    least-squares scale fit to the network log-depth."""
    torch = torch_cuda()
    kf = synth.make_keyframe(120, 90, 24)
    prm = params(n_gn=6, n_pcg=6, terms=dfl.DF_TERM_SEMI | dfl.DF_TERM_GRAD, scale_step=0,
                 solver=solver)
    k = create(kf)
    try:
        k.frame_update(to_dev(kf.mu_s), to_dev(kf.var_s))
        k.optimise(prm)
        out = torch.empty((kf.height, kf.width), dtype=torch.float32, device="cuda")
        k.fetch_depth(out, log_space=True)
        t_pre = k.get_state()
        x_pre = out.double().cpu().numpy()
        k.scale_fit_ls()
        k.fetch_depth(out, log_space=True)
        t = k.get_state()
        x = out.double().cpu().numpy()
    finally:
        k.close()
    xo, to, _ = oracle_solve(o, kf, prm)
    xo, to = o.ls_scale_fit(kf, xo, to)
    assert_parity(x, t, xo, to, what="table II")
    # the fit itself, from the GPU's own pre-fit state and the definition:
    # c = mean(mu_n - x) moves every x and t by the same c
    c = np.mean(kf.mu_n.astype(np.float64) - x_pre)
    assert abs(c) > 1e-2  # the scale-ambiguous solve leaves a real offset to fit
    assert abs((t - t_pre) - c) < 1e-6, (t - t_pre, c)
    assert np.allclose(x - x_pre, c, rtol=0, atol=1e-5)
    assert abs(np.mean(kf.mu_n.astype(np.float64) - x)) < 1e-5


@pytest.mark.parametrize("mode", [dfl.DF_MODE_STREAMING, dfl.DF_MODE_RESIDENT],
                         ids=["streaming", "resident"])
def test_gn_iterations_split_over_launches(o, mode):
    kf = synth.make_keyframe(140, 100, 25)
    prm = params(n_gn=6, n_pcg=4, solver=dfl.DF_SOLVER_FUSED)
    xo, to, ro = oracle_solve(o, kf, prm)
    try:
        for g in (1, 2, 4, 6):
            dfl.df_set_tuning(mode=mode, gn_per_launch=g)
            x, t, rep = solve(kf, prm)
            assert_parity(x, t, xo, to, what=f"gn_per_launch {g}")
            assert rep.iters_done == ro.iters_done == 24
    finally:
        dfl.df_set_tuning()


def test_autotune_picks_a_shape_and_restores_state(o):
    torch = torch_cuda()
    kfs = [synth.make_keyframe(W, H, 300 + i) for i, (W, H) in enumerate([(160, 120), (96, 64)])]
    prm = params(n_gn=4, n_pcg=3, solver=dfl.DF_SOLVER_FUSED)
    ks = [create(kf) for kf in kfs]
    try:
        for k, kf in zip(ks, kfs):
            k.frame_update(to_dev(kf.mu_s), to_dev(kf.var_s))
        before = [k.get_state(np.empty((kf.height, kf.width), np.float32)) for k, kf in zip(ks, kfs)]
        xs_before = []
        for k, kf in zip(ks, kfs):
            xb = np.empty((kf.height, kf.width), np.float32)
            k.get_state(xb)
            xs_before.append(xb)
        best, ms = dfl.df_autotune([k.handle for k in ks], prm)
        assert ms > 0 and best.mode in (1, 2)
        cur = dfl.df_get_tuning()
        assert (cur.mode, cur.vec, cur.tile_rows, cur.gn_per_launch) == (
            best.mode, best.vec, best.tile_rows, best.gn_per_launch)
        for k, kf, xb, tb in zip(ks, kfs, xs_before, before):
            xa = np.empty_like(xb)
            ta = k.get_state(xa)
            assert np.array_equal(xa, xb) and ta == tb  # the state is as before
        dfl.df_optimise_batch([k.handle for k in ks], prm, report=True)
        for k, kf in zip(ks, kfs):
            out = torch.empty((kf.height, kf.width), dtype=torch.float32, device="cuda")
            k.fetch_depth(out, log_space=True)
            t = k.get_state()
            xo, to, _ = oracle_solve(o, kf, prm)
            assert_parity(out.double().cpu().numpy(), t, xo, to, what="after autotune")
    finally:
        for k in ks:
            k.close()
        dfl.df_set_tuning()


def test_autotune_refuses_bad_lists_and_leaves_everything_as_it_was():
    """A NULL or repeated keyframe in the list: DF_EINVAL before anything is
    allocated or changed; the tuning and every keyframe's (x, t) stay as
    they were, and device memory in use is unchanged."""
    torch = torch_cuda()
    kfs = [synth.make_keyframe(64, 48, 310 + i) for i in range(2)]
    prm = params(n_gn=2, n_pcg=2, solver=dfl.DF_SOLVER_FUSED)
    ks = [create(kf) for kf in kfs]
    try:
        for k, kf in zip(ks, kfs):
            k.frame_update(to_dev(kf.mu_s), to_dev(kf.var_s))
            k.optimise(prm)
        before = []
        for k, kf in zip(ks, kfs):
            xb = np.empty((kf.height, kf.width), np.float32)
            before.append((xb, k.get_state(xb)))
        dfl.df_set_tuning(mode=1, vec=1, tile_rows=8)
        tun0 = dfl.df_get_tuning()
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        a, b = ks[0].handle, ks[1].handle
        for bad in ([a, None, b], [a, b, a], [None]):
            with pytest.raises(dfl.DFError) as ei:
                dfl.df_autotune(bad, prm)
            assert ei.value.status == dfl.DF_EINVAL
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0
        tun = dfl.df_get_tuning()
        assert (tun.mode, tun.vec, tun.tile_rows, tun.gn_per_launch) == (
            tun0.mode, tun0.vec, tun0.tile_rows, tun0.gn_per_launch)
        for k, (xb, tb) in zip(ks, before):
            xa = np.empty_like(xb)
            assert k.get_state(xa) == tb and np.array_equal(xa, xb)
    finally:
        for k in ks:
            k.close()
        dfl.df_set_tuning()


@pytest.mark.parametrize("sv", [(dfl.DF_SOLVER_LAUNCHES, 0), (dfl.DF_SOLVER_FUSED, 2),
                                (dfl.DF_SOLVER_FUSED, 1)], ids=["launches", "resident", "streaming"])
def test_frame_captured_in_a_cuda_graph(sv):
    """A frame's work (semi-dense update, solve, depth output) captured once
    in a CUDA graph and replayed gives the eager result."""
    torch = torch_cuda()
    solver, mode = sv
    kf, mus, vs = synth.make_sequence(96, 72, 26, n_frames=3)
    prm = params(n_gn=4, n_pcg=3, solver=solver)
    dfl.df_set_tuning(mode=mode)
    try:
        dmu, dvs = to_dev(mus), to_dev(vs)
        out = torch.empty((72, 96), dtype=torch.float32, device="cuda")
        eager = create(kf)
        try:
            for f in range(3):
                eager.frame_update(dmu[f], dvs[f])
                eager.optimise(prm)
            eager.fetch_depth(out, log_space=True)
            ref = out.clone()
        finally:
            eager.close()
        k = create(kf)
        try:
            mu_in = torch.empty_like(dmu[0])
            var_in = torch.empty_like(dvs[0])
            # warm-up outside the capture (uploads the fused kernel's plan)
            mu_in.copy_(dmu[0])
            var_in.copy_(dvs[0])
            k.set_state(to_dev(kf.mu_n), 0.0)
            k.optimise(prm)
            k.set_state(to_dev(kf.mu_n), 0.0)
            torch.cuda.synchronize()
            g = torch.cuda.CUDAGraph()
            s = torch.cuda.Stream()
            s.wait_stream(torch.cuda.current_stream())
            with torch.cuda.stream(s):
                with torch.cuda.graph(g, stream=s):
                    k.frame_update(mu_in, var_in)
                    k.optimise(prm)
                    k.fetch_depth(out, log_space=True)
            torch.cuda.current_stream().wait_stream(s)
            for f in range(3):
                mu_in.copy_(dmu[f])
                var_in.copy_(dvs[f])
                g.replay()
            torch.cuda.synchronize()
            assert torch.equal(out, ref)
        finally:
            k.close()
    finally:
        dfl.df_set_tuning()


def test_frame_captured_with_host_buffers():
    """Frame updates from pinned host buffers inside a CUDA graph capture take
    the direct upload (no copy stream in a capture); replays give the eager
    device-pointer result, also after uncaptured host updates made the
    keyframe's copy stream."""
    torch = torch_cuda()
    kf, mus, vs = synth.make_sequence(96, 72, 27, n_frames=3)
    prm = params(n_gn=4, n_pcg=3, solver=dfl.DF_SOLVER_FUSED)
    out = torch.empty((72, 96), dtype=torch.float32, device="cuda")
    eager = create(kf)
    try:
        for f in range(3):
            eager.frame_update(to_dev(mus[f]), to_dev(vs[f]))
            eager.optimise(prm)
        eager.fetch_depth(out, log_space=True)
        ref = out.clone()
    finally:
        eager.close()
    mu_h = torch.from_numpy(mus[0].copy()).pin_memory()
    var_h = torch.from_numpy(vs[0].copy()).pin_memory()
    k = create(kf)
    try:
        k.frame_update(mu_h, var_h)  # uncaptured host update: the copy stream path
        k.optimise(prm)
        k.set_state(to_dev(kf.mu_n), 0.0)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            with torch.cuda.graph(g, stream=s):
                k.frame_update(mu_h, var_h)
                k.optimise(prm)
                k.fetch_depth(out, log_space=True)
        torch.cuda.current_stream().wait_stream(s)
        torch.cuda.synchronize()
        for f in range(3):
            mu_h.copy_(torch.from_numpy(mus[f]))
            var_h.copy_(torch.from_numpy(vs[f]))
            g.replay()
            torch.cuda.synchronize()  # the graph reads the pinned buffers
        assert torch.equal(out, ref)
    finally:
        k.close()


def test_subnormal_variances_weigh_as_the_smallest_normal(solver):
    """The reciprocals of the IRLS weights flush subnormal operands: a
    variance below the smallest normal float must act exactly as that float
    does (the weight saturates at 1 / FLT_MIN), never as 0 or a NaN. One
    semi-dense pixel and one network-prior pixel carry such a variance, with
    a mean equal to the prior so the huge weight meets a zero residual."""
    import copy

    kf = synth.make_keyframe(96, 72, 11)
    p = int(np.flatnonzero(kf.var_s.ravel() > 0)[3])
    q = (kf.width * kf.height) // 2 + 5
    tiny, fmin = np.float32(1e-40), np.finfo(np.float32).tiny
    assert 0 < tiny < fmin

    def variant(v):
        k2 = copy.deepcopy(kf)
        k2.mu_s.ravel()[p] = k2.mu_n.ravel()[p]
        k2.var_s.ravel()[p] = v
        k2.var_n.ravel()[q] = v
        return k2

    prm = params(n_gn=4, n_pcg=4, solver=solver)
    x_sub, t_sub, rep_sub = solve(variant(tiny), prm)
    x_min, t_min, rep_min = solve(variant(fmin), prm)
    assert rep_sub.flags == rep_min.flags == 0
    assert np.isfinite(x_sub).all() and np.isfinite(t_sub)
    assert np.array_equal(x_sub, x_min) and t_sub == t_min
