"""The C ABI library without a GPU: it loads, exports every declared entry
point, and its host-side argument checks answer before touching the device."""
import ctypes as C

import numpy as np
import pytest

from paper_2207_12244_gb300 import _build, deepfusion as dfl


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return dfl.load()


def test_exports_every_declared_symbol(lib):
    names = dfl.header_functions()
    assert len(names) >= 19
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings_and_defaults(lib):
    assert dfl.df_status_str(dfl.DF_EINVAL) == "DF_EINVAL"
    assert dfl.df_status_str(dfl.DF_ETIMEOUT) == "DF_ETIMEOUT"
    p = dfl.df_default_params()
    assert (p.n_gn, p.n_pcg, p.loss, p.terms, p.scale_step, p.solver, p.tol, p.warm_gn) == (
        10, 3, dfl.DF_LOSS_HUBER, dfl.DF_TERMS_ALL, 1, dfl.DF_SOLVER_AUTO, 0.0, 0)
    assert abs(p.delta - 1.345) < 1e-6 and abs(p.warm_delta - 1.345) < 1e-6
    assert C.sizeof(dfl.df_solve_params) == 48  # the C struct's layout


def test_keyframe_bytes_and_budget(lib):
    b32 = dfl.df_keyframe_bytes(640, 480, dfl.DF_F32)
    b16 = dfl.df_keyframe_bytes(640, 480, dfl.DF_BF16)
    assert b32 > b16 > 640 * 480 * 40
    assert dfl.df_keyframe_bytes(0, 10) == 0 and dfl.df_keyframe_bytes(10, 10, 9) == 0
    assert dfl.df_memory_in_use() == 0
    dfl.df_set_memory_budget(1000)
    W, H = 8, 4
    z = np.zeros((H, W), np.float32)
    o = np.ones((H, W), np.float32)
    with pytest.raises(dfl.DFError) as e:
        dfl.df_keyframe_create(W, H, z, o, z, o, z, o)
    assert e.value.status == dfl.DF_EBUDGET
    dfl.df_set_memory_budget(0)
    assert dfl.df_memory_in_use() == 0


def test_invalid_arguments_rejected_on_host(lib):
    W, H = 6, 5
    z = np.zeros((H, W), np.float32)
    o = np.ones((H, W), np.float32)
    bad = o.copy()
    bad[2, 3] = -1.0
    for planes in ([z, bad, z, o, z, o], [z, o, z, bad, z, o], [z, o, z, o, z, bad]):
        with pytest.raises(dfl.DFError) as e:
            dfl.df_keyframe_create(W, H, *planes)
        assert e.value.status == dfl.DF_EINVAL
        assert "invalid network input" in str(e.value)
    nan = z.copy()
    nan[0, 0] = np.nan
    with pytest.raises(dfl.DFError) as e:
        dfl.df_keyframe_create(W, H, nan, o, z, o, z, o)
    assert e.value.status == dfl.DF_EINVAL
    # the ignored last column of var_gx and last row of var_gy may hold anything
    vx = o.copy()
    vx[:, -1] = -3.0
    vy = o.copy()
    vy[-1, :] = np.nan
    desc = dfl.df_keyframe_desc(0, H, 0)
    out = C.c_void_p()
    ptrs = [a.ctypes.data for a in (z, o, z, o, z, o)]
    assert lib.df_keyframe_create(C.byref(desc), *ptrs, 0, None, C.byref(out)) == dfl.DF_EINVAL
    desc = dfl.df_keyframe_desc(W, H, 7)
    assert lib.df_keyframe_create(C.byref(desc), *ptrs, 0, None, C.byref(out)) == dfl.DF_EINVAL
    assert lib.df_keyframe_create(None, *ptrs, 0, None, C.byref(out)) == dfl.DF_EINVAL
    assert lib.df_keyframe_create(C.byref(dfl.df_keyframe_desc(W, H, 0)), None, *ptrs[1:], 0,
                                  None, C.byref(out)) == dfl.DF_EINVAL
    assert "NULL" in dfl.df_last_error()


def test_null_keyframe_and_bad_params(lib):
    assert lib.df_optimise(None, None, None, None) == dfl.DF_EINVAL
    assert lib.df_frame_update(None, None, None, 0, None) == dfl.DF_EINVAL
    assert lib.df_fetch_depth(None, None, 0, 0, None) == dfl.DF_EINVAL
    lib.df_keyframe_destroy(None)  # NULL-safe
    bad = [dict(n_gn=-1), dict(n_pcg=-2), dict(loss=5), dict(terms=0), dict(terms=1),
           dict(terms=8), dict(solver=9), dict(tol=-1.0), dict(tol=float("inf")),
           dict(delta=float("nan")), dict(warm_gn=-1),
           dict(warm_gn=2, warm_delta=float("nan"))]
    arr = (C.c_void_p * 1)(None)
    for b in bad:
        p = dfl.df_default_params(**b)
        # batch checks the parameters before touching any keyframe
        assert lib.df_optimise_batch(arr, 0, C.byref(p), None, None) == dfl.DF_EINVAL, b
    assert lib.df_optimise_batch(None, 3, None, None, None) == dfl.DF_EINVAL
    assert lib.df_semi_to_log(None, None, None, None, -1, 0, None) == dfl.DF_EINVAL
    assert lib.df_semi_to_log(None, None, None, None, 0, 0, None) == dfl.DF_OK


def _codes(a, dtype):
    """float32 values as the element bits the library reads for each dtype."""
    a = np.asarray(a, np.float32)
    if dtype == dfl.DF_F32:
        return a
    if dtype == dfl.DF_F16:
        return a.astype(np.float16)
    return (a.view(np.uint32) >> 16).astype(np.uint16)  # bf16: upper half (exact here)


@pytest.mark.parametrize("dtype", [dfl.DF_F32, dfl.DF_BF16, dfl.DF_F16], ids=["f32", "bf16", "f16"])
def test_host_validation_matches_the_rule(lib, dtype):
    """The host check accepts exactly the planes whose means are finite and
    whose variances are finite and > 0, ignoring gx / var_gx in the last
    column and gy / var_gy in the last row; a rejection names the plane and
    the pixel."""
    W, H = 37, 11
    rng = np.random.default_rng(5)
    specials = [np.nan, np.inf, -np.inf, 0.0, -0.0, -2.0, 2.0 ** -130, 3.0]
    names = ["mu_net", "var_net", "gx", "var_gx", "gy", "var_gy"]
    base = [np.full((H, W), 0.5 if j % 2 == 0 else 1.5, np.float32) for j in range(6)]
    n_reject = 0
    for j in range(6):
        for val in specials:
            for (v, u) in [(int(rng.integers(H)), int(rng.integers(W))), (H - 1, W - 1),
                           (0, W - 1), (H - 1, 0)]:
                planes = [b.copy() for b in base]
                planes[j][v, u] = val
                fv = float(_codes(np.float32(val), dtype).astype(np.float32)) \
                    if dtype != dfl.DF_BF16 else float(np.float32(val))
                ignored = (j in (2, 3) and u == W - 1) or (j in (4, 5) and v == H - 1)
                ok_val = np.isfinite(fv) and (j % 2 == 0 or fv > 0.0)
                expect_reject = not ok_val and not ignored
                desc = dfl.df_keyframe_desc(W, H, dtype)
                out = C.c_void_p()
                codes = [np.ascontiguousarray(_codes(p, dtype)) for p in planes]
                st = lib.df_keyframe_create(C.byref(desc), *[c.ctypes.data for c in codes], 0,
                                            None, C.byref(out))
                if st == dfl.DF_OK:
                    lib.df_keyframe_destroy(out)
                msg = dfl.df_last_error()
                rejected = st == dfl.DF_EINVAL and "invalid network input" in msg
                assert rejected == expect_reject, (names[j], val, v, u, st, msg)
                if rejected:
                    n_reject += 1
                    assert f"{names[j]} at (u={u}, v={v})" in msg, msg
    assert n_reject > 50


def test_host_validation_of_large_planes_in_parallel(lib):
    """Planes large enough for the threaded check (6 x 1024 x 768 elements):
    a bad value anywhere is found and reported as the first bad pixel, and
    valid planes pass."""
    W, H = 1024, 768
    base = [np.full((H, W), 0.25 if j % 2 == 0 else 2.0, np.float32) for j in range(6)]
    desc = dfl.df_keyframe_desc(W, H, dfl.DF_F32)
    out = C.c_void_p()

    def create(planes):
        st = lib.df_keyframe_create(C.byref(desc), *[p.ctypes.data for p in planes], 0, None,
                                    C.byref(out))
        if st == dfl.DF_OK:
            lib.df_keyframe_destroy(out)
        return st, dfl.df_last_error()

    st, msg = create(base)
    assert not (st == dfl.DF_EINVAL and "invalid network input" in msg), msg
    for j, (v, u), val in [(5, (H - 2, W - 1), np.inf), (1, (700, 3), 0.0), (0, (383, 512), np.nan),
                           (3, (10, 1000), -1.0)]:
        planes = [b.copy() for b in base]
        planes[j][v, u] = val
        planes[2][H - 1, 5] = np.nan  # a later pixel (row H - 1) of an earlier plane
        st, msg = create(planes)
        assert st == dfl.DF_EINVAL and "invalid network input" in msg, msg
        names = ["mu_net", "var_net", "gx", "var_gx", "gy", "var_gy"]
        first = min([(v, u, j), (H - 1, 5, 2)])
        assert f"{names[first[2]]} at (u={first[1]}, v={first[0]})" in msg, msg


def _large_planes(W=1024, H=768, bad=None):
    planes = [np.full((H, W), 0.25 if j % 2 == 0 else 2.0, np.float32) for j in range(6)]
    if bad is not None:
        j, v, u, val = bad
        planes[j][v, u] = val
    return planes


def _create_status(lib, planes):
    H, W = planes[0].shape
    desc = dfl.df_keyframe_desc(W, H, dfl.DF_F32)
    out = C.c_void_p()
    st = lib.df_keyframe_create(C.byref(desc), *[p.ctypes.data for p in planes], 0, None,
                                C.byref(out))
    if st == dfl.DF_OK:
        lib.df_keyframe_destroy(out)
    return st, dfl.df_last_error()


def test_host_validation_from_concurrent_threads(lib):
    """Several host threads checking large planes at once (one holds the
    worker pool, the others check on their own threads): every call reports
    its own first bad pixel."""
    import threading

    cases = [(1, 700 - 9 * i, 3 + i, 0.0) for i in range(6)]
    results = [None] * len(cases)

    def work(i):
        planes = _large_planes(bad=cases[i])
        for _ in range(3):
            st, msg = _create_status(lib, planes)
            results[i] = (st, msg)

    ts = [threading.Thread(target=work, args=(i,)) for i in range(len(cases))]
    for t in ts:
        t.start()
    for t in ts:
        t.join(timeout=60)
        assert not t.is_alive()
    for (j, v, u, _), (st, msg) in zip(cases, results):
        assert st == dfl.DF_EINVAL and f"var_net at (u={u}, v={v})" in msg, msg


def _forked_child_check(q):
    lib = dfl.load()
    st, msg = _create_status(lib, _large_planes(bad=(4, 500, 17, np.inf)))
    q.put((st, msg))


def test_host_validation_in_a_forked_child(lib):
    """A child forked after the worker pool exists checks on its own thread
    (the pool's threads are not in the child) instead of waiting for them."""
    import multiprocessing as mp

    _create_status(lib, _large_planes())  # the pool exists in this process now
    ctx = mp.get_context("fork")
    q = ctx.Queue()
    p = ctx.Process(target=_forked_child_check, args=(q,))
    p.start()
    p.join(timeout=60)
    alive = p.is_alive()
    if alive:
        p.kill()
    assert not alive, "the forked child hung in the host check"
    st, msg = q.get(timeout=5)
    assert st == dfl.DF_EINVAL and "gy at (u=17, v=500)" in msg, msg


def test_noalloc_wrapper_refuses_buffers_it_would_overrun(lib):
    """The binding of df_optimise_noalloc checks dtypes, sizes, contiguity and
    devices before the call: a buffer of the wrong type or too few elements
    would be read or written out of bounds by the kernels."""
    import torch

    W, H = 8, 6
    ok = [torch.zeros(H, W) for _ in range(9)]
    t = torch.zeros(1, dtype=torch.float64)

    def call(planes, scale):
        dfl.df_optimise_noalloc(W, H, *planes, scale)

    cases = []
    for j in range(9):  # one plane of the wrong dtype, then one too small
        p = list(ok)
        p[j] = torch.zeros(H, W, dtype=torch.float16)
        cases.append((p, t, "float32"))
        p = list(ok)
        p[j] = torch.zeros(H * W - 1)
        cases.append((p, t, "fewer than"))
    cases.append((ok, torch.zeros(1, dtype=torch.float32), "float64"))
    cases.append((ok, torch.zeros(0, dtype=torch.float64), "float64"))
    p = list(ok)
    p[0] = torch.zeros(W, H).t()
    cases.append((p, t, "contiguous"))
    p = list(ok)
    p[6] = None
    cases.append((p, t, "go together"))
    p = list(ok)
    p[2] = None
    cases.append((p, t, "required"))
    p = list(ok)
    p[4] = np.zeros((H, W), np.float32)
    cases.append((p, t, "torch tensor"))
    cases.append((ok, t, "device buffers only"))  # host tensors
    for planes, scale, msg in cases:
        with pytest.raises((ValueError, TypeError)) as e:
            call(planes, scale)
        assert msg in str(e.value), (msg, str(e.value))
