"""Pins for the FP64 oracle: checks against facts fixed by the paper's cost
(Section II-C, Eqs. 5-8) and by mathematics, independent of the oracle's own
code. Each function takes an ``oracle.Oracle`` and raises AssertionError on a
mismatch, so the same pins run against the real oracle and against builds
with a planted mistake (tests/test_oracle_mutants.py).

What each pin fixes:
  cost_closed_form     hand-derived cost of one-pixel / scale perturbations of
                       a zero-residual state (every term, its whitening, its
                       neighbour index, Huber and Tukey branches, term bits)
  robust_weight        omega(u) = rho'(u) / (2u) by central differences
  dense_hessian        A, b of the depth step = Hessian / gradient of the cost
                       (second differences); PCG to convergence = Cholesky
  joint_optimum        alternation converges to the bordered (x, t) Cholesky
                       solution of the least-squares cost
  prior_only           network term alone: x = mu_n bitwise; one Jacobi-PCG
                       iteration from a perturbed start returns mu_n
  planar_recovery      noise-free piecewise-planar scene: x = ln D, t = ln s
  huber_scipy          robust cost: IRLS optimum = scipy BFGS optimum
  invariances          shifts of mu_s, of (mu_n, mu_s), and transposition
  monotone             cost never increases over scale and depth steps
  no_pairwise          semi + network only: closed-form joint optimum
  tukey_after_huber    Huber warm start then Tukey: the ends are the plain
                       solves; k + (n - k) iterations = two chained solves;
                       Tukey iterations never raise the Tukey cost
  ls_scale_fit         Table II fit: a constructed offset comes back exactly;
                       optimality, x - t kept, shift invariance
  semi_to_log          first-order log conversion vs Monte Carlo
"""
from __future__ import annotations

import types

import numpy as np

import oracle as orc
from paper_2207_12244_gb300 import synth

INF = float("inf")
DELTA = orc.HUBER_DELTA
TUKEY_C = 4.685


def _planes(W, H, rng, xs, ts, mask_frac=0.5, garbage=True):
    """A problem whose residuals all vanish at (xs, ts): mu_n = xs, g = exact
    forward differences, mu_s = xs - ts on a random mask."""
    kf = types.SimpleNamespace(width=W, height=H)
    X = xs.reshape(H, W)
    kf.mu_n = X.copy()
    kf.gx = np.zeros((H, W))
    kf.gy = np.zeros((H, W))
    kf.gx[:, :-1] = X[:, 1:] - X[:, :-1]
    kf.gy[:-1, :] = X[1:, :] - X[:-1, :]
    if garbage:  # entries the method must ignore
        kf.gx[:, -1] = 7.0
        kf.gy[-1, :] = -5.0
    kf.var_n = rng.uniform(0.1, 2.0, (H, W))
    kf.var_gx = rng.uniform(0.1, 2.0, (H, W))
    kf.var_gy = rng.uniform(0.1, 2.0, (H, W))
    m = rng.random((H, W)) < mask_frac
    kf.mu_s = np.where(m, X - ts, 0.0)
    kf.var_s = np.where(m, rng.uniform(0.1, 2.0, (H, W)), 0.0)
    if garbage:  # invalid semi-dense pixels in every encoding
        bad = np.argwhere(~m)
        for k, (v, u) in enumerate(bad):
            kind = k % 4
            if kind == 1:
                kf.var_s[v, u] = -1.0
                kf.mu_s[v, u] = 3.0
            elif kind == 2:
                kf.var_s[v, u] = np.nan
            elif kind == 3:
                kf.var_s[v, u] = 0.5
                kf.mu_s[v, u] = np.inf
    return kf, m


def _touch_weights(kf, m, j, terms=orc.TERMS_ALL):
    """Inverse variances of every term that contains pixel j (by hand)."""
    W, H = kf.width, kf.height
    v, u = divmod(j, W)
    w = []
    if terms & orc.TERM_SEMI and m[v, u]:
        w.append(1.0 / kf.var_s[v, u])
    if terms & orc.TERM_NET:
        w.append(1.0 / kf.var_n[v, u])
    if terms & orc.TERM_GRAD:
        if u < W - 1:
            w.append(1.0 / kf.var_gx[v, u])      # r_x at i   = x_{i+1} - x_i - gx_i
        if u > 0:
            w.append(1.0 / kf.var_gx[v, u - 1])  # r_x at i-1 = x_i - x_{i-1} - gx_{i-1}
        if v < H - 1:
            w.append(1.0 / kf.var_gy[v, u])
        if v > 0:
            w.append(1.0 / kf.var_gy[v - 1, u])
    return np.array(w)


def cost_closed_form(o):
    rng = np.random.default_rng(11)
    W, H = 5, 4
    xs = rng.normal(0.0, 1.0, W * H)
    ts = 0.3
    kf, m = _planes(W, H, rng, xs, ts)
    for delta in (INF, DELTA):
        assert abs(o.cost(kf, xs, ts, delta)) < 1e-24
    for j in range(W * H):
        w = _touch_weights(kf, m, j)
        # small step: every touched whitened residual is below delta
        eps = 1e-3
        x = xs.copy()
        x[j] += eps
        want = eps * eps * w.sum()
        for delta in (INF, DELTA):
            got = o.cost(kf, x, ts, delta)
            assert np.isclose(got, want, rtol=1e-8, atol=0), (j, delta, got, want)
        # large step: Huber's linear branch, 2 delta |u| - delta^2 per term
        eps = 40.0
        x = xs.copy()
        x[j] -= eps
        want = np.sum(2.0 * DELTA * eps * np.sqrt(w) - DELTA ** 2)
        got = o.cost(kf, x, ts, DELTA)
        assert np.isclose(got, want, rtol=1e-10), (j, got, want)
        assert np.isclose(o.cost(kf, x, ts, INF), eps * eps * w.sum(), rtol=1e-10)
        # Tukey saturates at c^2/3 per term
        got = o.cost(kf, x, ts, TUKEY_C, loss=orc.LOSS_TUKEY)
        assert np.isclose(got, len(w) * TUKEY_C ** 2 / 3.0, rtol=1e-12), (j, got)
        # term selection
        for terms in (orc.TERM_SEMI, orc.TERM_NET, orc.TERM_GRAD,
                      orc.TERM_SEMI | orc.TERM_GRAD, orc.TERM_SEMI | orc.TERM_NET):
            wt = _touch_weights(kf, m, j, terms)
            x = xs.copy()
            x[j] += 1e-3
            got = o.cost(kf, x, ts, INF, terms=terms)
            assert np.isclose(got, 1e-6 * wt.sum(), rtol=1e-8, atol=1e-30), (j, terms)
    # the scale enters only the semi-dense term, with the opposite sign of x
    sw = (1.0 / kf.var_s[m]).sum()
    for tau in (1e-3, -0.7):
        assert np.isclose(o.cost(kf, xs, ts + tau, INF), tau * tau * sw, rtol=1e-9)
    x = xs + 0.25
    assert np.isclose(o.cost(kf, x, ts + 0.25, INF, terms=orc.TERM_SEMI), 0.0, atol=1e-20)


def robust_weight(o):
    for loss, delta in ((orc.LOSS_HUBER, DELTA), (orc.LOSS_TUKEY, TUKEY_C)):
        for u in (-9.0, -3.1, -1.0, -0.2, 0.3, 1.2, 1.4, 2.5, 4.0, 8.0):
            h = 1e-6
            d = (o.rho(u + h, delta, loss) - o.rho(u - h, delta, loss)) / (2 * h)
            assert np.isclose(o.omega(u, delta, loss), d / (2 * u), rtol=1e-6, atol=1e-9), (loss, u)
        # continuity at the threshold
        a = o.rho(delta * (1 - 1e-12), delta, loss)
        b = o.rho(delta * (1 + 1e-12), delta, loss)
        assert abs(a - b) < 1e-9
    for u in (-3.0, 0.5, 10.0):
        assert o.omega(u, INF) == 1.0 and o.rho(u, INF) == u * u
        assert o.omega(u, 0.0) == 1.0


def _noisy(W, H, seed):
    kf = synth.make_keyframe(W, H, seed)
    return kf


def _dense_quadratic(o, kf, t, x0, terms=orc.TERMS_ALL):
    """Hessian/2 and -gradient/2 of the least-squares cost in x (t fixed),
    by exact second differences of the cost (a quadratic)."""
    N = kf.width * kf.height
    c = lambda x: o.cost(kf, x, t, INF, terms=terms)
    z = np.zeros(N)
    c0 = c(z)
    ce = np.empty(N)
    cm = np.empty(N)
    e = np.eye(N)
    for j in range(N):
        ce[j] = c(e[j])
        cm[j] = c(-e[j])
    A = np.empty((N, N))
    for j in range(N):
        for k in range(j, N):
            if j == k:
                A[j, j] = (c(2 * e[j]) - 2 * ce[j] + c0) / 2.0
            else:
                A[j, k] = A[k, j] = (c(e[j] + e[k]) - ce[j] - ce[k] + c0) / 2.0
    b = -(ce - cm) / 4.0
    return A, b


def dense_hessian(o):
    W, H = 6, 5
    kf = _noisy(W, H, 3)
    t = 0.2
    rng = np.random.default_rng(5)
    x0 = kf.mu_n.ravel().astype(np.float64) + rng.normal(0, 0.2, W * H)
    A, b = _dense_quadratic(o, kf, t, x0)
    diag, wx, wy, bb = o.assemble(kf, x0, t, INF)
    scale = np.abs(A).max()
    assert np.allclose(np.diag(A), diag, rtol=1e-7, atol=1e-9 * scale)
    N = W * H
    Ad = np.diag(diag)
    for i in range(N):
        v, u = divmod(i, W)
        if u < W - 1:
            Ad[i, i + 1] = Ad[i + 1, i] = -wx[i]
        else:
            assert wx[i] == 0.0
        if v < H - 1:
            Ad[i, i + W] = Ad[i + W, i] = -wy[i]
        else:
            assert wy[i] == 0.0
    assert np.allclose(Ad, A, rtol=1e-7, atol=1e-8 * scale)
    assert np.allclose(bb, b, rtol=1e-7, atol=1e-8 * np.abs(b).max())
    Lc = np.linalg.cholesky(A)
    xs = np.linalg.solve(Lc.T, np.linalg.solve(Lc, b))
    x, it, rn = o.pcg(W, H, diag, wx, wy, bb, x0, 300)
    assert np.allclose(x, xs, rtol=0, atol=1e-10 * np.abs(xs).max()), np.abs(x - xs).max()
    # the same through the full schedule (scale step off, one GN iteration)
    x2, t2, rep = o.optimise(kf, x0=x0, t0=t, n_gn=1, n_pcg=300, delta=INF, scale_step=False)
    assert t2 == t
    assert np.allclose(x2.ravel(), xs, rtol=0, atol=1e-10 * np.abs(xs).max())


def _bordered(o, kf):
    """Hessian/2 and -gradient/2 at 0 of the least-squares cost over (x, t),
    by exact second differences of the cost (a quadratic)."""
    N = kf.width * kf.height
    c = lambda y: o.cost(kf, y[:N], y[N], INF)
    n = N + 1
    e = np.eye(n)
    z = np.zeros(n)
    c0 = c(z)
    ce = np.array([c(e[j]) for j in range(n)])
    cm = np.array([c(-e[j]) for j in range(n)])
    A = np.empty((n, n))
    for j in range(n):
        for k in range(j, n):
            if j == k:
                A[j, j] = (c(2 * e[j]) - 2 * ce[j] + c0) / 2.0
            else:
                A[j, k] = A[k, j] = (c(e[j] + e[k]) - ce[j] - ce[k] + c0) / 2.0
    b = -(ce - cm) / 4.0
    return A, b


def joint_optimum(o):
    W, H = 6, 5
    kf = _noisy(W, H, 8)
    N = W * H
    A, b = _bordered(o, kf)
    ys = np.linalg.solve(A, b)
    np.linalg.cholesky(A)  # positive definite: the minimiser is unique
    x, t, rep = o.optimise(kf, n_gn=400, n_pcg=200, delta=INF)
    assert abs(t - ys[N]) < 1e-9, (t, ys[N])
    assert np.allclose(x.ravel(), ys[:N], rtol=0, atol=1e-9)


def joint_bordered(o):
    """The joint variant runs Jacobi-PCG on the bordered system itself: its
    first iterations equal textbook PCG on the (x, t) Hessian of the cost
    (built here from the cost alone), and it reaches that system's solution."""
    W, H = 6, 5
    kf = _noisy(W, H, 12)
    N = W * H
    K, b = _bordered(o, kf)
    ys = np.linalg.solve(K, b)
    rng = np.random.default_rng(4)
    y0 = np.concatenate([kf.mu_n.ravel().astype(np.float64) + rng.normal(0, 0.1, N), [0.3]])
    m = np.diag(K).copy()
    y, r = y0.copy(), b - K @ y0
    zv = r / m
    p = zv.copy()
    rho = r @ zv
    for j in range(1, 4):
        q = K @ p
        a = rho / (p @ q)
        y = y + a * p
        r = r - a * q
        x1, t1, rep = o.optimise(kf, x0=y0[:N], t0=y0[N], n_gn=1, n_pcg=j, delta=INF,
                                 scale_step=orc.SCALE_JOINT)
        assert rep.iters_done == j
        assert abs(t1 - y[N]) < 1e-10, (j, t1, y[N])
        assert np.allclose(x1.ravel(), y[:N], rtol=0, atol=1e-10), (j, np.abs(x1.ravel() - y[:N]).max())
        zv = r / m
        rho1 = r @ zv
        p = zv + (rho1 / rho) * p
        rho = rho1
    x, t, rep = o.optimise(kf, x0=y0[:N], t0=y0[N], n_gn=1, n_pcg=4 * (N + 1), delta=INF,
                           scale_step=orc.SCALE_JOINT)
    assert abs(t - ys[N]) < 1e-10 and np.allclose(x.ravel(), ys[:N], rtol=0, atol=1e-10)
    # without semi-dense pixels the border row is empty and t stays put
    k0 = types.SimpleNamespace(**vars(kf))
    k0.var_s = np.zeros_like(kf.var_s)
    x0j, t0j, _ = o.optimise(k0, t0=0.25, n_gn=2, n_pcg=5, delta=INF, scale_step=orc.SCALE_JOINT)
    x0a, t0a, _ = o.optimise(k0, t0=0.25, n_gn=2, n_pcg=5, delta=INF, scale_step=orc.SCALE_FIXED)
    assert t0j == 0.25 and np.allclose(x0j, x0a, rtol=0, atol=1e-13)


def prior_only(o):
    kf = _noisy(9, 7, 4)
    x, t, rep = o.optimise(kf, n_gn=3, n_pcg=4, terms=orc.TERM_NET)
    assert np.array_equal(x.ravel(), kf.mu_n.ravel().astype(np.float64))
    assert t == 0.0 and rep.iters_done == 0
    rng = np.random.default_rng(2)
    x0 = kf.mu_n.ravel() + rng.normal(0, 0.5, kf.n_pixels)
    for delta in (INF, DELTA):
        x, t, rep = o.optimise(kf, x0=x0, n_gn=1, n_pcg=1, terms=orc.TERM_NET, delta=delta)
        assert np.allclose(x.ravel(), kf.mu_n.ravel(), rtol=0, atol=1e-12)


def planar_recovery(o):
    W, H = 24, 16
    base = synth.make_keyframe(W, H, 21)
    L = base.log_depth_true
    kf = types.SimpleNamespace(width=W, height=H, mu_n=L.copy(), var_n=base.var_n,
                               var_gx=base.var_gx, var_gy=base.var_gy)
    kf.gx = np.zeros((H, W))
    kf.gy = np.zeros((H, W))
    kf.gx[:, :-1] = L[:, 1:] - L[:, :-1]
    kf.gy[:-1, :] = L[1:, :] - L[:-1, :]
    m = base.var_s > 0
    ts = base.scale_log_true
    kf.mu_s = np.where(m, L - ts, 0.0)
    kf.var_s = np.where(m, base.var_s, 0.0)
    x0 = np.full(W * H, L.mean())
    for delta in (INF, DELTA):
        x, t, rep = o.optimise(kf, x0=x0, n_gn=1000, n_pcg=100, delta=delta)
        assert abs(t - ts) < 1e-8, (delta, t, ts)
        assert np.allclose(x, L, rtol=0, atol=1e-8), np.abs(x - L).max()


def huber_scipy(o):
    from scipy.optimize import minimize

    W, H = 4, 4
    kf = _noisy(W, H, 30)
    kf.mu_n = kf.mu_n.astype(np.float64)
    kf.mu_n[1, 2] += 1.5   # network outliers
    kf.mu_n[3, 0] -= 1.2
    kf.mu_s = kf.mu_s.astype(np.float64)
    kf.var_s = kf.var_s.astype(np.float64)
    kf.var_s[0, :] = 0.01
    kf.mu_s[0, :] = kf.log_depth_true[0, :] - kf.scale_log_true
    kf.mu_s[0, 1] += 0.8   # semi-dense outlier
    kf.gx = kf.gx.astype(np.float64)
    kf.gx[2, 1] += 0.9     # gradient outlier
    N = W * H
    f = lambda y: o.cost(kf, y[:N], y[N], DELTA)
    x, t, rep = o.optimise(kf, n_gn=3000, n_pcg=60, delta=DELTA)
    y_irls = np.concatenate([x.ravel(), [t]])
    res = minimize(f, np.concatenate([kf.mu_n.ravel(), [0.0]]), method="BFGS",
                   options={"gtol": 1e-10, "maxiter": 20000})
    assert f(y_irls) <= res.fun + 1e-9 * max(1.0, abs(res.fun)), (f(y_irls), res.fun)
    assert np.allclose(y_irls, res.x, rtol=0, atol=1e-5), np.abs(y_irls - res.x).max()
    # the joint (x, t) variant of the GN iteration reaches the same minimiser
    xj, tj, _ = o.optimise(kf, n_gn=400, n_pcg=60, delta=DELTA, scale_step=orc.SCALE_JOINT)
    yj = np.concatenate([xj.ravel(), [tj]])
    assert f(yj) <= res.fun + 1e-9 * max(1.0, abs(res.fun)), (f(yj), res.fun)
    assert np.allclose(yj, res.x, rtol=0, atol=1e-5), np.abs(yj - res.x).max()
    # Huber must actually be active somewhere for this pin to mean anything
    assert abs(o.cost(kf, x, t, DELTA) - o.cost(kf, x, t, INF)) > 1e-3


def invariances(o):
    kf = _noisy(12, 9, 40)
    for delta in (INF, DELTA):
        x, t, _ = o.optimise(kf, n_gn=10, n_pcg=3, delta=delta)
        c = 0.37
        k1 = types.SimpleNamespace(**vars(kf))
        k1.mu_s = kf.mu_s.astype(np.float64) + c
        x1, t1, _ = o.optimise(k1, t0=-c, n_gn=10, n_pcg=3, delta=delta)
        assert abs(t1 - (t - c)) < 1e-10 and np.allclose(x1, x, rtol=0, atol=1e-10)
        k2 = types.SimpleNamespace(**vars(kf))
        k2.mu_s = kf.mu_s.astype(np.float64) + c
        k2.mu_n = kf.mu_n.astype(np.float64) + c
        x2, t2, _ = o.optimise(k2, n_gn=10, n_pcg=3, delta=delta)
        assert abs(t2 - t) < 1e-10 and np.allclose(x2, x + c, rtol=0, atol=1e-10)
        k3 = types.SimpleNamespace(width=kf.height, height=kf.width)
        for a, b in (("mu_n", "mu_n"), ("var_n", "var_n"), ("gx", "gy"), ("var_gx", "var_gy"),
                     ("gy", "gx"), ("var_gy", "var_gx"), ("mu_s", "mu_s"), ("var_s", "var_s")):
            setattr(k3, a, np.ascontiguousarray(getattr(kf, b).T))
        x3, t3, _ = o.optimise(k3, n_gn=10, n_pcg=3, delta=delta)
        assert abs(t3 - t) < 1e-10 and np.allclose(x3, x.T, rtol=0, atol=1e-10)


def monotone(o):
    kf = _noisy(32, 24, 50)
    rng = np.random.default_rng(1)
    for delta in (INF, DELTA):
        for x0 in (None, kf.mu_n.ravel() + rng.normal(0, 0.3, kf.n_pixels)):
            for npcg in (1, 3):
                for mode in (orc.SCALE_ALTERNATE, orc.SCALE_JOINT):
                    *_, tr = o.optimise(kf, x0=x0, n_gn=10, n_pcg=npcg, delta=delta, trace=True,
                                        scale_step=mode)
                    d = np.diff(tr)
                    assert np.all(d <= 1e-12 * tr[0]), (delta, npcg, mode, d.max())
                    assert tr[-1] < tr[0]


def no_pairwise(o):
    kf = _noisy(10, 8, 60)
    terms = orc.TERM_SEMI | orc.TERM_NET
    mu_n = kf.mu_n.astype(np.float64).ravel()
    vn = kf.var_n.astype(np.float64).ravel()
    vs = kf.var_s.astype(np.float64).ravel()
    mu_s = kf.mu_s.astype(np.float64).ravel()
    valid = vs > 0
    ws = np.where(valid, 1.0 / np.where(valid, vs, 1.0), 0.0)
    wn = 1.0 / vn
    h = ws * wn / (ws + wn)
    ts = np.sum(h * (mu_n - mu_s)) / np.sum(h)
    xs = (ws * (ts + mu_s) + wn * mu_n) / (ws + wn)
    x, t, _ = o.optimise(kf, n_gn=20000, n_pcg=1, delta=INF, terms=terms)
    assert abs(t - ts) < 1e-10, (t, ts)
    assert np.allclose(x.ravel(), xs, rtol=0, atol=1e-10)
    # one GN iteration: scale step from x = mu_n, then the exact per-pixel solve
    t1 = np.sum(ws * (mu_n - mu_s)) / np.sum(ws)
    x1 = (ws * (t1 + mu_s) + wn * mu_n) / (ws + wn)
    x, t, _ = o.optimise(kf, n_gn=1, n_pcg=1, delta=INF, terms=terms)
    assert abs(t - t1) < 1e-12 and np.allclose(x.ravel(), x1, rtol=0, atol=1e-12)


def tukey_after_huber(o):
    """The Huber-then-Tukey schedule (Section IV names Tukey's loss; being
    non-convex it is started from a Huber solve): warm_gn = n_gn is the
    Huber solve and warm_gn = 0 the Tukey solve, bit for bit; k Huber
    iterations followed by n - k Tukey ones equal a Huber solve of k
    iterations continued by a Tukey solve of n - k from its (x, t); and the
    Tukey iterations never increase the Tukey cost (IRLS on a loss concave
    in u^2 is majorise-minimise, and truncated CG decreases the majoriser)."""
    kf = _noisy(12, 9, 81)
    rng = np.random.default_rng(81)
    m = kf.var_s > 0
    out = rng.random(kf.mu_s.shape) < 0.15  # gross semi-dense outliers
    kf.mu_s = np.where(m & out, kf.mu_s + rng.choice([-1.5, 1.5], kf.mu_s.shape), kf.mu_s)
    n, k = 8, 3
    tk = dict(delta=TUKEY_C, loss=orc.LOSS_TUKEY, n_pcg=4)
    x_h, t_h, r_h = o.optimise(kf, n_gn=n, n_pcg=4, delta=DELTA)
    x_w, t_w, r_w = o.optimise(kf, n_gn=n, warm_gn=n, warm_delta=DELTA, **tk)
    assert np.array_equal(x_w, x_h) and t_w == t_h and r_w.iters_done == r_h.iters_done
    x_t, t_t, _ = o.optimise(kf, n_gn=n, **tk)
    x_0, t_0, _ = o.optimise(kf, n_gn=n, warm_gn=0, warm_delta=0.5, **tk)
    assert np.array_equal(x_0, x_t) and t_0 == t_t
    x1, t1, r1 = o.optimise(kf, n_gn=k, n_pcg=4, delta=DELTA)
    x2, t2, r2 = o.optimise(kf, x0=x1, t0=t1, n_gn=n - k, **tk)
    xs, ts, rs, tr = o.optimise(kf, n_gn=n, warm_gn=k, warm_delta=DELTA, trace=True, **tk)
    assert np.array_equal(xs, x2) and ts == t2
    assert rs.iters_done == r1.iters_done + r2.iters_done
    assert not np.array_equal(xs, x_t) and not np.array_equal(xs, x_h)
    d = np.diff(tr[2 * k:])
    assert np.all(d <= 1e-12 * tr[2 * k]), d.max()


def ls_scale_fit(o):
    """Table II's least-squares scale fit (reading: the shift c minimising
    sum_i (x_i + c - mu_n,i)^2 moves x and t together, so the semi-dense
    residuals x - t - mu_s are unchanged).

    Fixed by a constructed answer: x = mu_n - c0 + e with sum(e) = 0 exactly
    (e in 1/1024 steps, paired with its negation) must come back as x + c0
    and t0 + c0. Then, on an arbitrary x, three facts the definition fixes:
    the fitted x has zero mean offset from mu_n (first-order optimality) and
    a strictly smaller objective than any other shift; x - t is unchanged per
    pixel; shifting the input x by k leaves the fitted x unchanged."""
    W, H = 11, 7
    kf = _noisy(W, H, 71)
    N = W * H
    mu_n = kf.mu_n.astype(np.float64).ravel()
    rng = np.random.default_rng(71)
    half = rng.integers(-200, 201, N // 2) / 1024.0
    e = np.concatenate([half, -half, np.zeros(N - 2 * (N // 2))])
    rng.shuffle(e)
    c0, t0 = 0.375, -0.21
    x_in = mu_n - c0 + e
    xf, tf = o.ls_scale_fit(kf, x_in, t0)
    assert np.allclose(xf.ravel(), x_in + c0, rtol=0, atol=1e-13), np.abs(xf.ravel() - x_in - c0).max()
    assert abs(tf - (t0 + c0)) < 1e-13, (tf, t0 + c0)
    # an arbitrary start
    x_in = mu_n + rng.normal(0.8, 0.3, N)
    xf, tf = o.ls_scale_fit(kf, x_in, t0)
    xf = xf.ravel()
    assert abs(np.sum(xf - mu_n)) < 1e-11 * N
    obj = lambda c: np.sum((xf + c - mu_n) ** 2)
    for h in (1e-3, -1e-3, 0.1, -0.1):
        assert obj(h) > obj(0.0)
    assert np.allclose(xf - tf, x_in - t0, rtol=0, atol=1e-13)
    k = -1.7
    xk, tk = o.ls_scale_fit(kf, x_in + k, t0)
    assert np.allclose(xk.ravel(), xf, rtol=0, atol=1e-12)
    assert abs(tk - (tf - k)) < 1e-12


def semi_to_log(o):
    rng = np.random.default_rng(3)
    d = np.array([0.5, 1.0, 2.0, 4.5, -1.0, 0.0, 2.0, np.nan])
    sd = np.array([1e-3, 2e-3, 4e-3, 1e-2, 1e-3, 1e-3, -1.0, 1.0])
    mu, var = o.semi_to_log(d, sd * np.abs(sd))
    for i in range(4):
        s = np.log(d[i] + sd[i] * rng.normal(size=400000))
        assert abs(mu[i] - np.log(d[i])) < 1e-15
        assert np.isclose(var[i], s.var(), rtol=0.01), (i, var[i], s.var())
    assert np.all(mu[4:] == 0) and np.all(var[4:] == 0)


def within_10pct(o):
    """Section III-B's accuracy measure on a hand-made list: estimates at known
    relative offsets from the truth (well away from the 10% edge), and truths
    that do not count (zero, negative, NaN, infinite)."""
    g = np.array([1.0, 2.0, 0.7, 4.2, 3.0, 1.5, 2.5, 0.9, 0.0, -1.0, np.nan, np.inf, 5.0])
    off = np.array([0.0, 0.05, -0.05, 0.098, -0.098, 0.102, -0.11, 0.3, 0.0, 0.0, 0.0, 0.0, -0.5])
    with np.errstate(invalid="ignore", divide="ignore"):
        x = np.log(np.abs(g) * (1.0 + off))
    x[~np.isfinite(x)] = 0.0
    assert o.within(x, g, 0.1) == (5, 9)
    assert o.within(x, g, 0.2) == (7, 9)
    assert o.within(x, g, 0.0) == (1, 9)   # only g = 1, x = 0 is exact
    assert o.within(np.zeros(0), np.zeros(0), 0.1) == (0, 0)


def _rectified(delta_true, tx=0.2, fx=50.0, W=64, H=32):
    """Fronto-parallel plane, reference camera shifted along x (X_ref = X_key +
    (tx, 0, 0)), linear-ramp images: a keyframe point at depth Z appears
    fx tx / Z pixels further along x (the textbook disparity relation)."""
    cam = (fx, fx, W / 2.0, H / 2.0)
    u = np.arange(W, dtype=np.float64)[None, :]
    v = np.arange(H, dtype=np.float64)[:, None]
    img_key = (3.0 * u + 0.5 * v + 10.0) * np.ones((H, W))
    img_ref = img_key - 3.0 * delta_true
    return cam, img_key.astype(np.float32), img_ref.astype(np.float32), np.eye(3), np.array([tx, 0.0, 0.0])


def mvs_rectified(o):
    """Section II-B on rectified stereo in closed form: depth steps are
    disparities fx tx / d_min - j (1 px apart); with ramp images the error of
    every sample is 3 (disparity - true disparity), so the best step, its
    neighbour, the linearised sub-pixel fraction and sigma^2 = (J^T J)^-1
    are known exactly."""
    fx, tx = 50.0, 0.2
    B = fx * tx  # disparity x depth
    prm = dict(grad_min=1.0, d_min=0.5, d_max=10.0, ssd_max=1e9, max_steps=512)
    for dstar, (da_disp, db_disp) in ((8.0, (8.0, 9.0)), (8.3, (8.0, 9.0)), (7.8, (8.0, 7.0))):
        cam, ik, ir, R, t = _rectified(dstar, tx, fx)
        d, var, st, bs, mg, n = o.semi_dense(ik, ir, cam, R, t, **prm)
        da, db = B / da_disp, B / db_disp
        ea, eb = 3.0 * (da_disp - dstar), 3.0 * (db_disp - dstar)
        s = min(1.0, max(0.0, -ea / (eb - ea)))
        want_d = da + s * (db - da)
        want_var = (db - da) ** 2 / (5.0 * (eb - ea) ** 2)
        for (yy, xx) in ((16, 20), (10, 30), (20, 35)):
            assert st[yy, xx] == orc.MVS_OK, (dstar, st[yy, xx])
            assert bs[yy, xx] == int(round(B / prm["d_min"] - da_disp)), (dstar, bs[yy, xx])
            # the images are stored in float32 (values ~100 carry ~4e-6 rounding)
            assert abs(d[yy, xx] - want_d) < 1e-6 * want_d, (dstar, d[yy, xx], want_d)
            assert abs(var[yy, xx] - want_var) < 1e-5 * want_var, (dstar, var[yy, xx], want_var)
        # pixels whose samples leave the image, and the border rows, are not measured
        assert st[0, 20] == orc.MVS_FLAT and st[16, 63] == orc.MVS_FLAT
        assert st[16, 62] != orc.MVS_OK
    # too little texture: nothing is measured
    cam, ik, ir, R, t = _rectified(8.0, tx, fx)
    _, _, st, _, _, n = o.semi_dense(ik, ir, cam, R, t, **dict(prm, grad_min=4.0))
    assert n == 0 and np.all(st == orc.MVS_FLAT)


def mvs_fusion_and_interval(o):
    """A current estimate narrows the search to d +- 2 sigma and is fused with
    the measurement by the Gaussian product; an estimate wide enough to cover
    the whole range leaves the measurement unchanged before fusion."""
    fx, tx = 50.0, 0.2
    cam, ik, ir, R, t = _rectified(8.3, tx, fx)
    prm = dict(grad_min=1.0, d_min=0.5, d_max=10.0, ssd_max=1e9, max_steps=512)
    d0, v0, st0, _, _, _ = o.semi_dense(ik, ir, cam, R, t, **prm)
    H, W = ik.shape
    prior_d = np.full((H, W), 2.0)
    prior_v = np.full((H, W), 100.0)  # +-20 m: the whole range
    d1, v1, st1, _, _, _ = o.semi_dense(ik, ir, cam, R, t, depth=prior_d, var=prior_v, **prm)
    m = st0 == orc.MVS_OK
    assert np.array_equal(st1 == orc.MVS_OK, m)
    want_v = prior_v[m] * v0[m] / (prior_v[m] + v0[m])
    want_d = (prior_d[m] * v0[m] + d0[m] * prior_v[m]) / (prior_v[m] + v0[m])
    assert np.allclose(v1[m], want_v, rtol=1e-12) and np.allclose(d1[m], want_d, rtol=1e-12)
    # a tight estimate far from the truth: the measurement stays near it
    pd, pv = np.full((H, W), 1.6), np.full((H, W), 0.01 ** 2)
    d2, v2, st2, _, _, _ = o.semi_dense(ik, ir, cam, R, t, depth=pd, var=pv, **prm)
    k = st2 == orc.MVS_OK
    assert k.sum() > 0
    step = fx * tx / 1.6 ** 2  # pixels of disparity per metre of depth at 1.6 m
    assert np.all(np.abs(d2[k] - 1.6) <= 0.02 + 2.0 / step)
    # pixels without texture keep their estimate
    assert np.array_equal(d2[~k & (st2 == orc.MVS_FLAT)], pd[~k & (st2 == orc.MVS_FLAT)])


def mvs_scene(o):
    """On a noise-free textured scene (two views, known pose) the measured
    depths agree with the scene's true depth: most within 10 %, the median
    within a few per cent, and the stated sigma is not wildly optimistic."""
    sp = synth.make_stereo_pair(320, 240, 5)
    d, var, st, bs, mg, n = o.semi_dense(sp.img_key, sp.img_ref, sp.cam, sp.R, sp.t)
    m = st == orc.MVS_OK
    assert m.mean() > 0.15, m.mean()
    rel = np.abs(d[m] / sp.depth_true[m] - 1.0)
    assert np.median(rel) < 0.03 and np.mean(rel < 0.1) > 0.8, (np.median(rel), np.mean(rel < 0.1))
    z = np.abs(d[m] - sp.depth_true[m]) / np.sqrt(var[m])
    assert np.median(z) < 10.0


ALL = [cost_closed_form, robust_weight, dense_hessian, joint_optimum, joint_bordered, prior_only,
       planar_recovery, huber_scipy, invariances, monotone, no_pairwise, tukey_after_huber, ls_scale_fit,
       semi_to_log,
       within_10pct,
       mvs_rectified, mvs_fusion_and_interval, mvs_scene]
