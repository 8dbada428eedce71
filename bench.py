#!/usr/bin/env python
"""Throughput of the per-frame keyframe re-optimisation on GB300.

Default workload (one "step"): 64 keyframes of uneven sizes drawn from
{320x240, 512x384, 640x480, 1280x960} (30.5 Mpixel), each its own synthetic
scene, re-optimised together for one frame: keyframe (re)initialisation from
the network planes, the frame's semi-dense refresh, one batched solve of
10 Gauss-Newton x 3 PCG iterations (scale step, re-weighting / assembly,
PCG) in one persistent launch replayed from a CUDA graph with an autotuned
launch shape, and the depth output. Beside it the same keyframes are solved
by the plain path, one df_optimise launch per keyframe, and both results are
checked to agree.

Metric: Mpixel.iter/s = sum over keyframes of H*W*n_gn*n_pcg / time / 1e6.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload batch64|sequence|precision|serving|mvs]

With N > 1 (torchrun, one rank per GPU) every rank solves its own keyframes
(weak scaling, no collective on the data path); value = all ranks' units /
max-over-ranks time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import multiprocessing as mp
import os
import platform
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Mpixel·iter/s"
WORKLOAD = "sequence-640x480-100f-10x5-fp32"  # the default sequence workload


def sequence_name(args) -> str:
    """Name of the sequence workload a run measures (WORKLOAD by default)."""
    v = "" if getattr(args, "variant", "paper") == "paper" else f"-{args.variant}"
    return (f"sequence-{args.width}x{args.height}-{args.frames}f-"
            f"{args.n_gn}x{args.n_pcg}-fp32{v}")
SCALE_STEPS = {"fixed": 0, "alternate": 1, "joint": 2}  # DF_SCALE_* values
ALG_BYTES_PER_PCG_PX = 56  # canonical streaming model of one PCG iteration
ALG_BYTES_PER_GN_PX = 56   # scale step + re-weighting / assembly per GN iteration


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--solver", choices=["auto", "launches", "fused"], default="auto")
    ap.add_argument("--scale-step", choices=["alternate", "joint", "fixed"], default="alternate",
                    help="how t is solved: the paper's alternation, the joint (x, t) PCG, or fixed")
    ap.add_argument("--width", type=int, default=640)
    ap.add_argument("--height", type=int, default=480)
    ap.add_argument("--frames", type=int, default=100)
    ap.add_argument("--n-gn", type=int, default=None,
                    help="Gauss-Newton iterations per solve (default: the workload's, 10)")
    ap.add_argument("--n-pcg", type=int, default=None,
                    help="PCG iterations per GN iteration (default: the workload's, 5 for the "
                         "sequence, 3 for the keyframe workloads)")
    ap.add_argument("--variant", choices=["paper", "table2", "table3"], default="paper",
                    help="paper: the full cost with the alternating scale step; table2: semi-dense "
                         "+ gradient terms with the scale fixed, then the least-squares scale fit "
                         "to the network depth (Table II); table3: semi-dense + network terms, no "
                         "pairwise term (Table III)")
    ap.add_argument("--loss", choices=["huber", "lsq", "tukey", "huber-tukey"], default="huber",
                    help="robust loss: Huber (delta 1.345, the default), least squares, "
                         "Tukey's biweight (c 4.685), or 3 Huber GN iterations then Tukey")
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--mode", choices=["auto", "streaming", "resident"], default="auto",
                    help="fused kernel (launch shape)")
    ap.add_argument("--max-ctas", type=int, default=0, help="cap on the fused kernel's grid")
    ap.add_argument("--vec", type=int, default=0)
    ap.add_argument("--tile-rows", type=int, default=0)
    ap.add_argument("--assembly", type=int, choices=[0, 1, 2], default=0,
                    help="streaming kernel: where each GN iteration is assembled (0 auto, "
                         "1 a pass of the persistent kernel, 2 a kernel of its own)")
    ap.add_argument("--workload", choices=["batch64", "sequence", "precision", "serving", "mvs"],
                    default="batch64",
                    help="batch64: 64 keyframes of uneven sizes in one batched solve (default); "
                         "sequence: a 640x480 keyframe over 100 frames; precision: one "
                         "1920x1440 keyframe with reduced-precision network planes")
    ap.add_argument("--cnn-dtype", choices=["f32", "bf16", "f16"], default="bf16",
                    help="network-plane storage for --workload precision")
    ap.add_argument("--no-graph", action="store_true",
                    help="batch64: launch the batched solve eagerly instead of replaying a CUDA graph")
    ap.add_argument("--graph", action="store_true",
                    help="sequence: replay each frame's work (semi-dense update, solve, depth "
                         "output) from a CUDA graph captured once")
    ap.add_argument("--no-autotune", action="store_true",
                    help="batch64: keep the default launch shape instead of autotuning it")
    ap.add_argument("--rate", type=float, default=600.0, help="serving: frames/s offered")
    ap.add_argument("--requests", type=int, default=1200, help="serving: frames per run")
    args = ap.parse_args()
    keyframes = args.workload in ("batch64", "precision")
    if args.n_gn is None:
        args.n_gn = 10
    if args.n_pcg is None:
        args.n_pcg = 3 if keyframes else 5
    return args


# (delta, loss code, Huber warm-start GN iterations) of each --loss choice:
# the C ABI's df_solve_params fields and the oracle's keyword arguments take
# the same values
LOSSES = {"huber": (1.345, 0, 0), "lsq": (0.0, 0, 0), "tukey": (4.685, 1, 0),
          "huber-tukey": (4.685, 1, 3)}


def loss_params(args):
    delta, loss, warm = LOSSES[args.loss]
    kw = {"delta": delta, "loss": loss}
    if warm:
        kw.update(warm_gn=warm, warm_delta=1.345)
    return kw


# df_solve_params.terms of each --variant (DF_TERM_SEMI = 1, NET = 2, GRAD = 4)
VARIANT_TERMS = {"paper": 7, "table2": 5, "table3": 3}


def method_params(args):
    """The solve's method fields (loss, terms, scale step): the same keyword
    arguments for df_default_params and for the oracle's optimise."""
    kw = loss_params(args)
    kw["terms"] = VARIANT_TERMS[args.variant]
    kw["scale_step"] = SCALE_STEPS["fixed" if args.variant == "table2" else args.scale_step]
    return kw


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def _code_only(text: str) -> str:
    """C++ source without comments and with whitespace runs collapsed (string
    and character literals kept), so that comment or layout edits do not
    change the hash of the kernels' code."""
    out, i, n = [], 0, len(text)
    while i < n:
        c = text[i]
        if c in "\"'":
            j = i + 1
            while j < n and text[j] != c:
                j += 2 if text[j] == "\\" else 1
            out.append(text[i:j + 1])
            i = j + 1
        elif text.startswith("//", i):
            j = text.find("\n", i)
            i = n if j < 0 else j
        elif text.startswith("/*", i):
            j = text.find("*/", i + 2)
            i = n if j < 0 else j + 2
            out.append(" ")
        else:
            out.append(c)
            i += 1
    return " ".join("".join(out).split())


# The sources of the fused solvers, whose launches profiles/traffic.json
# records: the kernels, their launch plans and the device headers they use.
FUSED_SOURCES = ("df_exact.cuh", "df_fused.cu", "df_fused.cuh", "df_internal.cuh",
                 "df_resident.cu", "df_sync.cuh", "df_tma.cuh")


def lib_source_hash():
    """Hash of the fused solvers' code (comments and whitespace excluded):
    the key under which profiles/traffic.json records the ncu DRAM bytes."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2207_12244_gb300", "csrc")
    for n in sorted(os.listdir(csrc)):
        if n in FUSED_SOURCES:
            with open(os.path.join(csrc, n), encoding="utf-8") as f:
                h.update(n.encode())
                h.update(_code_only(f.read()).encode())
    return h.hexdigest()[:16]


def traffic_key(args, workload: str) -> str:
    """Key of a workload's dominant-kernel entry in profiles/traffic.json:
    the solver, the workload and every launch-shape or method flag that
    changes which kernel runs (a forced mode, grid cap, tile shape, the joint
    scale step)."""
    key = f"solve_{args.solver}_{workload}"  # the workload name carries a --variant
    if getattr(args, "scale_step", "alternate") != "alternate":
        key += f"_{args.scale_step}"
    if getattr(args, "loss", "huber") != "huber":
        key += f"_{args.loss}"
    if args.mode != "auto":
        key += f"_{args.mode}"
    for flag in ("max_ctas", "vec", "tile_rows", "assembly"):
        if getattr(args, flag, 0):
            key += f"_{flag}{getattr(args, flag)}"
    return key


def ncu_traffic(kernel_key: str):
    """Per-launch DRAM bytes of the dominant kernel from the committed ncu
    summary, if it was taken on the current kernel sources."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    e = d.get(kernel_key)
    if not e or e.get("source_hash") != lib_source_hash():
        return None
    return e.get("dram_bytes_per_launch")


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join("/tmp", f"df_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        time.sleep(0.25)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                c = [x.strip() for x in line.split(",")]
                if len(c) < 9:
                    continue
                try:
                    sm.append(float(c[1]))
                    smax = float(c[2])
                except ValueError:
                    continue
                for n, v in zip(names, c[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(n)
        os.remove(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


L2_NOTE = "flushed between steps (256 MB write)"


def sequence_config(args, ws):
    """config of the sequence workload (the same in both arms)."""
    return {"workload": sequence_name(args), "width": args.width, "height": args.height,
            "frames": args.frames, "n_gn": args.n_gn, "n_pcg": args.n_pcg, "loss": args.loss,
            "scale_step": args.scale_step, "variant": args.variant,
            "parallelism": f"replicas x{ws}", "l2": L2_NOTE}


def keyframe_shapes(args, rank):
    """(name, [(W, H)], network-plane dtype name) of a keyframe workload."""
    v = "" if args.variant == "paper" else f"-{args.variant}"
    if args.workload == "batch64":
        shapes = synth_batch_shapes(64, rank_seed(args.seed, rank))
        return f"batch64-uneven-{args.n_gn}x{args.n_pcg}-fp32{v}", shapes, "f32"
    return (f"keyframe-1920x1440-{args.n_gn}x{args.n_pcg}-{args.cnn_dtype}{v}", [(1920, 1440)],
            args.cnn_dtype)


def keyframe_seeds(args, rank, shapes):
    base = rank_seed(args.seed, rank)
    return [base + 17 * i for i in range(len(shapes))]


def keyframes_config(args, ws, rank=0):
    """config of the batch / large-keyframe workloads (the same in both arms)."""
    name, shapes, dt_name = keyframe_shapes(args, rank)
    return {"workload": name, "keyframes": len(shapes), "pixels": sum(W * H for W, H in shapes),
            "cnn_dtype": dt_name, "n_gn": args.n_gn, "n_pcg": args.n_pcg, "loss": args.loss,
            "scale_step": args.scale_step, "variant": args.variant,
            "parallelism": f"replicas x{ws}", "l2": L2_NOTE}


def synth_batch_shapes(n, seed):
    from paper_2207_12244_gb300 import synth

    return synth.batch_shapes(n, seed)


def rank_seed(base, rank):
    from paper_2207_12244_gb300 import replicas

    return replicas.rank_seed(base, rank)


def host_cpu():
    """(model name, usable cores) of this host."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.split(":")[0].strip() == "Model name":
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if not model:
        try:
            with open("/proc/cpuinfo") as f:
                for line in f:
                    if line.lower().startswith("model name"):
                        model = line.split(":", 1)[1].strip()
                        break
        except OSError:
            pass
    try:
        cores = len(os.sched_getaffinity(0))
    except AttributeError:
        cores = os.cpu_count() or 1
    return f"{model or 'unknown'} ({platform.machine()})", cores


def _shares(sizes, n_workers):
    """Largest-first greedy split of jobs over workers (balanced work)."""
    loads = [0] * n_workers
    shares = [[] for _ in range(n_workers)]
    for i in sorted(range(len(sizes)), key=lambda j: -sizes[j]):
        w = min(range(n_workers), key=lambda k: loads[k])
        shares[w].append(i)
        loads[w] += sizes[i]
    return [sh for sh in shares if sh]


def _oracle_worker(conn, jobs, solve_kw):
    """Pool worker: generate its keyframes once, then solve them all with the
    oracle (single thread) whenever the parent asks; reply the busy time."""
    import oracle
    from paper_2207_12244_gb300 import synth

    o = oracle.get()
    solve_kw = dict(solve_kw)
    ls_fit = solve_kw.pop("ls_fit", False)
    kfs = [synth.make_keyframe(W, H, seed) for W, H, seed in jobs]
    conn.send(0.0)
    while True:
        msg = conn.recv()
        if msg is None:
            break
        t0 = time.perf_counter()
        for kf in kfs:
            x, t, _ = o.optimise(kf, **solve_kw)
            if ls_fit:  # Table II: the scale fitted to the network depth
                o.ls_scale_fit(kf, x, t)
        conn.send(time.perf_counter() - t0)
    conn.close()


class OraclePool:
    """The oracle over independent keyframes on every host core: one spawned
    process per core, each solving a fixed share of the keyframes (the
    arithmetic of each solve is the oracle's, unchanged)."""

    def __init__(self, jobs, solve_kw, n_workers):
        import oracle

        oracle.build()  # once, before the workers load it
        ctx = mp.get_context("spawn")
        self.shares = _shares([W * H for W, H, _ in jobs], max(1, n_workers))
        self.procs, self.conns = [], []
        for share in self.shares:
            a, b = ctx.Pipe()
            p = ctx.Process(target=_oracle_worker, args=(b, [jobs[i] for i in share], solve_kw),
                            daemon=True)
            p.start()
            b.close()
            self.procs.append(p)
            self.conns.append(a)
        for c in self.conns:
            c.recv()

    def solve_all(self):
        """Wall time of one pass over every keyframe, and each worker's busy time."""
        t0 = time.perf_counter()
        for c in self.conns:
            c.send(1)
        busy = [c.recv() for c in self.conns]
        return time.perf_counter() - t0, busy

    def close(self):
        for c in self.conns:
            try:
                c.send(None)
            except OSError:
                pass
        for p in self.procs:
            p.join(timeout=30)
            if p.is_alive():
                p.terminate()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def keyframe_pool(args, rank, n_workers=None):
    """An OraclePool over the keyframes of a batch / large-keyframe workload."""
    _, shapes, _ = keyframe_shapes(args, rank)
    seeds = keyframe_seeds(args, rank, shapes)
    jobs = [(W, H, sd) for (W, H), sd in zip(shapes, seeds)]
    kw = dict(n_gn=args.n_gn, n_pcg=args.n_pcg, **method_params(args))
    kw["ls_fit"] = args.variant == "table2"
    model, cores = host_cpu()
    n = min(cores, len(jobs)) if n_workers is None else n_workers
    return OraclePool(jobs, kw, n), model, cores


def keyframes_cpu_baseline(args, rank, passes=1):
    """The oracle on every host core over the workload's keyframes: `passes`
    timed passes over all of them (a batch pass is ~20 s of CPU work)."""
    pool, model, cores = keyframe_pool(args, rank)
    _, shapes, _ = keyframe_shapes(args, rank)
    units = sum(W * H for W, H in shapes) * args.n_gn * args.n_pcg
    with pool:
        walls, busy = [], []
        for _ in range(passes):
            w, b = pool.solve_all()
            walls.append(w)
            busy.extend(b)
    return {"value": units * passes / sum(walls) / 1e6, "unit": METRIC,
            "cores": len(pool.shares), "kind": "oracle", "cpu_model": model, "host_cores": cores,
            "single_thread_value": units * passes / sum(busy) / 1e6,
            "sample": f"{passes} pass(es) over all {len(shapes)} keyframes of the workload, "
                      f"{args.n_gn}x{args.n_pcg}, FP64 on the FP32 inputs; one spawned process "
                      f"per core, each a fixed share of the keyframes; {sum(walls):.1f} s wall, "
                      f"{sum(busy):.1f} s of CPU work; single_thread_value = the same work over "
                      f"the workers' summed busy time"}


def _sequence_reference(args, kf, mus, vs, n_frames):
    """The oracle over the first frames of a warm-started sequence, one frame
    per step: (per-step seconds of the timed steps)."""
    import oracle

    o = oracle.get()
    x = kf.mu_n.astype(np.float64).ravel()
    t = 0.0
    times = []

    class _V:
        pass

    view = _V()
    for n in ("width", "height", "mu_n", "var_n", "gx", "var_gx", "gy", "var_gy"):
        setattr(view, n, getattr(kf, n))
    for step in range(args.warmup + args.steps):
        view.mu_s, view.var_s = mus[step % n_frames], vs[step % n_frames]
        t0 = time.perf_counter()
        xr, t, _ = o.optimise(view, x0=x, t0=t, n_gn=args.n_gn, n_pcg=args.n_pcg,
                               **method_params(args))
        if args.variant == "table2":
            xr, t = o.ls_scale_fit(view, xr, t)
        dt = time.perf_counter() - t0
        x = xr.ravel()
        if step >= args.warmup:
            times.append(dt)
    return times


def run_reference(args, ws, rank):
    """The reference arm: the oracle (FP64, CPU) on the same workload and
    config as our arm, on the host cores of this machine. Rank 0 only."""
    if rank != 0:
        return
    from paper_2207_12244_gb300 import synth

    model, cores = host_cpu()
    line = {"impl": "reference", "metric": METRIC, "unit": METRIC, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "l2_note": "config.l2 states how our arm times the GPU; the oracle runs on the host"}
    if args.workload in ("batch64", "precision"):
        line["config"] = keyframes_config(args, ws)
        pool, model, cores = keyframe_pool(args, rank)
        _, shapes, _ = keyframe_shapes(args, rank)
        units = sum(W * H for W, H in shapes) * args.n_gn * args.n_pcg
        with pool:
            for _ in range(args.warmup):
                pool.solve_all()
            walls = [pool.solve_all()[0] for _ in range(args.steps)]
        value = units * len(walls) / sum(walls) / 1e6
        n_used = len(pool.shares)
        sample = (f"every step: all {len(shapes)} keyframes of the workload, {args.n_gn}x"
                  f"{args.n_pcg}, one spawned process per core with a fixed share of them")
    elif args.workload == "mvs":  # one stereo update (first reference view) per step
        import oracle

        o = oracle.get()
        W, H = args.width, args.height
        p = synth.make_stereo_pair(W, H, rank_seed(args.seed, 0), baseline=0.03, view=0)
        walls = []
        for step in range(args.warmup + args.steps):
            t0 = time.perf_counter()
            o.semi_dense(p.img_key, p.img_ref, p.cam, p.R, p.t)
            if step >= args.warmup:
                walls.append(time.perf_counter() - t0)
        line.update({"metric": "Mpixel/s", "unit": "Mpixel/s", "config": mvs_config(args, ws)})
        value = W * H * len(walls) / sum(walls) / 1e6
        n_used = 1
        sample = f"one {W}x{H} stereo update (first reference view) per step, FP64"
    else:
        if args.workload == "serving":  # the frames of the first 640x480 stream, in order
            kf, mus, vs = synth.make_sequence(640, 480, rank_seed(args.seed, 0), n_frames=8)
            n_frames = 8
            px_iters = 640 * 480 * 10 * 5
            args.n_gn, args.n_pcg = 10, 5
            line["config"] = serving_config(args, ws)
            sample = "the frames of one 640x480 stream in order, 10x5 per frame, warm-started"
        else:
            kf, mus, vs = synth.make_sequence(args.width, args.height, args.seed, args.frames)
            n_frames = args.frames
            px_iters = args.width * args.height * args.n_gn * args.n_pcg
            line["config"] = sequence_config(args, ws)
            sample = (f"{args.steps} timed frames (after {args.warmup} warm-up) of the "
                      f"{args.width}x{args.height} sequence, {args.n_gn}x{args.n_pcg} per frame, "
                      "warm-started; one frame per step (frames depend on each other)")
        times = _sequence_reference(args, kf, mus, vs, n_frames)
        walls = times
        value = px_iters * len(times) / sum(times) / 1e6
        n_used = 1
    line.update({
        "value": value, "ms_per_step": 1e3 * sum(walls) / len(walls),
        "cpu_baseline": {"value": value, "unit": line["unit"], "cores": n_used, "kind": "oracle",
                         "cpu_model": model, "host_cores": cores, "sample": sample},
        "e2e": {"value": value, "unit": line["unit"], "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    })
    print(json.dumps(line), flush=True)


def cpu_baseline(args, kf, mus, vs):
    """The oracle on the sequence (frames depend on each other: one core)."""
    import oracle

    o = oracle.get()
    x = kf.mu_n.astype(np.float64).ravel()
    t = 0.0

    class _V:
        pass

    view = _V()
    for n in ("width", "height", "mu_n", "var_n", "gx", "var_gx", "gy", "var_gy"):
        setattr(view, n, getattr(kf, n))
    n = 0
    t_start = time.perf_counter()
    while True:
        view.mu_s, view.var_s = mus[n % args.frames], vs[n % args.frames]
        xr, t, _ = o.optimise(view, x0=x, t0=t, n_gn=args.n_gn, n_pcg=args.n_pcg,
                               **method_params(args))
        if args.variant == "table2":
            xr, t = o.ls_scale_fit(view, xr, t)
        x = xr.ravel()
        n += 1
        el = time.perf_counter() - t_start
        if el >= args.cpu_seconds or n >= args.frames:
            break
    px_iters = args.width * args.height * args.n_gn * args.n_pcg * n
    model, cores = host_cpu()
    return {"value": px_iters / el / 1e6, "unit": METRIC, "cores": 1, "kind": "oracle",
            "cpu_model": model, "host_cores": cores,
            "sample": f"first {n} frames of the same {args.width}x{args.height} sequence, "
                      f"{args.n_gn}x{args.n_pcg} per frame, warm-started, {el:.1f} s single-thread "
                      "(each frame starts from the previous one's result, so one core)"}


def mvs_config(args, ws):
    W, H, F = args.width, args.height, min(args.frames, 8)
    return {"workload": f"mvs-{W}x{H}-{F}views", "width": W, "height": H, "views": F,
            "parallelism": f"replicas x{ws}", "l2": L2_NOTE}


def serving_config(args, ws):
    return {"workload": "serving-32streams-640x480+1280x960-poisson-10x5",
            "offered_frames_per_s": args.rate, "frames": args.requests,
            "budget_bytes": 40 << 30, "parallelism": f"replicas x{ws}"}


def run_serving(args, ws, rank, dev, torch, dfl, replicas, synth):
    """32 camera streams (16 at 640x480, 16 at 1280x960), Poisson frame
    arrivals at --rate frames/s, device-resident keyframes admitted under a
    40 GB budget, 10 GN x 5 PCG per frame: continuous batching vs one launch
    per frame, same arrival schedule."""
    from paper_2207_12244_gb300 import serving

    sizes = [(640, 480)] * 16 + [(1280, 960)] * 16
    my = replicas.shard(len(sizes), rank, ws)
    F = 8
    seqs = [synth.make_sequence(W, H, replicas.rank_seed(args.seed, 0) + 31 * i, n_frames=F)
            for i, (W, H) in enumerate(sizes) if i in my]
    frames = [[(torch.from_numpy(m[f]).to(dev), torch.from_numpy(v[f]).to(dev)) for f in range(F)]
              for _, m, v in seqs]
    cnn = [[torch.from_numpy(p).to(dev) for p in kf.cnn_planes] for kf, _, _ in seqs]
    prm = dfl.df_default_params(n_gn=10, n_pcg=5)
    n_req = max(1, args.requests * len(my) // len(sizes))
    rate = args.rate * len(my) / len(sizes)
    t, s = serving.poisson_schedule(n_req, rate, len(my), seed=args.seed + rank)
    px = np.array([kf.width * kf.height for kf, _, _ in seqs])
    results = {}
    for mode in ("batched", "plain"):
        srv = dfl.df_server_create(memory_budget=40 << 30, max_batch=64, max_inflight=2,
                                   batching=(mode == "batched"), params=prm)
        try:
            sids = [dfl.df_server_open_stream(srv, kf.width, kf.height, *c)
                    for (kf, _, _), c in zip(seqs, cnn)]
            # warm-up: args.warmup rounds of one frame per stream
            for _ in range(max(1, args.warmup)):
                ws_t, ws_s = serving.poisson_schedule(len(sids), 1e6, len(sids), seed=1)
                serving.run(srv, sids, frames, ws_t, np.arange(len(sids)))
            torch.cuda.synchronize()
            st = serving.run(srv, sids, frames, t, s)
        finally:
            dfl.df_server_destroy(srv)
        units = float(px[s].sum()) * 50
        results[mode] = {"p50_ms": st.p50_ms, "p99_ms": st.p99_ms, "mean_ms": st.mean_ms,
                         "max_ms": st.max_ms, "mean_batch": st.mean_batch,
                         "frames_per_s": st.throughput_rps,
                         "mpx_iter_per_s": units / st.wall_s / 1e6, "wall_s": st.wall_s}
    # job-wide: slowest rank's wall time, everybody's work
    wall = replicas.max_over_ranks(results["batched"]["wall_s"], device=dev)
    units_all = replicas.sum_over_ranks(float(px[s].sum()) * 50, device=dev)
    if rank == 0:
        line = {
            "metric": METRIC, "value": units_all / wall / 1e6, "unit": METRIC, "n_gpus": ws,
            "steps": 1, "warmup": max(1, args.warmup), "ms_per_step": 1e3 * wall,
            "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded piecewise-planar scenes; no dataset)",
            "config": serving_config(args, ws),
            "update_latency_ms": {"batched": results["batched"], "plain": results["plain"],
                                  "what": "arrival (submit) to finished (event seen), host clock"},
            "e2e": None, "roofline": None, "cpu_baseline": None,
        }
        print(json.dumps(line), flush=True)


# FP32 operations of one epipolar step of the stereo search, counted from
# the kernel source: the step's depth (9), and per sample (x5) the projection
# (12 + 6), the bilinear read (14), the error and its square (3).
MVS_FLOPS_PER_STEP = 9 + 5 * (12 + 6 + 14 + 3)
# nominal FP32 FMA peak of the part: SMs x 128 lanes x 2 flops x max clock
FP32_LANES_PER_SM = 128


def run_mvs(args, ws, rank, dev, torch, dfl, replicas, synth):
    """Semi-dense stereo (Section II-B): one step = a keyframe image against
    a run of reference views, one df_mvs_update each (search + fusion),
    starting from no estimate."""
    W, H, F = args.width, args.height, min(args.frames, 8)
    seed = replicas.rank_seed(args.seed, rank)
    pairs = [synth.make_stereo_pair(W, H, seed, baseline=0.03 + 0.01 * (v % 4), view=v)
             for v in range(F)]
    name = f"mvs-{W}x{H}-{F}views"
    key_d = torch.from_numpy(pairs[0].img_key).to(dev)
    refs_d = [torch.from_numpy(p.img_ref).to(dev) for p in pairs]
    depth = torch.zeros((H, W), dtype=torch.float32, device=dev)
    var = torch.zeros((H, W), dtype=torch.float32, device=dev)
    stream = torch.cuda.Stream(dev)
    sptr = stream.cuda_stream
    m = dfl.SemiDense(W, H)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(F)]

    def step(record, key, refs, d, v):
        d.zero_()
        v.zero_()
        for f, p in enumerate(pairs):
            if record:
                evs[f][0].record(stream)
            m.update(key, refs[f], p.cam, p.R, p.t, d, v, stream=sptr)
            if record:
                evs[f][1].record(stream)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step(False, key_d, refs_d, depth, var)
    torch.cuda.synchronize()
    # work count of one step (outside the timed region)
    steps_per_update = []
    with torch.cuda.stream(stream):
        depth.zero_()
        var.zero_()
        for f, p in enumerate(pairs):
            m.update(key_d, refs_d[f], p.cam, p.R, p.t, depth, var, stream=sptr)
            steps_per_update.append(m.last_steps(stream=sptr))
    step_ms, upd_ms = [], []
    launches0 = dfl.df_kernel_launches()
    with ClockSampler(dev.index) as clk:
        for _ in range(args.steps):
            flush.fill_(1.0)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(stream):
                e0.record(stream)
                step(True, key_d, refs_d, depth, var)
                e1.record(stream)
            torch.cuda.synchronize()
            step_ms.append(e0.elapsed_time(e1))
            upd_ms.extend(a.elapsed_time(b) for a, b in evs)
    launches = dfl.df_kernel_launches() - launches0
    clocks = clk.summary()
    total_ms = replicas.max_over_ranks(sum(step_ms), device=dev)
    units = W * H * F
    value = units * args.steps * ws / (total_ms / 1e3) / 1e6
    flops = MVS_FLOPS_PER_STEP * float(np.mean(steps_per_update))
    upd_s = statistics.mean(upd_ms) / 1e3
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    peak = sms * FP32_LANES_PER_SM * 2 * 2.07e9 / 1e12
    achieved = flops / upd_s / 1e12
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": None,
                "peak_kind": "derived: SMs x 128 FP32 lanes x 2 x 2.07 GHz (nominal FMA rate)",
                "region": "df_mvs_update (one reference view)",
                "alg_flops_per_launch": flops, "steps_per_launch": float(np.mean(steps_per_update))}
    e2e = None
    if not args.no_e2e:
        key_h = torch.from_numpy(pairs[0].img_key).pin_memory()
        refs_h = [torch.from_numpy(p.img_ref).pin_memory() for p in pairs]
        out_h = torch.empty((2, H, W), dtype=torch.float32).pin_memory()
        kd = torch.empty_like(key_d)
        rd = [torch.empty_like(r) for r in refs_d]
        tms = []
        for it in range(args.steps + 1):
            flush.fill_(1.0)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            with torch.cuda.stream(stream):
                kd.copy_(key_h, non_blocking=True)
                for r, h in zip(rd, refs_h):
                    r.copy_(h, non_blocking=True)
                step(False, kd, rd, depth, var)
                out_h[0].copy_(depth, non_blocking=True)
                out_h[1].copy_(var, non_blocking=True)
            torch.cuda.synchronize()
            if it:
                tms.append(1e3 * (time.perf_counter() - t0))
        tot = replicas.max_over_ranks(sum(tms), device=dev)
        e2e = {"value": units * args.steps * ws / (tot / 1e3) / 1e6, "unit": "Mpixel/s",
               "h2d_bytes_per_step": int(4 * W * H * (F + 1)), "d2h_bytes_per_step": int(8 * W * H),
               "ms_per_step": tot / args.steps}
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        import oracle

        o = oracle.get()
        p = pairs[0]
        t0 = time.perf_counter()
        o.semi_dense(p.img_key, p.img_ref, p.cam, p.R, p.t)
        el = time.perf_counter() - t0
        model, host_cores = host_cpu()
        cpu = {"value": W * H / el / 1e6, "unit": "Mpixel/s", "cores": 1, "kind": "oracle",
               "cpu_model": model, "host_cores": host_cores,
               "sample": f"one {W}x{H} update (first reference view), {el:.2f} s single-thread FP64"}
    m.close()
    if rank == 0:
        line = {
            "metric": "Mpixel/s", "value": value, "unit": "Mpixel/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (two rendered views of a textured piecewise-planar scene)",
            "config": mvs_config(args, ws),
            "clocks": clocks, "e2e": e2e, "gpu_launches": launches, "roofline": roofline,
            "cpu_baseline": cpu,
            "update_latency_ms": {"p50": float(np.percentile(upd_ms, 50)),
                                  "p99": float(np.percentile(upd_ms, 99)),
                                  "what": "one df_mvs_update, device time"},
        }
        print(json.dumps(line), flush=True)


def _flat_views(flat, per, shapes):
    """Per keyframe, `per` consecutive (H, W) views of one flat tensor."""
    out, o = [], 0
    for W, H in shapes:
        vs = []
        for _ in range(per):
            vs.append(flat[o:o + W * H].view(H, W))
            o += W * H
        out.append(vs)
    return out


def keyframes_e2e_pipelined(args, torch, dfl, dev, kfs, shapes, tdt, handles, ks, stream, solve,
                            ls_fit, flush, steps, warmup, barrier):
    """End-to-end steps as a caller with pinned host buffers runs them back
    to back: every step copies all its inputs (network planes and
    semi-dense frames) from pinned host memory to the device and its depth
    maps back, on copy streams, through two device staging sets, so that
    step k+1's upload and step k-1's download overlap step k's solve.
    Returns (wall ms for `steps` steps, from the first upload to the last
    download, the host copy of the last step's depth maps)."""
    px = sum(W * H for W, H in shapes)
    hcnn = torch.empty(6 * px, dtype=tdt).pin_memory()
    hsemi = torch.empty(2 * px, dtype=torch.float32).pin_memory()
    hout = [torch.empty(px, dtype=torch.float32).pin_memory() for _ in range(2)]
    for kf, vc, vsm in zip(kfs, _flat_views(hcnn, 6, shapes), _flat_views(hsemi, 2, shapes)):
        for dst, p in zip(vc, kf.cnn_planes):
            dst.copy_(torch.from_numpy(p).to(tdt))
        vsm[0].copy_(torch.from_numpy(kf.mu_s))
        vsm[1].copy_(torch.from_numpy(kf.var_s))
    dcnn = [torch.empty(6 * px, dtype=tdt, device=dev) for _ in range(2)]
    dsemi = [torch.empty(2 * px, dtype=torch.float32, device=dev) for _ in range(2)]
    dout = [torch.empty(px, dtype=torch.float32, device=dev) for _ in range(2)]
    dc = [_flat_views(d, 6, shapes) for d in dcnn]
    dmu = [[v[0] for v in _flat_views(d, 2, shapes)] for d in dsemi]
    dvar = [[v[1] for v in _flat_views(d, 2, shapes)] for d in dsemi]
    do = [[v[0] for v in _flat_views(d, 1, shapes)] for d in dout]
    sptr = stream.cuda_stream
    up, down = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
    ev_up, ev_in_free, ev_out, ev_out_free = ([torch.cuda.Event() for _ in range(2)]
                                              for _ in range(4))

    def enqueue(k):
        b = k & 1
        if k >= 2:  # step k-2 has read this staging set's inputs
            up.wait_event(ev_in_free[b])
        with torch.cuda.stream(up):
            dcnn[b].copy_(hcnn, non_blocking=True)
            dsemi[b].copy_(hsemi, non_blocking=True)
        ev_up[b].record(up)
        stream.wait_event(ev_up[b])
        with torch.cuda.stream(stream):
            flush.fill_(1.0)
            dfl.df_keyframe_reset_batch(handles, dc[b], stream=sptr)
            dfl.df_frame_update_batch(handles, dmu[b], dvar[b], stream=sptr)
        ev_in_free[b].record(stream)
        if k >= 2:  # step k-2's depth maps have left this staging set
            stream.wait_event(ev_out_free[b])
        with torch.cuda.stream(stream):
            solve()
            if ls_fit:
                for kk in ks:
                    kk.scale_fit_ls(stream=sptr)
            dfl.df_fetch_depth_batch(handles, do[b], stream=sptr)
        ev_out[b].record(stream)
        down.wait_event(ev_out[b])
        with torch.cuda.stream(down):
            hout[b].copy_(dout[b], non_blocking=True)
        ev_out_free[b].record(down)

    for k in range(warmup):
        enqueue(k)
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    for k in range(steps):
        enqueue(k)
    torch.cuda.synchronize()
    ms = 1e3 * (time.perf_counter() - t0)
    return ms, hout[(steps - 1) & 1]


def run_keyframes(args, ws, rank, dev, torch, dfl, replicas, synth):
    """Batched / large-keyframe workloads: one solve of all keyframes per step.

    For the 64-keyframe batch a second, plain leg solves the same keyframes
    from the same state with one df_optimise launch per keyframe; both legs'
    depth maps are compared after the timed regions."""
    import torch.distributed as dist

    n_gn, n_pcg = args.n_gn, args.n_pcg
    name, shapes, dt_name = keyframe_shapes(args, rank)
    code = {"f32": dfl.DF_F32, "bf16": dfl.DF_BF16, "f16": dfl.DF_F16}[dt_name]
    tdt = {"f32": torch.float32, "bf16": torch.bfloat16, "f16": torch.float16}[dt_name]
    seeds = keyframe_seeds(args, rank, shapes)
    kfs = [synth.make_keyframe(W, H, sd) for (W, H), sd in zip(shapes, seeds)]
    cnn_d = [[torch.from_numpy(p).to(tdt).to(dev) for p in kf.cnn_planes] for kf in kfs]
    semi_d = [(torch.from_numpy(kf.mu_s).to(dev), torch.from_numpy(kf.var_s).to(dev)) for kf in kfs]
    outs = [torch.empty((kf.height, kf.width), dtype=torch.float32, device=dev) for kf in kfs]
    solver = {"auto": dfl.DF_SOLVER_AUTO, "launches": dfl.DF_SOLVER_LAUNCHES,
              "fused": dfl.DF_SOLVER_FUSED}[args.solver]
    prm = dfl.df_default_params(n_gn=n_gn, n_pcg=n_pcg, solver=solver, **method_params(args))
    ls_fit = args.variant == "table2"
    stream = torch.cuda.Stream(dev)
    sptr = stream.cuda_stream
    ks = [dfl.Keyframe(kf.width, kf.height, *c, cnn_dtype=code, stream=sptr)
          for kf, c in zip(kfs, cnn_d)]
    handles = [k.handle for k in ks]
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))

    def forced_tuning():
        dfl.df_set_tuning(mode={"auto": 0, "streaming": 1, "resident": 2}[args.mode],
                          vec=args.vec, tile_rows=args.tile_rows, max_ctas=args.max_ctas,
                          assembly=args.assembly)

    graph = None
    graph_launches = 0
    tuning = None

    def solve():
        if graph is not None:
            graph.replay()
        else:
            dfl.df_optimise_batch(handles, prm, stream=sptr)

    mu_d = [m for m, _ in semi_d]
    var_d = [v for _, v in semi_d]

    def load_frame():
        # keyframe (re)initialisation from the network planes, then the
        # frame's semi-dense planes: a few batched launches for all keyframes
        dfl.df_keyframe_reset_batch(handles, cnn_d, stream=sptr)
        dfl.df_frame_update_batch(handles, mu_d, var_d, stream=sptr)

    io_graphs = None  # (reset + frame update, depth output) captured with the solve

    def output():
        # Table II: the scale fitted to the network depth after the
        # scale-ambiguous solve; then the depth maps
        if ls_fit:
            for k in ks:
                k.scale_fit_ls(stream=sptr)
        dfl.df_fetch_depth_batch(handles, outs, stream=sptr)

    def step(record):
        if io_graphs is not None:
            io_graphs[0].replay()
        else:
            load_frame()
        if record:
            ev[0].record(stream)
        solve()
        if record:
            ev[1].record(stream)
        if io_graphs is not None:
            io_graphs[1].replay()
        else:
            output()

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step(False)
    torch.cuda.synchronize()
    use_graph = args.workload == "batch64" and not args.no_graph and args.solver != "launches"
    if args.workload == "batch64" and not args.no_autotune and args.solver != "launches" \
            and args.mode == "auto" and not (args.vec or args.tile_rows or args.max_ctas
                                             or args.assembly):
        # launch shape (kernel, tile rows, vector width, GN iterations per
        # launch) picked by timing the candidates on this batch
        best, best_ms = dfl.df_autotune(handles, prm, stream=sptr)
        tuning = {"mode": best.mode, "vec": best.vec, "tile_rows": best.tile_rows,
                  "max_ctas": best.max_ctas, "gn_per_launch": best.gn_per_launch,
                  "assembly": best.assembly, "autotune_ms": best_ms}
    if use_graph:
        # the batched solve captured once in a CUDA graph, replayed per step
        dfl.df_batch_prepare(handles, stream=sptr)
        with torch.cuda.stream(stream):
            step(False)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        g_load = torch.cuda.CUDAGraph()
        g_fetch = torch.cuda.CUDAGraph()
        cap0 = dfl.df_kernel_launches()
        with torch.cuda.stream(stream):
            with torch.cuda.graph(g, stream=stream):
                dfl.df_optimise_batch(handles, prm, stream=sptr)
            # the per-frame bookkeeping too: device buffers, so nothing is
            # uploaded and every step replays the same launches
            with torch.cuda.graph(g_load, stream=stream):
                load_frame()
            with torch.cuda.graph(g_fetch, stream=stream):
                output()
        torch.cuda.synchronize()
        graph_launches = dfl.df_kernel_launches() - cap0  # kernels in the graphs
        graph = g
        io_graphs = (g_load, g_fetch)
        with torch.cuda.stream(stream):
            for _ in range(args.warmup):
                step(False)
        torch.cuda.synchronize()
    step_ms, solve_ms = [], []
    launches0 = dfl.df_kernel_launches()
    with ClockSampler(dev.index) as clk:
        for _ in range(args.steps):
            flush.fill_(1.0)
            if ws > 1:
                dist.barrier()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(stream):
                e0.record(stream)
                step(True)
                e1.record(stream)
            torch.cuda.synchronize()
            step_ms.append(e0.elapsed_time(e1))
            solve_ms.append(ev[0].elapsed_time(ev[1]))
        if ws > 1:
            dist.barrier()
    # the library counts its own launches; a replayed graph's kernels are
    # counted from the capture, once per timed replay
    launches = dfl.df_kernel_launches() - launches0 + graph_launches * args.steps
    clocks = clk.summary()
    total_ms = replicas.max_over_ranks(sum(step_ms), device=dev)
    px = sum(W * H for W, H in shapes)
    # the PCG iterations a step executes, from the solve reports of one more
    # (untimed) step from the same state: all n_gn x n_pcg of them unless a
    # depth step stops early (the diagonal system of --variant table3 is
    # solved exactly by its first iteration)
    with torch.cuda.stream(stream):
        load_frame()
        reps = dfl.df_optimise_batch(handles, prm, stream=sptr, report=True)
    torch.cuda.synchronize()
    iters = [int(r.iters_done) for r in reps]
    units = sum(W * H * it for (W, H), it in zip(shapes, iters))
    value = units * args.steps * ws / (total_ms / 1e3) / 1e6
    gn_bytes = ALG_BYTES_PER_GN_PX if code == dfl.DF_F32 else ALG_BYTES_PER_GN_PX - 12
    alg = units * ALG_BYTES_PER_PCG_PX + px * n_gn * gn_bytes
    peak, peak_kind = peaks()
    solve_s = statistics.mean(solve_ms) / 1e3
    achieved = alg / solve_s / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": ncu_traffic(traffic_key(args, name)),
                "peak_kind": peak_kind, "region": "df_optimise_batch (all keyframes, one frame)",
                "alg_bytes_per_launch": alg,
                "pcg_iterations": {"nominal_per_keyframe": n_gn * n_pcg,
                                   "executed_mean": float(np.mean(iters))}}
    e2e = None
    if not args.no_e2e:
        cnn_h = [[torch.from_numpy(p).to(tdt).pin_memory() for p in kf.cnn_planes] for kf in kfs]
        semi_h = [(torch.from_numpy(kf.mu_s).pin_memory(), torch.from_numpy(kf.var_s).pin_memory())
                  for kf in kfs]
        outs_h = [torch.empty((kf.height, kf.width), dtype=torch.float32).pin_memory() for kf in kfs]

        mu_h = [m for m, _ in semi_h]
        var_h = [v for _, v in semi_h]

        def step_host():
            dfl.df_keyframe_reset_batch(handles, cnn_h, stream=sptr)
            dfl.df_frame_update_batch(handles, mu_h, var_h, stream=sptr)
            solve()
            if ls_fit:
                for k in ks:
                    k.scale_fit_ls(stream=sptr)
            dfl.df_fetch_depth_batch(handles, outs_h, stream=sptr)

        with torch.cuda.stream(stream):
            step_host()
        torch.cuda.synchronize()
        e2e_graph = None
        if graph is not None:
            # the whole host-buffer step replayed from a CUDA graph: the
            # batched calls read the pinned inputs and write the pinned depth
            # maps directly, so every replay still moves this step's bytes
            # between host and device
            try:
                e2e_graph = torch.cuda.CUDAGraph()
                with torch.cuda.stream(stream):
                    with torch.cuda.graph(e2e_graph, stream=stream):
                        dfl.df_keyframe_reset_batch(handles, cnn_h, stream=sptr)
                        dfl.df_frame_update_batch(handles, mu_h, var_h, stream=sptr)
                        dfl.df_optimise_batch(handles, prm, stream=sptr)
                        if ls_fit:
                            for k in ks:
                                k.scale_fit_ls(stream=sptr)
                        dfl.df_fetch_depth_batch(handles, outs_h, stream=sptr)
                torch.cuda.synchronize()
                with torch.cuda.stream(stream):
                    e2e_graph.replay()
                torch.cuda.synchronize()
            except (RuntimeError, dfl.DFError) as exc:  # capture refused: eager steps
                print(f"bench: host-buffer step not captured ({exc}); timing it eagerly",
                      file=sys.stderr)
                e2e_graph = None
                torch.cuda.synchronize()
        tms = []
        for _ in range(args.steps):
            flush.fill_(1.0)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            with torch.cuda.stream(stream):
                if e2e_graph is not None:
                    e2e_graph.replay()
                else:
                    step_host()
            torch.cuda.synchronize()
            tms.append(1e3 * (time.perf_counter() - t0))
        tot = replicas.max_over_ranks(sum(tms), device=dev)
        serial = {"value": units * args.steps * ws / (tot / 1e3) / 1e6,
                  "ms_per_step": tot / args.steps, "cuda_graph": e2e_graph is not None,
                  "what": "one step at a time (host wall time per step): the batched calls "
                          "read the pinned inputs and write the pinned depth maps directly"}
        e2e_graph = None
        pipe_ms, last_h = keyframes_e2e_pipelined(
            args, torch, dfl, dev, kfs, shapes, tdt, handles, ks, stream, solve, ls_fit, flush,
            args.steps, args.warmup, lambda: dist.barrier() if ws > 1 else None)
        ref = torch.cat([o.reshape(-1) for o in outs]).cpu()
        if not torch.equal(last_h, ref):  # same kernels, same inputs: the same bits
            raise RuntimeError("bench: pipelined end-to-end depth maps differ from the "
                               "device-buffer steps'")
        ptot = replicas.max_over_ranks(pipe_ms, device=dev)
        esz = 4 if code == dfl.DF_F32 else 2
        e2e = {"value": units * args.steps * ws / (ptot / 1e3) / 1e6, "unit": METRIC,
               "h2d_bytes_per_step": int(px * (6 * esz + 8)), "d2h_bytes_per_step": int(px * 4),
               "ms_per_step": ptot / args.steps,
               "what": "host wall time of the steps back to back, from the first upload to "
                       "the last download: every step copies its network planes and "
                       "semi-dense frames from pinned host memory and its depth maps back "
                       "(copy streams, two device staging sets; step k+1's upload and step "
                       "k-1's download overlap step k's solve)",
               "serial": serial}

    # the batched result of one more (untimed) step, kept for the comparison
    with torch.cuda.stream(stream):
        step(False)
    torch.cuda.synchronize()
    batched_depth = [o.clone() for o in outs]

    plain = None
    if args.workload == "batch64":
        # the plain path: one df_optimise launch per keyframe, in list order,
        # with the library's default launch shape (not the batch's tuning)
        forced_tuning()
        evk = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in ks]

        def plain_solve(record):
            for j, k in enumerate(ks):
                if record:
                    evk[j][0].record(stream)
                k.optimise(prm, stream=sptr)
                if ls_fit:
                    k.scale_fit_ls(stream=sptr)
                if record:
                    evk[j][1].record(stream)

        with torch.cuda.stream(stream):
            for _ in range(args.warmup):
                load_frame()
                plain_solve(False)
        torch.cuda.synchronize()
        plain_ms, per_kf_ms = [], []
        p_launches0 = dfl.df_kernel_launches()
        for _ in range(args.steps):
            flush.fill_(1.0)
            if ws > 1:
                dist.barrier()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(stream):
                load_frame()
                e0.record(stream)
                plain_solve(True)
                e1.record(stream)
            torch.cuda.synchronize()
            plain_ms.append(e0.elapsed_time(e1))
            per_kf_ms.extend(a.elapsed_time(b) for a, b in evk)
        p_launches = dfl.df_kernel_launches() - p_launches0
        # same accuracy: the plain leg's depth against the batched leg's
        dfl.df_fetch_depth_batch(handles, outs, stream=sptr)
        torch.cuda.synchronize()
        diff = max(float(((o.double() / b.double()) - 1.0).abs().max())
                   for o, b in zip(outs, batched_depth))
        plain_tot = replicas.max_over_ranks(sum(plain_ms), device=dev)
        plain = {"p50": float(np.percentile(plain_ms, 50)), "p99": float(np.percentile(plain_ms, 99)),
                 "value": units * args.steps * ws / (plain_tot / 1e3) / 1e6, "unit": METRIC,
                 "per_keyframe_p50": float(np.percentile(per_kf_ms, 50)),
                 "per_keyframe_p99": float(np.percentile(per_kf_ms, 99)),
                 "gpu_launches_per_step": p_launches / args.steps,
                 "max_rel_depth_diff_vs_batched": diff,
                 "same_accuracy": bool(diff <= 1e-4),
                 "what": f"the same {len(ks)} keyframes from the same state, one df_optimise "
                         "launch per keyframe (default launch shape), eager; p50/p99 = device "
                         "time until all keyframes are solved; per_keyframe = one launch"}
        if diff > 1e-4:
            raise RuntimeError(f"plain and batched depth maps differ by {diff:.3g} (> 1e-4)")

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        cpu = keyframes_cpu_baseline(args, rank)
    used_graph = graph is not None
    if used_graph:
        graph = None
        io_graphs = None
        dfl.df_batch_release(handles)
    forced_tuning()
    for k in ks:
        k.close()
    if rank == 0:
        lat = {"p50": float(np.percentile(solve_ms, 50)), "p99": float(np.percentile(solve_ms, 99)),
               "what": "one batched solve of every keyframe, device time"}
        if plain is not None:
            lat = {"batched": lat, "plain": plain}
        line = {
            "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded piecewise-planar scenes; no dataset)",
            "config": keyframes_config(args, ws, rank),
            "launch": {"solver": args.solver, "cuda_graph": used_graph, "autotuned": tuning,
                       "kernel_mode": args.mode, "max_ctas": args.max_ctas,
                       "vec": args.vec, "tile_rows": args.tile_rows, "assembly": args.assembly},
            "clocks": clocks, "e2e": e2e, "gpu_launches": launches, "roofline": roofline,
            "cpu_baseline": cpu,
            "update_latency_ms": lat,
            "hbm_frac": roofline["frac"],
        }
        print(json.dumps(line), flush=True)


def main():
    args = parse()
    ws, rank, local = dist_env()
    if args.impl == "reference":
        run_reference(args, ws, rank)
        return

    import torch
    import torch.distributed as dist

    from paper_2207_12244_gb300 import _build
    from paper_2207_12244_gb300 import deepfusion as dfl
    from paper_2207_12244_gb300 import replicas
    from paper_2207_12244_gb300 import synth

    if ws > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    if rank == 0:
        _build.build()
    if ws > 1:
        dist.barrier()
    dfl.load()
    dfl.df_set_tuning(mode={"auto": 0, "streaming": 1, "resident": 2}[args.mode],
                      vec=args.vec, tile_rows=args.tile_rows, max_ctas=args.max_ctas,
                      assembly=args.assembly)
    if args.workload == "serving":
        run_serving(args, ws, rank, dev, torch, dfl, replicas, synth)
        if ws > 1:
            dist.barrier()
            dist.destroy_process_group()
        return
    if args.workload == "mvs":
        run_mvs(args, ws, rank, dev, torch, dfl, replicas, synth)
        if ws > 1:
            dist.barrier()
            dist.destroy_process_group()
        return
    if args.workload != "sequence":
        run_keyframes(args, ws, rank, dev, torch, dfl, replicas, synth)
        if ws > 1:
            dist.barrier()
            dist.destroy_process_group()
        return

    W, H, F = args.width, args.height, args.frames
    kf, mus, vs = synth.make_sequence(W, H, replicas.rank_seed(args.seed, rank), F)
    cnn_d = [torch.from_numpy(p).to(dev) for p in kf.cnn_planes]
    mus_d = torch.from_numpy(mus).to(dev)
    vs_d = torch.from_numpy(vs).to(dev)
    out_d = torch.empty((F, H, W), dtype=torch.float32, device=dev)
    solver = {"auto": dfl.DF_SOLVER_AUTO, "launches": dfl.DF_SOLVER_LAUNCHES,
              "fused": dfl.DF_SOLVER_FUSED}[args.solver]
    prm = dfl.df_default_params(n_gn=args.n_gn, n_pcg=args.n_pcg, solver=solver,
                                **method_params(args))
    ls_fit = args.variant == "table2"
    dfl.df_set_tuning(mode={"auto": 0, "streaming": 1, "resident": 2}[args.mode],
                      vec=args.vec, tile_rows=args.tile_rows, max_ctas=args.max_ctas,
                      assembly=args.assembly)
    stream = torch.cuda.Stream(dev)
    sptr = stream.cuda_stream
    k = dfl.Keyframe(W, H, *cnn_d, stream=sptr)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MB > L2

    ev_opt = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(F)]

    # one frame's work (semi-dense update, solve, depth output) captured once
    # in a CUDA graph on fixed buffers and replayed per frame
    graph = None
    graph_launches = 0
    mu_in = torch.empty_like(mus_d[0])
    var_in = torch.empty_like(vs_d[0])
    out_fix = torch.empty((H, W), dtype=torch.float32, device=dev)

    def step(record_solve: bool):
        k.reset(*cnn_d, stream=sptr)
        for f in range(F):
            if graph is not None:
                mu_in.copy_(mus_d[f], non_blocking=True)
                var_in.copy_(vs_d[f], non_blocking=True)
                if record_solve:
                    ev_opt[f][0].record(stream)
                graph.replay()
                if record_solve:
                    ev_opt[f][1].record(stream)
                out_d[f].copy_(out_fix, non_blocking=True)
            else:
                k.frame_update(mus_d[f], vs_d[f], stream=sptr)
                if record_solve:
                    ev_opt[f][0].record(stream)
                k.optimise(prm, stream=sptr)
                if record_solve:
                    ev_opt[f][1].record(stream)
                if ls_fit:  # Table II: the scale fitted to the network depth
                    k.scale_fit_ls(stream=sptr)
                k.fetch_depth(out_d[f], stream=sptr)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step(False)
    torch.cuda.synchronize()
    if args.graph:
        g = torch.cuda.CUDAGraph()
        cap0 = dfl.df_kernel_launches()
        with torch.cuda.stream(stream):
            with torch.cuda.graph(g, stream=stream):
                k.frame_update(mu_in, var_in, stream=sptr)
                k.optimise(prm, stream=sptr)
                if ls_fit:
                    k.scale_fit_ls(stream=sptr)
                k.fetch_depth(out_fix, stream=sptr)
        torch.cuda.synchronize()
        graph_launches = dfl.df_kernel_launches() - cap0
        graph = g
        with torch.cuda.stream(stream):
            for _ in range(args.warmup):
                step(False)
        torch.cuda.synchronize()

    step_ms, solve_ms = [], []
    launches0 = dfl.df_kernel_launches()
    with ClockSampler(dev.index) as clk:
        for _ in range(args.steps):
            flush.fill_(1.0)  # evict the previous step's working set from L2
            if ws > 1:
                dist.barrier()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(stream):
                e0.record(stream)
                step(True)
                e1.record(stream)
            torch.cuda.synchronize()
            step_ms.append(e0.elapsed_time(e1))
            solve_ms.extend(a.elapsed_time(b) for a, b in ev_opt)
        if ws > 1:
            dist.barrier()
    # a replayed graph's kernels are counted from its capture, once per frame
    launches = dfl.df_kernel_launches() - launches0 + graph_launches * F * args.steps
    clocks = clk.summary()
    total_ms = replicas.max_over_ranks(sum(step_ms), device=dev)
    # the PCG iterations a step executes (solve reports of one more, untimed
    # step): n_gn x n_pcg per frame unless a depth step stops early
    iters = []
    with torch.cuda.stream(stream):
        k.reset(*cnn_d, stream=sptr)
        for f in range(F):
            k.frame_update(mus_d[f], vs_d[f], stream=sptr)
            iters.append(int(k.optimise(prm, stream=sptr, report=True).iters_done))
            if ls_fit:
                k.scale_fit_ls(stream=sptr)
    torch.cuda.synchronize()
    units_per_step = W * H * sum(iters)
    value = units_per_step * args.steps * ws / (total_ms / 1e3) / 1e6

    # dominant region: the solve of one frame (all its kernels)
    solve_avg_s = statistics.mean(solve_ms) / 1e3
    alg_bytes = W * H * (float(np.mean(iters)) * ALG_BYTES_PER_PCG_PX +
                         args.n_gn * ALG_BYTES_PER_GN_PX)
    peak, peak_kind = peaks()
    achieved = alg_bytes / solve_avg_s / 1e9
    kernel_key = traffic_key(args, sequence_name(args))
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": ncu_traffic(kernel_key),
                "peak_kind": peak_kind, "region": "df_optimise (one frame's solve)",
                "alg_bytes_per_launch": alg_bytes,
                "pcg_iterations": {"nominal_per_frame": args.n_gn * args.n_pcg,
                                   "executed_mean": float(np.mean(iters))}}
    lat = np.percentile(np.array(solve_ms), [50, 99])

    # end to end through the public API with host (pinned) buffers
    e2e = None
    if not args.no_e2e:
        cnn_h = [torch.from_numpy(p).pin_memory() for p in kf.cnn_planes]
        mus_h = torch.from_numpy(mus).pin_memory()
        vs_h = torch.from_numpy(vs).pin_memory()
        out_h = torch.empty((F, H, W), dtype=torch.float32).pin_memory()

        def step_host():
            k.reset(*cnn_h, stream=sptr)
            for f in range(F):
                k.frame_update(mus_h[f], vs_h[f], stream=sptr)
                k.optimise(prm, stream=sptr)
                if ls_fit:
                    k.scale_fit_ls(stream=sptr)
                k.fetch_depth(out_h[f], stream=sptr)

        step_host()
        torch.cuda.synchronize()
        e2e_ms = []
        for _ in range(args.steps):
            flush.fill_(1.0)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            step_host()
            torch.cuda.synchronize()
            e2e_ms.append(1e3 * (time.perf_counter() - t0))
        tot = replicas.max_over_ranks(sum(e2e_ms), device=dev)
        e2e = {"value": units_per_step * args.steps * ws / (tot / 1e3) / 1e6, "unit": METRIC,
               "h2d_bytes_per_step": int(sum(p.nbytes for p in kf.cnn_planes) + mus.nbytes + vs.nbytes),
               "d2h_bytes_per_step": int(F * H * W * 4), "ms_per_step": tot / args.steps}

    # accuracy of the fused depth after the last frame (Section III-B's
    # measure, outside the timed region), next to the network prior alone
    truth_d = torch.from_numpy(np.exp(kf.log_depth_true).astype(np.float32)).to(dev)
    with torch.cuda.stream(stream):
        step(False)
    torch.cuda.synchronize()
    graph = None  # the accuracy check and the host-buffer leg run eagerly
    n_in, n_valid = k.depth_accuracy(truth_d, 0.1, stream=sptr)
    k.reset(*cnn_d, stream=sptr)
    n_in0, _ = k.depth_accuracy(truth_d, 0.1, stream=sptr)
    accuracy = {"within_10pct": n_in / n_valid, "cnn_prior_within_10pct": n_in0 / n_valid,
                "what": "fraction of pixels within 10% of the synthetic ground-truth depth "
                        "after the last frame (Section III-B measure)"}

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        cpu = cpu_baseline(args, kf, mus, vs)

    k.close()
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded piecewise-planar scenes; no dataset)",
            "config": sequence_config(args, ws),
            "launch": {"solver": args.solver, "cuda_graph": bool(args.graph),
                       "kernel_mode": args.mode, "max_ctas": args.max_ctas,
                       "vec": args.vec, "tile_rows": args.tile_rows, "assembly": args.assembly},
            "clocks": clocks, "e2e": e2e, "gpu_launches": launches, "roofline": roofline,
            "cpu_baseline": cpu, "accuracy": accuracy,
            "update_latency_ms": {"p50": float(lat[0]), "p99": float(lat[1]),
                                  "what": "one frame's df_optimise, device time"},
            "hbm_frac": roofline["frac"],
        }
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
