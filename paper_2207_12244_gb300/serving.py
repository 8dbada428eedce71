"""Driver of the serving layer: Poisson frame arrivals from many camera
streams, submitted to a df_server and collected as they finish.

The scheduling itself (admission, per-stream queues, continuous batching,
overlapping launches) is native code in the library (df_server_*); this
module only generates arrival times, submits the frames when their time
comes, polls completions and summarises latency.
"""
from __future__ import annotations

import time
from dataclasses import dataclass
from typing import List, Sequence

import numpy as np

from . import deepfusion as dfl


@dataclass
class Stats:
    n: int
    wall_s: float
    p50_ms: float
    p99_ms: float
    mean_ms: float
    max_ms: float
    mean_batch: float
    throughput_rps: float


def poisson_schedule(n_requests: int, rate_hz: float, n_streams: int, seed: int):
    """(arrival time in s, stream index) of n_requests frames: a Poisson
    process of the total rate, each arrival from a uniformly drawn stream
    (equivalently, independent per-stream Poisson processes)."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate_hz, n_requests))
    s = rng.integers(0, n_streams, n_requests)
    return t, s


def run(srv, stream_ids: Sequence[int], frames: Sequence[Sequence[tuple]], arrivals,
        streams_of_arrival, time_limit_s: float = 120.0) -> Stats:
    """Submit frames at their arrival times (busy-waiting on the host clock),
    drive the scheduler, return latency statistics (arrival -> finished).

    frames[k] is the list of (mu_semi, var_semi) buffers of stream k, used in
    turn; they must stay alive until the run returns."""
    n = len(arrivals)
    nexts = [0] * len(stream_ids)
    lat, batch = [], []
    t0 = time.perf_counter()
    i = 0
    deadline = t0 + time_limit_s
    while (i < n or dfl.df_server_pending(srv) > 0) and time.perf_counter() < deadline:
        now = time.perf_counter() - t0
        while i < n and arrivals[i] <= now:
            k = int(streams_of_arrival[i])
            mu, var = frames[k][nexts[k] % len(frames[k])]
            nexts[k] += 1
            dfl.df_server_submit(srv, stream_ids[k], mu, var, i)
            i += 1
        for c in dfl.df_server_progress(srv):
            if c.status != dfl.DF_OK:
                raise RuntimeError(f"frame {c.tag} of stream {c.stream_id}: status {c.status}")
            lat.append((c.t_done_ns - c.t_submit_ns) / 1e6)
            batch.append(c.batch_size)
    wall = time.perf_counter() - t0
    if i < n or dfl.df_server_pending(srv) > 0:
        raise RuntimeError("serving run did not finish within its time limit")
    a = np.array(lat)
    return Stats(len(a), wall, float(np.percentile(a, 50)), float(np.percentile(a, 99)),
                 float(a.mean()), float(a.max()), float(np.mean(batch)), len(a) / wall)
