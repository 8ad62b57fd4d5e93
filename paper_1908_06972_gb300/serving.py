"""Replay of a request trace through the request server (``pft_server_*``).

Admission, batching and all device work happen in the library's server; this module only
hands requests over at their arrival times, keeps the server stepping, and turns the
completion records into latencies.  Arrival times and completion times share the
server clock (``pft_server_clock``; completions are timed by CUDA events).
"""
import time
from dataclasses import dataclass, field

import numpy as np


def poisson_arrivals(rate, count, seed):
    """Arrival times (seconds from the start) of a Poisson process of the given rate."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate, count))


@dataclass
class Request:
    t: float          # arrival, seconds after the start of the replay
    ring: int
    level: int
    scale: float
    coeffs: np.ndarray  # uint64 [chunks][2][level][N], coefficient form
    out: np.ndarray     # uint64 [2][level - 2][N], filled on completion
    tag: int


@dataclass
class Result:
    latencies: dict = field(default_factory=dict)  # tag -> seconds from arrival to completion
    done: dict = field(default_factory=dict)       # tag -> completion record
    makespan: float = 0.0                          # first arrival to last completion
    max_active: int = 0
    peak_bytes: int = 0
    iterations: int = 0

    def throughput(self):
        return len(self.latencies) / self.makespan if self.makespan > 0 else 0.0

    def percentile(self, p):
        return float(np.percentile(np.fromiter(self.latencies.values(), float), p))


class _Native:
    """The library's server entry points (the default back end of replay)."""

    def __init__(self):
        from . import (pft_server_clock, pft_server_get_stats, pft_server_poll, pft_server_step,
                       pft_server_submit)
        self.submit, self.step, self.poll = pft_server_submit, pft_server_step, pft_server_poll
        self.clock, self.stats = pft_server_clock, pft_server_get_stats


def replay(srv, requests, api=None, sleep=time.sleep, idle_wait=0.002, timeout=900.0):
    """Submit each request once the server clock passes its arrival time, stepping the
    server in between, until every request has completed.  ``requests`` must be sorted by
    arrival.  ``api`` replaces the native entry points (tests use a simulated server).
    Raises TimeoutError if requests are still open ``timeout`` seconds after the start."""
    api = api or _Native()
    reqs = list(requests)
    assert all(reqs[i].t <= reqs[i + 1].t for i in range(len(reqs) - 1)), "requests must be sorted by arrival"
    by_tag = {r.tag: r for r in reqs}
    assert len(by_tag) == len(reqs), "tags must be unique"
    res = Result()
    t0 = api.clock(srv)
    nxt, pending = 0, 0
    while nxt < len(reqs) or pending > 0:
        now = api.clock(srv) - t0
        if now > timeout:
            raise TimeoutError("%d requests still open after %.0f s" % (pending + len(reqs) - nxt, now))
        while nxt < len(reqs) and reqs[nxt].t <= now:
            r = reqs[nxt]
            api.submit(srv, r.ring, r.coeffs, r.level, r.scale, r.out, r.tag)
            nxt += 1
            pending += 1
        if pending == 0:
            sleep(max(0.0, min(reqs[nxt].t - now, 0.05)))
            continue
        api.step(srv)
        for d in api.poll(srv):
            r = by_tag[d["tag"]]
            res.done[r.tag] = d
            res.latencies[r.tag] = d["t_done"] - (t0 + r.t)
            pending -= 1
        st = api.stats(srv)
        if pending > 0 and st["active"] == 0 and st["waiting"] == 0:
            sleep(idle_wait)  # only score copies in flight: nothing to queue until they land
    st = api.stats(srv)
    res.max_active, res.peak_bytes, res.iterations = st["max_active"], st["peak_bytes"], st["iterations"]
    if reqs:
        res.makespan = max(d["t_done"] for d in res.done.values()) - (t0 + reqs[0].t)
    return res
