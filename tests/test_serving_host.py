"""Host logic of the trace replay (no GPU): a simulated server with a virtual clock stands
in for the library's request server."""
import numpy as np
import pytest

from paper_1908_06972_gb300 import serving


class FakeServer:
    """Arrival-order admission of at most `cap` requests; each needs `stages` steps of `dt`
    seconds; a request completes at the end of its last step."""

    def __init__(self, cap, stages, dt):
        self.cap, self.stages, self.dt = cap, stages, dt
        self.t = 100.0  # the server clock does not start at zero
        self.waiting, self.active, self.done = [], [], []
        self.submitted = {}
        self.max_active = 0
        self.iterations = 0

    # the entry points replay() calls
    def clock(self, srv):
        return self.t

    def submit(self, srv, ring, coeffs, level, scale, out, tag):
        self.submitted[tag] = self.t
        self.waiting.append([tag, self.stages])

    def step(self, srv):
        while self.waiting and len(self.active) < self.cap:
            self.active.append(self.waiting.pop(0))
        self.max_active = max(self.max_active, len(self.active))
        if self.active:
            self.t += self.dt
            self.iterations += 1
            for a in self.active:
                a[1] -= 1
            for a in [a for a in self.active if a[1] == 0]:
                self.done.append({"tag": a[0], "t_done": self.t, "ring": 0, "level": 1, "scale": 1.0,
                                  "t_submit": self.submitted[a[0]]})
                self.active.remove(a)
        return len(self.waiting) + len(self.active)

    def poll(self, srv):
        d, self.done = self.done, []
        return d

    def stats(self, srv):
        return {"active": len(self.active), "waiting": len(self.waiting), "max_active": self.max_active,
                "peak_bytes": 0, "iterations": self.iterations}

    def sleep(self, s):
        self.t += max(s, 1e-4)


def make_requests(times):
    z = np.zeros(1, np.uint64)
    return [serving.Request(t=float(t), ring=0, level=3, scale=1.0, coeffs=z, out=z, tag=i)
            for i, t in enumerate(times)]


def test_poisson_arrivals_rate_and_seed():
    a = serving.poisson_arrivals(200.0, 20000, seed=5)
    assert np.all(np.diff(a) > 0)
    assert abs(a[-1] / 20000 - 1 / 200.0) < 0.03 / 200.0 * 5
    assert np.array_equal(a, serving.poisson_arrivals(200.0, 20000, seed=5))


def test_replay_waits_for_arrivals_and_measures_latency():
    fake = FakeServer(cap=2, stages=3, dt=0.01)
    times = [0.0, 0.001, 0.002, 0.5, 0.5005]
    res = serving.replay(None, make_requests(times), api=fake, sleep=fake.sleep)
    assert sorted(res.latencies) == list(range(5))
    for tag, t in enumerate(times):
        assert fake.submitted[tag] >= 100.0 + t - 1e-12  # never submitted before its arrival
        assert res.latencies[tag] == pytest.approx(res.done[tag]["t_done"] - (100.0 + t))
    # requests 0 and 1 share the first three iterations; 2 waits for a free slot
    assert res.latencies[0] == pytest.approx(0.03)
    assert res.latencies[2] > res.latencies[1]
    assert res.max_active == 2
    assert res.makespan == pytest.approx(max(d["t_done"] for d in res.done.values()) - 100.0)
    assert res.throughput() == pytest.approx(5 / res.makespan)
    lat = np.array([res.latencies[i] for i in range(5)])
    assert res.percentile(50) == pytest.approx(np.median(lat))


def test_replay_rejects_unsorted_trace():
    fake = FakeServer(cap=1, stages=1, dt=0.01)
    with pytest.raises(AssertionError):
        serving.replay(None, make_requests([0.2, 0.1]), api=fake, sleep=fake.sleep)


def test_replay_times_out_on_a_server_that_never_completes():
    fake = FakeServer(cap=1, stages=10 ** 9, dt=1.0)
    with pytest.raises(TimeoutError):
        serving.replay(None, make_requests([0.0]), api=fake, sleep=fake.sleep, timeout=50.0)
