"""Continuous-batching server logic on the host (no GPU): a fake backend completes each
launch after a time proportional to its pixels, one launch after another."""
import numpy as np
import pytest

from paper_1811_02168_gb300.serve import FakeBackend, Request, Server


def _requests(n, rate, seed, lo=64, hi=512):
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for i in range(n):
        t += rng.exponential(1.0 / rate)
        H, W = (int(v) for v in rng.integers(lo, hi, 2))
        out.append(Request(i, t, H, W, theta=2.0, sigma=30.0, K=4))
    return out


def test_every_request_completes_and_latency_is_positive():
    reqs = _requests(60, rate=2000.0, seed=1)
    be = FakeBackend(sec_per_pixel=2e-9)
    st = Server(be, hbm_budget_bytes=1 << 30).run(reqs)
    assert st.requests == 60
    assert all(r.done >= r.arrival for r in reqs)
    assert sorted(be.admitted) == list(range(60))
    assert st.pct(50) <= st.pct(99)


def test_hbm_budget_is_never_exceeded_and_requests_wait():
    reqs = _requests(40, rate=5000.0, seed=2, lo=200, hi=400)
    budget = 3 * 8 * 400 * 400          # room for about three of the largest requests
    be = FakeBackend(sec_per_pixel=5e-9)
    st = Server(be, hbm_budget_bytes=budget).run(reqs)
    assert st.requests == 40
    assert be.max_live_bytes <= budget
    assert st.hbm_high_water <= budget
    assert st.waited_for_budget > 0


def test_continuous_batching_groups_arrivals_while_the_gpu_is_busy():
    reqs = _requests(80, rate=20000.0, seed=3)     # arrivals much faster than service
    be = FakeBackend(sec_per_pixel=1e-8)
    st = Server(be, hbm_budget_bytes=1 << 30, max_batch=16, max_inflight=2).run(reqs)
    sizes = [len(l) for l in be.launched]
    assert max(sizes) > 1 and max(sizes) <= 16
    assert st.max_inflight_seen <= 2
    assert st.launches < 80
    # arrival order is kept across launches
    flat = [rid for l in be.launched for rid in l]
    assert flat == sorted(flat)


def test_one_at_a_time_mode_launches_single_requests():
    reqs = _requests(20, rate=5000.0, seed=4)
    be = FakeBackend(sec_per_pixel=1e-9)
    Server(be, hbm_budget_bytes=1 << 30, batching=False).run(reqs)
    assert all(len(l) == 1 for l in be.launched)


def test_request_larger_than_the_budget_is_refused():
    r = Request(0, 0.0, 1000, 1000, 2.0, 30.0, 4)
    with pytest.raises(ValueError):
        Server(FakeBackend(), hbm_budget_bytes=1000).run([r])


class _FailingBackend(FakeBackend):
    """FakeBackend whose admit of chosen requests, chosen launches (by index) and completion
    queries of chosen launches raise, as a failing device call would."""

    def __init__(self, bad_admit=(), bad_launch=(), bad_done=(), **kw):
        super().__init__(**kw)
        self.bad_admit, self.bad_launch, self.bad_done = set(bad_admit), set(bad_launch), set(bad_done)
        self.n_launch = 0
        self.handles = {}

    def admit(self, r):
        if r.rid in self.bad_admit:
            raise RuntimeError("upload failed")
        super().admit(r)

    def launch(self, rs):
        n = self.n_launch
        self.n_launch += 1
        if n in self.bad_launch:
            raise RuntimeError("launch failed")
        h = super().launch(rs)
        self.handles[n] = h
        return (n, h)

    def done(self, h):
        n, t = h
        if n in self.bad_done:
            raise RuntimeError("completion query failed")
        return super().done(t)


def test_backend_failures_fail_only_their_requests():
    """An upload, a launch and a completion query that fail (errors raised by a fake of the
    failing call, on the host) fail exactly the requests they concern; every other request
    completes, the failed ones release their budget and device state, and the loop ends."""
    reqs = _requests(60, rate=20000.0, seed=9)
    be = _FailingBackend(bad_admit={3, 17}, bad_launch={1}, bad_done={2}, sec_per_pixel=2e-9)
    st = Server(be, hbm_budget_bytes=1 << 30, max_batch=8).run(reqs)
    failed = [r for r in reqs if r.error]
    assert st.failed == len(failed) and st.requests + st.failed == len(reqs)
    assert {3, 17} <= {r.rid for r in failed}
    assert {r.rid for r in failed if "upload" in r.error} == {3, 17}
    assert any("launch failed" in r.error for r in failed)
    assert any("completion query failed" in r.error for r in failed)
    assert all(r.done == r.done for r in reqs if not r.error)        # served: a completion time
    assert all(r.done != r.done for r in failed)                       # failed: none (NaN)
    assert be.live_bytes == 0                                          # all device state released
    assert st.summary()["failed"] == len(failed)
