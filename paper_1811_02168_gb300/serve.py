"""Continuous-batching server for bilateral-filtering requests: the Python model of the
library's native serving loop (``fbf_server_*``, a worker thread in the library, which the
benchmark uses).  This one keeps the same policy with a pluggable device backend, so the
admission, budget and batching logic can be tested on the CPU (``FakeBackend``), and runs
on the GPU through ``TorchBackend``.

Requests (an image plus theta, sigma and K) arrive over time.  The loop:

  * admits waiting requests in arrival order while their device buffers (input + output,
    8 bytes per pixel) fit the HBM budget and the next launch has room;
  * starts the device copy of each admitted image at once (upload stream);
  * launches everything admitted so far as ONE batched launch (compute stream, one
    persistent kernel per radius class) whenever fewer than ``max_inflight`` launches are
    on the GPU -- requests that arrive while others run join the next launch instead of
    waiting for a fixed batch to fill (continuous batching);
  * copies results back (download stream, after the launch) and, when a launch's results are on
    the host, records each request's latency (completion - arrival) and frees its budget;
  * a backend error (an upload, a launch, a completion query) fails only the requests it
    concerns: they are counted as failed, their budget and device state are released, and
    the loop goes on with the others.

Plans (the fitted K, T, c per (theta, sigma, K)) are cached, so the FP64 fit runs once per
parameter set.  The device work is the library's batched path (``binding.Batch``); the
server itself only orders host calls.  A backend object isolates the device so the
admission/batching logic can be tested without a GPU (``FakeBackend``).
"""
from __future__ import annotations

import collections
import math
import time
from dataclasses import dataclass, field


@dataclass
class Request:
    rid: int
    arrival: float            # seconds from the start of the run
    H: int
    W: int
    theta: float
    sigma: float
    K: int
    host_in: object = None    # host image (backend specific)
    host_out: object = None
    admitted: float = math.nan
    launched: float = math.nan
    done: float = math.nan
    dev: object = None        # backend state
    error: str = ""           # why the request failed ("" if it did not)

    @property
    def nbytes(self) -> int:
        return 8 * self.H * self.W

    @property
    def latency(self) -> float:
        return self.done - self.arrival


@dataclass
class ServeStats:
    requests: int = 0
    pixels: int = 0
    wall_s: float = 0.0
    latencies: list = field(default_factory=list)
    # per served request: (latency, arrival -> admitted, admitted -> launched,
    # launched -> result on the host, pixels, requests in its launch)
    trace: list = field(default_factory=list)
    launches: int = 0
    max_inflight_seen: int = 0
    hbm_high_water: int = 0
    waited_for_budget: int = 0
    failed: int = 0

    def pct(self, q: float) -> float:
        if not self.latencies:
            return math.nan
        xs = sorted(self.latencies)
        i = min(len(xs) - 1, max(0, int(math.ceil(q / 100.0 * len(xs))) - 1))
        return xs[i]

    def summary(self) -> dict:
        return {"requests": self.requests, "pixels": self.pixels, "wall_s": self.wall_s,
                "mpix_per_s": self.pixels / self.wall_s / 1e6 if self.wall_s > 0 else math.nan,
                "p50_ms": 1e3 * self.pct(50), "p99_ms": 1e3 * self.pct(99),
                "launches": self.launches, "max_inflight": self.max_inflight_seen,
                "hbm_high_water_bytes": self.hbm_high_water,
                "waited_for_budget": self.waited_for_budget, "failed": self.failed,
                "slowest_1pct": self.tail_breakdown(99)}

    def tail_breakdown(self, q: float) -> dict:
        """Mean parts of the latency of the requests at or above the q-th percentile."""
        if not self.trace:
            return {}
        cut = self.pct(q)
        tail = [t for t in self.trace if t[0] >= cut]
        n = len(tail)
        return {"requests": n,
                "queued_ms": 1e3 * sum(t[1] for t in tail) / n,
                "wait_for_launch_ms": 1e3 * sum(t[2] for t in tail) / n,
                "launch_to_result_ms": 1e3 * sum(t[3] for t in tail) / n,
                "mpix": sum(t[4] for t in tail) / n / 1e6,
                "batch_requests": sum(t[5] for t in tail) / n}


class Server:
    def __init__(self, backend, hbm_budget_bytes: int, max_batch: int = 64, max_inflight: int = 2,
                 batching: bool = True):
        self.be = backend
        self.budget = int(hbm_budget_bytes)
        self.max_batch = max_batch if batching else 1
        self.max_inflight = max_inflight
        self.batching = batching

    def run(self, requests: list[Request], clock=time.perf_counter, idle_sleep: float = 5e-5) -> ServeStats:
        reqs = sorted(requests, key=lambda r: r.arrival)
        for r in reqs:
            if r.nbytes > self.budget:
                raise ValueError(f"request {r.rid} needs {r.nbytes} bytes, over the HBM budget")
        st = ServeStats()
        waiting = collections.deque()
        admitted: list[Request] = []
        inflight: list[tuple[object, list[Request]]] = []
        used = 0
        i = 0
        t0 = clock()

        def fail(rs, err, release=True):
            nonlocal used
            for r in rs:
                r.error = f"{type(err).__name__}: {err}"
                st.failed += 1
                used -= r.nbytes
                if release:
                    self.be.release(r)

        while i < len(reqs) or waiting or admitted or inflight:
            now = clock() - t0
            busy = False
            while i < len(reqs) and reqs[i].arrival <= now:
                waiting.append(reqs[i])
                i += 1
            # admission: arrival order, HBM budget, room in the next launch
            while waiting and len(admitted) < self.max_batch:
                r = waiting[0]
                if used + r.nbytes > self.budget:
                    st.waited_for_budget += 1
                    break
                waiting.popleft()
                used += r.nbytes
                st.hbm_high_water = max(st.hbm_high_water, used)
                r.admitted = now
                try:
                    self.be.admit(r)
                except Exception as e:       # the backend cleaned up; nothing to release
                    fail([r], e, release=False)
                else:
                    admitted.append(r)
                busy = True
            # continuous batching: launch what is admitted whenever a launch slot is free
            if admitted and len(inflight) < self.max_inflight:
                for r in admitted:
                    r.launched = now
                try:
                    h = self.be.launch(admitted)
                except Exception as e:
                    fail(admitted, e)
                else:
                    inflight.append((h, admitted))
                    st.launches += 1
                    st.max_inflight_seen = max(st.max_inflight_seen, len(inflight))
                admitted = []
                busy = True
            # completions (results on the host)
            still = []
            for h, rs in inflight:
                try:
                    finished = self.be.done(h)
                except Exception as e:
                    fail(rs, e)
                    busy = True
                    continue
                if finished:
                    t = clock() - t0
                    for r in rs:
                        r.done = t
                        st.latencies.append(r.latency)
                        st.trace.append((r.latency, r.admitted - r.arrival, r.launched - r.admitted,
                                         t - r.launched, r.H * r.W, len(rs)))
                        st.requests += 1
                        st.pixels += r.H * r.W
                        used -= r.nbytes
                        self.be.release(r)
                    busy = True
                else:
                    still.append((h, rs))
            inflight = still
            if not busy:
                if idle_sleep > 0:
                    time.sleep(idle_sleep)
        st.wall_s = clock() - t0
        return st


class TorchBackend:
    """Device backend on the library's batched path: inputs copied in on an upload stream as
    soon as a request is admitted, one batched launch per server launch on the compute
    stream, results copied back on a download stream.  Uploads never queue behind a
    download (which waits for its launch to finish), so admission overlaps compute.
    ``precision`` selects the form every request is filtered in (FBF_FP32, FBF_FP16_TC,
    FBF_BF16_TC)."""

    def __init__(self, binding, device=0, precision=0):
        import torch
        self.torch = torch
        self.B = binding
        self.dev = torch.device("cuda", device)
        self.h2d = torch.cuda.Stream(self.dev)
        self.d2h = torch.cuda.Stream(self.dev)
        self.compute = torch.cuda.Stream(self.dev)
        self.plans = {}
        self.precision = precision
        self.batch = binding.Batch(4096)

    def plan(self, theta, sigma, K):
        key = (theta, sigma, K)
        if key not in self.plans:
            self.plans[key] = self.B.Plan(sigma, 255, theta, K=K, precision=self.precision)
        return self.plans[key]

    def admit(self, r: Request):
        torch = self.torch
        with torch.cuda.stream(self.h2d):
            x = torch.empty((r.H, r.W), dtype=torch.float32, device=self.dev)
            y = torch.empty((r.H, r.W), dtype=torch.float32, device=self.dev)
            x.copy_(r.host_in, non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(self.h2d)
        r.dev = (x, y, ev)

    def launch(self, rs: list[Request]):
        try:
            return self._launch(rs)
        except Exception:
            # wait for what was queued; images left in the batch's queue (a submit that
            # failed before the launch) must not run with the next launch: a new batch
            self.torch.cuda.synchronize(self.dev)
            if self.batch.pending() > 0:
                self.batch.close()
                self.batch = self.B.Batch(4096)
            raise

    def _launch(self, rs: list[Request]):
        torch = self.torch
        for r in rs:
            x, y, ev = r.dev
            self.compute.wait_event(ev)
            x.record_stream(self.compute)
            y.record_stream(self.compute)
            self.batch.submit(self.plan(r.theta, r.sigma, r.K), x, y)
        self.batch.launch(self.compute)
        k_done = torch.cuda.Event()
        k_done.record(self.compute)
        self.d2h.wait_event(k_done)
        with torch.cuda.stream(self.d2h):
            for r in rs:
                r.dev[1].record_stream(self.d2h)
                r.host_out.copy_(r.dev[1], non_blocking=True)
            done = torch.cuda.Event()
            done.record(self.d2h)
        return done

    def done(self, h) -> bool:
        return h.query()

    def release(self, r: Request):
        r.dev = None


class FakeBackend:
    """Backend without a device: a launch completes `cost(pixels)` seconds after it starts,
    launches run one after another (like one compute stream).  For tests of the loop."""

    def __init__(self, sec_per_pixel: float = 1e-9, clock=time.perf_counter):
        self.spp = sec_per_pixel
        self.clock = clock
        self.busy_until = 0.0
        self.admitted = []
        self.launched = []
        self.live_bytes = 0
        self.max_live_bytes = 0

    def admit(self, r):
        self.admitted.append(r.rid)
        self.live_bytes += r.nbytes
        self.max_live_bytes = max(self.max_live_bytes, self.live_bytes)

    def launch(self, rs):
        now = self.clock()
        start = max(now, self.busy_until)
        self.busy_until = start + self.spp * sum(r.H * r.W for r in rs)
        self.launched.append([r.rid for r in rs])
        return self.busy_until

    def done(self, h) -> bool:
        return self.clock() >= h

    def release(self, r):
        self.live_bytes -= r.nbytes
