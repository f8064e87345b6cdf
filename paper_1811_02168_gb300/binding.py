"""Thin Python binding of ``libfbf.so`` (ctypes).  Argument marshalling only: every step
of the filter runs in the library's kernels; PyTorch provides device memory and streams.

The functions mirror the C ABI in ``include/fbf.h`` name for name (``fbf_plan``,
``fbf_filter``, ...), raising :class:`FbfError` on a non-zero return code.  ``Plan`` and
``bilateral_filter`` are small conveniences on top.
There is no fallback: if the library is missing or cannot be loaded, loading raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfbf.so")

FBF_OK, FBF_EINVAL, FBF_ENOMEM, FBF_ECUDA, FBF_ETIMEDOUT, FBF_EBUSY = 0, 1, 2, 3, 4, 5
FBF_PENDING, FBF_DONE, FBF_EUNSUPPORTED = 6, 7, 8
FBF_FP32 = 0
FBF_FP16_TC = 1
FBF_BF16_TC = 2
FBF_BF16 = FBF_TF32_TC = FBF_BF16_TC   # the problem statement's names for the compensated form
FBF_FAST = 3                          # FBF_FP32 or FBF_BF16_TC, whichever is faster at the radius
FBF_FAST_FP32_MAX_RADIUS = 6
FBF_FLAG_FIXED_PERIOD = 1
FBF_MAX_K = 64
FBF_MAX_RADIUS = 48

_CODES = {0: "FBF_OK", 1: "FBF_EINVAL", 2: "FBF_ENOMEM", 3: "FBF_ECUDA", 4: "FBF_ETIMEDOUT",
          5: "FBF_EBUSY", 6: "FBF_PENDING", 7: "FBF_DONE", 8: "FBF_EUNSUPPORTED"}


class FbfError(RuntimeError):
    def __init__(self, code: int, func: str, msg: str):
        super().__init__(f"{func} -> {_CODES.get(code, code)}: {msg}")
        self.code = code


_lib = None
_lock = threading.Lock()

_c_double_p = ctypes.POINTER(ctypes.c_double)
_c_int_p = ctypes.POINTER(ctypes.c_int)
_c_void_pp = ctypes.POINTER(ctypes.c_void_p)
_c_u64_p = ctypes.POINTER(ctypes.c_uint64)


class ServerStats(ctypes.Structure):
    """Mirror of fbf_server_stats_t."""
    _fields_ = [("requests", ctypes.c_uint64), ("pixels", ctypes.c_uint64), ("launches", ctypes.c_uint64),
                ("failed", ctypes.c_uint64), ("hbm_high_water", ctypes.c_uint64),
                ("waited_for_budget", ctypes.c_uint64), ("max_inflight_seen", ctypes.c_uint32),
                ("wall_s", ctypes.c_double), ("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double),
                ("tail_requests", ctypes.c_double), ("tail_queued_ms", ctypes.c_double),
                ("tail_wait_for_launch_ms", ctypes.c_double), ("tail_launch_to_result_ms", ctypes.c_double),
                ("tail_mpix", ctypes.c_double), ("tail_batch", ctypes.c_double)]

# name -> (restype, argtypes); mirrors include/fbf.h
SIGNATURES = {
    "fbf_plan": (ctypes.c_int, [_c_void_pp, ctypes.c_double, ctypes.c_int, ctypes.c_double,
                                ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_int]),
    "fbf_plan_from_samples": (ctypes.c_int, [_c_void_pp, _c_double_p, ctypes.c_int, ctypes.c_double,
                                             ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_int]),
    "fbf_plan_info": (ctypes.c_int, [ctypes.c_void_p, _c_int_p, _c_int_p, _c_double_p, _c_double_p,
                                     _c_double_p]),
    "fbf_plan_radius": (ctypes.c_int, [ctypes.c_void_p, _c_int_p]),
    "fbf_plan_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "fbf_filter": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                  ctypes.c_int, ctypes.c_size_t, ctypes.c_void_p]),
    "fbf_filter_noalloc": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                          ctypes.c_int, ctypes.c_size_t, ctypes.c_void_p]),
    "fbf_brute_filter": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                        ctypes.c_size_t, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                        ctypes.c_void_p]),
    "fbf_lut_build": (ctypes.c_int, [_c_void_pp, ctypes.c_int, _c_double_p, ctypes.c_int, _c_double_p,
                                     ctypes.c_int]),
    "fbf_lut_entry": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, _c_int_p, _c_int_p]),
    "fbf_lut_lookup": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double, ctypes.c_double, _c_int_p, _c_int_p]),
    "fbf_plan_from_lut": (ctypes.c_int, [_c_void_pp, ctypes.c_void_p, ctypes.c_double, ctypes.c_double,
                                         ctypes.c_double, ctypes.c_int]),
    "fbf_lut_save": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_char_p]),
    "fbf_lut_load": (ctypes.c_int, [_c_void_pp, ctypes.c_char_p]),
    "fbf_lut_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "fbf_batch_create": (ctypes.c_int, [_c_void_pp, ctypes.c_int, ctypes.c_int]),
    "fbf_batch_submit": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_int, ctypes.c_int, ctypes.c_size_t,
                                        ctypes.POINTER(ctypes.c_uint64)]),
    "fbf_submit": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                  ctypes.c_int, ctypes.c_size_t, ctypes.POINTER(ctypes.c_uint64)]),
    "fbf_poll": (ctypes.c_int, [ctypes.c_uint64, _c_int_p]),
    "fbf_wait": (ctypes.c_int, [ctypes.c_uint64, ctypes.c_double]),
    "fbf_launch": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "fbf_batch_capture": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "fbf_batch_replay": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_uint64)]),
    "fbf_batch_poll": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, _c_int_p]),
    "fbf_batch_wait": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_double]),
    "fbf_batch_pending": (ctypes.c_int, [ctypes.c_void_p, _c_int_p]),
    "fbf_batch_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "fbf_filter_host": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                       ctypes.c_int, ctypes.c_size_t, ctypes.c_void_p]),
    "fbf_server_create": (ctypes.c_int, [_c_void_pp, ctypes.c_int, ctypes.c_int, ctypes.c_uint64, ctypes.c_int,
                                         ctypes.c_int]),
    "fbf_server_submit": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                         ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                         ctypes.c_int, ctypes.c_double, _c_u64_p]),
    "fbf_server_replay": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, _c_double_p, _c_void_pp, _c_void_pp,
                                         _c_int_p, _c_int_p, _c_double_p, _c_double_p, _c_int_p, _c_int_p,
                                         _c_double_p, _c_u64_p]),
    "fbf_server_poll": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, _c_int_p]),
    "fbf_server_drain": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double]),
    "fbf_server_stats": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ServerStats)]),
    "fbf_server_reset_stats": (ctypes.c_int, [ctypes.c_void_p]),
    "fbf_server_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "fbf_device_errors": (ctypes.c_int, [_c_int_p, ctypes.c_int]),
    "fbf_last_error": (ctypes.c_char_p, []),
    "fbf_version": (ctypes.c_char_p, []),
    "fbf_debug_set_wait_limit": (ctypes.c_int, [ctypes.c_int]),
    "fbf_debug_server_inject": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int]),
    "fbf_debug_fp32_peak": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_longlong,
                                           ctypes.c_void_p, ctypes.c_void_p, _c_double_p]),
    "fbf_debug_error_curve": (ctypes.c_int, [_c_double_p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                             _c_double_p]),
}


def lib() -> ctypes.CDLL:
    """Load libfbf.so (once).  Raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise ImportError(f"{LIB_PATH} is missing: build it with "
                                  "`python -c 'import __graft_entry__ as g; g.build()'`")
            L = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def _check(rc: int, func: str):
    if rc != FBF_OK:
        raise FbfError(rc, func, lib().fbf_last_error().decode())


# ----------------------------------------------------------------------------- ABI mirrors

def fbf_plan(sigma: float, R: int, theta: float, K: int = 0, eps: float = 0.0,
             precision: int = FBF_FP32, flags: int = 0) -> int:
    h = ctypes.c_void_p()
    _check(lib().fbf_plan(ctypes.byref(h), sigma, R, theta, K, eps, precision, flags), "fbf_plan")
    return h.value


def fbf_plan_from_samples(b, R: int, theta: float, K: int = 0, eps: float = 0.0,
                          precision: int = FBF_FP32, flags: int = 0) -> int:
    arr = (ctypes.c_double * (2 * R + 1))(*[float(x) for x in b])
    h = ctypes.c_void_p()
    _check(lib().fbf_plan_from_samples(ctypes.byref(h), arr, R, theta, K, eps, precision, flags),
           "fbf_plan_from_samples")
    return h.value


def fbf_plan_info(plan: int):
    K, T = ctypes.c_int(), ctypes.c_int()
    E, dm = ctypes.c_double(), ctypes.c_double()
    _check(lib().fbf_plan_info(plan, ctypes.byref(K), ctypes.byref(T), None, ctypes.byref(E),
                               ctypes.byref(dm)), "fbf_plan_info")
    c = (ctypes.c_double * max(1, K.value))()
    _check(lib().fbf_plan_info(plan, None, None, c, None, None), "fbf_plan_info")
    return K.value, T.value, [c[i] for i in range(K.value)], E.value, dm.value


def fbf_plan_radius(plan: int) -> int:
    r = ctypes.c_int()
    _check(lib().fbf_plan_radius(plan, ctypes.byref(r)), "fbf_plan_radius")
    return r.value


def fbf_plan_destroy(plan: int) -> None:
    _check(lib().fbf_plan_destroy(plan), "fbf_plan_destroy")


def fbf_filter(plan: int, d_in: int, d_out: int, H: int, W: int, pitch_elems: int,
               stream: int = 0) -> None:
    _check(lib().fbf_filter(plan, d_in, d_out, H, W, pitch_elems, stream), "fbf_filter")


def fbf_filter_noalloc(plan: int, d_in: int, d_out: int, H: int, W: int, pitch_elems: int,
                       stream: int = 0) -> None:
    _check(lib().fbf_filter_noalloc(plan, d_in, d_out, H, W, pitch_elems, stream), "fbf_filter_noalloc")


FBF_BATCH_AUTOTUNE = 1


def fbf_batch_create(max_images: int, flags: int = 0) -> int:
    h = ctypes.c_void_p()
    _check(lib().fbf_batch_create(ctypes.byref(h), max_images, flags), "fbf_batch_create")
    return h.value


def fbf_batch_submit(batch: int, plan: int, d_in: int, d_out: int, H: int, W: int, pitch_elems: int) -> int:
    t = ctypes.c_uint64()
    _check(lib().fbf_batch_submit(batch, plan, d_in, d_out, H, W, pitch_elems, ctypes.byref(t)),
           "fbf_batch_submit")
    return t.value


def fbf_submit(plan: int, d_in: int, d_out: int, H: int, W: int, pitch_elems: int) -> int:
    """Queue one image on the current device's implicit queue; returns its ticket."""
    t = ctypes.c_uint64()
    _check(lib().fbf_submit(plan, d_in, d_out, H, W, pitch_elems, ctypes.byref(t)), "fbf_submit")
    return t.value


def fbf_poll(ticket: int) -> int:
    """FBF_DONE or FBF_PENDING for a ticket of fbf_submit (launching its queue if needed)."""
    st = ctypes.c_int()
    _check(lib().fbf_poll(ticket, ctypes.byref(st)), "fbf_poll")
    return st.value


def fbf_wait(ticket: int, timeout_s: float) -> None:
    _check(lib().fbf_wait(ticket, timeout_s), "fbf_wait")


def fbf_launch(batch: int, stream: int = 0) -> None:
    _check(lib().fbf_launch(batch, stream), "fbf_launch")


def fbf_batch_capture(batch: int, stream: int = 0) -> None:
    _check(lib().fbf_batch_capture(batch, stream), "fbf_batch_capture")


def fbf_batch_replay(batch: int, stream: int = 0) -> int:
    t = ctypes.c_uint64()
    _check(lib().fbf_batch_replay(batch, stream, ctypes.byref(t)), "fbf_batch_replay")
    return t.value


def fbf_batch_poll(batch: int, ticket: int) -> int:
    st = ctypes.c_int()
    _check(lib().fbf_batch_poll(batch, ticket, ctypes.byref(st)), "fbf_batch_poll")
    return st.value


def fbf_batch_wait(batch: int, ticket: int, timeout_s: float) -> None:
    _check(lib().fbf_batch_wait(batch, ticket, timeout_s), "fbf_batch_wait")


def fbf_batch_pending(batch: int) -> int:
    n = ctypes.c_int()
    _check(lib().fbf_batch_pending(batch, ctypes.byref(n)), "fbf_batch_pending")
    return n.value


def fbf_batch_destroy(batch: int) -> None:
    _check(lib().fbf_batch_destroy(batch), "fbf_batch_destroy")


def fbf_filter_host(plan: int, host_in: int, host_out: int, H: int, W: int, pitch_elems: int,
                    stream: int = 0) -> None:
    _check(lib().fbf_filter_host(plan, host_in, host_out, H, W, pitch_elems, stream), "fbf_filter_host")


def fbf_server_create(device: int, precision: int, hbm_budget_bytes: int, max_batch: int,
                      max_inflight: int) -> int:
    h = ctypes.c_void_p()
    _check(lib().fbf_server_create(ctypes.byref(h), device, precision, hbm_budget_bytes, max_batch,
                                   max_inflight), "fbf_server_create")
    return h.value


def fbf_server_submit(server: int, host_in: int, host_out: int, H: int, W: int, theta: float, sigma: float,
                      R: int, K: int, eps: float = 0.0) -> int:
    t = ctypes.c_uint64()
    _check(lib().fbf_server_submit(server, host_in, host_out, H, W, theta, sigma, R, K, eps, ctypes.byref(t)),
           "fbf_server_submit")
    return t.value


def fbf_server_replay(server: int, arrival_s, host_in, host_out, H, W, theta, sigma, R, K, eps) -> list:
    n = len(arrival_s)
    arr = lambda ct, xs: (ct * n)(*xs)   # noqa: E731
    tickets = (ctypes.c_uint64 * n)()
    _check(lib().fbf_server_replay(server, n, arr(ctypes.c_double, arrival_s), arr(ctypes.c_void_p, host_in),
                                   arr(ctypes.c_void_p, host_out), arr(ctypes.c_int, H), arr(ctypes.c_int, W),
                                   arr(ctypes.c_double, theta), arr(ctypes.c_double, sigma),
                                   arr(ctypes.c_int, R), arr(ctypes.c_int, K), arr(ctypes.c_double, eps),
                                   tickets), "fbf_server_replay")
    return list(tickets)


def fbf_server_poll(server: int, ticket: int) -> int:
    st = ctypes.c_int()
    _check(lib().fbf_server_poll(server, ticket, ctypes.byref(st)), "fbf_server_poll")
    return st.value


def fbf_server_drain(server: int, timeout_s: float = 60.0) -> None:
    _check(lib().fbf_server_drain(server, timeout_s), "fbf_server_drain")


def fbf_server_stats(server: int) -> dict:
    st = ServerStats()
    _check(lib().fbf_server_stats(server, ctypes.byref(st)), "fbf_server_stats")
    return {name: getattr(st, name) for name, _ in ServerStats._fields_}


def fbf_server_reset_stats(server: int) -> None:
    _check(lib().fbf_server_reset_stats(server), "fbf_server_reset_stats")


def fbf_server_destroy(server: int) -> None:
    _check(lib().fbf_server_destroy(server), "fbf_server_destroy")


def fbf_device_errors(clear: bool = False) -> int:
    f = ctypes.c_int()
    _check(lib().fbf_device_errors(ctypes.byref(f), 1 if clear else 0), "fbf_device_errors")
    return f.value


def fbf_brute_filter(d_in: int, d_out: int, H: int, W: int, pitch_elems: int, theta: float, sigma: float,
                     R: int = 255, stream: int = 0) -> None:
    """Eq. (1) with the Gaussian range kernel, evaluated directly on the device (device
    pointers, asynchronous on `stream`)."""
    _check(lib().fbf_brute_filter(d_in, d_out, H, W, pitch_elems, theta, sigma, R, stream), "fbf_brute_filter")


class Lut:
    """Owns an ``fbf_lut_t``: Algorithm 1 on a (sigma, eps) grid, bilinear lookup off the grid."""

    def __init__(self, R: int = 255, sigmas=None, eps=None, path: str | None = None):
        h = ctypes.c_void_p()
        if path is not None:
            _check(lib().fbf_lut_load(ctypes.byref(h), os.fsencode(path)), "fbf_lut_load")
        else:
            s = (ctypes.c_double * len(sigmas))(*sigmas)
            e = (ctypes.c_double * len(eps))(*eps)
            _check(lib().fbf_lut_build(ctypes.byref(h), R, s, len(sigmas), e, len(eps)), "fbf_lut_build")
        self.handle = h.value
        self.R = R

    def entry(self, i: int, j: int):
        K, T = ctypes.c_int(), ctypes.c_int()
        _check(lib().fbf_lut_entry(self.handle, i, j, ctypes.byref(K), ctypes.byref(T)), "fbf_lut_entry")
        return K.value, T.value

    def lookup(self, sigma: float, eps: float):
        K, T = ctypes.c_int(), ctypes.c_int()
        _check(lib().fbf_lut_lookup(self.handle, sigma, eps, ctypes.byref(K), ctypes.byref(T)), "fbf_lut_lookup")
        return K.value, T.value

    def plan(self, sigma: float, eps: float, theta: float, precision: int = FBF_FP32) -> "Plan":
        h = ctypes.c_void_p()
        _check(lib().fbf_plan_from_lut(ctypes.byref(h), self.handle, sigma, eps, theta, precision),
               "fbf_plan_from_lut")
        return Plan._adopt(h.value, sigma, self.R, theta, precision)

    def save(self, path: str) -> None:
        _check(lib().fbf_lut_save(self.handle, os.fsencode(path)), "fbf_lut_save")

    def close(self):
        if getattr(self, "handle", None):
            lib().fbf_lut_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def fbf_last_error() -> str:
    return lib().fbf_last_error().decode()


def fbf_version() -> str:
    return lib().fbf_version().decode()


def fbf_debug_server_inject(server: int, stage: int, count: int) -> None:
    """Test aid: the server's next `count` uploads (stage 1) or launches (stage 2) fail."""
    _check(lib().fbf_debug_server_inject(server, stage, count), "fbf_debug_server_inject")


def fbf_debug_set_wait_limit(polls: int) -> None:
    """Test aid: make the kernels' pipeline waits give up after `polls` polls (0 = normal)."""
    _check(lib().fbf_debug_set_wait_limit(polls), "fbf_debug_set_wait_limit")


def fbf_debug_fp32_peak(pairs: bool, blocks: int, threads: int, iters: int, d_out: int, stream) -> float:
    """Launch the FP32 multiply-add rate probe on `stream`; returns the launch's flop count."""
    flop = ctypes.c_double(0.0)
    _check(lib().fbf_debug_fp32_peak(1 if pairs else 0, blocks, threads, iters, ctypes.c_void_p(d_out),
                                     ctypes.c_void_p(stream), ctypes.byref(flop)), "fbf_debug_fp32_peak")
    return flop.value


def fbf_debug_error_curve(b, R: int, T: int, Kc: int):
    arr = (ctypes.c_double * (2 * R + 1))(*[float(x) for x in b])
    out = (ctypes.c_double * Kc)()
    _check(lib().fbf_debug_error_curve(arr, R, T, Kc, out), "fbf_debug_error_curve")
    return [out[i] for i in range(Kc)]


# ----------------------------------------------------------------------------- conveniences

class Plan:
    """Owns an ``fbf_plan_t``.  Fitted parameters are read back once."""

    def __init__(self, sigma: float | None = None, R: int = 255, theta: float = 3.0, K: int = 0,
                 eps: float = 0.0, precision: int = FBF_FP32, flags: int = 0, samples=None):
        if samples is not None:
            self.handle = fbf_plan_from_samples(samples, R, theta, K, eps, precision, flags)
        else:
            self.handle = fbf_plan(sigma, R, theta, K, eps, precision, flags)
        self.sigma, self.R, self.theta, self.precision, self.flags = sigma, R, theta, precision, flags
        self.K, self.T, self.c, self.E, self.delta_max = fbf_plan_info(self.handle)
        self.radius = fbf_plan_radius(self.handle)

    @classmethod
    def _adopt(cls, handle: int, sigma, R: int, theta: float, precision: int) -> "Plan":
        p = cls.__new__(cls)
        p.handle = handle
        p.sigma, p.R, p.theta, p.precision, p.flags = sigma, R, theta, precision, 0
        p.K, p.T, p.c, p.E, p.delta_max = fbf_plan_info(handle)
        p.radius = fbf_plan_radius(handle)
        return p

    def close(self):
        if getattr(self, "handle", None):
            fbf_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __repr__(self):
        return (f"Plan(sigma={self.sigma}, R={self.R}, theta={self.theta}, K={self.K}, T={self.T}, "
                f"E={self.E:.3g}, precision={self.precision})")


def bilateral_filter(plan: Plan, image, out=None, stream=None):
    """f_BF of one 2-D float32 image.

    ``image`` is a torch tensor.  On the GPU it is filtered in device memory on the current
    (or given) stream, asynchronously, into ``out`` or a new device tensor, which is
    returned.  On the host it goes through ``fbf_filter_host``, the end-to-end path: the image
    is taken page-locked (copied into pinned memory if it is not) and the result is a pinned
    tensor, so the kernel reads and writes host memory directly; returns when the result is
    on the host.
    """
    import torch
    if image.dim() != 2 or image.dtype != torch.float32:
        raise ValueError("image must be a 2-D float32 tensor")
    if not image.is_cuda:
        src = image if image.is_pinned() else image.pin_memory()
        if src.stride(1) != 1:
            src = src.contiguous().pin_memory()
        H, W = src.shape
        res = out if out is not None else torch.empty((H, W), dtype=torch.float32, pin_memory=True)
        if res.is_cuda or res.stride(1) != 1 or res.stride(0) != src.stride(0):
            raise ValueError("out must be a host tensor with the input's row stride")
        st = stream if stream is not None else torch.cuda.current_stream()
        fbf_filter_host(plan.handle, src.data_ptr(), res.data_ptr(), H, W, src.stride(0), st.cuda_stream)
        return res
    dev_in = image if image.stride(1) == 1 else image.contiguous()
    H, W = dev_in.shape
    dev_out = out if (out is not None and out.is_cuda) else torch.empty((H, W), device=dev_in.device,
                                                                        dtype=torch.float32)
    if dev_out.stride(0) != dev_in.stride(0) or dev_out.stride(1) != 1:
        raise ValueError("out must have the input's row stride")
    st = stream if stream is not None else torch.cuda.current_stream(dev_in.device)
    fbf_filter(plan.handle, dev_in.data_ptr(), dev_out.data_ptr(), H, W, dev_in.stride(0),
               st.cuda_stream)
    return dev_out


class Batch:
    """Owns an ``fbf_batch_t``: queue device images with ``submit``, run them with
    ``launch`` (or ``capture`` once and ``replay``), and query tickets."""

    def __init__(self, max_images: int, autotune: bool = False):
        self.handle = fbf_batch_create(max_images, FBF_BATCH_AUTOTUNE if autotune else 0)
        self._keep = []          # plans referenced by queued images stay alive

    def submit(self, plan: Plan, x, y) -> int:
        """x, y: 2-D float32 CUDA tensors with equal row strides."""
        if x.stride(1) != 1 or y.stride(1) != 1 or x.stride(0) != y.stride(0):
            raise ValueError("x and y need unit column stride and equal row strides")
        self._keep.append(plan)
        H, W = x.shape
        return fbf_batch_submit(self.handle, plan.handle, x.data_ptr(), y.data_ptr(), H, W, x.stride(0))

    def launch(self, stream=None):
        import torch
        st = stream if stream is not None else torch.cuda.current_stream()
        fbf_launch(self.handle, st.cuda_stream)
        self._keep.clear()       # the launch copied the plans' parameters

    def capture(self, stream=None):
        import torch
        st = stream if stream is not None else torch.cuda.current_stream()
        fbf_batch_capture(self.handle, st.cuda_stream)
        self._keep.clear()

    def replay(self, stream=None) -> int:
        import torch
        st = stream if stream is not None else torch.cuda.current_stream()
        return fbf_batch_replay(self.handle, st.cuda_stream)

    def poll(self, ticket: int) -> int:
        return fbf_batch_poll(self.handle, ticket)

    def wait(self, ticket: int, timeout_s: float = 60.0) -> None:
        fbf_batch_wait(self.handle, ticket, timeout_s)

    def pending(self) -> int:
        return fbf_batch_pending(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            fbf_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Owns an ``fbf_server_t`` (continuous batching under an HBM budget, served by a native
    worker thread).  Host tensors passed to ``submit`` / ``replay`` must be pinned, float32,
    contiguous, and stay alive until their request is done."""

    def __init__(self, precision: int = FBF_FP32, hbm_budget_bytes: int = 40 << 30, max_batch: int = 64,
                 max_inflight: int = 2, device: int = 0):
        self.handle = fbf_server_create(device, precision, hbm_budget_bytes, max_batch, max_inflight)

    @staticmethod
    def _host(t):
        if not (t.is_pinned() and t.is_contiguous() and t.dtype.itemsize == 4):
            raise ValueError("host images must be pinned, contiguous float32 tensors")
        return t.data_ptr()

    def submit(self, host_in, host_out, theta: float, sigma: float, K: int = 0, eps: float = 0.0,
               R: int = 255) -> int:
        H, W = host_in.shape
        if tuple(host_out.shape) != (H, W):
            raise ValueError("host_out must have the shape of host_in")
        return fbf_server_submit(self.handle, self._host(host_in), self._host(host_out), H, W, theta, sigma,
                                 R, K, eps)

    def replay(self, arrivals, host_in, host_out, theta, sigma, K, eps=None, R: int = 255) -> list:
        """Submit request i at arrivals[i] seconds after the call (open-loop load)."""
        n = len(arrivals)
        eps = eps if eps is not None else [0.0] * n
        return fbf_server_replay(self.handle, list(arrivals), [self._host(x) for x in host_in],
                                 [self._host(y) for y in host_out], [x.shape[0] for x in host_in],
                                 [x.shape[1] for x in host_in], list(theta), list(sigma), [R] * n, list(K),
                                 list(eps))

    def poll(self, ticket: int) -> int:
        return fbf_server_poll(self.handle, ticket)

    def drain(self, timeout_s: float = 600.0) -> None:
        fbf_server_drain(self.handle, timeout_s)

    def stats(self) -> dict:
        return fbf_server_stats(self.handle)

    def reset_stats(self) -> None:
        fbf_server_reset_stats(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            fbf_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
