"""C-ABI library on the host (no GPU): it loads, exports every symbol include/*.h
declares, its FP64 fitter matches the oracle's, and bad arguments are rejected with the
documented codes before any device work."""
import ctypes
import glob
import math
import os
import re

import numpy as np
import pytest

from oracle import fit as ofit
from paper_1811_02168_gb300 import binding as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1811_02168_gb300 import build
    build.build()
    B.lib()


def _declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(fbf_\w+)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


def test_exports_every_declared_symbol():
    names = _declared_symbols()
    assert "fbf_plan" in names and "fbf_filter" in names
    L = ctypes.CDLL(B.LIB_PATH)
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing
    assert set(names) <= set(B.SIGNATURES), "binding lacks a mirror for a declared symbol"


def test_binding_constants_equal_the_header():
    """Every integer constant the binding mirrors has the header's value (error codes,
    statuses, precision forms, flags, limits)."""
    defined = {}
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        for m in re.finditer(r"^#define\s+(FBF_\w+)\s+\(?(\d+)u?(?:\s*<<\s*(\d+))?\)?", open(h).read(), flags=re.M):
            defined[m.group(1)] = int(m.group(2)) << int(m.group(3) or 0)
        for m in re.finditer(r"^#define\s+(FBF_\w+)\s+(FBF_\w+)\s*$", open(h).read(), flags=re.M):
            defined[m.group(1)] = defined[m.group(2)]   # another name for a defined constant
    mirrored = {n: getattr(B, n) for n in dir(B) if n.startswith("FBF_") and isinstance(getattr(B, n), int)}
    assert {"FBF_OK", "FBF_EINVAL", "FBF_EUNSUPPORTED", "FBF_FP32", "FBF_BF16_TC", "FBF_MAX_K"} <= set(mirrored)
    unknown = sorted(set(mirrored) - set(defined))
    assert not unknown, f"binding constants the header does not define: {unknown}"
    wrong = {n: (v, defined[n]) for n, v in mirrored.items() if defined[n] != v}
    assert not wrong, wrong


def _phi_hat(c, T, R):
    t = np.arange(-R, R + 1)
    return ofit.phi_hat(t, c, T)


@pytest.mark.parametrize("sigma,K", [(50.0, 4), (30.0, 4), (10.0, 16), (80.0, 8), (15.0, 5)])
def test_fitter_fixed_K_matches_oracle(sigma, K):
    """eq. (5)/(6) with K fixed: same T, same E, same phi_hat on Lambda."""
    R, theta = 255, 3.0
    p = B.Plan(sigma, R, theta, K=K)
    o = ofit.make_plan(sigma, R, K=K)
    assert p.K == o.K == K
    assert p.T == o.T
    assert abs(p.E - o.E) <= 1e-9 * max(1.0, o.E) + 1e-14
    np.testing.assert_allclose(_phi_hat(p.c, p.T, R), _phi_hat(o.c, o.T, R), rtol=0, atol=1e-10)
    assert abs(p.delta_max - o.delta_max) < 1e-10


def test_fitter_fig1_T203():
    """Fig. 1: K = 4, sigma = 50, R = 255 gives T = 203."""
    assert B.Plan(50.0, 255, 2.0, K=4).T == 203


@pytest.mark.parametrize("sigma,eps", [(10.0, 0.01), (30.0, 0.01), (80.0, 0.01), (30.0, 0.1),
                                       (50.0, 1e-3)])
def test_fitter_algorithm1_matches_oracle(sigma, eps):
    """Algorithm 1: same K*, T* and error."""
    R = 255
    p = B.Plan(sigma, R, 5.0, eps=eps)
    o = ofit.make_plan(sigma, R, eps=eps)
    assert (p.K, p.T) == (o.K, o.T)
    assert p.E <= eps
    np.testing.assert_allclose(_phi_hat(p.c, p.T, R), _phi_hat(o.c, o.T, R), rtol=0, atol=1e-10)


def test_fitter_roundoff_region_phi_hat_agrees():
    """K = 16, sigma = 80: E is at FP64 round-off for many T; compare through phi_hat."""
    R = 255
    p = B.Plan(80.0, R, 5.0, K=16)
    o = ofit.make_plan(80.0, R, K=16)
    assert p.E < 1e-15 and o.E < 1e-15
    np.testing.assert_allclose(_phi_hat(p.c, p.T, R), ofit.kernel_samples(80.0, R), rtol=0, atol=1e-9)


def test_error_curve_matches_oracle_including_rank_deficient():
    """E(K,T) from the C++ folded Householder reduction against NumPy lstsq on the full
    (2R+1) x K system.  Rank-deficient T (K > T+1) must agree exactly up to round-off;
    at large T the columns are ill-conditioned and two backward-stable solvers may differ
    by about eps * cond(A) * ||b||^2."""
    R, sigma = 255, 20.0
    b = ofit.kernel_samples(sigma, R)
    for T in (1, 2, 5, 40, 150, 700):
        E = B.fbf_debug_error_curve(b, R, T, 10)
        for K in range(1, 11):
            Eo, _ = ofit.kernel_error(K, T, b, R)
            A = ofit.design_matrix(K, T, R)
            s = np.linalg.svd(A, compute_uv=False)
            s = s[s > s[0] * 1e-12]
            tol = 1e-10 * max(1.0, Eo) + 8 * np.finfo(float).eps * (s[0] / s[-1]) * float(b @ b)
            assert abs(E[K - 1] - Eo) <= tol, (T, K, E[K - 1], Eo)


def test_fixed_period_flag_is_T_equals_R():
    """FBF model (Section III): T = R, only the least-squares step; matches the oracle."""
    R = 255
    p = B.Plan(40.0, R, 3.0, K=4, flags=B.FBF_FLAG_FIXED_PERIOD)
    o = ofit.make_plan(40.0, R, K=4, T=R)
    assert p.T == R
    np.testing.assert_allclose(_phi_hat(p.c, p.T, R), _phi_hat(o.c, o.T, R), rtol=0, atol=1e-12)


def test_non_gaussian_kernel_from_samples():
    """Any range kernel (Sections I, IV): the exponential kernel exp(-|t|/s)."""
    R, s = 255, 25.0
    kern = lambda t: np.exp(-np.abs(t) / s)  # noqa: E731
    b = kern(np.arange(-R, R + 1))
    p = B.Plan(None, R, 3.0, K=10, samples=b)
    o = ofit.make_plan(None, R, K=10, kernel=kern)
    assert p.T == o.T
    np.testing.assert_allclose(_phi_hat(p.c, p.T, R), _phi_hat(o.c, o.T, R), rtol=0, atol=1e-10)


@pytest.mark.parametrize("args,code", [
    (dict(sigma=0.0, R=255, theta=3.0, K=4), B.FBF_EINVAL),
    (dict(sigma=-1.0, R=255, theta=3.0, K=4), B.FBF_EINVAL),
    (dict(sigma=30.0, R=0, theta=3.0, K=4), B.FBF_EINVAL),
    (dict(sigma=30.0, R=255, theta=0.0, K=4), B.FBF_EINVAL),
    (dict(sigma=30.0, R=255, theta=3.0, K=0, eps=0.0), B.FBF_EINVAL),
    (dict(sigma=30.0, R=255, theta=3.0, K=-2), B.FBF_EINVAL),
    (dict(sigma=30.0, R=255, theta=3.0, K=4, precision=99), B.FBF_EINVAL),
    (dict(sigma=30.0, R=255, theta=3.0, K=4, flags=1 << 20), B.FBF_EINVAL),
    (dict(sigma=30.0, R=255, theta=17.0, K=4), B.FBF_EUNSUPPORTED),
    (dict(sigma=30.0, R=255, theta=3.0, K=B.FBF_MAX_K + 1), B.FBF_EUNSUPPORTED),
])
def test_plan_rejects_bad_arguments(args, code):
    with pytest.raises(B.FbfError) as ei:
        B.fbf_plan(**args)
    assert ei.value.code == code
    assert B.fbf_last_error()


def test_filter_rejects_bad_arguments_without_touching_the_device():
    p = B.Plan(30.0, 255, 3.0, K=4)
    cases = [
        (dict(d_in=0, d_out=1 << 20, H=4, W=4, pitch_elems=4), B.FBF_EINVAL),
        (dict(d_in=1 << 20, d_out=0, H=4, W=4, pitch_elems=4), B.FBF_EINVAL),
        (dict(d_in=1 << 20, d_out=1 << 24, H=0, W=4, pitch_elems=4), B.FBF_EINVAL),
        (dict(d_in=1 << 20, d_out=1 << 24, H=4, W=-1, pitch_elems=4), B.FBF_EINVAL),
        (dict(d_in=1 << 20, d_out=1 << 24, H=4, W=8, pitch_elems=4), B.FBF_EINVAL),
        (dict(d_in=1 << 20, d_out=(1 << 20) + 16, H=4, W=4, pitch_elems=4), B.FBF_EINVAL),
    ]
    for kw, code in cases:
        with pytest.raises(B.FbfError) as ei:
            B.fbf_filter(p.handle, **kw)
        assert ei.value.code == code
    with pytest.raises(B.FbfError):
        B.fbf_filter(0, 1 << 20, 1 << 24, 4, 4, 4)


def test_plan_info_null_plan():
    with pytest.raises(B.FbfError) as ei:
        B.fbf_plan_info(0)
    assert ei.value.code == B.FBF_EINVAL


def test_batch_host_side_queue_and_bounded_wait():
    """Batch bookkeeping needs no GPU until a launch: queueing, the max_images bound
    (FBF_EBUSY), argument checks, and a bounded wait on a launch that never happens."""
    p = B.Plan(30.0, 255, 3.0, K=4)
    b = B.fbf_batch_create(2, 0)
    try:
        t0 = B.fbf_batch_submit(b, p.handle, 1 << 20, 1 << 30, 16, 16, 16)
        t1 = B.fbf_batch_submit(b, p.handle, 1 << 21, 1 << 31, 8, 9, 9)
        assert t0 == t1                       # same pending launch
        assert B.fbf_batch_pending(b) == 2
        with pytest.raises(B.FbfError) as ei:
            B.fbf_batch_submit(b, p.handle, 1 << 22, 1 << 32, 4, 4, 4)
        assert ei.value.code == B.FBF_EBUSY
        for kw in (dict(d_in=0), dict(H=0), dict(pitch_elems=2)):
            args = dict(d_in=1 << 23, d_out=1 << 33, H=4, W=4, pitch_elems=4)
            args.update(kw)
            with pytest.raises(B.FbfError) as ei:
                B.fbf_batch_submit(b, p.handle, args["d_in"], args["d_out"], args["H"], args["W"],
                                   args["pitch_elems"])
            assert ei.value.code in (B.FBF_EINVAL, B.FBF_EBUSY)
        assert B.fbf_batch_poll(b, t0) == B.FBF_PENDING
        with pytest.raises(B.FbfError) as ei:
            B.fbf_batch_wait(b, t0, 0.05)
        assert ei.value.code == B.FBF_ETIMEDOUT
    finally:
        B.fbf_batch_destroy(b)
    with pytest.raises(B.FbfError):
        B.fbf_batch_create(0, 0)


def test_implicit_queue_host_side():
    """fbf_submit / fbf_poll / fbf_wait (no batch handle): a ticket that no fbf_submit
    returned is refused on the host; without a GPU, fbf_submit reports the CUDA failure
    instead of queueing."""
    for bad in (0, 5, (70 << 48) | 1):
        with pytest.raises(B.FbfError) as ei:
            B.fbf_poll(bad)
        assert ei.value.code == B.FBF_EINVAL
        with pytest.raises(B.FbfError) as ei:
            B.fbf_wait(bad, 0.01)
        assert ei.value.code == B.FBF_EINVAL
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        return
    p = B.Plan(30.0, 255, 3.0, K=4)
    with pytest.raises(B.FbfError) as ei:
        B.fbf_submit(p.handle, 1 << 20, 1 << 30, 16, 16, 16)
    assert ei.value.code == B.FBF_ECUDA


def test_precision_names_of_the_problem_statement():
    """FBF_BF16 and FBF_TF32_TC name the compensated BF16 / TF32 tensor-core form."""
    hdr = open(os.path.join(ROOT, "include", "fbf.h")).read()
    assert "#define FBF_BF16       FBF_BF16_TC" in hdr and "#define FBF_TF32_TC    FBF_BF16_TC" in hdr
    assert B.FBF_BF16 == B.FBF_TF32_TC == B.FBF_BF16_TC
    p = B.Plan(30.0, 255, 3.0, K=4, precision=B.FBF_TF32_TC)
    assert p.K == 4


def test_fast_form_takes_fp32_where_tensor_cores_cannot():
    """FBF_FAST is resolved when the plan is made: beyond the tensor-core radius limit it is
    the FP32 form (a plan FBF_BF16_TC refuses), and any other precision value is refused."""
    with pytest.raises(B.FbfError) as ei:
        B.Plan(30.0, 255, 16.0, K=4, precision=B.FBF_BF16_TC)      # r = 48 > FBF_MAX_RADIUS_TC
    assert ei.value.code == B.FBF_EUNSUPPORTED
    for theta in (2.0, 5.0, 10.0, 16.0):                          # r = 6, 15, 30, 48
        assert B.Plan(30.0, 255, theta, K=4, precision=B.FBF_FAST).K == 4
    with pytest.raises(B.FbfError) as ei:
        B.Plan(30.0, 255, 2.0, K=4, precision=7)
    assert ei.value.code == B.FBF_EINVAL


def test_failed_launch_empties_the_queue():
    """A launch or capture that fails (here: no CUDA device) still empties the queue, so
    images whose buffers the caller frees after the error are never launched later.  The
    pointers are fake, so this runs only where no GPU is visible."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("fake device pointers: only without a GPU")
    p = B.Plan(30.0, 255, 3.0, K=4)
    b = B.fbf_batch_create(2, 0)
    try:
        for call in (lambda: B.fbf_launch(b, 0), lambda: B.fbf_batch_capture(b, 0)):
            B.fbf_batch_submit(b, p.handle, 1 << 20, 1 << 30, 16, 16, 16)
            assert B.fbf_batch_pending(b) == 1
            with pytest.raises(B.FbfError):
                call()
            assert B.fbf_batch_pending(b) == 0
    finally:
        B.fbf_batch_destroy(b)


def test_brute_filter_argument_errors():
    from paper_1811_02168_gb300 import binding as B
    L = B.lib()
    x = ctypes.c_void_p(16)
    y = ctypes.c_void_p(1 << 20)
    assert L.fbf_brute_filter(None, y, 4, 4, 4, 2.0, 30.0, 255, None) == B.FBF_EINVAL
    assert L.fbf_brute_filter(x, y, 0, 4, 4, 2.0, 30.0, 255, None) == B.FBF_EINVAL
    assert L.fbf_brute_filter(x, y, 4, 4, 3, 2.0, 30.0, 255, None) == B.FBF_EINVAL
    assert L.fbf_brute_filter(x, y, 4, 4, 4, 0.0, 30.0, 255, None) == B.FBF_EINVAL
    assert L.fbf_brute_filter(x, y, 4, 4, 4, 2.0, -1.0, 255, None) == B.FBF_EINVAL
    assert L.fbf_brute_filter(x, y, 4, 4, 4, 2.0, 30.0, 0, None) == B.FBF_EINVAL
    assert L.fbf_brute_filter(x, x, 4, 4, 4, 2.0, 30.0, 255, None) == B.FBF_EINVAL   # overlap
    assert L.fbf_brute_filter(x, y, 4, 4, 4, 17.0, 30.0, 255, None) == B.FBF_EUNSUPPORTED   # r = 51
    far = ctypes.c_void_p(1 << 40)
    H = 65535 * 32 + 1                                                   # grid y above 65535
    assert L.fbf_brute_filter(x, far, H, 1, 1, 2.0, 30.0, 255, None) == B.FBF_EUNSUPPORTED

def test_server_argument_errors():
    """fbf_server_create rejects bad arguments before touching a device; the other entry
    points reject a NULL server."""
    import ctypes
    from paper_1811_02168_gb300 import binding as B
    L = B.lib()
    h = ctypes.c_void_p()
    assert L.fbf_server_create(ctypes.byref(h), 0, 99, 1 << 20, 4, 2) == B.FBF_EINVAL      # form
    assert L.fbf_server_create(ctypes.byref(h), 0, B.FBF_FP32, 0, 4, 2) == B.FBF_EINVAL    # budget
    assert L.fbf_server_create(ctypes.byref(h), 0, B.FBF_FP32, 1 << 20, 0, 2) == B.FBF_EINVAL
    assert L.fbf_server_create(ctypes.byref(h), 0, B.FBF_FP32, 1 << 20, 4, 0) == B.FBF_EINVAL
    assert L.fbf_server_create(None, 0, B.FBF_FP32, 1 << 20, 4, 2) == B.FBF_EINVAL
    t = ctypes.c_uint64()
    st = ctypes.c_int()
    assert L.fbf_server_submit(None, None, None, 8, 8, 2.0, 30.0, 255, 4, 0.0, ctypes.byref(t)) == B.FBF_EINVAL
    assert L.fbf_server_poll(None, 1, ctypes.byref(st)) == B.FBF_EINVAL
    assert L.fbf_server_drain(None, 1.0) == B.FBF_EINVAL
    assert L.fbf_server_stats(None, None) == B.FBF_EINVAL
    assert L.fbf_server_reset_stats(None) == B.FBF_EINVAL
    assert L.fbf_server_destroy(None) == B.FBF_OK
    assert ctypes.sizeof(B.ServerStats) == 128

def test_filter_host_argument_errors():
    """fbf_filter_host rejects bad arguments before any device work."""
    import ctypes
    from paper_1811_02168_gb300 import binding as B
    L = B.lib()
    p = B.Plan(30.0, 255, 2.0, K=4)
    buf = (ctypes.c_float * 64)()
    a = ctypes.addressof(buf)
    assert L.fbf_filter_host(None, a, a, 8, 8, 8, None) == B.FBF_EINVAL
    assert L.fbf_filter_host(p.handle, None, a, 8, 8, 8, None) == B.FBF_EINVAL
    assert L.fbf_filter_host(p.handle, a, a, 0, 8, 8, None) == B.FBF_EINVAL
    assert L.fbf_filter_host(p.handle, a, a, 8, 8, 7, None) == B.FBF_EINVAL       # pitch < W
    assert L.fbf_filter_host(p.handle, a, a + 4, 8, 8, 8, None) == B.FBF_EINVAL   # partial overlap



def test_nvtx_ranges_on_the_host_stages():
    """Host-side stages carry NVTX ranges (plan, filter, host call, batch launch / capture /
    replay, serving admission, launch and completion) for timeline tools."""
    src = ""
    for f in glob.glob(os.path.join(ROOT, "paper_1811_02168_gb300", "csrc", "*.c*")):
        src += open(f).read()
    for name in ("fbf_plan", "fbf_filter", "fbf_filter_host", "fbf_launch", "fbf_batch_capture",
                 "fbf_batch_replay", "fbf_server admit: upload", "fbf_server launch", "fbf_server complete"):
        assert f'NvtxRange tr("{name}")' in src, name
