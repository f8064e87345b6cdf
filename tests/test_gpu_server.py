"""The native serving loop (fbf_server_*) on the GPU: every served result equals the same
request filtered alone by fbf_filter (within the FP32 tolerance; only the order of
split-tile partial sums can differ between a batched and a lone launch), whatever else
was in flight; admission respects the HBM budget; max_batch = 1 gives one launch per
request.  FP32 and both tensor-core forms."""
import numpy as np
import pytest

from paper_1811_02168_gb300.synth import voronoi_image

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
TOL = 5e-3


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1811_02168_gb300 import build
    build.build()
    from paper_1811_02168_gb300 import binding
    binding.lib()
    return binding


def _requests(n, seed):
    """Bursts of ten simultaneous arrivals, 5 ms apart: the worker admits a burst's requests
    while it issues their uploads (tens of microseconds), so they share launches."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        t = 0.005 * (i // 10)
        H, W = (int(v) for v in rng.integers(40, 400, 2))
        out.append(dict(t=t, H=H, W=W, theta=float(rng.choice([2.0, 5.0, 10.0])),
                        sigma=float(rng.choice([10.0, 30.0, 80.0])), K=int(rng.choice([4, 8])),
                        img=voronoi_image(H, W, 8, 30.0, 10.0, seed=1000 + i)))
    return out


def _alone(B, plans, r, precision):
    key = (r["theta"], r["sigma"], r["K"])
    if key not in plans:
        plans[key] = B.Plan(r["sigma"], 255, r["theta"], K=r["K"], precision=precision)
    x = torch.from_numpy(r["img"]).cuda()
    y = torch.empty_like(x)
    B.fbf_filter(plans[key].handle, x.data_ptr(), y.data_ptr(), r["H"], r["W"], r["W"],
                 torch.cuda.current_stream().cuda_stream)
    return y.cpu()


def _close(got, ref):
    # ill-conditioned plans can produce large outputs; compare relative to their magnitude
    return float((got - ref).abs().max()) <= TOL * max(1.0, float(ref.abs().max()) / 255.0)


@pytest.mark.parametrize("form", ["fp32", "bf16_tc", "fp16_tc"])
def test_served_equals_alone(B, form):
    prec = {"fp32": B.FBF_FP32, "bf16_tc": B.FBF_BF16_TC, "fp16_tc": B.FBF_FP16_TC}[form]
    reqs = _requests(40, 3)
    hin = [torch.from_numpy(r["img"]).pin_memory() for r in reqs]
    hout = [torch.full((r["H"], r["W"]), -1.0).pin_memory() for r in reqs]
    srv = B.Server(precision=prec, hbm_budget_bytes=1 << 30, max_batch=8, max_inflight=2)
    tickets = srv.replay([r["t"] for r in reqs], hin, hout, [r["theta"] for r in reqs],
                         [r["sigma"] for r in reqs], [r["K"] for r in reqs])
    srv.drain(120.0)
    st = srv.stats()
    assert all(srv.poll(t) == B.FBF_DONE for t in tickets)
    srv.close()
    assert st["requests"] == len(reqs) and st["failed"] == 0
    assert st["launches"] < len(reqs)                    # requests were batched
    assert st["pixels"] == sum(r["H"] * r["W"] for r in reqs)
    assert 0 < st["p50_ms"] <= st["p99_ms"]
    plans = {}
    for r, y in zip(reqs, hout):
        assert _close(y, _alone(B, plans, r, prec)), (r["H"], r["W"], r["theta"], r["sigma"], r["K"])


def test_budget_and_one_request_per_launch(B):
    reqs = _requests(16, 4)
    img = voronoi_image(768, 768, 30, 30.0, 10.0, seed=2000)
    for r in reqs:                                       # equal sizes: the budget holds exactly two
        r["H"], r["W"], r["img"] = 768, 768, img
    budget = 2 * 8 * 768 * 768
    hin = [torch.from_numpy(img).pin_memory()] * len(reqs)
    hout = [torch.zeros((768, 768)).pin_memory() for _ in reqs]
    srv = B.Server(precision=B.FBF_FP32, hbm_budget_bytes=budget, max_batch=1, max_inflight=2)
    # every request arrives at once: the budget, not the arrival rate, must hold them back
    srv.replay([0.0] * len(reqs), hin, hout, [r["theta"] for r in reqs], [r["sigma"] for r in reqs],
               [r["K"] for r in reqs])
    srv.drain(120.0)
    st = srv.stats()
    srv.close()
    assert st["requests"] == len(reqs)
    assert st["launches"] == len(reqs)                   # max_batch = 1
    assert st["hbm_high_water"] <= budget
    assert st["waited_for_budget"] > 0
    plans = {}
    for r, y in zip(reqs, hout):
        assert _close(y, _alone(B, plans, r, B.FBF_FP32))


def test_errors(B):
    srv = B.Server(precision=B.FBF_FP32, hbm_budget_bytes=1 << 20, max_batch=4, max_inflight=1)
    x = torch.zeros((512, 512)).pin_memory()             # 2 MiB of device buffers > 1 MiB budget
    with pytest.raises(B.FbfError) as e:
        srv.submit(x, x.clone().pin_memory(), 3.0, 30.0, K=4)
    assert e.value.code == B.FBF_EINVAL
    with pytest.raises(B.FbfError):
        srv.poll(12345)
    srv.close()


@pytest.mark.parametrize("form,tol", [("fp32", TOL), ("bf16_tc", 0.5)])
def test_served_in_a_mix_matches_the_oracle(B, form, tol):
    """Requests served in shared launches with others (bursts of ten) are compared element
    by element with the FP64 Fourier oracle at the form's tolerance (relative to the output's
    magnitude beyond [0, 255], as for the other served-path checks)."""
    from oracle import fit as ofit
    from oracle import filters as ofl
    prec = {"fp32": B.FBF_FP32, "bf16_tc": B.FBF_BF16_TC}[form]
    reqs = _requests(30, 8)
    hin = [torch.from_numpy(r["img"]).pin_memory() for r in reqs]
    hout = [torch.full((r["H"], r["W"]), -1.0).pin_memory() for r in reqs]
    srv = B.Server(precision=prec, hbm_budget_bytes=1 << 30, max_batch=8, max_inflight=2)
    srv.replay([r["t"] for r in reqs], hin, hout, [r["theta"] for r in reqs], [r["sigma"] for r in reqs],
               [r["K"] for r in reqs])
    srv.drain(120.0)
    st = srv.stats()
    srv.close()
    assert st["requests"] == len(reqs) and st["launches"] < len(reqs)
    for i in (0, 7, 13, 22):
        r = reqs[i]
        op = ofit.make_plan(r["sigma"], 255, K=r["K"])
        ref = ofl.fourier_bf(r["img"].astype(np.float64), r["theta"], op.c, op.T)
        scale = max(1.0, float(np.abs(ref).max()) / 255.0)
        err = float(np.abs(hout[i].numpy() - ref).max())
        assert err <= tol * scale, (i, r["H"], r["W"], r["theta"], r["sigma"], r["K"], err)


def test_injected_failures_fail_only_their_requests(B):
    """Failure handling of the native loop, driven on the host (fbf_debug_server_inject: no
    device fault): with a budget of exactly two images, three failing uploads and then a
    failing batched launch end only their own requests with FBF_ECUDA; their buffers and
    budget come back (otherwise later requests could never be admitted and the drain would
    time out), the batch left with queued images is made anew, and every other request is
    served with fbf_filter's result."""
    n, H, W = 14, 256, 256
    imgs = [voronoi_image(H, W, 10, 30.0, 10.0, seed=3000 + i) for i in range(n)]
    hin = [torch.from_numpy(im).pin_memory() for im in imgs]
    hout = [torch.full((H, W), -1.0).pin_memory() for _ in range(n)]
    srv = B.Server(precision=B.FBF_FP32, hbm_budget_bytes=2 * 8 * H * W, max_batch=4, max_inflight=2)
    B.fbf_debug_server_inject(srv.handle, 1, 3)
    first = srv.replay([0.0] * 7, hin[:7], hout[:7], [3.0] * 7, [30.0] * 7, [4] * 7)
    srv.drain(60.0)
    st1 = [srv.poll(t) for t in first]
    assert st1.count(B.FBF_ECUDA) == 3 and st1.count(B.FBF_DONE) == 4, st1
    B.fbf_debug_server_inject(srv.handle, 2, 1)
    second = srv.replay([0.0] * 7, hin[7:], hout[7:], [3.0] * 7, [30.0] * 7, [4] * 7)
    srv.drain(60.0)
    st2 = [srv.poll(t) for t in second]
    stats = srv.stats()
    srv.close()
    failed2 = st2.count(B.FBF_ECUDA)
    assert 1 <= failed2 <= 4 and st2.count(B.FBF_DONE) == 7 - failed2, st2
    assert stats["failed"] == 3 + failed2 and stats["requests"] == n - 3 - failed2
    plans = {}
    for i, s in enumerate(st1 + st2):
        if s == B.FBF_DONE:
            r = dict(theta=3.0, sigma=30.0, K=4, H=H, W=W, img=imgs[i])
            assert _close(hout[i], _alone(B, plans, r, B.FBF_FP32)), i
