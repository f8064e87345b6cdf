"""Served requests on the GPU: each result equals the same request filtered alone by
fbf_filter, within the FP32 tolerance, although it was batched with whatever else had
arrived (continuous batching) and its copies overlapped other launches.  Both the FP32 form
and the compensated BF16 tensor-core form (the form the Poisson-stream bench serves): only
the order of split-tile partial sums can differ between a batched and a lone launch."""
import numpy as np
import pytest

from paper_1811_02168_gb300.serve import Request, Server, TorchBackend
from paper_1811_02168_gb300.synth import voronoi_image

pytestmark = pytest.mark.gpu
TOL = 5e-3
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1811_02168_gb300 import build
    build.build()
    from paper_1811_02168_gb300 import binding
    binding.lib()
    return binding


@pytest.mark.parametrize("form", ["fp32", "bf16_tc"])
def test_served_results_equal_alone_results(B, form):
    rng = np.random.default_rng(77)
    reqs = []
    for i in range(24):
        t = 0.01 * (i // 6)          # bursts of six simultaneous arrivals: they share launches
        H, W = (int(v) for v in rng.integers(48, 320, 2))
        theta = float(rng.choice([2.0, 5.0, 10.0]))
        sigma = float(rng.choice([10.0, 30.0, 80.0]))
        K = int(rng.choice([4, 8]))
        img = voronoi_image(H, W, 8, 30.0, 10.0, seed=500 + i)
        r = Request(i, t, H, W, theta, sigma, K)
        r.host_in = torch.from_numpy(img).pin_memory()
        r.host_out = torch.empty((H, W), dtype=torch.float32).pin_memory()
        reqs.append(r)
    be = TorchBackend(B, precision=B.FBF_FP32 if form == "fp32" else B.FBF_BF16_TC)
    st = Server(be, hbm_budget_bytes=1 << 30, max_batch=8, max_inflight=2).run(reqs)
    assert st.requests == len(reqs)
    assert st.launches < len(reqs)          # requests were batched
    for r in reqs:
        plan = be.plan(r.theta, r.sigma, r.K)
        x = r.host_in.cuda()
        y = torch.empty_like(x)
        B.fbf_filter(plan.handle, x.data_ptr(), y.data_ptr(), r.H, r.W, r.W,
                     torch.cuda.current_stream().cuda_stream)
        alone = y.cpu()
        assert float((r.host_out - alone).abs().max()) <= TOL
