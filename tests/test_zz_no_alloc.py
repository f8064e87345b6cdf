"""The allocation-free entry point fbf_filter_noalloc, through the C ABI (GPU).

Some callers cannot allocate device memory while they filter -- their memory belongs to
another allocator, or a cudaMalloc/cudaFree (which may synchronise the device) would break
their latency budget.  fbf_filter_noalloc runs the same FP32 kernel as fbf_filter but takes
its scratch from a fixed array compiled into the library.  Its results must match
fbf_filter's within the tolerance of the other GPU tests, on consecutive calls that reuse
that array (the second call sees what the first left in it).  This file is collected last
so that a run stopping at the first failure has already run every other test; it also
passes when run alone in a fresh process, where its first call performs the set-up.
"""
import numpy as np
import pytest

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


@pytest.mark.parametrize("H,W,theta,sigma,K,eps", [
    (333, 517, 5.0, 30.0, 0, 0.01),     # radius 15 configuration, K from Algorithm 1
    (700, 260, 10.0, 10.0, 16, 0.0),    # radius 30 configuration, 16 terms
])
def test_noalloc_matches_fbf_filter_on_two_calls_in_a_row(B, H, W, theta, sigma, K, eps):
    img = voronoi_image(H, W, 25, 40.0, 10.0, seed=H + W)
    plan = B.Plan(sigma, 255, theta, K=K, eps=eps)
    x = torch.from_numpy(img).cuda()
    st = torch.cuda.current_stream()
    ref = torch.full_like(x, -1.0)
    B.fbf_filter(plan.handle, x.data_ptr(), ref.data_ptr(), H, W, W, st.cuda_stream)
    outs = []
    for _ in range(2):
        y = torch.full_like(x, -1.0)
        B.fbf_filter_noalloc(plan.handle, x.data_ptr(), y.data_ptr(), H, W, W, st.cuda_stream)
        outs.append(y)
    st.synchronize()
    r = ref.cpu().numpy()
    for y in outs:
        err = float(np.abs(y.cpu().numpy() - r).max())
        assert err <= TOL, err


def test_noalloc_rejects_images_beyond_its_scratch(B):
    """An image that needs more tile counters than the fixed array holds is refused on
    the host, before any device work (the pointers are never dereferenced)."""
    plan = B.Plan(30.0, 255, 5.0, K=4)
    H = W = 40000
    with pytest.raises(B.FbfError) as ei:
        B.fbf_filter_noalloc(plan.handle, 1 << 36, 1 << 40, H, W, W, 0)
    assert ei.value.code == B.FBF_EUNSUPPORTED
    assert "tiles" in B.fbf_last_error()


def test_noalloc_allocates_no_device_memory(B):
    """After one warm-up call, a call on a stream not used before, with an image size not
    seen before, leaves the device's free memory unchanged: no workspace is created for the
    new stream and nothing is allocated (buffers and stream are made before the reading)."""
    plan = B.Plan(10.0, 255, 10.0, K=16)
    img = voronoi_image(256, 200, 10, 40.0, 10.0, seed=1)
    x = torch.from_numpy(img).cuda()
    y = torch.empty_like(x)
    st = torch.cuda.current_stream()
    B.fbf_filter_noalloc(plan.handle, x.data_ptr(), y.data_ptr(), 256, 200, 200, st.cuda_stream)
    st.synchronize()
    img2 = voronoi_image(900, 700, 30, 40.0, 10.0, seed=2)
    x2 = torch.from_numpy(img2).cuda()
    y2 = torch.full_like(x2, -1.0)
    ref = torch.full_like(x2, -1.0)
    side = torch.cuda.Stream()
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    B.fbf_filter_noalloc(plan.handle, x2.data_ptr(), y2.data_ptr(), 900, 700, 700, side.cuda_stream)
    side.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
    B.fbf_filter(plan.handle, x2.data_ptr(), ref.data_ptr(), 900, 700, 700, st.cuda_stream)
    st.synchronize()
    assert float((y2 - ref).abs().max()) <= TOL
