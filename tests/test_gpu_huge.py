"""An image with more pixels than a 32-bit index holds (32768 x 70000 = 2.29e9), in every form,
sampled against eq. (1) with phi_hat evaluated directly (the oracle's per-pixel form).  The
image is a 1024 x 1024 Voronoi mosaic tiled over the plane plus a coarse ramp, so that it is
cheap to build but not periodic in the tile; 9.2 GB per buffer on the device."""
import numpy as np
import pytest

from oracle import fit as ofit
from oracle import filters as ofl
from paper_1811_02168_gb300.synth import voronoi_image

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
H, W = 32768, 70000


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    free, _ = torch.cuda.mem_get_info()
    if free < 24 * (1 << 30):
        pytest.skip("needs 24 GB of free device memory")
    from paper_1811_02168_gb300 import build
    build.build()
    from paper_1811_02168_gb300 import binding
    binding.lib()
    return binding


@pytest.fixture(scope="module")
def image():
    base = torch.from_numpy(voronoi_image(1024, 1024, 60, 0.0, 8.0, seed=77)).cuda()
    x = base.repeat(H // 1024, (W + 1023) // 1024)[:, :W].contiguous()
    ramp = (torch.arange(W, device="cuda", dtype=torch.float32) * (40.0 / W)).floor()
    x = torch.clamp(x + ramp[None, :], 0.0, 255.0)
    assert x.numel() > 2 ** 31
    return x


def _points():
    rng = np.random.default_rng(11)
    pts = [(int(a), int(b)) for a, b in zip(rng.integers(0, H, 40), rng.integers(0, W, 40))]
    pts += [(0, 0), (H - 1, W - 1), (H - 1, 0), (0, W - 1), (H // 2, W - 1), (30000, 65535),
            (32767, 65536), (16384, 65600)]
    return pts


@pytest.mark.parametrize("form,tol", [("fp32", 5e-3), ("fp16_tc", 0.5), ("bf16_tc", 0.5)])
def test_beyond_32_bit_pixel_indices(B, image, form, tol):
    prec = {"fp32": B.FBF_FP32, "fp16_tc": B.FBF_FP16_TC, "bf16_tc": B.FBF_BF16_TC}[form]
    theta, sigma, K = 3.0, 30.0, 4
    plan = B.Plan(sigma, 255, theta, K=K, precision=prec)
    y = torch.empty_like(image)
    B.fbf_filter(plan.handle, image.data_ptr(), y.data_ptr(), H, W, W, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert B.fbf_device_errors(True) == 0
    pts = _points()
    r = ofl.spatial_radius(theta)
    op = ofit.make_plan(sigma, 255, K=K)
    for (py, px) in pts:
        y0, y1, x0, x1 = max(0, py - r), min(H, py + r + 1), max(0, px - r), min(W, px + r + 1)
        win = image[y0:y1, x0:x1].cpu().numpy().astype(np.float64)
        # the (2r+1)^2 window around the point, cut at the image border like the image itself:
        # eq. (1) at the point sees exactly these neighbours
        ref = ofl.fourier_bf_at(win, theta, op.c, op.T, [(py - y0, px - x0)])[0]
        got = float(y[py, px])
        assert abs(got - ref) <= tol, (form, py, px, got, ref)
    del y
