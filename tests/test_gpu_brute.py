"""Direct eq. (1) kernel (fbf_brute_filter) against the FP64 oracle's brute force, through the
C ABI; and the PSNR of the Fourier filter against it (Section III).

Tolerance 2e-3 gray levels: FP32 sums of up to (2r+1)^2 = 961 weighted terms (the FP32 form's
5e-3 bound is for the same arithmetic depth)."""
import numpy as np
import pytest

from oracle import filters as ofl
from oracle import fit as ofit
from paper_1811_02168_gb300.synth import voronoi_image

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
TOL = 2e-3


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1811_02168_gb300 import build
    build.build()
    from paper_1811_02168_gb300 import binding
    binding.lib()
    return binding


def _brute(B, img, theta, sigma, R=255):
    x = torch.from_numpy(np.ascontiguousarray(img, np.float32)).cuda()
    y = torch.full_like(x, -9.0)
    H, W = img.shape
    B.fbf_brute_filter(x.data_ptr(), y.data_ptr(), H, W, W, theta, sigma, R, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return y.cpu().numpy()


@pytest.mark.parametrize("shape,theta,sigma", [((64, 80), 2.0, 30.0), ((33, 47), 1.0, 10.0), ((70, 66), 3.3, 80.0),
                                               ((1, 1), 2.0, 30.0), ((5, 200), 5.0, 20.0), ((97, 41), 5.0, 50.0)])
def test_brute_against_oracle(B, shape, theta, sigma):
    img = voronoi_image(shape[0], shape[1], 9, 40.0, 10.0, seed=shape[0] * 3 + shape[1])
    ref = ofl.brute_bf(img.astype(np.float64), theta, sigma)
    out = _brute(B, img, theta, sigma)
    assert float(np.abs(out - ref).max()) <= TOL


def test_brute_interior_tiles(B):
    # tiles whose window lies inside the image take the table path without bounds checks
    img = voronoi_image(160, 150, 20, 40.0, 10.0, seed=11)
    ref = ofl.brute_bf(img.astype(np.float64), 2.0, 25.0)
    assert float(np.abs(_brute(B, img, 2.0, 25.0) - ref).max()) <= TOL


def test_brute_non_integer_and_wide_range(B):
    rng = np.random.default_rng(4)
    img = (voronoi_image(60, 75, 9, 30.0, 10.0, seed=5) + rng.uniform(0, 0.999, (60, 75))).astype(np.float32)
    ref = ofl.brute_bf(img.astype(np.float64), 2.0, 30.0)
    assert float(np.abs(_brute(B, img, 2.0, 30.0) - ref).max()) <= TOL
    # 12-bit integer data: values above the table range take the expf path
    img12 = np.rint(voronoi_image(50, 64, 9, 40.0, 10.0, seed=6) * 16.0).astype(np.float32)
    ref12 = ofl.brute_bf(img12.astype(np.float64), 1.5, 300.0)
    out12 = _brute(B, img12, 1.5, 300.0, R=4095)
    assert float(np.abs(out12 - ref12).max()) <= 16 * TOL


def test_brute_large_sampled(B):
    img = voronoi_image(1024, 1024, 200, 40.0, 10.0, seed=1000)
    out = _brute(B, img, 5.0, 30.0)
    rng = np.random.default_rng(9)
    pts = [(int(a), int(b)) for a, b in zip(rng.integers(0, 1024, 150), rng.integers(0, 1024, 150))]
    pts += [(0, 0), (1023, 1023), (0, 1023), (1023, 0), (511, 0), (15, 16), (1008, 500)]
    ref = ofl.brute_bf_at(img.astype(np.float64), 5.0, 30.0, pts)
    got = np.array([out[p] for p in pts])
    assert float(np.abs(got - ref).max()) <= TOL


def test_fourier_psnr_against_brute(B):
    """PSNR of the FP32 Fourier filter against the GPU brute force equals the FP64 oracle's
    PSNR of fourier_bf against brute_bf (Section III's accuracy measure)."""
    img = voronoi_image(128, 160, 15, 40.0, 10.0, seed=21)
    theta, sigma, K = 3.0, 30.0, 5
    plan = B.Plan(sigma, 255, theta, K=K)
    x = torch.from_numpy(img).cuda()
    y = torch.empty_like(x)
    B.fbf_filter(plan.handle, x.data_ptr(), y.data_ptr(), 128, 160, 160, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    gpu = ofl.psnr(y.cpu().numpy(), _brute(B, img, theta, sigma))
    op = ofit.make_plan(sigma, 255, K=K)
    cpu = ofl.psnr(ofl.fourier_bf(img.astype(np.float64), theta, op.c, op.T), ofl.brute_bf(img.astype(np.float64), theta, sigma))
    assert gpu > 40.0
    assert abs(gpu - cpu) < 0.05, (gpu, cpu)
