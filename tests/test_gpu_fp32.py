"""GPU parity of the FP32 fused kernel against the FP64 oracle, through the C ABI.

Tolerance: max abs error <= 5e-3 gray levels (0..255 scale) against the FP64 Fourier
oracle.  Whole images are compared element by element at sizes the oracle finishes in
seconds (several tiles plus ragged tails); full-size workloads are compared on sampled
pixels that the oracle evaluates one by one (eq. (1) with phi_hat over each window).
"""
import numpy as np
import pytest

from oracle import fit as ofit
from oracle import filters as ofl
from paper_1811_02168_gb300.synth import (voronoi_image, workload_small, workload_sigma_sweep,
                                          workload_large)

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


def _gpu(B, plan, img, pitch=None, stream=None):
    H, W = img.shape
    if pitch is None or pitch == W:
        x = torch.from_numpy(np.ascontiguousarray(img, np.float32)).cuda()
        y = torch.full_like(x, -7.0)
        pe = W
    else:
        xb = torch.zeros((H, pitch), dtype=torch.float32, device="cuda")
        xb[:, :W] = torch.from_numpy(np.ascontiguousarray(img, np.float32)).cuda()
        x = xb
        y = torch.full((H, pitch), -7.0, dtype=torch.float32, device="cuda")
        pe = pitch
    st = stream or torch.cuda.current_stream()
    B.fbf_filter(plan.handle, x.data_ptr(), y.data_ptr(), H, W, pe, st.cuda_stream)
    st.synchronize()
    out = y.cpu().numpy()
    if pe != W:
        assert np.all(out[:, W:] == -7.0), "kernel wrote outside the image"
        out = out[:, :W]
    return out


def _oracle_plan(sigma, K=None, eps=None):
    return ofit.make_plan(sigma, 255, K=K, eps=eps)


def test_small_workload_whole_image(B):
    """256x256, theta 3, sigma 30, K 4: every pixel against the FP64 Fourier oracle."""
    job = workload_small()
    img = job.image()
    plan = B.Plan(job.sigma, 255, job.theta, K=job.K)
    op = _oracle_plan(job.sigma, K=job.K)
    assert (plan.K, plan.T) == (op.K, op.T)
    ref = ofl.fourier_bf(img.astype(np.float64), job.theta, op.c, op.T)
    out = _gpu(B, plan, img)
    err = np.abs(out - ref).max()
    assert err <= TOL, err


@pytest.mark.parametrize("sigma", [10.0, 30.0, 80.0])
def test_sigma_sweep_ragged_whole_image(B, sigma):
    """theta 5, K from eps 0.01 (the sigma sweep), on a 300 x 419 image: ragged in x and y."""
    img = voronoi_image(300, 419, 30, 40.0, 10.0, seed=101)
    plan = B.Plan(sigma, 255, 5.0, eps=0.01)
    op = _oracle_plan(sigma, eps=0.01)
    assert (plan.K, plan.T) == (op.K, op.T)
    ref = ofl.fourier_bf(img.astype(np.float64), 5.0, op.c, op.T)
    out = _gpu(B, plan, img)
    err = np.abs(out - ref).max()
    assert err <= TOL, (sigma, err)


def _sample_points(H, W, n, seed):
    rng = np.random.default_rng(seed)
    pts = [(0, 0), (0, W - 1), (H - 1, 0), (H - 1, W - 1), (H // 2, 0), (0, W // 2)]
    pts += list(zip(rng.integers(0, H, n), rng.integers(0, W, n)))
    return np.array(pts)


@pytest.mark.parametrize("sigma", [10.0, 30.0, 80.0])
def test_sigma_sweep_full_size_sampled(B, sigma):
    """The 1024 x 1024 sigma-sweep workload at full size, in the benchmark's launch
    configuration; 400 sampled pixels (corners and edges included) against eq. (1) with
    phi_hat evaluated directly over each pixel's window."""
    job = [j for j in workload_sigma_sweep() if j.sigma == sigma][0]
    img = job.image()
    plan = B.Plan(job.sigma, 255, job.theta, eps=job.eps)
    op = _oracle_plan(job.sigma, eps=job.eps)
    out = _gpu(B, plan, img)
    pts = _sample_points(job.H, job.W, 400, seed=int(sigma))
    ref = ofl.fourier_bf_at(img.astype(np.float64), job.theta, op.c, op.T, pts)
    err = np.abs(out[pts[:, 0], pts[:, 1]] - ref).max()
    assert err <= TOL, err
    assert np.isfinite(out).all()


def test_large_workload_sampled(B):
    """4096 x 4096, theta 10 (61 x 61 window), sigma 10, K 16: sampled pixels."""
    job = workload_large()
    img = job.image()
    plan = B.Plan(job.sigma, 255, job.theta, K=job.K)
    op = _oracle_plan(job.sigma, K=job.K)
    out = _gpu(B, plan, img)
    pts = _sample_points(job.H, job.W, 120, seed=5)
    ref = ofl.fourier_bf_at(img.astype(np.float64), job.theta, op.c, op.T, pts)
    err = np.abs(out[pts[:, 0], pts[:, 1]] - ref).max()
    assert err <= TOL, err


@pytest.mark.parametrize("H,W,theta", [(1, 1, 2.0), (1, 57, 3.0), (61, 1, 3.0), (5, 7, 5.0),
                                       (33, 31, 10.0), (130, 97, 1.5), (129, 65, 2.0),
                                       (70, 200, 16.0), (40, 45, 0.3)])
def test_edge_shapes(B, H, W, theta):
    """Degenerate and ragged shapes: single pixel, single row/column, images smaller than
    the window, a radius that uses a wider kernel instantiation (theta 1.5 -> r 5), the
    largest supported radius (theta 16 -> r 48), and r = 1."""
    img = voronoi_image(H, W, 5, 30.0, 10.0, seed=H * 1000 + W)
    plan = B.Plan(30.0, 255, theta, K=5)
    op = _oracle_plan(30.0, K=5)
    ref = ofl.fourier_bf(img.astype(np.float64), theta, op.c, op.T)
    out = _gpu(B, plan, img)
    err = np.abs(out - ref).max()
    assert err <= TOL, err


def test_pitch_larger_than_width(B):
    img = voronoi_image(77, 90, 8, 30.0, 10.0, seed=3)
    plan = B.Plan(30.0, 255, 3.0, K=6)
    op = _oracle_plan(30.0, K=6)
    ref = ofl.fourier_bf(img.astype(np.float64), 3.0, op.c, op.T)
    out = _gpu(B, plan, img, pitch=128)
    assert np.abs(out - ref).max() <= TOL


def test_constant_image_is_fixed_point(B):
    img = np.full((150, 170), 93.0, np.float32)
    plan = B.Plan(30.0, 255, 5.0, eps=0.01)
    out = _gpu(B, plan, img)
    assert np.abs(out - 93.0).max() <= 1e-3


def test_K1_is_normalised_gaussian_blur(B):
    """K = 1 reduces eq. (1) to the zero-padded normalised Gaussian blur."""
    img = voronoi_image(90, 110, 10, 30.0, 10.0, seed=9)
    plan = B.Plan(30.0, 255, 2.0, K=1)
    out = _gpu(B, plan, img)
    ref = ofl.gaussian_blur_normalised(img.astype(np.float64), 2.0)
    assert np.abs(out - ref).max() <= TOL


def test_fixed_period_fbf_model(B):
    """T = R (the fixed-period model the paper compares against)."""
    img = voronoi_image(64, 80, 8, 30.0, 10.0, seed=12)
    plan = B.Plan(40.0, 255, 3.0, K=4, flags=B.FBF_FLAG_FIXED_PERIOD)
    op = ofit.make_plan(40.0, 255, K=4, T=255)
    ref = ofl.fourier_bf(img.astype(np.float64), 3.0, op.c, op.T)
    assert np.abs(_gpu(B, plan, img) - ref).max() <= TOL


def test_non_gaussian_range_kernel(B):
    R, s = 255, 25.0
    kern = lambda t: np.exp(-np.abs(t) / s)  # noqa: E731
    img = voronoi_image(70, 66, 8, 30.0, 10.0, seed=13)
    plan = B.Plan(None, R, 3.0, K=10, samples=kern(np.arange(-R, R + 1)))
    op = ofit.make_plan(None, R, K=10, kernel=kern)
    ref = ofl.fourier_bf(img.astype(np.float64), 3.0, op.c, op.T)
    assert np.abs(_gpu(B, plan, img) - ref).max() <= TOL


def test_deterministic_and_side_stream(B):
    img = voronoi_image(200, 260, 20, 30.0, 10.0, seed=21)
    plan = B.Plan(10.0, 255, 5.0, eps=0.01)
    a = _gpu(B, plan, img)
    s = torch.cuda.Stream()
    b = _gpu(B, plan, img, stream=s)
    assert np.array_equal(a, b)


def test_host_end_to_end_api(B):
    """bilateral_filter: a host tensor takes the end-to-end call (page-locked, filtered by
    the kernel in host memory, returned on the host), a device tensor the device call; both
    give fbf_filter's bits."""
    img = voronoi_image(120, 140, 10, 30.0, 10.0, seed=4)
    plan = B.Plan(30.0, 255, 3.0, K=4)
    ref = _gpu(B, plan, img)
    res = B.bilateral_filter(plan, torch.from_numpy(img))
    assert not res.is_cuda
    assert np.array_equal(res.numpy(), ref)
    dev = B.bilateral_filter(plan, torch.from_numpy(img).cuda())
    assert dev.is_cuda
    assert np.array_equal(dev.cpu().numpy(), ref)


def test_non_integer_input_uses_the_general_phase_path(B):
    """Values that are not integers (Section II treats integer intensities; the library
    filters any float input with the same formula) against the oracle's cos(k nu f)."""
    rng = np.random.default_rng(31)
    img = (voronoi_image(150, 170, 12, 30.0, 10.0, seed=31) * 0.9 +
           rng.uniform(0.0, 0.999, (150, 170))).astype(np.float32)
    plan = B.Plan(20.0, 255, 3.0, K=8)
    op = _oracle_plan(20.0, K=8)
    ref = ofl.fourier_bf(img.astype(np.float64), 3.0, op.c, op.T)
    assert np.abs(_gpu(B, plan, img) - ref).max() <= TOL


def test_ten_bit_image(B):
    """R = 1023: intensities above the kernels' 256-entry term tables take the general
    phase path; the fit covers Lambda = {-1023..1023}."""
    R = 1023
    img = np.rint(voronoi_image(96, 130, 10, 30.0, 10.0, seed=7) * 4.0).clip(0, R).astype(np.float32)
    plan = B.Plan(120.0, R, 2.0, K=6)
    op = ofit.make_plan(120.0, R, K=6)
    assert (plan.K, plan.T) == (op.K, op.T)
    ref = ofl.fourier_bf(img.astype(np.float64), 2.0, op.c, op.T)
    assert np.abs(_gpu(B, plan, img) - ref).max() <= 4 * TOL   # scale: 4x the 8-bit range


@pytest.mark.parametrize("H,W,theta,K", [(2050, 1000, 10.0, 4), (2100, 760, 8.0, 5), (1640, 600, 16.0, 3)])
def test_carried_rows_whole_image(B, H, W, theta, K):
    """Images with at least three tiles per SM at r > 15 take the kernel that carries the
    x-pass halo rows down each strip (r = 30, 24 and 48 instantiations; ragged in x and y):
    every pixel against the FP64 oracle, and against the allocation-free entry point, which
    always convolves every halo row (the two differ only in where the split tiles' partial
    sums are cut)."""
    img = voronoi_image(H, W, 120, 40.0, 12.0, seed=H + W)
    plan = B.Plan(30.0, 255, theta, K=K)
    op = _oracle_plan(30.0, K=K)
    assert (plan.K, plan.T) == (op.K, op.T)
    ref = ofl.fourier_bf(img.astype(np.float64), theta, op.c, op.T)
    out = _gpu(B, plan, img)
    assert np.abs(out - ref).max() <= TOL
    x = torch.from_numpy(img).cuda()
    y = torch.full_like(x, -7.0)
    st = torch.cuda.current_stream()
    B.fbf_filter_noalloc(plan.handle, x.data_ptr(), y.data_ptr(), H, W, W, st.cuda_stream)
    st.synchronize()
    assert np.abs(y.cpu().numpy() - out).max() <= 1e-3


def test_carried_rows_mixed_phase_paths(B):
    """Carried rows cross from tiles with non-integer values (general phase path) into
    8-bit tiles (term tables) and back: every pixel against the oracle."""
    H, W = 2048, 1024
    img = voronoi_image(H, W, 100, 40.0, 10.0, seed=77)
    rng = np.random.default_rng(78)
    img[700:900] = (img[700:900] * 0.9 + rng.uniform(0.0, 0.999, (200, W))).astype(np.float32)
    plan = B.Plan(20.0, 255, 10.0, K=4)
    op = _oracle_plan(20.0, K=4)
    ref = ofl.fourier_bf(img.astype(np.float64), 10.0, op.c, op.T)
    assert np.abs(_gpu(B, plan, img) - ref).max() <= TOL
