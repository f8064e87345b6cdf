"""fbf_filter_host (host memory in, host memory out: read and written by the kernel directly
for distinct page-locked buffers, else staged in bands with the copies overlapped) gives
fbf_filter's result.  Bands are whole tile rows and each band's launch reads its halo
rows from the whole image, so the only difference from one launch over the whole image is
the order of split-tile partial sums (stream-K splits fall elsewhere).  Each result is
within its own rounding error of the exact one, which small bilateral denominators amplify
(FP32: 5.8e-4 against the FP64 oracle on the sigma sweep), so the two may differ by that
much: the bound is 1e-3 gray levels for FP32, a fifth of its tolerance (observed: 2e-4),
and 1e-2 for the tensor-core forms, whose errors against the oracle are larger (up to 4.2
for FP16_TC at r = 30; observed difference 1.2e-3).
Cases: page-locked (direct), in place and pageable (staged: one band and several, a ragged
last band, widths that are not a multiple of 4 so the device rows are padded), a host pitch
above the width, FP32 and the tensor-core forms; one case also against the FP64 oracle."""
import numpy as np
import pytest

from oracle import fit as ofit
from oracle import filters as ofl
from paper_1811_02168_gb300.synth import voronoi_image

pytestmark = pytest.mark.gpu
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


def _device(B, plan, img):
    x = torch.from_numpy(img).cuda()
    y = torch.empty_like(x)
    st = torch.cuda.current_stream()
    B.fbf_filter(plan.handle, x.data_ptr(), y.data_ptr(), img.shape[0], img.shape[1], img.shape[1],
                 st.cuda_stream)
    st.synchronize()
    return y.cpu().numpy()


def _host(B, plan, img, pitch=None, inplace=False, pinned=True):
    """pinned: the kernel reads and writes the host buffers directly; pageable (or in place):
    the image is staged through device memory in bands."""
    H, W = img.shape
    pitch = pitch or W
    src = torch.full((H, pitch), -3.0)
    src = src.pin_memory() if pinned else src
    src[:, :W] = torch.from_numpy(img)
    dst = src if inplace else torch.full((H, pitch), -9.0)
    dst = dst.pin_memory() if (pinned and not inplace) else dst
    B.fbf_filter_host(plan.handle, src.data_ptr(), dst.data_ptr(), H, W, pitch,
                      torch.cuda.current_stream().cuda_stream)
    out = dst.numpy()
    if not inplace and pitch > W:
        assert np.all(out[:, W:] == -9.0), "wrote outside the image"
    return out[:, :W].copy()


@pytest.mark.parametrize("prec", ["fp32", "bf16_tc", "fp16_tc"])
@pytest.mark.parametrize("theta,sigma,K,H,W", [
    (2.0, 30.0, 4, 200, 131),       # one band (r = 6)
    (5.0, 10.0, 12, 2300, 2050),    # r = 15: FP32 4 bands, tensor-core forms 2; width not a multiple of 4
    (10.0, 10.0, 16, 2085, 4099),   # r = 30: FP32 4 bands, tensor-core forms 3; ragged last band
    (10.0, 30.0, 8, 4096, 1024),    # r = 30, FP32: bands of 1408 rows (11 x 128) whose launches
                                    # carry rows in 96-row tiles, the last tile row past the band
])
def test_host_call_equals_device_call(B, prec, theta, sigma, K, H, W):
    form = {"fp32": B.FBF_FP32, "bf16_tc": B.FBF_BF16_TC, "fp16_tc": B.FBF_FP16_TC}[prec]
    img = voronoi_image(H, W, 20, 40.0, 10.0, seed=H + W)
    plan = B.Plan(sigma, 255, theta, K=K, precision=form)
    ref = _device(B, plan, img)
    got = _host(B, plan, img)
    tol = (1e-3 if prec == "fp32" else 1e-2) * max(1.0, float(np.abs(ref).max()) / 255.0)
    assert float(np.abs(got - ref).max()) <= tol
    got = _host(B, plan, img, pitch=W + 13)
    assert float(np.abs(got - ref).max()) <= tol
    got = _host(B, plan, img, inplace=True)
    assert float(np.abs(got - ref).max()) <= tol
    got = _host(B, plan, img, pitch=W + 3, pinned=False)
    assert float(np.abs(got - ref).max()) <= tol
    assert B.fbf_device_errors(True) == 0


def test_host_call_against_oracle(B):
    img = voronoi_image(700, 150, 15, 40.0, 10.0, seed=31)
    plan = B.Plan(30.0, 255, 4.0, K=6)
    got = _host(B, plan, img)
    op = ofit.make_plan(30.0, 255, K=6)
    ref = ofl.fourier_bf(img.astype(np.float64), 4.0, op.c, op.T)
    assert float(np.abs(got - ref).max()) <= 5e-3


def test_host_call_rejects_partial_overlap(B):
    plan = B.Plan(30.0, 255, 2.0, K=4)
    buf = torch.zeros(64 * 64 + 64).pin_memory()
    with pytest.raises(B.FbfError) as e:
        B.fbf_filter_host(plan.handle, buf.data_ptr(), buf.data_ptr() + 4 * 64, 64, 64, 64,
                          torch.cuda.current_stream().cuda_stream)
    assert e.value.code == B.FBF_EINVAL
