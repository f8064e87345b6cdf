"""The kernels' bounded waits giving up, on the GPU, without any fault: a test hook
(fbf_debug_set_wait_limit) turns the waits inside each kernel's own pipeline into a few
non-blocking polls, so that they run out.  Each launch must then return, report its bit in
fbf_device_errors (bit 1: the FP32 kernel's wait for a TMA box of the f halo; bit 0: a
tensor-core kernel's mbarrier wait), leave the context usable and its tensor memory freed,
and the next normal call must be clean and match the FP64 oracle."""
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


def _filter(B, plan, x):
    y = torch.full_like(x, -1.0)
    H, W = x.shape
    st = torch.cuda.current_stream()
    B.fbf_filter(plan.handle, x.data_ptr(), y.data_ptr(), H, W, W, st.cuda_stream)
    st.synchronize()
    return y


def _gave_up(B, run):
    """Run `run` with the pipeline waits limited to one poll; return the error word."""
    assert B.fbf_device_errors(True) == 0
    B.fbf_debug_set_wait_limit(1)
    try:
        run()
        torch.cuda.synchronize()
    finally:
        B.fbf_debug_set_wait_limit(0)
    return B.fbf_device_errors(True)


@pytest.mark.parametrize("form,bit,tol", [("fp32", 2, 5e-3), ("bf16_tc", 1, 0.5), ("fp16_tc", 1, 0.5)])
def test_single_image_waits_give_up_then_clean(B, form, bit, tol):
    prec = {"fp32": B.FBF_FP32, "bf16_tc": B.FBF_BF16_TC, "fp16_tc": B.FBF_FP16_TC}[form]
    img = voronoi_image(512, 512, 60, 40.0, 10.0, seed=91)     # r = 15: the FP32 form stages by TMA
    plan = B.Plan(30.0, 255, 5.0, eps=0.01, precision=prec)
    x = torch.from_numpy(img).cuda()
    flags = _gave_up(B, lambda: _filter(B, plan, x))
    assert flags & bit, flags
    y = _filter(B, plan, x)                                      # normal limits again
    assert B.fbf_device_errors(True) == 0
    op = ofit.make_plan(30.0, 255, eps=0.01)
    ref = ofl.fourier_bf(img.astype(np.float64), 5.0, op.c, op.T)
    assert float(np.abs(y.cpu().numpy() - ref).max()) <= tol


def test_batched_tensor_core_wait_gives_up_then_clean(B):
    """The work-list tensor-core kernel (a batch of BF16_TC plans); a batch whose launch
    gave up is replaced by a new one (its split-tile counters are left behind)."""
    imgs = [voronoi_image(300 + 37 * i, 260, 20, 40.0, 10.0, seed=95 + i) for i in range(3)]
    plan = B.Plan(30.0, 255, 2.0, K=5, precision=B.FBF_BF16_TC)
    xs = [torch.from_numpy(im).cuda() for im in imgs]

    def launch():
        batch = B.Batch(4)
        ys = [torch.full_like(x, -1.0) for x in xs]
        t = 0
        for x, y in zip(xs, ys):
            t = batch.submit(plan, x, y)
        batch.launch()
        batch.wait(t, 60.0)
        batch.close()
        return ys

    assert _gave_up(B, launch) & 1
    ys = launch()
    assert B.fbf_device_errors(True) == 0
    op = ofit.make_plan(30.0, 255, K=5)
    for im, y in zip(imgs, ys):
        ref = ofl.fourier_bf(im.astype(np.float64), 2.0, op.c, op.T)
        assert float(np.abs(y.cpu().numpy() - ref).max()) <= 0.5
