"""A plan from the K*/T* lookup table (bilinear in (sigma, log 1/eps), Section II's closing
remark on Fig. 2), filtering on the GPU: the result equals the FP64 oracle's filter with the
looked-up K and T and the least-squares c at that T (eq. 5), in every precision form."""
import numpy as np
import pytest

from oracle import fit as ofit
from oracle import filters as ofl
from paper_1811_02168_gb300.synth import voronoi_image

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
TOL = {"fp32": 5e-3, "bf16_tc": 0.5, "fp16_tc": 0.5}


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1811_02168_gb300 import build
    build.build()
    from paper_1811_02168_gb300 import binding
    binding.lib()
    return binding


@pytest.mark.parametrize("form", ["fp32", "bf16_tc", "fp16_tc"])
def test_lut_plan_filters_like_the_oracle(B, form):
    prec = {"fp32": B.FBF_FP32, "bf16_tc": B.FBF_BF16_TC, "fp16_tc": B.FBF_FP16_TC}[form]
    lut = B.Lut(255, [10.0, 20.0, 40.0, 80.0], [0.1, 0.01, 0.001])
    sigma, eps, theta = 27.0, 0.004, 3.0                  # off the grid in both directions
    K, T = lut.lookup(sigma, eps)
    plan = lut.plan(sigma, eps, theta, precision=prec)
    assert (plan.K, plan.T) == (K, T)
    img = voronoi_image(180, 211, 12, 40.0, 10.0, seed=27)
    x = torch.from_numpy(img).cuda()
    y = torch.empty_like(x)
    B.fbf_filter(plan.handle, x.data_ptr(), y.data_ptr(), 180, 211, 211, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    op = ofit.make_plan(sigma, 255, K=K, T=T)
    ref = ofl.fourier_bf(img.astype(np.float64), theta, op.c, op.T)
    assert float(np.abs(y.cpu().numpy() - ref).max()) <= TOL[form]
    lut.close()
