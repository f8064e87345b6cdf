"""The FP32 kernel's two ways of staging the f halo give the same bits.

Single images at r <= 15 whose base address and row stride are 16-byte aligned are staged
by TMA (a 2-D tensor map of the image, the next tile's box loaded while the current tile is
filtered, elements outside the image arriving as NaN); other images by plain loads.  The
arithmetic after staging is the same, so the outputs must be identical bit for bit, and
both within the FP32 tolerance of the FP64 oracle.  Cases: a packed image whose width is
not a multiple of 4 (plain) against the same image at a padded pitch (TMA), and a base
pointer one float past a 16-byte boundary (plain) against an aligned one (TMA); radii 3 to
15, borders on every side, several tiles per CTA and split tiles.
"""
import numpy as np
import pytest

from oracle import fit as ofit
from oracle import filters as ofl
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


def _run(B, plan, img, pitch, offset):
    """Filter img stored at row stride `pitch` starting `offset` floats into a buffer."""
    H, W = img.shape
    buf = torch.full((offset + H * pitch + 8,), -5.0, dtype=torch.float32, device="cuda")
    view = buf[offset:offset + H * pitch].view(H, pitch)
    view[:, :W] = torch.from_numpy(np.ascontiguousarray(img, np.float32)).cuda()
    out = torch.full((offset + H * pitch + 8,), -7.0, dtype=torch.float32, device="cuda")
    oview = out[offset:offset + H * pitch].view(H, pitch)
    st = torch.cuda.current_stream()
    B.fbf_filter(plan.handle, view.data_ptr(), oview.data_ptr(), H, W, pitch, st.cuda_stream)
    st.synchronize()
    o = out.cpu().numpy()
    assert np.all(o[:offset] == -7.0) and np.all(o[offset + H * pitch:] == -7.0)
    res = oview.cpu().numpy()
    if pitch > W:
        assert np.all(res[:, W:] == -7.0), "kernel wrote outside the image"
    return res[:, :W]


@pytest.mark.parametrize("theta,sigma,K,H,W", [
    (1.0, 30.0, 4, 150, 131),     # r = 3
    (2.0, 20.0, 5, 233, 203),     # r = 6
    (3.0, 30.0, 6, 211, 157),     # r = 9
    (5.0, 10.0, 12, 301, 259),    # r = 15, K = 12 (many split tiles)
    (5.0, 80.0, 4, 97, 45),       # r = 15, a single column of tiles, halo past both sides
])
def test_tma_and_plain_staging_agree(B, theta, sigma, K, H, W):
    img = voronoi_image(H, W, 12, 40.0, 10.0, seed=int(100 * theta + sigma + K))
    plan = B.Plan(sigma, 255, theta, K=K)
    assert W % 4 != 0
    packed = _run(B, plan, img, W, 0)                  # row stride not 16-byte aligned: plain
    pitched = _run(B, plan, img, (W + 3) // 4 * 4, 0)  # aligned: TMA
    shifted = _run(B, plan, img, (W + 3) // 4 * 4, 1)  # base 4 bytes past alignment: plain
    assert np.array_equal(packed, pitched)
    assert np.array_equal(shifted, pitched)
    assert B.fbf_device_errors(True) == 0
    op = ofit.make_plan(sigma, 255, K=K)
    ref = ofl.fourier_bf(img.astype(np.float64), theta, op.c, op.T)
    assert float(np.abs(pitched - ref).max()) <= TOL


def test_tma_non_integer_image(B):
    """Non-integer values take the sincospi path; NaN-marked outside pixels must still count
    as absent there."""
    rng = np.random.default_rng(5)
    img = (voronoi_image(120, 100, 9, 30.0, 10.0, seed=9) + rng.uniform(-0.5, 0.5, (120, 100))).clip(0, 255)
    img = img.astype(np.float32)
    plan = B.Plan(30.0, 255, 4.0, K=6)
    pitched = _run(B, plan, img, 100, 0)               # aligned: TMA
    packed = _run(B, plan, img[:, :99].copy(), 99, 0)  # plain, one column narrower
    op = ofit.make_plan(30.0, 255, K=6)
    ref = ofl.fourier_bf(img.astype(np.float64), 4.0, op.c, op.T)
    ref99 = ofl.fourier_bf(img[:, :99].astype(np.float64), 4.0, op.c, op.T)
    assert float(np.abs(pitched - ref).max()) <= TOL
    assert float(np.abs(packed - ref99).max()) <= TOL


@pytest.mark.parametrize("H,W,theta", [(1, 4, 2.0), (2, 8, 3.0), (61, 4, 3.0), (5, 8, 5.0),
                                       (3, 200, 5.0), (33, 32, 5.0), (130, 96, 1.5)])
def test_tma_edge_shapes(B, H, W, theta):
    """Degenerate shapes on the TMA path (aligned rows, r <= 15): a single row, images
    smaller than the window and than one box, so that most of each box is outside the image
    (NaN-filled); bit-identical to the plain staging and within the tolerance of the oracle."""
    img = voronoi_image(H, W, 5, 30.0, 10.0, seed=H * 1000 + W + 7)
    plan = B.Plan(30.0, 255, theta, K=5)
    tma = _run(B, plan, img, W, 0)          # aligned: TMA
    plain = _run(B, plan, img, W, 1)        # base one float past alignment: plain
    assert np.array_equal(tma, plain)
    op = ofit.make_plan(30.0, 255, K=5)
    ref = ofl.fourier_bf(img.astype(np.float64), theta, op.c, op.T)
    assert float(np.abs(tma - ref).max()) <= TOL
