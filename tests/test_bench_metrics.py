"""The bench's roofline arithmetic (host only): the algorithmic work per pixel, the FP32
peak from unit counts and clock, the dense tensor-core work, and which FP32 instantiation a
workload runs."""
import os
import sys
from types import SimpleNamespace

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_flops_per_pixel_formula():
    """F(K, r) = 4 (4K - 3)(2r + 1) + 16K: 4K - 3 blurred images (k = 0 has f and the
    constant image; k >= 1 four images, the constant image's blur being one of k = 0's),
    two separable passes of 2r + 1 taps at 2 flop, plus generation and recombination."""
    assert bench._flops_per_px(16, 30) == 4 * 61 * 61 + 256 == 15140
    assert bench._flops_per_px(12, 15) == 4 * 45 * 31 + 192 == 5772
    assert bench._flops_per_px(4, 15) == 4 * 13 * 31 + 64 == 1676
    assert bench._flops_per_px(1, 3) == 4 * 1 * 7 + 16


def test_fp32_peak_is_units_times_clock():
    peak, src = bench._fp32_peak_tflops(152)
    mhz = float(src.split(" x ")[-1].split(" MHz")[0])
    assert abs(peak - 152 * 128 * 2 * mhz * 1e6 / 1e12) < 1e-9
    assert 60.0 < peak < 90.0          # GB300: about 80.5 TFLOP/s at 2070 MHz


def test_dense_tensor_work_counts_padding_and_compensation():
    """One 128 x 64 tile, K = 1 (one image pair): x pass M 128 x N KY x K KX and y pass
    M 128 x N 64 x K KY per image, TF32 y pass counted twice; the compensated form adds
    two x-pass products and an FP16 y pass."""
    r = 15
    kx = (128 + 2 * r + 15) // 16 * 16
    ky = (64 + 2 * r + 15) // 16 * 16
    x = 2 * 128 * ky * kx
    y = 2 * (2 * 128 * 64 * ky)
    # K = 1: 4K - 2 = 2 images (the pair (1, f - m)); one tile
    assert bench._tc_mma_flops(1, r, 64, 128) == 2 * (x + y)
    comp = bench._tc_mma_flops(1, r, 64, 128, compensated=True)
    assert comp == 2 * (3 * x + y + 2 * 128 * 64 * ky)
    # H = 128, W = 256: 2 x 2 tiles of 128 (x) by 64 (y); K = 4: 14 images
    assert bench._tc_mma_flops(4, r, 128, 256) == 4 * (4 * 4 - 2) * (x + y)


def test_fp32_instantiation_name():
    plan15 = SimpleNamespace(radius=15)
    plan30 = SimpleNamespace(radius=30)
    job = SimpleNamespace(W=1024, H=1024)
    odd = SimpleNamespace(W=1023, H=1024)
    assert bench._fp32_kernel_name([plan15], [job]) == "fbf_fp32_tma_kernel"
    assert bench._fp32_kernel_name([plan30], [job]) == "fbf_fp32_kernel"
    assert bench._fp32_kernel_name([plan15], [odd]) == "fbf_fp32_kernel"
    # r > 15 with at least three 32 x 96 tiles per SM: rows carried down the strips; r <= 15
    # never carries
    big = SimpleNamespace(W=4096, H=4096)
    assert bench._fp32_kernel_name([plan30], [big]) == "fbf_fp32_carry_kernel"
    assert bench._fp32_kernel_name([plan30], [big], sm_count=2000) == "fbf_fp32_kernel"
    assert bench._fp32_kernel_name([plan15], [big]) == "fbf_fp32_tma_kernel"
    assert bench._fp32_kernel_name([SimpleNamespace(radius=9)], [big]) == "fbf_fp32_tma_kernel"


def test_serve_size_classes_cover_every_request():
    """The serving workload generates one image per size-class pair for the whole grid, so any
    request side the Poisson stream, the backlog or a rate sweep draws snaps to a generated
    class (a short run once drew a class the stream and backlog had not)."""
    import numpy as np
    grid = bench._size_classes(512, 4096, 12)
    assert grid[0] == 512 and grid[-1] == 4096 and len(set(grid)) == 12
    assert all(a < b for a, b in zip(grid, grid[1:]))
    rng = np.random.default_rng(0)
    for v in np.exp(rng.uniform(np.log(512), np.log(4096), 2000)):
        assert bench._snap_log(float(v), 512, 4096, 12) in grid


def test_host_sampler_records_load_and_stops():
    """The serving bench's host sampler (load average, CPU clocks where exposed) samples once
    a second on its own thread and stops on request."""
    import time
    h = bench.HostSampler()
    h.start()
    time.sleep(1.3)
    rec = h.stop()
    assert rec["samples"] >= 1 and rec["load1_max"] >= 0.0
    assert rec["cpu_mhz_median"] is None or rec["cpu_mhz_median"] > 0
