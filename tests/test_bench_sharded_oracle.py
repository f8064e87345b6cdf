"""The CPU baseline's sharded oracle: row bands with r halo rows on spawned processes give
exactly the whole-image oracle (the halo covers every neighbour a kept row's window reads;
band edges that are image borders stay borders), for a sample of all rows and for a prefix
whose last band ends inside the image."""
import os
import sys
from types import SimpleNamespace

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402
from oracle import filters as ofl, fit as ofit  # noqa: E402
from paper_1811_02168_gb300.synth import voronoi_image  # noqa: E402


def test_row_bands_equal_whole_image_oracle():
    img = voronoi_image(53, 41, 9, 30.0, 10.0, seed=5)
    job = SimpleNamespace(theta=2.0, sigma=30.0, K=5, eps=None)
    plan = ofit.make_plan(job.sigma, 255, K=job.K)
    whole = ofl.fourier_bf(img.astype(np.float64), job.theta, plan.c, plan.T)
    sh = bench._ShardedOracle(3)
    try:
        out, dt = sh.run(img, job, 53)             # bands of 18, 18, 17 rows; r = 6
        assert out.shape == whole.shape and dt > 0
        assert np.array_equal(out, whole)
        part, _ = sh.run(img, job, 20)             # 3 bands of 7/7/6 rows, the last ends at row 20
        assert part.shape == (20, 41)
        assert np.array_equal(part, whole[:20])
    finally:
        sh.close()
