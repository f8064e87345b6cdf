"""FP64 CPU oracle for Optimized Fourier Bilateral Filtering (Ghosh, Nair, Chaudhury,
IEEE SPL 25(10), 2018).

TEST INFRASTRUCTURE ONLY.  Nothing in the product package imports, links or runs this
package; only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline legs of
``bench.py`` may.  It shares no code with the CUDA path: plain NumPy in float64, written
from the paper's equations, slow on purpose and easy to check by eye.

Modules
  fit      -- eq. (2) range kernel samples, eq. (3) cosine series, eq. (4)/(5) kernel
              error and least squares, eq. (6) period optimisation, Algorithm 1.
  filters  -- eq. (1) brute-force bilateral filter, the Fourier (channel) form of eq. (1)
              with the approximated range kernel, a per-pixel sampler, PSNR.

Every function is pinned by ``tests/test_oracle_pins.py`` against what the paper or the
mathematics fixes (Fig. 1's argmin, Prop. 2, closed forms, library routines, invariants).
"""
from .fit import (range_kernel, kernel_samples, design_matrix, kernel_error,
                  optimal_period, algorithm1, make_plan, phi_hat, OraclePlan,
                  ROUNDOFF_FLOOR_REL)
from .filters import (spatial_radius, spatial_taps, brute_bf, fourier_bf,
                      fourier_bf_at, brute_bf_at, gaussian_blur_normalised, psnr,
                      prop1_bound)

__all__ = [
    "range_kernel", "kernel_samples", "design_matrix", "kernel_error", "optimal_period",
    "algorithm1", "make_plan", "phi_hat", "OraclePlan", "ROUNDOFF_FLOOR_REL",
    "spatial_radius", "spatial_taps", "brute_bf", "fourier_bf", "fourier_bf_at",
    "brute_bf_at", "gaussian_blur_normalised", "psnr", "prop1_bound",
]
