"""Oracle: range-kernel approximation and parameter optimisation (FP64, NumPy).

TEST INFRASTRUCTURE ONLY -- see the package docstring.  Parity pins: tests/test_oracle_pins.py.

Notation follows Section II of the paper:
  * phi(t) = exp(-t^2 / (2 sigma^2))                       eq. (2)
  * phi_hat(t) = sum_{k=0}^{K-1} c_k cos(2 pi k t/(2T+1))   eq. (3)
  * Lambda = {-R, ..., R}; b(i) = phi(i-R-1); A(i,j) = cos(nu (i-R-1)(j-1)), nu = 2 pi/(2T+1)
    (the definition of A and b in Section II, just before eq. (5))
  * E(K,T) = min_c ||A c - b||^2                             eq. (5), the error of eq. (4)
  * e(K) = min_{T in N} E(K,T)                               eq. (6)
  * Algorithm 1: smallest K with e(K) <= eps, and its T.

Readings where the paper is silent:
  * T_max is only "large" (Section II, text after Prop. 2): T_max = 4R; if the optimum sits
    above T_max/2 the scan is repeated with T_max doubled.
  * Round-off ties: for large K, E(K,T) reaches FP64 round-off for many T and the argmin
    becomes noise.  Errors are floored at ROUNDOFF_FLOOR_REL * ||b||^2 and, among the
    T that reach the minimum of the floored error, the smallest T is taken.  Algorithm 1's
    "<=" update takes the largest T on exact ties; exact ties above the floor do not occur
    in floating point, so the two differ only at the floor.
  * Rank deficiency (K > T+1: columns k and 2T+1-k coincide): minimum-norm least squares
    (NumPy lstsq).  phi_hat on Lambda is the same for every minimiser.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

ROUNDOFF_FLOOR_REL = 1e-20


def range_kernel(t, sigma: float):
    """Gaussian range kernel phi(t) = exp(-t^2/(2 sigma^2)), eq. (2)."""
    t = np.asarray(t, dtype=np.float64)
    return np.exp(-(t * t) / (2.0 * sigma * sigma))


def kernel_samples(sigma: float, R: int, kernel=None):
    """b(i) = phi(i - R - 1) for i = 1..2R+1, i.e. phi on Lambda = {-R..R} (Section II).

    ``kernel`` (optional) replaces the Gaussian by any even range kernel given as a
    callable of t; the paper notes the fit works for non-Gaussian kernels (Sections I, IV).
    """
    t = np.arange(-R, R + 1, dtype=np.float64)
    if kernel is None:
        return range_kernel(t, sigma)
    return np.asarray(kernel(t), dtype=np.float64)


def design_matrix(K: int, T: int, R: int):
    """A(i,j) = cos(nu (i-R-1)(j-1)), nu = 2 pi/(2T+1), size (2R+1) x K (Section II).

    t = i-R-1 and k = j-1 are integers, so the angle nu t k is reduced exactly, as the
    integer (t k) mod (2T+1) times nu.  Columns that coincide in exact arithmetic
    (k and 2T+1-k when K > T+1) then coincide in floating point too; evaluating cos at
    the unreduced angle leaves ~1e-13 differences that least squares would fit.
    """
    P = 2 * T + 1
    t = np.arange(-R, R + 1, dtype=np.int64)[:, None]
    k = np.arange(K, dtype=np.int64)[None, :]
    return np.cos((2.0 * math.pi / P) * np.mod(t * k, P).astype(np.float64))


def kernel_error(K: int, T: int, b, R: int):
    """E(K,T) = min_c ||A c - b||^2 (eq. 5) and a minimiser c (minimum norm).

    Returns (E, c).  E is recomputed from the residual rather than taken from lstsq,
    which returns no residual for rank-deficient A.
    """
    A = design_matrix(K, T, R)
    c, *_ = np.linalg.lstsq(A, b, rcond=None)
    res = A @ c - b
    return float(res @ res), c


def optimal_period(K: int, b, R: int, T_max: int | None = None):
    """e(K) = min_{T} E(K,T) over T = 1..T_max (eq. 6), with the floor/tie reading above.

    Returns (T_star, E_star, c_star, E_curve) where E_curve[T-1] = E(K,T).
    """
    if T_max is None:
        T_max = 4 * R
    floor = ROUNDOFF_FLOOR_REL * float(np.dot(b, b))
    while True:
        curve = np.empty(T_max)
        coefs = []
        for T in range(1, T_max + 1):
            E, c = kernel_error(K, T, b, R)
            curve[T - 1] = E
            coefs.append(c)
        floored = np.maximum(curve, floor)
        T_star = int(np.argmin(floored)) + 1          # first index = smallest T on ties
        if T_star <= T_max // 2:
            return T_star, float(curve[T_star - 1]), coefs[T_star - 1], curve
        T_max *= 2


def algorithm1(b, R: int, eps: float, T_max: int | None = None, K_limit: int | None = None):
    """Algorithm 1: smallest K with e(K) <= eps, the period T* reaching it, and e.

    The loop is the paper's: K = 1, 2, ...; for each K scan T = 1..T_max and keep the
    (K,T) whose error is <= min(e, eps).  The floor/tie reading of the module docstring
    replaces the "<=" tie rule at the floor.  Prop. 2 guarantees termination by K = 2R+1.
    """
    if eps <= 0:
        raise ValueError("eps must be positive")
    if K_limit is None:
        K_limit = 2 * R + 1
    floor = ROUNDOFF_FLOOR_REL * float(np.dot(b, b))
    K = 0
    e = math.inf
    best = None
    while e > eps:
        K += 1
        if K > K_limit:
            raise RuntimeError("Algorithm 1 did not reach eps within K_limit")
        T_star, E_star, c_star, _ = optimal_period(K, b, R, T_max)
        if max(E_star, floor) <= eps:
            e = E_star
            best = (K, T_star, E_star, c_star)
    return best


def phi_hat(t, c, T: int):
    """phi_hat(t) = sum_k c_k cos(2 pi k t/(2T+1)), eq. (3)."""
    t = np.asarray(t, dtype=np.float64)
    P = 2 * T + 1
    nu = 2.0 * math.pi / P
    integral = bool(np.all(t == np.round(t))) and t.size > 0 and np.max(np.abs(t)) < 2 ** 40
    out = np.zeros_like(t)
    for k, ck in enumerate(np.asarray(c, dtype=np.float64)):
        if integral:   # exact reduction of the angle, as in design_matrix
            ang = nu * np.mod(np.round(t).astype(np.int64) * k, P).astype(np.float64)
        else:
            ang = nu * k * t
        out = out + ck * np.cos(ang)
    return out


@dataclass
class OraclePlan:
    sigma: float
    R: int
    K: int
    T: int
    c: np.ndarray
    E: float
    delta_max: float = field(default=math.nan)

    @property
    def nu(self) -> float:
        return 2.0 * math.pi / (2 * self.T + 1)


def make_plan(sigma: float, R: int = 255, K: int | None = None, eps: float | None = None,
              kernel=None, T: int | None = None, T_max: int | None = None) -> OraclePlan:
    """(K, T, c) for the filter.

    * eps given, K None  -> Algorithm 1.
    * K given, T None    -> T = argmin_T E(K,T) (the Fig. 1 construction).
    * K and T given      -> only the least-squares step (eq. 5); T = R is the fixed-period
                            FBF model the paper compares against.
    delta_max = max over Lambda of |phi_hat - phi| (used by the Prop. 1 bound).
    """
    b = kernel_samples(sigma, R, kernel)
    if K is None:
        if eps is None:
            raise ValueError("give K or eps")
        K, T, E, c = algorithm1(b, R, eps, T_max)
    elif T is None:
        T, E, c, _ = optimal_period(K, b, R, T_max)
    else:
        E, c = kernel_error(K, T, b, R)
    t = np.arange(-R, R + 1, dtype=np.float64)
    delta = float(np.max(np.abs(phi_hat(t, c, T) - b)))
    return OraclePlan(sigma=sigma, R=R, K=int(K), T=int(T), c=np.asarray(c, np.float64),
                      E=float(E), delta_max=delta)
