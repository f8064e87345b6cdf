"""Oracle: bilateral filtering in FP64 (NumPy).

TEST INFRASTRUCTURE ONLY -- see the package docstring.  Parity pins: tests/test_oracle_pins.py.

  * brute_bf       -- eq. (1) with the kernels of eq. (2), evaluated directly over the
                      square window |j_x|, |j_y| <= r, r = ceil(3 theta) (the (6 theta+1)^2
                      window whose cost Section I states).
  * fourier_bf     -- eq. (1) with phi replaced by phi_hat of eq. (3).  Expanding
                      cos(k nu (f(i-j) - f(i))) = cos(k nu f(i-j)) cos(k nu f(i))
                                               + sin(k nu f(i-j)) sin(k nu f(i))
                      turns numerator and denominator into Gaussian convolutions of the
                      images cos(k nu f), sin(k nu f), f cos(k nu f), f sin(k nu f) (Section II,
                      the remark after eq. (3)).  Each convolution is done here as a plain
                      separable shift-and-add over the 2r+1 taps.
  * fourier_bf_at  -- the same quantity at a list of pixels, by evaluating eq. (1) with
                      phi_hat directly over each pixel's window (for sampled checks of large
                      images).
  * psnr           -- 10 log10(255^2 / MSE) (Section III).

Readings where the paper is silent: neighbours outside the image are absent from both sums of
eq. (1), which is zero padding of every channel including the constant one; a pixel whose
denominator is <= 0 keeps its input value.
"""
from __future__ import annotations

import math

import numpy as np

from .fit import range_kernel, phi_hat


def spatial_radius(theta: float) -> int:
    """r = ceil(3 theta): the window is (2r+1)^2 = (6 theta + 1)^2 for integer theta."""
    return int(math.ceil(3.0 * theta - 1e-12))


def spatial_taps(theta: float):
    """g(x) = exp(-x^2/(2 theta^2)) for |x| <= r; omega(j) = g(j_x) g(j_y) (eq. 2)."""
    r = spatial_radius(theta)
    x = np.arange(-r, r + 1, dtype=np.float64)
    return np.exp(-(x * x) / (2.0 * theta * theta))


def _shift(img, dy: int, dx: int):
    """out(y,x) = img(y-dy, x-dx) with zeros where (y-dy, x-dx) is outside the image."""
    H, W = img.shape
    out = np.zeros_like(img)
    ys, yd = (slice(0, H - dy), slice(dy, H)) if dy >= 0 else (slice(-dy, H), slice(0, H + dy))
    xs, xd = (slice(0, W - dx), slice(dx, W)) if dx >= 0 else (slice(-dx, W), slice(0, W + dx))
    if (ys.stop - ys.start) > 0 and (xs.stop - xs.start) > 0:
        out[yd, xd] = img[ys, xs]
    return out


def _gauss_conv(img, g):
    """sum_j omega(j) img(i - j) with omega(j) = g(j_x) g(j_y): x pass then y pass."""
    r = (len(g) - 1) // 2
    tmp = np.zeros_like(img)
    for jx in range(-r, r + 1):
        tmp += g[jx + r] * _shift(img, 0, jx)
    out = np.zeros_like(img)
    for jy in range(-r, r + 1):
        out += g[jy + r] * _shift(tmp, jy, 0)
    return out


def brute_bf(f, theta: float, sigma: float | None = None, range_fn=None):
    """Eq. (1) by direct summation over the (2r+1)^2 window.

    range_fn(t) is the range kernel; default the Gaussian phi of eq. (2) with ``sigma``.
    Returns the filtered image (float64).
    """
    f = np.asarray(f, dtype=np.float64)
    if range_fn is None:
        range_fn = lambda t: range_kernel(t, sigma)  # noqa: E731
    g = spatial_taps(theta)
    r = (len(g) - 1) // 2
    ones = np.ones_like(f)
    num = np.zeros_like(f)
    den = np.zeros_like(f)
    for jy in range(-r, r + 1):
        for jx in range(-r, r + 1):
            fj = _shift(f, jy, jx)            # f(i - j)
            inside = _shift(ones, jy, jx)     # 1 where i - j is in the image
            w = g[jy + r] * g[jx + r] * range_fn(fj - f) * inside
            num += w * fj
            den += w
    return np.where(den > 0, num / np.where(den > 0, den, 1.0), f)


def fourier_bf(f, theta: float, c, T: int, return_parts: bool = False):
    """Eq. (1) with phi_hat (eq. 3) as range kernel, via Gaussian convolutions (Section II).

    num(i) = sum_k c_k [cos(k nu f(i)) (omega*(f cos(k nu f)))(i) + sin(k nu f(i)) (omega*(f sin(k nu f)))(i)]
    den(i) = sum_k c_k [cos(k nu f(i)) (omega*cos(k nu f))(i)     + sin(k nu f(i)) (omega*sin(k nu f))(i)]
    with nu = 2 pi/(2T+1) and * the zero-padded convolution.  Output num/den.
    """
    f = np.asarray(f, dtype=np.float64)
    c = np.asarray(c, dtype=np.float64)
    g = spatial_taps(theta)
    nu = 2.0 * math.pi / (2 * T + 1)
    num = np.zeros_like(f)
    den = np.zeros_like(f)
    for k, ck in enumerate(c):
        C = np.cos(k * nu * f)
        S = np.sin(k * nu * f)
        num += ck * (C * _gauss_conv(f * C, g) + S * _gauss_conv(f * S, g))
        den += ck * (C * _gauss_conv(C, g) + S * _gauss_conv(S, g))
    out = np.where(den > 0, num / np.where(den > 0, den, 1.0), f)
    if return_parts:
        return out, num, den
    return out


def _window_at(f, theta, points, range_fn):
    f = np.asarray(f, dtype=np.float64)
    H, W = f.shape
    g = spatial_taps(theta)
    r = (len(g) - 1) // 2
    pts = np.asarray(points, dtype=np.int64).reshape(-1, 2)
    py, px = pts[:, 0], pts[:, 1]
    fi = f[py, px]
    num = np.zeros(len(pts))
    den = np.zeros(len(pts))
    for jy in range(-r, r + 1):
        qy = py - jy
        for jx in range(-r, r + 1):
            qx = px - jx
            ok = (qy >= 0) & (qy < H) & (qx >= 0) & (qx < W)
            fj = np.where(ok, f[np.clip(qy, 0, H - 1), np.clip(qx, 0, W - 1)], 0.0)
            w = np.where(ok, g[jy + r] * g[jx + r] * range_fn(fj - fi), 0.0)
            num += w * fj
            den += w
    return np.where(den > 0, num / np.where(den > 0, den, 1.0), fi)


def fourier_bf_at(f, theta: float, c, T: int, points):
    """Eq. (1) with phi_hat as range kernel, evaluated directly at pixels ``points`` (N x 2, (y, x))."""
    return _window_at(f, theta, points, lambda t: phi_hat(t, c, T))


def brute_bf_at(f, theta: float, sigma: float, points):
    """Eq. (1) with the Gaussian phi, evaluated directly at pixels ``points``."""
    return _window_at(f, theta, points, lambda t: range_kernel(t, sigma))


def gaussian_blur_normalised(f, theta: float):
    """(omega * f) / (omega * 1): the limit of eq. (1) when the range kernel is constant."""
    f = np.asarray(f, dtype=np.float64)
    g = spatial_taps(theta)
    return _gauss_conv(f, g) / _gauss_conv(np.ones_like(f), g)


def psnr(a, b, peak: float = 255.0) -> float:
    """10 log10(peak^2 / MSE) (Section III)."""
    mse = float(np.mean((np.asarray(a, np.float64) - np.asarray(b, np.float64)) ** 2))
    return math.inf if mse == 0 else 10.0 * math.log10(peak * peak / mse)


def prop1_bound(R: int, delta_max: float, theta: float) -> float:
    """A usable form of Prop. 1: |f_hat_BF - f_BF| <= R delta W / (1 - delta W).

    delta = max over Lambda of |phi_hat - phi| and W = sum_j omega(j) over the window with
    omega(0) = 1.  Numerator and denominator of eq. (1) move by at most R delta W and
    delta W, and the exact denominator is at least omega(0) phi(0) = 1; the paper states the
    bound with eps and omega(0) and defers the proof to its supplement.  Returns inf when
    delta W >= 1 (no bound).
    """
    g = spatial_taps(theta)
    Wsum = float(np.sum(g) ** 2)
    x = delta_max * Wsum
    return math.inf if x >= 1.0 else R * x / (1.0 - x)
