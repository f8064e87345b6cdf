"""The oracle's pins catch plausible slips (CPU only).

Each case plants one mistake in a copy of an oracle module -- its source with one textual
change, executed as a separate module whose functions then replace the real ones for the
duration of the test -- and requires that at least one pin of ``test_oracle_pins.py``
fails.  The slips are the kind a careful reading of the paper can still produce: the
period 2T instead of 2T + 1 (eq. 3), a dropped k = 0 term, the factor 2 of eq. (2) lost,
an off-by-one in Lambda or in the argmin over T (eq. 6), the norm instead of the squared
norm (eq. 5), a sign in the sine channels, a transposed image axis, a periodic instead of a
zero-padded border, the outside neighbours counted in the denominator of eq. (1), a floor
instead of a ceiling in r, 20 instead of 10 in the PSNR.  An unmutated copy must pass every
pin (so a failure is the slip's, not the harness's).
"""
import inspect
import sys
import types

import numpy as np
import pytest

import test_oracle_pins as pins
from oracle import filters, fit

# Pins that finish in well under a second; the slower ones run only when none of these fails.
FAST = [
    ("fig1_argmin_T_is_203", pins.test_fig1_argmin_T_is_203, ()),
    ("ls_closed_form_at_T_equals_R", pins.test_ls_closed_form_at_T_equals_R, ()),
    ("prop2_error_vanishes", pins.test_prop2_error_vanishes_at_T_R_K_R_plus_1, ()),
    ("K1_is_mean", pins.test_K1_is_mean, ()),
    ("roundoff_floor_picks_smallest_T", pins.test_roundoff_floor_picks_smallest_T, ()),
    ("spatial_radius", pins.test_spatial_radius, ()),
    ("brute_constant_image_unchanged", pins.test_brute_constant_image_unchanged, ()),
    ("brute_large_sigma_is_gaussian_blur", pins.test_brute_large_sigma_is_gaussian_blur, ()),
    ("brute_tiny_sigma_is_identity", pins.test_brute_tiny_sigma_is_identity_on_integer_image, ()),
    ("brute_step_edge_closed_form", pins.test_brute_step_edge_closed_form, ()),
    ("fourier_equals_brute_with_phi_hat", pins.test_fourier_equals_brute_with_phi_hat,
     ((13, 17), 2.0, 5)),
    ("fourier_K1_is_normalised_blur", pins.test_fourier_K1_is_normalised_blur, ()),
    ("psnr_definition", pins.test_psnr_definition, ()),
    ("optimised_period_beats_fixed_period", pins.test_optimised_period_beats_fixed_period_in_psnr,
     (2.0, 20.0)),
]
SLOW = [
    ("prop2_monotone_in_K", pins.test_prop2_monotone_in_K, ()),
    ("fourier_converges_and_prop1_bound", pins.test_fourier_converges_to_brute_and_prop1_bound, ()),
    ("psnr_band_at_eps_0_1", pins.test_psnr_band_at_eps_0_1, ()),
    ("algorithm1_trends", pins.test_algorithm1_trends, ()),
]

# (module, id, text in the module's source, replacement)
MUTATIONS = [
    (fit, "eq2_factor_2_dropped",
     "return np.exp(-(t * t) / (2.0 * sigma * sigma))",
     "return np.exp(-(t * t) / (sigma * sigma))"),
    (fit, "lambda_shifted",
     "t = np.arange(-R, R + 1, dtype=np.float64)\n    if kernel is None:",
     "t = np.arange(0, 2 * R + 1, dtype=np.float64)\n    if kernel is None:"),
    (fit, "A_period_2T",
     "P = 2 * T + 1\n    t = np.arange(-R, R + 1, dtype=np.int64)",
     "P = 2 * T\n    t = np.arange(-R, R + 1, dtype=np.int64)"),
    (fit, "A_k0_column_dropped",
     "k = np.arange(K, dtype=np.int64)[None, :]",
     "k = np.arange(1, K + 1, dtype=np.int64)[None, :]"),
    (fit, "A_angle_t_plus_k",
     "np.mod(t * k, P)", "np.mod(t + k, P)"),
    (fit, "E_is_norm_not_squared",
     "return float(res @ res), c", "return float(np.sqrt(res @ res)), c"),
    (fit, "argmin_T_off_by_one",
     "T_star = int(np.argmin(floored)) + 1", "T_star = int(np.argmin(floored))"),
    (fit, "phi_hat_nu_pi",
     "nu = 2.0 * math.pi / P\n    integral", "nu = math.pi / P\n    integral"),
    (fit, "phi_hat_c0_dropped",
     "for k, ck in enumerate(np.asarray(c, dtype=np.float64)):",
     "for k, ck in list(enumerate(np.asarray(c, dtype=np.float64)))[1:]:"),
    (filters, "r_floor_not_ceil",
     "math.ceil(3.0 * theta - 1e-12)", "math.floor(3.0 * theta + 1e-12)"),
    (filters, "g_factor_2_dropped",
     "np.exp(-(x * x) / (2.0 * theta * theta))", "np.exp(-(x * x) / (theta * theta))"),
    (filters, "periodic_border",
     "def _shift(img, dy: int, dx: int):\n",
     "def _shift(img, dy: int, dx: int):\n    return np.roll(img, (dy, dx), axis=(0, 1))\n\n\n"
     "def _unused_shift(img, dy: int, dx: int):\n"),
    (filters, "y_pass_along_x",
     "out += g[jy + r] * _shift(tmp, jy, 0)", "out += g[jy + r] * _shift(tmp, 0, jy)"),
    (filters, "brute_outside_counted",
     "w = g[jy + r] * g[jx + r] * range_fn(fj - f) * inside",
     "w = g[jy + r] * g[jx + r] * range_fn(fj - f)"),
    (filters, "brute_range_of_value_not_difference",
     "range_fn(fj - f) * inside", "range_fn(fj) * inside"),
    (filters, "fourier_sine_sign",
     "num += ck * (C * _gauss_conv(f * C, g) + S * _gauss_conv(f * S, g))",
     "num += ck * (C * _gauss_conv(f * C, g) - S * _gauss_conv(f * S, g))"),
    (filters, "fourier_den_sine_dropped",
     "den += ck * (C * _gauss_conv(C, g) + S * _gauss_conv(S, g))",
     "den += ck * (C * _gauss_conv(C, g))"),
    (filters, "fourier_nu_2T",
     "nu = 2.0 * math.pi / (2 * T + 1)\n    num", "nu = 2.0 * math.pi / (2 * T)\n    num"),
    (filters, "window_at_y_tap_for_x",
     "g[jy + r] * g[jx + r] * range_fn(fj - fi)", "g[jy + r] * g[jy + r] * range_fn(fj - fi)"),
    (filters, "psnr_20_log",
     "10.0 * math.log10(peak * peak / mse)", "20.0 * math.log10(peak * peak / mse)"),
]


def _install_mutant(monkeypatch, module, old, new):
    """Execute ``module``'s source with ``old`` replaced by ``new`` (exactly one occurrence)
    and patch every function and class it defines over the real module's; a mutated fit
    also replaces the names that filters imported from it."""
    src = inspect.getsource(module)
    assert src.count(old) == 1, f"mutation text not found exactly once in {module.__name__}"
    name = module.__name__ + "_mutant"
    mutant = types.ModuleType(name)
    mutant.__package__ = module.__package__
    mutant.__file__ = module.__file__
    monkeypatch.setitem(sys.modules, name, mutant)
    exec(compile(src.replace(old, new), f"<{name}>", "exec"), mutant.__dict__)
    for attr, val in vars(mutant).items():
        if ((inspect.isfunction(val) or inspect.isclass(val)) and hasattr(module, attr)
                and getattr(val, "__module__", None) == name):
            monkeypatch.setattr(module, attr, val)
            if module is fit and hasattr(filters, attr):
                monkeypatch.setattr(filters, attr, val)


def _failing_pins(stop_at_first=True):
    failed = []
    for group in (FAST, SLOW):
        for pin_name, pin, args in group:
            try:
                pin(*args)
            except (AssertionError, ArithmeticError, ValueError, IndexError, RuntimeError,
                    KeyError, np.linalg.LinAlgError):
                failed.append(pin_name)
                if stop_at_first:
                    return failed
        if failed:
            break
    return failed


@pytest.mark.parametrize("module", [fit, filters], ids=["fit", "filters"])
def test_unmutated_copy_passes_every_pin(monkeypatch, module):
    _install_mutant(monkeypatch, module, "import numpy as np\n", "import numpy as np\n")
    assert _failing_pins(stop_at_first=False) == []


@pytest.mark.parametrize("module,old,new", [m[:1] + m[2:] for m in MUTATIONS],
                         ids=[m[1] for m in MUTATIONS])
def test_pins_catch_planted_slip(monkeypatch, module, old, new):
    _install_mutant(monkeypatch, module, old, new)
    assert _failing_pins(), "no pin fails with this slip in the oracle"
