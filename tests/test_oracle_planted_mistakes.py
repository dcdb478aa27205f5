"""Planted mistakes in the 2-D oracle: each must fail at least one pin.

The oracle's source text is mutated in memory (one plausible slip at a time:
the over-relaxation weight, the iterate fed to a step, the B0 axis, a dropped
constant, a sign, a dropped weighting, the prox denominator), loaded as a
fresh module, and its functions patched into ``oracle.pd_oracle`` for the
duration of one test.  The pins of ``tests/test_oracle_pins.py`` then run
against the mutated oracle; the test passes only if one of them fails.  The
unmutated oracle passes every pin used here (that file runs them as tests).
"""

import inspect
import sys
import types

import numpy as np
import pytest

from oracle import pd_oracle as O

import test_oracle_pins as pins  # noqa: E402  (tests/ is on sys.path under pytest's rootdir conftest)

# (name, original text, mutated text, occurrence to replace: 1 = the first only)
MUTATIONS = [
    ("theta_zero", "theta: float = 1.0,", "theta: float = 0.0,"),
    ("chi_instead_of_chibar_in_p", "(Wt * apply_D(chi_bar, Dk))", "(Wt * apply_D(chi, Dk))"),
    ("b0_axis_swapped", "kpar2 = (ky * ky) if b0_axis == 0 else (kx * kx)",
     "kpar2 = (kx * kx) if b0_axis == 0 else (ky * ky)"),
    ("one_third_dropped", "D[nz] = 1.0 / 3.0 - kpar2[nz] / k2[nz]", "D[nz] = -kpar2[nz] / k2[nz]"),
    ("adjoint_sign_of_y_term", "out[..., 1:, :] += b[..., :-1, :]\n    out[..., :-1, :] -= b[..., :-1, :]",
     "out[..., 1:, :] -= b[..., :-1, :]\n    out[..., :-1, :] += b[..., :-1, :]"),
    ("data_weight_dropped", "(Wt * apply_D(chi_bar, Dk))", "(apply_D(chi_bar, Dk))"),
    ("q_from_chi", "gx, gy = grad(chi_bar)", "gx, gy = grad(chi)"),
    ("prox_denominator", "return (v - sigma * b) / (1.0 + sigma / lam)",
     "return (v - sigma * b) / (1.0 + sigma * lam)"),
    ("unweighted_field", "    b = Wt * f\n", "    b = f\n"),  # first occurrence: pd_solve's
]


def _pin_runs():
    """The pins a mutated oracle is run against, cheapest first."""
    return [
        ("hand fractions of D(k)", pins.test_dipole_kernel_matches_hand_fractions),
        ("adjoint identities", pins.test_adjoint_identities_random),
        ("first iterate closed form", pins.test_first_iterate_closed_form),
        ("linear case, N=2", lambda: pins.test_linear_case_per_frequency_matrix_power(2)),
        ("linear case, N=17", lambda: pins.test_linear_case_per_frequency_matrix_power(17)),
        ("fixed points", pins.test_fixed_points_zero_field_and_empty_mask),
        ("gap/KKT one hole", lambda: pins.test_gap_stationarity_and_kkt_8x8(0, 50.0, "one_hole")),
        ("gap/KKT weighted", lambda: pins.test_gap_stationarity_and_kkt_8x8(3, 20.0, "weighted")),
        ("gap/KKT random mask", lambda: pins.test_gap_stationarity_and_kkt_8x8(2, 50.0, "random")),
    ]


def _mutated_module(monkeypatch, old, new):
    src = inspect.getsource(O)
    assert src.count(old) >= 1, f"mutation target not found: {old!r}"
    mod = types.ModuleType("pd_oracle_mutated")
    mod.__dict__["__file__"] = O.__file__
    monkeypatch.setitem(sys.modules, mod.__name__, mod)  # dataclasses resolve their module
    exec(compile(src.replace(old, new, 1), "<mutated pd_oracle>", "exec"), mod.__dict__)
    return mod


@pytest.mark.parametrize("name,old,new", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_planted_mistake_fails_a_pin(monkeypatch, name, old, new):
    mod = _mutated_module(monkeypatch, old, new)
    for attr, val in vars(mod).items():
        if isinstance(val, (types.FunctionType, type)) and getattr(val, "__module__", None) == "pd_oracle_mutated":
            monkeypatch.setattr(O, attr, val)
    failed = []
    for label, run in _pin_runs():
        try:
            with np.errstate(all="ignore"):
                run()
        except AssertionError:
            failed.append(label)
            break
    assert failed, f"planted mistake {name!r} passed every pin"


def test_harness_control_unmutated_copy_passes_every_pin(monkeypatch):
    """The same patching with an unchanged copy of the oracle: no pin may fail (so a failure
    above comes from the planted mistake, not from the harness)."""
    mod = _mutated_module(monkeypatch, "theta: float = 1.0,", "theta: float = 1.0,")
    for attr, val in vars(mod).items():
        if isinstance(val, (types.FunctionType, type)) and getattr(val, "__module__", None) == "pd_oracle_mutated":
            monkeypatch.setattr(O, attr, val)
    assert O.pd_solve is mod.pd_solve
    for _, run in _pin_runs():
        run()
