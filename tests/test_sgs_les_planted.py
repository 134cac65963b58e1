"""Planted one-line mistakes in a copy of the LES-step oracle (oracle/les.py):
each must fail at least one of its pins (tests/test_sgs_les_oracle.py), and
the unchanged source must pass them all.  The copies are built from the
source text in memory; nothing on disk changes."""
import types

import pytest

import oracle.les as les_src
import tests.test_sgs_les_oracle as pins

MUTANTS = {
    "subfilter stress with the wrong sign": ("flux = flux + np.asarray(tau", "flux = flux - np.asarray(tau"),
    "Runge-Kutta zeta coefficients swapped": ("RK3_ZETA = (0.0, -17.0 / 60.0, -5.0 / 12.0)",
                                              "RK3_ZETA = (0.0, -5.0 / 12.0, -17.0 / 60.0)"),
    "projection weight of one cell instead of two half cells": ("return (y[2:] - y[:-2]) / 2.0",
                                                               "return (y[2:] - y[1:-1])"),
    "y Laplacian without the factor 2": ("fy = 2.0 / (hm + hp)", "fy = 1.0 / (hm + hp)"),
    "forcing on the wrong component": ("        if i == 0:\n            acc += forcing",
                                       "        if i == 1:\n            acc += forcing"),
    "advective flux u_i u_i instead of u_i u_j": ("flux = u[i] * u[j]", "flux = u[i] * u[i]"),
    "wall value of u_2 taken from the filtered field": ("        u[1, row] = 0.0\n        for c in (0, 2):",
                                                         "        for c in (0, 1, 2):"),
    "difference symbol at half the wavenumber": ("s = np.sin(2.0 * np.pi * m / n) / h", "s = np.sin(np.pi * m / n) / h"),
}


def _pin_calls():
    return [
        lambda: pins.test_projection_forms_agree(),
        lambda: pins.test_projection_is_the_hodge_split((16, 13, 12)),
        lambda: pins.test_poiseuille_is_steady("rk3"),
        lambda: pins.test_couette_with_wall_values_is_steady("rk3"),
        lambda: pins.test_single_mode_decays_by_the_scheme_amplification(
            "rk3", lambda z: 1 + z + z * z / 2 + z ** 3 / 6),
        lambda: pins.test_rhs_closed_form_uniform_grid(),
        lambda: pins.test_subfilter_term_enters_by_its_divergence(),
    ]


def _module_from(source: str):
    mod = types.ModuleType("oracle.les_planted")
    mod.__package__ = "oracle"
    exec(compile(source, "les_planted.py", "exec"), mod.__dict__)
    return mod


def _failures(mod, monkeypatch):
    monkeypatch.setattr(pins, "L", mod)
    failed = 0
    for call in _pin_calls():
        try:
            call()
        except (AssertionError, ValueError, FloatingPointError):
            failed += 1
    return failed


def test_unchanged_source_passes(monkeypatch):
    src = open(les_src.__file__).read()
    assert _failures(_module_from(src), monkeypatch) == 0


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_fails_a_pin(name, monkeypatch):
    old, new = MUTANTS[name]
    src = open(les_src.__file__).read()
    assert src.count(old) == 1, name
    assert _failures(_module_from(src.replace(old, new)), monkeypatch) >= 1, name
