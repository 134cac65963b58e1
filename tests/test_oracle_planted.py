"""Planted mistakes in the C oracle (oracle/oracle.c), on the CPU.

Each case changes one line of a copy of oracle.c into a plausible mistake,
compiles the copy with the oracle's own flags, and runs the relevant pins of
tests/test_oracle_pins.py against it in a subprocess (ORACLE_LIB names the
copy): at least one pin must fail.  The unchanged source, compiled and run the
same way, passes the same pins, so a failure is the mistake's doing.

  kernel width        exp(-3 s^2 / Delta^2) for the Gaussian of Eq. 2 (the
                      transfer function exp(-k^2 Delta^2 / 24) no longer holds)
  no normalisation    periodic rows not divided by their sum (a constant is no
                      longer preserved where Delta / h is small)
  swapped sampling    the two weights of the linear interpolation to the LES
                      nodes (the discretization operator of Sec. 3) exchanged
  wall parity         u2 even and u1, u3 odd instead of Eq. 7 (a constant
                      u1 is no longer preserved at the walls)
  no product term     T_ij = bar(u_i u_j) without - bar(u_i) bar(u_j) (Eq. 6)
  pair parity         bar(u_i u_j) filtered with the parity of u_i alone instead
                      of p_i p_j (the separable and the direct three-dimensional
                      evaluations no longer agree)
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "oracle.c")

PLANTS = {
    "kernel_width": ("exp(-6.0 * s * s / (delta * delta))", "exp(-3.0 * s * s / (delta * delta))",
                     "test_periodic_transfer_function"),
    "no_normalisation": ("for (int ip = 0; ip < n; ip++) F[(size_t)i * n + ip] /= norm;",
                         "for (int ip = 0; ip < n; ip++) F[(size_t)i * n + ip] /= 1.0 + 0.0 * norm;",
                         "test_periodic_rows_normalised"),
    "swapped_sampling": ("A[(size_t)X * n + ip] = (1.0 - theta) * F[(size_t)i0 * n + ip]\n"
                         "                                    + theta * F[(size_t)i1 * n + ip];",
                         "A[(size_t)X * n + ip] = theta * F[(size_t)i0 * n + ip]\n"
                         "                                    + (1.0 - theta) * F[(size_t)i1 * n + ip];",
                         "test_periodic_sampling_is_linear_interpolation"),
    "wall_parity": ("int p = (c == 1) ? -1 : 1;", "int p = (c == 1) ? 1 : -1;",
                    "test_constant_and_mean_profile or test_mirror_symmetric or test_tau_closed_form"),
    "no_product_term": ("tau[q * nl + o] = uu[o] - ubar[a * nl + o] * ubar[b * nl + o];", "tau[q * nl + o] = uu[o];",
                        "test_tau_closed_form_single_modes or test_separable_equals_direct3d"),
    "pair_parity": ("const double *Ay = comp_parity(ext, a) * comp_parity(ext, b) > 0 ? Ayp : Aym;",
                    "const double *Ay = comp_parity(ext, a) > 0 ? Ayp : Aym;",
                    "test_separable_equals_direct3d"),
}


def _build(tmp_path, name, old=None, new=None):
    src = open(SRC).read()
    if old is not None:
        assert src.count(old) == 1, f"{name}: the planted line is not unique in oracle.c"
        src = src.replace(old, new)
    c = tmp_path / f"{name}.c"
    c.write_text(src)
    so = tmp_path / f"lib{name}.so"
    subprocess.check_call(["gcc", "-O2", "-std=c99", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared", str(c),
                           "-o", str(so), "-lm"])
    return str(so)


def _pins(lib, selector):
    env = dict(os.environ, ORACLE_LIB=lib, OMP_NUM_THREADS="4")
    r = subprocess.run([sys.executable, "-m", "pytest", os.path.join(ROOT, "tests", "test_oracle_pins.py"), "-q",
                        "-p", "no:cacheprovider", "-m", "not gpu", "-k", selector],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    return r.returncode, r.stdout[-2000:]


@pytest.mark.parametrize("name", sorted(PLANTS))
def test_planted_oracle_mistake_fails_a_pin(name, tmp_path):
    old, new, selector = PLANTS[name]
    rc, out = _pins(_build(tmp_path, "control"), selector)
    assert rc == 0, f"the unchanged oracle fails its pins:\n{out}"
    rc, out = _pins(_build(tmp_path, name, old, new), selector)
    assert rc == 1, f"planted mistake '{name}' passed the pins ({selector}):\n{out}"
