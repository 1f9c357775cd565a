"""The oracle pins are strong enough to catch plausible mistakes.

Each case plants one mistake in a copy of the oracle source (on the CPU, in a
temporary directory), rebuilds it, and runs the pin suites against it: at
least one pin must fail.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "sh_oracle.c")

MUTATIONS = {
    "dropped Condon-Shortley sign": ("const double sgn = (m & 1) ? -1.0 : 1.0;", "const double sgn = 1.0;"),
    "wrong recurrence coefficient": ("((2.0 * l - 1.0) * ct", "((2.0 * l + 1.0) * ct"),
    "transposed atan2 operands": ("atan2(y, x)", "atan2(x, y)"),
    "missing conjugate in Eq. 10": ("sa * conj(Yp[a])", "sa * Yp[a]"),
    "inverted factorial ratio": ("factorial(l - m) / factorial(l + m)", "factorial(l + m) / factorial(l - m)"),
    "m ordering reversed": ("row[l * l + l + m] = v;", "row[l * l + l - m] = v;"),
    "r = 0 convention lost": ("row[0] = 1.0 / sqrt(4.0 * ORACLE_PI);", "row[0] = 0.0;"),
    "minimum image by floor": ("rint(d[c] / box)", "floor(d[c] / box)"),
    "Lagrange stencil shifted": ("int i0 = (int)floor(t) - 1;", "int i0 = (int)floor(t);"),
    "spinor upper sign dropped": ("const double cu = s * sqrt(l + s * mj + 0.5) * pre",
                                  "const double cu = sqrt(l + s * mj + 0.5) * pre"),
    "spinor components swapped": ("mu = (int)lround(mj - 0.5), md = (int)lround(mj + 0.5)",
                                  "mu = (int)lround(mj + 0.5), md = (int)lround(mj - 0.5)"),
    "spinor normalisation": ("const double pre = 1.0 / sqrt(2.0 * l + 1.0);",
                                      "const double pre = 1.0 / sqrt(2.0 * l + 2.0);"),
    "radial index off by one": ("((int64_t)s * radial_lstride + l) * n_rad", "((int64_t)s * radial_lstride + l + 1) * n_rad"),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(tmp_path, name):
    old, new = MUTATIONS[name]
    src = open(SRC).read()
    assert src.count(old) >= 1, f"mutation anchor not found: {old!r}"
    mutated = tmp_path / "sh_oracle.c"
    mutated.write_text(src.replace(old, new))
    env = dict(os.environ, SHM_ORACLE_SRC=str(mutated), SHM_ORACLE_BUILD_DIR=str(tmp_path / "build"))
    cmd = [sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
           os.path.join(ROOT, "tests", "test_oracle_pins.py"),
           os.path.join(ROOT, "tests", "test_oracle_projector_pins.py"),
           os.path.join(ROOT, "tests", "test_oracle_spinor_pins.py")]
    res = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert res.returncode != 0, f"mutation '{name}' survived every pin:\n{res.stdout[-2000:]}"
