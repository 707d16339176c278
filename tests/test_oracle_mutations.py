"""The pins catch plausible mistakes in the oracle: each case compiles a copy of the oracle's C source with
one deliberate error (on the CPU, into a temporary directory) and runs the pin tests against it in a
subprocess; at least one pin must fail.  The correct source passes the same run (tests/test_oracle_pins.py
in the ordinary suite)."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "lbve_oracle.c")

MUTATIONS = {
    # the u.u term of the equilibrium dropped
    "dropped_uu_term": ("(cu * cu - cs2 * uu) / (2.0 * cs2 * cs2)", "(cu * cu) / (2.0 * cs2 * cs2)"),
    # a merged point keeps the newer half's time instead of the older one's
    "merge_keeps_newer_time": ("merged.tp = o1->tp;", "merged.tp = o2->tp;"),
    # merged factors multiplied in the wrong order (earlier factor on the left)
    "merge_factor_order": ("mat_mul(d, o2->F, o1->F, merged.F);", "mat_mul(d, o1->F, o2->F, merged.F);"),
    # the non-Newtonian stress enters the forcing with the wrong sign
    "flipped_stress_sign": ("const double Fi = ch->w[i] * (-stress /", "const double Fi = ch->w[i] * (stress /"),
    # -d_t'B formed as 2 E kappa E^T instead of E kappa E^T plus its transpose
    "missing_transpose": ("(M[a * d + b] + M[b * d + a])", "(M[a * d + b] + M[a * d + b])"),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_fails_a_pin(name, tmp_path):
    old, new = MUTATIONS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site of {name} not unique"
    mutated = tmp_path / "lbve_oracle_mutated.c"
    mutated.write_text(src.replace(old, new))
    lib = tmp_path / "liblbve_oracle_mutated.so"
    subprocess.run(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-o", str(lib), str(mutated), "-lm"], check=True)
    env = dict(os.environ, LBVE_ORACLE_LIB=str(lib))
    out = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                          os.path.join(ROOT, "tests", "test_oracle_pins.py")],
                         capture_output=True, text=True, env=env, cwd=ROOT, timeout=900)
    assert out.returncode == 1, f"{name}: no pin failed\n{out.stdout[-1500:]}"
    assert "failed" in out.stdout
