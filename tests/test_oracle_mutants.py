"""Mutation tests of the oracle's pins: each case plants one plausible mistake in a copy of
the oracle (a dropped term, a wrong index, a wrong power or sign), builds the copy, and runs
the pins that must catch it in a child pytest with that copy loaded.  A pin set that still
passes on a planted mistake would not pin the oracle's arithmetic.  CPU only."""
import os
import re
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ORACLE = os.path.join(ROOT, "oracle")

ADAPTIVE_PIN = ["tests/test_oracle_recon.py::test_adaptive_ct_worked_examples"]
POSITIVITY_PINS = ["tests/test_oracle_positivity.py"]

# (name, replaced text, replacement, pins that must fail)
MUTANTS = [
    # TENO8A adaptive cutoff (Section 2.4, Eqs. shock_indicator and cut-off_adjust)
    ("epsilon with xi instead of xi^2", "(1.0 - 0.9 * Cr) * xi * xi;", "(1.0 - 0.9 * Cr) * xi;", ADAPTIVE_PIN),
    ("eta window shifted left", "int c = q - 1;", "int c = q - 2;", ADAPTIVE_PIN),
    ("eta window shifted right", "int c = q - 1;", "int c = q;", ADAPTIVE_PIN),
    ("(1 - m)^3 in g", "T g = om * om * om * om * (1.0 + 4.0 * m);", "T g = om * om * om * (1.0 + 4.0 * m);",
     ADAPTIVE_PIN),
    # positivity-preserving flux limiter (Section 4.4)
    ("density factor dropped", "if (rh < eps) th =", "if (false && rh < eps) th =", POSITIVITY_PINS),
    ("pressure factor dropped", "if (p1 < eps) tp =", "if (false && p1 < eps) tp =", POSITIVITY_PINS),
    ("one-sided signs flipped", "sgn_mu[2] = {-mu, mu};", "sgn_mu[2] = {mu, -mu};", POSITIVITY_PINS),
    ("2 dim factor of the one-sided split missing", "const double mu = 2.0 * D * dt / g.dx[a];",
     "const double mu = dt / g.dx[a];", POSITIVITY_PINS),
    ("min for max in the Lax-Friedrichs alpha", "const double alpha = std::fmax(sp[0], sp[1]);",
     "const double alpha = std::fmin(sp[0], sp[1]);", POSITIVITY_PINS),
]


def build_mutant(tmp, idx, old, new):
    d = os.path.join(tmp, "m%d" % idx)
    os.makedirs(d)
    for f in os.listdir(ORACLE):
        if f.endswith((".hpp", ".h", ".cpp")):
            shutil.copy(os.path.join(ORACLE, f), d)
    hpp = os.path.join(d, "tenom_oracle.hpp")
    src = open(hpp).read()
    assert src.count(old) == 1, "mutation site not unique: %r" % old
    open(hpp, "w").write(src.replace(old, new))
    so = os.path.join(d, "liboracle_mutant.so")
    cmd = ["g++", "-std=c++17", "-O0", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-o", so,
           os.path.join(d, "oracle_capi.cpp")]
    return so, subprocess.Popen(cmd, cwd=d, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)


@pytest.fixture(scope="module")
def mutant_libs(tmp_path_factory):
    tmp = str(tmp_path_factory.mktemp("oracle_mutants"))
    jobs = [build_mutant(tmp, i, old, new) for i, (_, old, new, _) in enumerate(MUTANTS)]
    libs = []
    for so, p in jobs:
        out, _ = p.communicate()
        assert p.returncode == 0, out.decode(errors="replace")
        libs.append(so)
    return libs


def run_pins(so, pins):
    env = dict(os.environ, TENOM_ORACLE_LIB=so)
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "--tb=no", "-p", "no:cacheprovider"] + pins,
                       cwd=ROOT, env=env, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True, timeout=600)
    m = re.search(r"(\d+) failed", r.stdout)
    return (int(m.group(1)) if m else 0), r.stdout


@pytest.mark.parametrize("i", range(len(MUTANTS)), ids=[m[0] for m in MUTANTS])
def test_planted_mistake_is_caught(mutant_libs, i):
    name, _, _, pins = MUTANTS[i]
    failed, out = run_pins(mutant_libs[i], pins)
    assert failed >= 1, "planted mistake '%s' passed every pin:\n%s" % (name, out[-2000:])


def test_unmutated_copy_passes(tmp_path):
    """Control: the same build of an unchanged copy passes the same pins."""
    so, p = build_mutant(str(tmp_path), 0, "int c = q - 1;", "int c = q - 1;")
    out, _ = p.communicate()
    assert p.returncode == 0, out
    failed, out = run_pins(so, ADAPTIVE_PIN + POSITIVITY_PINS)
    assert failed == 0, out[-2000:]
