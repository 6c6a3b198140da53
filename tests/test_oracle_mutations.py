"""The oracle's pins catch plausible mistakes: each case plants one mistake in a temporary copy of
oracle/ (a sign, an operand, a convention, a policy rule) and runs the pin that must fail on
it.  A pin that still passes on the mutated oracle would not tell a wrong oracle from a right
one."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CASES = [
    # (file, original text, planted mistake, the pin that must fail)
    ("oracle/pair_dual.c", "dvec D = v_normalize(v_cross(nB, nA));", "dvec D = v_normalize(v_cross(nA, nB));",
     "test_closed_form_pairs"),                                   # line direction of the listing
    ("oracle/pair_dual.c", "r.g[i] = a.g[i] * b.v + a.v * b.g[i];", "r.g[i] = a.g[i] * b.v - a.v * b.g[i];",
     "test_dual_gradient_matches_central_differences"),           # product rule of the duals
    ("oracle/pair_dual.c", "int lone_sign = (pos == 1) ? 1 : -1;", "int lone_sign = (pos == 1) ? -1 : 1;",
     "test_closed_form_pairs"),                                   # the 2:1 cut case
    ("oracle/ttie_oracle.py",
     "g = (2 * a * b * b)[:, None] * ev.dtc[:, 0] + (2 * b * a * a)[:, None] * ev.dtc[:, 1]",
     "g = (2 * a * a * b)[:, None] * ev.dtc[:, 0] + (2 * b * b * a)[:, None] * ev.dtc[:, 1]",
     "test_eq3_gradient_is_gradient_of_T"),                       # Eq. 3
    ("oracle/ttie_oracle.py", "H = p1 + p2 + clamp_psd(p3)", "H = clamp_psd(p1 + p2 + p3)",
     "test_psd_projection_properties"),                           # the per-part projection of §1.1
    ("oracle/exact.py", "return max(tA) > min(tB) and min(tA) < max(tB)",
     "return max(tA) >= min(tB) and min(tA) <= max(tB)", "test_closed_form_pairs"),   # touching
    ("oracle/ttie_oracle.py", "if nt == 0 or Et <= E + prm.armijo_c * a * slope or fewer:",
     "if nt == 0 or Et <= E - prm.armijo_c * a * slope or fewer:", "test_line_search_rule"),    # Armijo
    ("oracle/ttie_oracle.py", "fewer = prm.ls_rule == \"fewer\" and n0 is not None and nt < n0 and Et <= E",
     "fewer = prm.ls_rule == \"fewer\" and n0 is not None and nt <= n0 and Et <= E",
     "test_line_search_rule"),                                    # the fewer-pairs acceptance
    ("oracle/elastic.py", "K = k * (P + (1.0 - L / l) * (np.eye(3) - P))",
     "K = k * (P + (1.0 - l / L) * (np.eye(3) - P))", "test_spring_hessian_central_differences"),
]


def _copy(tmp_path):
    for d in ("oracle", "ttie_inputs"):
        shutil.copytree(os.path.join(ROOT, d), tmp_path / d, ignore=shutil.ignore_patterns("_build", "__pycache__"))
    (tmp_path / "tests").mkdir()
    shutil.copytree(os.path.join(ROOT, "tests", "golden"), tmp_path / "tests" / "golden")
    for f in ("test_oracle.py", "conftest.py"):
        shutil.copy(os.path.join(ROOT, "tests", f), tmp_path / "tests" / f)
    if os.path.exists(os.path.join(ROOT, "pytest.ini")):
        shutil.copy(os.path.join(ROOT, "pytest.ini"), tmp_path / "pytest.ini")


def _run(tmp_path, pins):
    return subprocess.run([sys.executable, "-m", "pytest", "tests/test_oracle.py", "-q", "-p", "no:cacheprovider",
                           "-k", " or ".join(pins)], cwd=tmp_path, capture_output=True, text=True, timeout=600)


def test_pins_pass_on_the_copied_oracle(tmp_path):
    """Control: the same pins pass on an unchanged copy, so a failure below is the mistake's."""
    _copy(tmp_path)
    r = _run(tmp_path, sorted({c[3] for c in CASES}))
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-2000:]


@pytest.mark.parametrize("case", range(len(CASES)), ids=[c[3] + "-%d" % i for i, c in enumerate(CASES)])
def test_pin_catches_planted_mistake(tmp_path, case):
    path, old, new, pin = CASES[case]
    _copy(tmp_path)
    src = (tmp_path / path).read_text()
    assert src.count(old) == 1, "the oracle changed: update this case"
    (tmp_path / path).write_text(src.replace(old, new))
    r = _run(tmp_path, [pin])
    assert r.returncode == 1 and "failed" in r.stdout, r.stdout[-2000:] + r.stderr[-2000:]
