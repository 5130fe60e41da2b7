"""How strong the oracle's pins are: each case plants one plausible mistake in
a copy of the C oracle (a wrong sign, index, axis or operand, a dropped term,
a wrong constant of a reading) and runs the CPU pin tests against the copy;
every case must make at least one pin fail.  About 25 s per case with eight
pytest-xdist workers, so the module runs only with HJBP_ORACLE_MUTANTS=1.

Planted changes that no pin can see, left out of the table:
- clamping the cell index to n - 1 instead of n - 2 (R2): the extra corners
  then carry weight 0 and are skipped, so every result is the same;
- breaking exact ties of the colours towards the higher colour (R10): exact
  ties of phi^j do not occur on the pinned problems;
- making the other target parts zero-cost terminals of a patch under state
  constraints: on every problem tried the values move by less than 1e-13,
  because a patch's nodes next to another part's target reach their own part
  as cheaply.
"""
import os
import shutil
import subprocess
import sys

import pytest

from tests._oracle_mutants_table import MUTANTS

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

pytestmark = [pytest.mark.slow,
              pytest.mark.skipif(os.environ.get("HJBP_ORACLE_MUTANTS") != "1",
                                 reason="planted-error runs take minutes: set HJBP_ORACLE_MUTANTS=1")]


def _copy(tmp, mutate=None):
    """The oracle, the problem descriptions and the CPU pin tests under tmp,
    the oracle's C source with mutate = (old, new) applied once."""
    ignore = shutil.ignore_patterns("__pycache__", "liboracle.so*")
    shutil.copytree(os.path.join(ROOT, "oracle"), os.path.join(tmp, "oracle"), ignore=ignore)
    shutil.copytree(os.path.join(ROOT, "workloads"), os.path.join(tmp, "workloads"), ignore=ignore)
    os.makedirs(os.path.join(tmp, "tests", "golden"))
    here = os.path.join(ROOT, "tests")
    for f in os.listdir(here):
        pin = f.startswith("test_oracle_") and f != os.path.basename(__file__)
        if pin or f in ("__init__.py", "conftest.py", "_indep.py"):
            shutil.copy(os.path.join(here, f), os.path.join(tmp, "tests", f))
    shutil.copy(os.path.join(here, "golden", "paper_patchy_errors.txt"), os.path.join(tmp, "tests", "golden"))
    shutil.copy(os.path.join(ROOT, "pytest.ini"), tmp)
    if mutate:
        src = os.path.join(tmp, "oracle", "hjbp_oracle.c")
        text = open(src).read()
        old, new = mutate
        assert old in text, "the planted change no longer matches the oracle's source"
        open(src, "w").write(text.replace(old, new, 1))


def _pins(tmp):
    cmd = [sys.executable, "-m", "pytest", "tests", "-x", "-q", "-p", "no:cacheprovider"]
    try:
        import xdist  # noqa: F401
        cmd += ["-n", "8"]
    except ImportError:
        pass
    return subprocess.run(cmd, cwd=tmp, capture_output=True, text=True, timeout=7200)


def test_unplanted_copy_passes(tmp_path):
    _copy(str(tmp_path))
    r = _pins(str(tmp_path))
    assert r.returncode == 0, r.stdout[-3000:]


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_error_fails_a_pin(name, tmp_path):
    _copy(str(tmp_path), MUTANTS[name])
    r = _pins(str(tmp_path))
    # a pin ran and failed (with -x under xdist the exit status is 2, so read
    # the summary line rather than the status; a collection error is not it)
    last = r.stdout.strip().splitlines()[-1] if r.stdout.strip() else ""
    assert r.returncode != 0 and " failed" in last and "error" not in last, \
        f"{name}: no pin failed\n" + r.stdout[-3000:]
