"""The oracle's pins are sensitive: each plausible mistake planted in the
oracle (tests/oracle_mutations.py; in memory, in a child pytest process, on
the CPU) fails at least one pin of the oracle's own test files, by an
assertion.  A mistake no pin catches fails this test."""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

from oracle_mutations import MUTATIONS

HERE = os.path.dirname(os.path.abspath(__file__))
# fastest files first: each child stops at its first failure
PINS = ["test_oracle_cfl.py", "test_oracle_boundaries.py", "test_oracle_pins.py", "test_oracle_split1.py", "test_oracle_physics.py"]


def run_pins(mutation):
    env = dict(os.environ, DVBM_ORACLE_MUTATION=mutation, PYTHONPATH=os.pathsep.join([HERE, os.path.dirname(HERE)]),
               OMP_NUM_THREADS="2")
    cmd = [sys.executable, "-m", "pytest", "-p", "oracle_mutations", "-p", "no:cacheprovider", "-x", "-q",
           "--tb=line", "-m", "not gpu", *[os.path.join(HERE, p) for p in PINS]]
    r = subprocess.run(cmd, cwd=os.path.dirname(HERE), env=env, capture_output=True, text=True, timeout=900)
    return mutation, r.returncode, r.stdout[-2000:]


@pytest.fixture(scope="module")
def outcomes():
    with ThreadPoolExecutor(max_workers=min(4, os.cpu_count() or 1)) as ex:
        return {m: (rc, out) for m, rc, out in ex.map(run_pins, MUTATIONS)}


@pytest.mark.parametrize("mutation", MUTATIONS)
def test_planted_mistake_fails_a_pin(outcomes, mutation):
    rc, out = outcomes[mutation]
    assert rc == 1, f"{mutation}: pins exit {rc}\n{out}"  # 1 = tests failed (not a crash or a usage error)
    assert "AssertionError" in out or "assert" in out, f"{mutation}: failed without an assertion\n{out}"
