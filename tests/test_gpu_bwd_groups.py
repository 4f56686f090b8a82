"""The two-group variant of the tensor-core backward (8 warps, 32 Gaussians
per thread and batch) against the oracle.

The library picks the backward's group count once per process from
FHGS_BWD_GROUPS (default 4), so the variant's parity cases run in a child
process with FHGS_BWD_GROUPS=2: the tensor-core backward parity tests at
every D split, on the same bars as the default kernel.
"""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_two_group_backward_parity():
    env = dict(os.environ, FHGS_BWD_GROUPS="2")
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-m", "gpu",
                        os.path.join(ROOT, "tests", "test_gpu_tc.py"), "-k", "test_tc_backward_small"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert "3 passed" in r.stdout, r.stdout[-2000:]
