"""The checked build (librelnn_checked.so, compiled with -DRELNN_CHECKED): every gathered row index and
output row of the fused kernels is tested on the device; a failing one raises RELNN_DEV_BOUNDS and the
access is skipped, so a bad plan or input would end as RELNN_EDEVICE instead of a memory fault. Here
the rule parity suites run against that build on valid inputs (the checks must stay silent and the
results must match the FP64 oracle as with the regular build), in a child process that loads it."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(args):
    env = dict(os.environ, RELNN_LIB="checked")
    return subprocess.run([sys.executable, *args], cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)


def test_checked_build_is_the_one_loaded(gpu):
    r = _run(["-c", "from paper_2605_24207_b300 import relnn as R; import sys; "
                    "sys.exit(0 if R.lib().relnn_build_flags() & 1 else 3)"])
    assert r.returncode == 0, r.stdout + r.stderr


def test_parity_suites_under_checked_build(gpu):
    r = _run(["-m", "pytest", "-q", "-x", "-m", "gpu", "-p", "no:cacheprovider",
              "tests/test_gpu_agg.py", "tests/test_gpu_rule.py", "tests/test_gpu_program.py"])
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
