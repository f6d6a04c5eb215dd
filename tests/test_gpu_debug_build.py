"""The bounds-checked debug build (libladder_debug.so, LADDER_BOUNDS_CHECK=1):
device-side checks of array indexes and plane offsets that record
LADDER_E_BOUNDS in the status word instead of faulting -- the stand-in for a
memory checker on GPUs where none can run.  Small parity cases of every
kernel family run on it in a process of their own (a process loads one
build of the library); they must pass with no check failing."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

HERE = os.path.dirname(os.path.abspath(__file__))


def test_parity_cases_pass_on_the_debug_build():
    env = dict(os.environ, LADDER_DEBUG_BUILD="1")
    res = subprocess.run([sys.executable, os.path.join(HERE, "debug_parity_job.py")], capture_output=True, text=True,
                         env=env, timeout=900)
    assert res.returncode == 0, res.stdout[-2000:] + res.stderr[-4000:]
    assert "debug build ok" in res.stdout
