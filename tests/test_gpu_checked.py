"""The bounds-checked build (-DAPX_CHECKED): device-side index checks on the
FFT and direct-core shared-memory accesses, the output words and the
tensor-memory columns report APX_ERR_CHECK instead of touching memory out of
range.  A slice of the parity suite runs against that build in a child
process (the library is loaded once per process) and must stay clean and
exact."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_parity_subset_clean_under_checked_build():
    from paper_1201_3018_gb300 import build
    lib = build.build(checked=True)
    env = dict(os.environ, APX_LIB=lib)
    cmd = [sys.executable, "-m", "pytest", "-q", "-x", "-m", "gpu", "-p", "no:cacheprovider",
           "tests/test_gpu_parity.py::test_full_precision", "tests/test_gpu_parity.py::test_auto_selection",
           "tests/test_gpu_tc.py::test_filterbank_matches_oracle",
           "tests/test_gpu_fused.py::test_one_launch_equals_three_launch_form",
           "tests/test_gpu_parity.py::test_paper_literal_form_matches_oracle", "-k", "not 16384"]
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=1200)
    assert r.returncode == 0, r.stdout[-4000:] + r.stderr[-2000:]
    import re
    m = re.search(r"(\d+) passed", r.stdout)
    assert m and int(m.group(1)) >= 80, r.stdout[-2000:]   # parity, filterbank, one-launch and literal cases
