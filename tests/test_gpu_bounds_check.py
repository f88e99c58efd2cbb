"""The bounds-checked build (-DCWT_BOUNDS_CHECK, csrc/check.cuh): every
shared-memory access of the kernels and the spectrum indices of the sparse
passes are checked on the device; an out-of-range one is recorded and turned
into CWT_EDEVICE, without the access being made.  This builds that variant
and runs small cases of every kernel family under it in a fresh process
(tests/bounds_check_cases.py), expecting no violation and oracle-correct
results."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

pytestmark = pytest.mark.gpu


def test_every_kernel_family_runs_clean_under_bounds_checks():
    import importlib.util
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    spec = importlib.util.spec_from_file_location(
        "_cwt_build", os.path.join(ROOT, "paper_2506_07793_gb300", "build.py"))
    b = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(b)
    lib = b.build(check=True)
    env = dict(os.environ, CWT_GB300_LIB=lib)
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "bounds_check_cases.py")],
                       capture_output=True, text=True, env=env, cwd=ROOT, timeout=1200)
    print(r.stdout)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert "ALL CASES PASSED UNDER BOUNDS CHECKS" in r.stdout
