"""The GPU suite once more against the bounds-checked build (DCEM_CHECKS).

In that build every marked index (traversal nodes and leaves, stack slots,
segment-log rows and slots, work lists, candidate and hash slots, triangle
ids) is checked against its array before use; an index out of range is
counted, replaced by an in-range one and reported as DCEM_ERR_CHECK by the
call, so a latent out-of-bounds access shows as a failing test instead of a
device fault. Every GPU test must pass unchanged with it.
"""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_gpu_suite_under_bounds_checks():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2112_07115_gb300 import build
    lib = build.build(checks=True)
    assert os.path.exists(lib)
    env = dict(os.environ)
    env["DCEM_LIB_VARIANT"] = "checks"
    r = subprocess.run([sys.executable, "-m", "pytest", "tests", "-m", "gpu", "-x", "-q", "-p", "no:cacheprovider",
                        "--ignore", os.path.join("tests", "test_gpu_checks.py")],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=1800)
    assert r.returncode == 0, r.stdout[-4000:] + r.stderr[-2000:]
    assert " passed" in r.stdout
