"""The bounds-checked build (every global-memory index of every kernel checked
against its buffer, the first failure recorded instead of faulting) runs the
kernel families on small cases, including ragged and strip-walk sizes, with
results equal to the oracle's and no access out of range."""
import json
import os
import subprocess
import sys

import pytest
import torch

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_bounds_checked_build_records_no_out_of_range_access():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1908_07341_gb300 import build
    path = build.build(debug_bounds=True)
    env = dict(os.environ, SHK_LIBRARY=path, PYTHONPATH=ROOT)
    r = subprocess.run([sys.executable, "-m", "tests.bounds_cases"], cwd=ROOT, env=env, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    out = json.loads(r.stdout.strip().splitlines()[-1])
    assert out["status"] == 0 and out["site"] == 0, out
    assert len(out["checked"]) == 13
