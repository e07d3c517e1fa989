"""Shared-memory bounds of the pass kernels, checked in a separate build.

compute-sanitizer is not available on the GPU pool. The checked build of the
library (-DSNLM_CHECKED, `python -m paper_1407_2343_gb300.build --checked`) places
guard words after every warp's shared-memory rows; each unit writes them before its
first shared-memory store and verifies them after its last, and a damaged guard is
recorded in the device failure word (SNLM_ERR_CHECK) without any fault. The cases
(tests/checked_run.py, run in a process of its own against the checked library)
cover every pass variant class: uint8 / float16 / float32, box and Gaussian, S from
0 to 128, K from 0 to 7, lines shorter than a window, a single pixel, and the
batched persistent kernel; each must leave the guards intact and match the oracle.
"""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_checked_build_keeps_every_shared_memory_guard():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1407_2343_gb300 import build

    lib = build.build(checked=True)
    env = dict(os.environ, SNLM_LIBRARY=lib)
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "checked_run.py")], env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    results = json.loads(r.stdout.strip().splitlines()[-1])
    assert len(results) >= 9
    for c in results:
        assert c["device_error"] == 0, c
        assert c.get("status", 0) == 0, c
        assert c["max_abs"] <= 1e-4, c
