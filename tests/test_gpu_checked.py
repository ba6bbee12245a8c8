"""The bounds-checked build: the merge kernel with every global load and
store checked against the job's buffers (-DLW_CHECKED), run on parity cases
of every entry point (one CTA and grids, both layouts, six linkages, a
pinned host matrix, a batch, the entry point without allocation, an
n = 16384 grid run).  A kernel access outside its buffers would fail the
call with its source line; none may occur, and every result must still
equal the oracle's.  The library is built here on first use and loaded in
a child process (LW_CHECKED=1 selects it).
"""
import os
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - collected on CPU machines
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1709_06816_gb300 import build as lw_build  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


def test_checked_build_runs_clean():
    lw_build.build(checked=True)
    env = dict(os.environ, LW_CHECKED="1")
    r = subprocess.run([sys.executable, os.path.join(HERE, "checked_cases.py")], env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert "checked ok" in r.stdout, r.stdout[-3000:]
