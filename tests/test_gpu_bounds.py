"""Memory safety of the direct kernels with the bounds-checked library build
(liblbm_check.so, -DLBM_BOUNDS_CHECK): every global access of the step, export, set-up and
exchange kernels is checked against the array it belongs to and an access outside it is
skipped and reported by lbm_sync.  compute-sanitizer is closed on this machine; this is the
stand-in.  The cases (tests/sanitizer_cases.py) cover every boundary type, stencil, storage
precision, streaming pattern and collision; the checked build must report nothing and give
the bits of the normal build."""
import os
import re
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(lib):
    env = dict(os.environ)
    if lib:
        env["LBM_LIBRARY"] = lib
    r = subprocess.run([sys.executable, "-m", "tests.sanitizer_cases"], capture_output=True, text=True,
                       timeout=900, cwd=ROOT, env=env)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-3000:]
    m = re.search(r"(\d+) lattices stepped, populations sha256 ([0-9a-f]+)", r.stdout)
    assert m, r.stdout
    return int(m.group(1)), m.group(2)


def test_checked_build_reports_no_bad_access_and_same_bits():
    from paper_2305_09910_gb300 import build

    build.build()
    checked = build.build(variant="check")
    n_chk, h_chk = _run(checked)
    n, h = _run(None)
    assert n_chk == n >= 40
    assert h_chk == h
