"""The small parity suites rerun against libmapsq_checked.so, the build whose
kernels check their device indexes (a failed check sets a status bit and
skips the access; the call then fails).  Every join, star join, SELECT and
query of those suites must stay exact and raise no bounds error."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CHECKED = os.path.join(ROOT, "paper_1702_03484_gb300", "libmapsq_checked.so")


def test_parity_suites_under_the_checked_build():
    assert os.path.exists(CHECKED), "build() makes libmapsq_checked.so beside libmapsq.so"
    env = dict(os.environ, MAPSQ_LIB=CHECKED)
    info = subprocess.run([sys.executable, "-c", "from paper_1702_03484_gb300 import mapsq; "
                           "print(mapsq.lib().mapsq_build_info().decode())"],
                          env=env, cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert info.stdout.strip() == "sm_103a checked", info.stderr[-2000:]
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-m", "gpu", "-p", "no:cacheprovider",
                        "tests/test_gpu_join.py", "tests/test_gpu_star.py", "tests/test_gpu_select.py",
                        "tests/test_gpu_query.py", "-k", "not autotune and not full_size and not slices"],
                       env=env, cwd=ROOT, capture_output=True, text=True, timeout=1500)
    assert r.returncode == 0, r.stdout[-4000:] + r.stderr[-2000:]
