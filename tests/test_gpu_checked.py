"""The tracking chain built with every subscript of its workspace and input
arrays range-checked on the device (build.py --checked; selected at run time
by TPCT_CHECKED=1).  The parity tests of the single sector, the central
event and the collision batches, the hand-worked tracklet fixture and the
edge cases run on that build; each of them asserts a clean device status, so
an index outside its array anywhere in the chain (TPCT_E_BOUNDS) fails them.
The checked build stands in for a memory checker on this GPU: it reports the
first bad index instead of faulting."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_parity_suite_under_the_bounds_checked_build():
    import paper_2502_09138_gb300.build as b
    lib = b.build(checked=True)
    env = dict(os.environ, TPCT_CHECKED="1")
    probe = subprocess.run([sys.executable, "-c", "import paper_2502_09138_gb300.binding as B; print(B.LIB_PATH)"],
                           cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert probe.returncode == 0 and probe.stdout.strip() == lib, probe.stdout + probe.stderr
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-m", "gpu", "-p", "no:cacheprovider",
                        "tests/test_gpu_parity.py", "tests/test_gpu_tracklet_fixture.py",
                        "tests/test_gpu_edge_cases.py"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=1800)
    assert r.returncode == 0, r.stdout[-4000:] + r.stderr[-2000:]
