"""The bounds-check build (-DFEM_DEBUG_BOUNDS), the stand-in for a memory checker:
the patch kernels test every index they take from plan data (node ids of the
closure, element ids, closure-local node indices, accumulator targets, row
offsets and CSR positions) before the access, skip a bad one and report it as
FEM_ERR_INDEX.  Run in a child process, since the library is chosen when the
package is imported.  No access is ever made out of bounds: the planted id is
tested before the load it would feed."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

HERE = os.path.dirname(os.path.abspath(__file__))


def test_bounds_check_build():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    env = dict(os.environ, FEM_DEBUG_BOUNDS="1")
    r = subprocess.run([sys.executable, os.path.join(HERE, "debug_bounds_run.py")], env=env, capture_output=True,
                       text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    out = json.loads(r.stdout.strip().splitlines()[-1])
    assert out["lib"].endswith(os.path.join("_build", "debug", "libfem.so"))
    assert out["clean"] and all(out["clean"].values()), out["clean"]
    assert out["planted"] == "FEM_ERR_INDEX"
    assert out["after"]
