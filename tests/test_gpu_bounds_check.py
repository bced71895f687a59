"""The bounds-check build (libdobfs_bc.so, -DDOBFS_BOUNDS_CHECK).

Run in a child process (bc_worker.py) so that this process keeps the normal
library: on valid graphs the checked build returns the oracle's results with
no check firing; on a graph with a column corrupted on purpose (a value just
past n, inside the build's allocation slack) every path fails with
DOBFS_ERR_BOUNDS and the library stays usable. The normal build refuses the
corrupting debug call.
"""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

HERE = os.path.dirname(os.path.abspath(__file__))


def test_bounds_check_build():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1503_04359_b300 import build
    build.build(bounds_check=True)
    env = dict(os.environ, DOBFS_BOUNDS_CHECK="1")
    r = subprocess.run([sys.executable, os.path.join(HERE, "bc_worker.py")], env=env, capture_output=True,
                       text=True, timeout=900)
    print(r.stdout)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.strip().endswith("OK")


def test_normal_build_refuses_debug_call():
    from paper_1503_04359_b300 import build, dobfs
    import dobfs_inputs as inputs
    build.build()
    assert dobfs.LIB_PATH.endswith("libdobfs.so")
    dobfs.load()
    dobfs.use_torch_allocator()
    g = dobfs.rmat_graph(inputs.rmat(8))
    with pytest.raises(dobfs.DobfsError) as e:
        dobfs.dobfs_debug_set_column(g.handle, 0, 1)
    assert e.value.status == dobfs.DOBFS_ERR_INVALID
    g.close()
