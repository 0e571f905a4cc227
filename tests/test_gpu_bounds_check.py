"""The bounds-checked build (libfrpcpf_checked.so: every partner index read
from the connectivity is checked on the device before use, and an index out
of range ends the run with FR_EBOUNDS instead of an access outside the
arrays) runs the GPU parity suites with no check firing: the residual, RK4,
preconditioning, tile-variant, batch, partitioned-march and adjoint parity
tests pass on it, and every field they create is destroyed with a status
free of FR_EBOUNDS (the package reads it at destruction under
FRP_BOUNDS_CHECK=1; the tests' conftest fails the test otherwise)."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.gpu
@pytest.mark.parametrize("suite,select", [
    ("tests/test_gpu_parity.py", "rhs_parity or march or pseudo or tile_variants or noflux"),
    ("tests/test_gpu_adjoint.py", ""),
    ("tests/test_gpu_batch.py", ""),
    ("tests/test_gpu_partition.py", ""),
])
def test_parity_suites_pass_on_the_bounds_checked_build(suite, select):
    from paper_2006_10967_gb300 import build
    build.build(checked=True)
    env = dict(os.environ, FRP_BOUNDS_CHECK="1")
    probe = subprocess.run([sys.executable, "-c", "import paper_2006_10967_gb300._capi as c; c.lib(); print(c.LIB_PATH)"],
                           cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert probe.stdout.strip().endswith("libfrpcpf_checked.so"), probe.stdout + probe.stderr
    cmd = [sys.executable, "-m", "pytest", suite, "-m", "gpu", "-q", "-x", "-p", "no:cacheprovider"]
    if select:
        cmd += ["-k", select]
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=1500)
    tail = "\n".join(r.stdout.splitlines()[-15:])
    assert r.returncode == 0, tail
    assert " passed" in tail and "failed" not in tail, tail
