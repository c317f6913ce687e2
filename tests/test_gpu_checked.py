"""The bounds-checked build (librbffd_checked.so) on the GPU.

Every computed index of every kernel is tested before its access; a
violation is recorded and redirected instead of performed.  The checked
pipeline (checked_pipeline.py, its own process under RBFFD_CHECKED=1) runs
every stage on small node sets -- stencils, every weight kernel, assembly,
transpose, the Jacobi-scaled and multigrid solves, both adjoint hierarchies,
the explicit loop, every batched mode -- against the oracle, and reads the
violation records after each stage: none may appear, and the self-check
probes must each record theirs.
"""

import json
import os
import subprocess
import sys

import pytest

from conftest import ROOT

pytestmark = pytest.mark.gpu


def test_checked_pipeline_has_no_violations(lib):
    from paper_2107_03632_gb300 import _build

    _build.build(checked=True)
    env = dict(os.environ, RBFFD_CHECKED="1")
    env.pop("RBFFD_WEIGHTS", None)
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "checked_pipeline.py")], env=env,
                       capture_output=True, text=True, timeout=1200)
    assert r.returncode == 0, r.stderr[-4000:]
    report = json.loads(r.stdout.strip().splitlines()[-1])
    stages = report["stages"]
    print(f"checked build: {len(stages)} stages")
    for name, entry in stages.items():
        print(f"  {name}: {entry}")
    assert report["checked"] == 1
    assert not report["failures"], report["failures"]
    # every part ran (a part that raised is listed in failures above)
    for must in ("probe index", "stencils noalloc", "weights autotune", "adjoint galerkin m=6 n=56",
                 "explicit m=2 n=12", "batched mg-persistent rhs=3", "batched mg-device-loop rhs=4"):
        assert must in stages, must
    assert sum(1 for k in stages if k.startswith("weights ")) >= 25
