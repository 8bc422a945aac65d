"""The bounds-checked debug build (libdg_elliptic_debug.so, `build.py --debug`, loaded with
DG_DEBUG_BUILD=1): built on the GPU machine, it runs small Poisson (FP64 and mixed, two levels: the
gather, the residual written into the subdomain vectors, the scatter) and puncture solves (the
linearized subdomain solver) with every set-up-table index in range, and reaches the release
build's solutions (same launch shapes: the checks change no arithmetic). The release build answers
-1 (no checks)."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

dgg = pytest.importorskip("paper_2111_06767_gb300")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

_CHILD = r"""
import json, sys
sys.path.insert(0, sys.argv[1])
import numpy as np, torch
import workloads
import paper_2111_06767_gb300 as dgg
out = {"before": dgg.debug_bounds_check()}
for prec in ("fp64", "mixed"):
    d = dgg.Domain(n=(4, 4, 2), N=5, precision=prec, mg_levels=2, overlap=2)
    x, y, z = d.coordinates()
    b = d.rhs(workloads.gaussian_source(3)(x, y, z).contiguous())
    u = torch.zeros_like(b)
    rep = d.solve(b, u, 1e-10)
    out["poisson_" + prec] = [rep.status, u.cpu().numpy().tolist()]
dp = dgg.Domain((-20.0,) * 3, (20.0,) * 3, (3, 3, 3), 5, precision="mixed", overlap=2, problem="puncture",
                punctures=workloads.BINARY_PUNCTURES)
up = torch.zeros(dp.n_dof, dtype=torch.float64, device="cuda")
rep = dp.solve(None, up, 1e-10, opts=dgg.solve_opts(linear_tol=1e-4))
out["puncture"] = [rep.status, up.cpu().numpy().tolist()]
out["after"] = dgg.debug_bounds_check()
print(json.dumps(out))
"""


def _run(env_extra):
    env = dict(os.environ, **env_extra)
    res = subprocess.run([sys.executable, "-c", _CHILD, ROOT], capture_output=True, text=True, env=env, timeout=900,
                         check=True, cwd=ROOT)
    return json.loads([l for l in res.stdout.splitlines() if l.startswith("{")][-1])


def test_debug_build_solves_with_every_index_in_range():
    subprocess.run([sys.executable, os.path.join(ROOT, "paper_2111_06767_gb300", "build.py"), "--debug"], check=True,
                   timeout=900, capture_output=True)
    # fixed launch shapes in both processes (the autotuner's timing could pick different ones)
    rel = _run({"DG_DEBUG_BUILD": "0", "DG_AUTOTUNE": "0"})
    dbg = _run({"DG_DEBUG_BUILD": "1", "DG_AUTOTUNE": "0"})
    assert rel["before"] == -1 and rel["after"] == -1
    assert dbg["before"] == 0 and dbg["after"] == 0
    for key in ("poisson_fp64", "poisson_mixed", "puncture"):
        assert rel[key][0] == 0 and dbg[key][0] == 0, key
        a, b = np.array(rel[key][1]), np.array(dbg[key][1])
        assert np.linalg.norm(a - b) <= 1e-12 * np.linalg.norm(a), key
