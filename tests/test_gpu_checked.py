"""Bounds-checked build (libfds_checked.so, -DFDS_CHECKS): every
index-mapped gather and scatter checks its index against the buffer it
addresses.  The whole path (FP64 build and solve, the learned-rank mixed
build with tensor-core products and CUDA-graph sweeps, the Woodbury form,
the field through the skeletons) runs with no access out of range, and
gives the unchecked library's answers."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

from gpu_util import fdslib, torch_cuda

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROG = r"""
import json, sys
import numpy as np
import torch
import workloads
from paper_2411_18026_gb300 import fds, learned
out = sys.argv[1]
xy = workloads.star(4096, 0.25, 6, rot=0.3)
om = workloads.omega_for_kTa(12.0)
kinds, ang = workloads.plane_wave_set(3)
prm = learned.load_params()
res, viol = {}, {}
cases = {
    "fp64": {},
    "mixed": dict(precision=fds.FDS_MIXED, ir_tol=1e-10, mlp_params=prm, merge_c64=True,
                  fw_engine=fds.FDS_FW_TENSOR, c64_engine=fds.FDS_C64_TENSOR, use_graph=1),
    "mr2005": dict(variant=fds.FDS_VARIANT_MR2005),
    "single": dict(top_level=-1),
}
for name, kw in cases.items():
    h = fds.fds_build(xy, om, 2.0, 1.0, 1e-9, **kw)
    F = fds.fds_rhs_plane_wave(h, kinds, ang)
    res[name] = fds.fds_solve(h, F)
    if name == "fp64":
        d = torch.tensor(np.ascontiguousarray(res[name].T), device="cuda")
        pts = np.array([[1.6, 0.2], [-0.3, 1.9], [0.1, -2.4]])
        res["field"] = fds.fds_field(h, d, kinds, ang, pts, compressed=True)
    h.close()
    viol[name] = fds.fds_bounds_violations()
np.savez(out, **res)
print(json.dumps(viol))
"""


def test_checked_library_no_out_of_range_access(tmp_path):
    torch_cuda()
    fds = fdslib()
    from paper_2411_18026_gb300 import build
    lib = build.build(checked=True)
    # the default library has no checks
    with pytest.raises(fds.FdsError) as e:
        fds.fds_bounds_violations()
    assert e.value.code == fds.FDS_ERR_STATE
    out = str(tmp_path / "checked.npz")
    env = dict(os.environ, FDS_LIB=lib, PYTHONPATH=ROOT + os.pathsep + os.environ.get("PYTHONPATH", ""))
    r = subprocess.run([sys.executable, "-c", PROG, out], env=env, cwd=ROOT, capture_output=True, text=True,
                       timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    viol = json.loads(r.stdout.strip().splitlines()[-1])
    assert viol == {"fp64": 0, "mixed": 0, "mr2005": 0, "single": 0}, viol
    got = np.load(out)
    # the same cases through the unchecked library
    import workloads
    from paper_2411_18026_gb300 import learned
    import torch
    xy = workloads.star(4096, 0.25, 6, rot=0.3)
    om = workloads.omega_for_kTa(12.0)
    kinds, ang = workloads.plane_wave_set(3)
    h = fds.fds_build(xy, om, 2.0, 1.0, 1e-9)
    F = fds.fds_rhs_plane_wave(h, kinds, ang)
    x = fds.fds_solve(h, F)
    d = torch.tensor(np.ascontiguousarray(x.T), device="cuda")
    fld = fds.fds_field(h, d, kinds, ang, np.array([[1.6, 0.2], [-0.3, 1.9], [0.1, -2.4]]), compressed=True)
    h.close()
    # two builds agree to rounding times the condition number (the tile
    # evaluator's atomics add in no fixed order; measured 6.7e-12)
    assert np.linalg.norm(got["fp64"] - x) <= 1e-10 * np.linalg.norm(x)
    assert np.abs(got["field"] - fld).max() <= 1e-10 * np.abs(fld).max()
    for name in ("mixed", "mr2005", "single"):
        assert np.linalg.norm(got[name] - x) <= 1e-8 * np.linalg.norm(x), name
