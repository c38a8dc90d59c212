"""The bounds-checked build of the library on the small parity cases.

`_build.build_bounds_checked()` compiles the library with -DHDG_BOUNDS_CHECK:
the guarded device indices (trace gathers of the applies and the back-solve,
the row-blocks and outputs of the trace apply, the bulk copies of the
pipelined apply, the element-side products and face sums of the level-mesh
apply) are checked, the first failure is recorded as a site code and the
access is skipped, without a trap. A fresh interpreter loads that library and
runs uniform and level meshes through every apply precision, the pipelined
apply, single and batched solves with both Krylov bases, and the back-solve;
every result must still match the oracle and no check may have failed.
"""
import json
import os
import subprocess
import sys

import pytest
import torch

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import json, math, sys
import numpy as np
import torch
sys.path.insert(0, sys.argv[1])
import paper_2302_10917_gb300 as pkg
from paper_2302_10917_gb300 import _build
pkg.load_library(_build.LIB_BOUNDS_CHECK)
from paper_2302_10917_gb300 import Problem
from paper_2302_10917_gb300 import workloads as wl
from oracle.hdg import HDGProblem
from oracle.levels import LevelHDGProblem

def rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))

out = {"bounds": [], "err": {}}
for (n, m, p, beta) in ((3, 4, 2, (0.8, -0.3)), (2, 8, 3, (50 * math.cos(0.3), 50 * math.sin(0.3)))):
    kap = wl.random_kappa(2 * n * n, seed=n + m)
    ora = HDGProblem(n, m, p, beta=beta, kappa=kap)
    pts, _ = ora.quad_points()
    g = np.random.default_rng([wl.MASTER_SEED, 211, n, m])
    f = g.standard_normal(pts.shape[:2])
    S_el, g_o, ghat = ora.condense(f, None)
    Sa = ora.assemble_S(S_el)
    x_dir = np.linalg.solve(Sa, g_o)
    pr = Problem(n, m, p, beta=beta, kappa=kap)
    pr.set_source(torch.from_numpy(f))
    pr.condense(keep_factors=True, store_fp32=True, store_df64=True)
    key = f"n{n}m{m}p{p}"
    S = pr.schur().cpu().numpy()
    out["err"][key + "_S"] = max(rel(S[e], S_el[e]) for e in range(S.shape[0]))
    v = g.standard_normal(ora.mesh.N_tr)
    out["err"][key + "_apply64"] = rel(pr.apply(torch.from_numpy(v)).cpu().numpy(), Sa @ v)
    zp = ora.apply_Dinv(Sa @ v)
    for prec in (48, 33):
        out["err"][key + f"_apply{prec}"] = rel(pr.apply(torch.from_numpy(v), precond=True, prec=prec).cpu().numpy(), zp)
    X = g.standard_normal((3, ora.mesh.N_tr))
    Y = pr.apply(torch.from_numpy(X)).cpu().numpy()
    out["err"][key + "_mrhs"] = rel(Y, X @ Sa.T)
    try:
        pr.set_apply_shape(2, bulk_warps=1)
        hi = v.astype(np.float32)
        xs = torch.from_numpy(np.stack([hi, (v - hi).astype(np.float32)], axis=1))
        y = pr.apply(xs, precond=True, prec=49).cpu().numpy().astype(np.float64)
        out["err"][key + "_bulk"] = rel(y[:, 0] + y[:, 1], zp)
        pr.set_apply_shape(2)
    except pkg.HDGError:
        pass
    for mode in (0, 1, 2):
        for basis in (0, 1):
            x, rep, st = pr.solve(pr.rhs(), tol=1e-10, restart=30, mode=mode, basis=basis, orth=3)
            out["err"][key + f"_solve{mode}{basis}"] = rel(x.cpu().numpy(), x_dir)
    u, q = pr.recover(torch.from_numpy(x_dir))
    u_o, q_o = ora.recover(x_dir, f, ghat)
    out["err"][key + "_recover"] = max(rel(u.cpu().numpy(), u_o), rel(q.cpu().numpy(), q_o))
    out["bounds"].append(pr.bounds_error())
    pr.close()
# batched solve (several sources) and a level mesh
n, m, p, beta = 2, 2, 2, (1.0, 0.5)
pr = Problem(n, m, p, beta=beta, kappa=1.0)
F = torch.from_numpy(np.random.default_rng(5).standard_normal((3, pr.info["N"], pr.info["n_qp"])))
pr.set_source(F)
pr.condense(keep_factors=True, store_df64=True)
for basis in (0, 1):
    x, rep, st = pr.solve(pr.rhs(), tol=1e-10, restart=20, mode=2, basis=basis)
    out["err"][f"batched{basis}"] = rep["rel_residual"]
pr.recover(x)
out["bounds"].append(pr.bounds_error())
pr.close()
lev = np.array([0, 1, 2, 1, 0, 2, 1, 1], dtype=np.int8)
ora = LevelHDGProblem(2, lev, 2, beta=(1.0, -0.5), kappa=1.0)
f = np.random.default_rng(7).standard_normal(ora.qoff[-1])
S_lv, g_lv, gh_lv = ora.condense(f)
x_dir = np.linalg.solve(ora.assemble_S(S_lv), g_lv)
pr = Problem(2, 1, 2, beta=(1.0, -0.5), kappa=1.0, levels=lev)
pr.set_source(torch.from_numpy(f))
pr.condense(keep_factors=True, store_fp32=True, store_df64=True)
v = np.random.default_rng(8).standard_normal(ora.N_tr)
out["err"]["level_apply"] = rel(pr.apply(torch.from_numpy(v)).cpu().numpy(), ora.assemble_S(S_lv) @ v)
for mode in (0, 2):
    x, rep, st = pr.solve(pr.rhs(), tol=1e-12, restart=30, mode=mode)
    out["err"][f"level_solve{mode}"] = rel(x.cpu().numpy(), x_dir)
pr.recover(x)
out["bounds"].append(pr.bounds_error())
pr.close()
print(json.dumps(out))
"""


def test_bounds_checked_build_passes_the_small_parity_cases():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2302_10917_gb300 import _build
    _build.build_bounds_checked()
    res = subprocess.run([sys.executable, "-c", SCRIPT, ROOT], cwd=ROOT, capture_output=True, text=True, timeout=900)
    assert res.returncode == 0, res.stderr[-3000:]
    out = json.loads(res.stdout.strip().splitlines()[-1])
    assert out["bounds"] == [0] * len(out["bounds"]), out["bounds"]
    err = out["err"]
    for k, v in err.items():
        if k.startswith("batched"):
            assert v <= 1e-10, (k, v)
        elif k.endswith("apply33") or k.endswith("_bulk"):
            assert v < (5e-5 if k.endswith("apply33") else 1e-12), (k, v)
        elif "solve" in k:
            assert v < 1e-8, (k, v)
        else:
            assert v < 1e-11, (k, v)
