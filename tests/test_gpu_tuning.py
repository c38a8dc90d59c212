"""Launch-shape autotuner (hdg_autotune): it must pick shapes from its
candidate sets, leave the trace-operator apply bit for bit unchanged (the
apply's arithmetic does not depend on its block shape), and solves after
tuning must still match the oracle's direct solve and be reproducible."""
import math

import numpy as np
import pytest
import torch

from oracle.hdg import HDGProblem
from paper_2302_10917_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def rel(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300)


@pytest.mark.parametrize("n,m,p,beta", [(3, 4, 2, (0.8, -0.3)), (2, 8, 3, (50 * math.cos(0.3), 50 * math.sin(0.3)))])
def test_autotune_choices_and_solves(n, m, p, beta):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2302_10917_gb300 import Problem
    kappa = wl.random_kappa(2 * n * n, seed=11 * n + m)
    ora = HDGProblem(n, m, p, beta=beta, kappa=kappa)
    pts, _ = ora.quad_points()
    g = np.random.default_rng([wl.MASTER_SEED, 131, n, m, p])
    f = g.standard_normal(pts.shape[:2])
    S_el, g_ora, _ = ora.condense(f)
    x_ref = np.linalg.solve(ora.assemble_S(S_el), g_ora)
    pr = Problem(n, m, p, beta=beta, kappa=kappa)
    pr.set_source(torch.from_numpy(f))
    pr.condense(keep_factors=True, store_df64=True, store_fp32=True)
    gv = pr.rhs()
    v = torch.from_numpy(g.standard_normal(pr.info["N_tr"])).cuda()
    y_before = pr.apply(v, precond=True, prec=48)
    for mode in (2, 1, 0):
        rep = pr.autotune(mode=mode, restart=40)
        P1 = m * p + 1
        assert rep["apply_edges_per_block"] * P1 <= 512 and rep["apply_threads"] % 32 == 0
        assert rep["mdot_blocks"] in (608, 1216, 2432) and rep["update_blocks"] in (608, 1216, 2432, 4864)
        assert rep["apply_ms"] > 0 and rep["default_ms"] > 0
        x1, r1, st1 = pr.solve(gv, tol=1e-10, restart=40, mode=mode, orth=1)
        x2, r2, st2 = pr.solve(gv, tol=1e-10, restart=40, mode=mode, orth=1)
        assert st1 == 0 and r1["converged"] == 1
        assert torch.equal(x1, x2)
        assert rel(x1.cpu().numpy(), x_ref) < 1e-8
    assert torch.equal(pr.apply(v, precond=True, prec=48), y_before)
    pr.close()
