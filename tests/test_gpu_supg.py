"""SUPG stabilisation (Sec. 3.4) on the GPU path against the oracle: Schur
blocks of every element (FP64 and split-FP32 condensation), right-hand sides
with the SUPG load, the solution against the oracle's direct solve, and
polynomial exactness (the SUPG residual vanishes for the exact solution).

Tolerance of the Schur blocks and right-hand sides: 5e-11 relative (1e-12 without SUPG). The
consistency term -tau_s kappa (a . grad w, Lap u) of the SUPG residual lowers
the smallest singular value of A_u: at m = 8, p = 3, beta = 50, kappa ~ 1 the
measured cond(A_u) grows from 1.2e2 to 5.6e4 and that of the oracle's full
3Q system from 1.2e5 to 3.5e8, so the two LU factorisations (different
formulations, pivot orders and rounding) legitimately differ by up to about
cond x 1e-16; measured 2.3e-11 (the bound keeps 2x slack). The polynomial-exactness test below pins the
SUPG terms independently of that conditioning.
"""
import math

import numpy as np
import pytest
import torch

from oracle.hdg import HDGProblem
from oracle.problems import polynomial, random_polynomial
from paper_2302_10917_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

B1 = (50.0 * math.cos(0.3), 50.0 * math.sin(0.3))
CASES = [("m4p2", 2, 4, 2, (1.0, 0.5), 1e-3), ("m2p3", 2, 2, 3, (0.9, -0.4), 0.05), ("m8p3", 2, 8, 3, B1, 1.0),
         ("m1p2", 3, 1, 2, (1.0, 1.0), 1e-5)]


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.mark.parametrize("cid,n,m,p,beta,kscale", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("split", [False, True])
def test_supg_condensation_rhs_and_solve(cid, n, m, p, beta, kscale, split):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2302_10917_gb300 import Problem
    kappa = kscale * wl.random_kappa(2 * n * n, seed=3 * n + m + p)
    ora = HDGProblem(n, m, p, beta=beta, kappa=kappa, supg=True)
    pts, _ = ora.quad_points()
    bpts, _ = ora.bnd_quad_points()
    g = np.random.default_rng([wl.MASTER_SEED, 173, n, m, p])
    f = g.standard_normal(pts.shape[:2])
    gD = g.standard_normal(bpts.shape[:2])
    S_el, g_ora, ghat = ora.condense(f, gD)
    pr = Problem(n, m, p, beta=beta, kappa=kappa, supg=True)
    pr.set_source(torch.from_numpy(f), torch.from_numpy(gD))
    pr.condense(keep_factors=True, store_df64=True, split_update=split)
    S = pr.schur().cpu().numpy()
    for e in range(S.shape[0]):
        assert rel(S[e], S_el[e]) < 5e-11, e
    gv = pr.rhs()
    assert rel(gv.cpu().numpy(), g_ora) < 5e-11        # -C A^-1 R: the same conditioning as S
    Sa = ora.assemble_S(S_el)
    x, rep, st = pr.solve(gv, tol=1e-11, restart=60, mode=2, orth=1, maxit=40000)
    assert st == 0, (rep, np.linalg.cond(Sa))
    x_ref = np.linalg.solve(Sa, g_ora)
    assert rel(x.cpu().numpy(), x_ref) < 1e-8, np.linalg.cond(Sa)
    u, q = pr.recover(x)
    u_o, q_o = ora.recover(x_ref, f, ghat)
    assert rel(u.cpu().numpy(), u_o) < 1e-8
    pr.close()


@pytest.mark.parametrize("n,m,p", [(3, 2, 2), (2, 2, 3)])
def test_supg_polynomial_exactness_gpu(n, m, p):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2302_10917_gb300 import Problem
    kap, beta = 0.05, (0.9, -0.4)
    ora = HDGProblem(n, m, p, beta=beta, kappa=kap)
    u, gr, f = polynomial(random_polynomial(p, seed=41 + p), kap, beta)
    pts, _ = ora.quad_points()
    bpts, _ = ora.bnd_quad_points()
    pr = Problem(n, m, p, beta=beta, kappa=kap, supg=True)
    pr.set_source(torch.from_numpy(f(pts[..., 0], pts[..., 1])), torch.from_numpy(u(bpts[..., 0], bpts[..., 1])))
    pr.condense(split_update=True, store_df64=True)
    x, rep, st = pr.solve(pr.rhs(), tol=1e-13, restart=120, mode=0, maxit=40000)
    assert st == 0, rep
    uu, qq = pr.recover(x)
    eu, eq = ora.l2_errors(uu.cpu().numpy(), qq.cpu().numpy(), u, gr)
    assert eu < 1e-10 and eq < 1e-9, (eu, eq)
    pr.close()


def test_gradient_refused_with_supg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2302_10917_gb300 import HDG_ERR_STATE, HDGError, Problem
    pr = Problem(2, 2, 2, beta=(1.0, 0.0), kappa=1.0, supg=True)
    N, Q = pr.info["N"], pr.info["Q"]
    pr.set_source(torch.ones(N, pr.info["n_qp"], dtype=torch.float64))
    pr.condense()
    x, _, _ = pr.solve(pr.rhs(), tol=1e-10)
    u, _ = pr.recover(x)
    with pytest.raises(HDGError) as ei:
        pr.gradient(x, u, torch.zeros_like(u), torch.zeros_like(x))
    assert ei.value.status == HDG_ERR_STATE and "SUPG" in str(ei.value)
    pr.close()
