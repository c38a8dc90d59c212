"""Discrete adjoint and gradient (hdg_set_kappa, hdg_transpose, hdg_adjoint_rhs,
hdg_adjoint_recover, hdg_gradient and the autograd.Function on top of them).

Against the CPU oracle (oracle/adjoint.py, the full 3Q-unknown local systems):
the adjoint right-hand side, the trace adjoint nu, the element adjoint mu and
both gradients, on the same seeded inputs. The forward and adjoint GPU solves
run GMRES to a 1e-13 relative residual against the oracle's direct solves,
so the tolerances are 1e-9 (states) and 1e-8 (gradients), relative in the max
norm. Without the oracle: central differences of J through the GPU path along
20 seeded directions, and torch.autograd.gradcheck on a tiny case.
"""
import math

import numpy as np
import pytest
import torch

from oracle.adjoint import gradient as oracle_gradient
from oracle.hdg import HDGProblem
from paper_2302_10917_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

B1 = (50.0 * math.cos(0.3), 50.0 * math.sin(0.3))
CASES = [
    # id, n, m, p, beta
    ("m2p2", 2, 2, 2, (0.7, -0.4)),
    ("m4p2", 3, 4, 2, (1.0, 0.5)),       # the element of the gradient workload (m = 4, p = 2)
    ("m8p3", 2, 8, 3, B1),               # Q = 325: pivots across 21 LU panels
    ("n1", 1, 1, 1, (0.3, 0.2)),
    ("p4diff", 2, 2, 4, (0.0, 0.0)),
]
TIGHT = 1e-13


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.fixture(scope="module", params=CASES, ids=[c[0] for c in CASES])
def case(request):
    _need_gpu()
    from paper_2302_10917_gb300 import Problem
    cid, n, m, p, beta = request.param
    N = 2 * n * n
    kappa = wl.random_kappa(N, seed=7 * n + m + p)
    ora = HDGProblem(n, m, p, beta=beta, kappa=kappa)
    gpu = Problem(n, m, p, beta=beta, kappa=kappa)
    pts, _ = ora.quad_points()
    bpts, _ = ora.bnd_quad_points()
    g = np.random.default_rng([wl.MASTER_SEED, 83, n, m, p])
    f = g.standard_normal(pts.shape[:2])
    gD = g.standard_normal(bpts.shape[:2])
    r = g.standard_normal((N, ora.mesh.Q))          # dJ/du of J = sum r . u
    gk, gf, u_o, st = oracle_gradient(ora, f, r, gD, return_state=True)
    gpu.set_source(torch.from_numpy(f), torch.from_numpy(gD))
    gpu.condense(keep_factors=True, store_df64=True, store_fp32=True)
    x, rep, status = gpu.solve(gpu.rhs(), tol=TIGHT, restart=60)
    assert status == 0, rep
    u, _ = gpu.recover(x)
    torch.cuda.synchronize()
    yield dict(ora=ora, gpu=gpu, f=f, gD=gD, r=torch.from_numpy(r).cuda(), x=x, u=u, u_o=u_o,
               gk=gk, gf=gf, st=st, rng=g)
    gpu.close()


def test_transposed_apply_matches_oracle_and_transposes_back(case):
    ora, gpu = case["ora"], case["gpu"]
    S_el, _, _ = ora.condense(case["f"], case["gD"])
    St = ora.assemble_S(S_el).T
    v = case["rng"].standard_normal(ora.mesh.N_tr)
    vt = torch.from_numpy(v).cuda()
    y0 = gpu.apply(vt)
    y0p = gpu.apply(vt, precond=True)
    gpu.transpose()
    try:
        assert rel(gpu.apply(vt).cpu().numpy(), St @ v) < 1e-12
        assert rel(gpu.apply(vt, precond=True).cpu().numpy(), ora.apply_Dinv(St @ v)) < 1e-12
    finally:
        gpu.transpose()
    # transposing twice restores every stored copy bit for bit
    assert torch.equal(gpu.apply(vt), y0) and torch.equal(gpu.apply(vt, precond=True), y0p)


def test_adjoint_rhs_matches_oracle(case):
    g = case["gpu"].adjoint_rhs(case["r"]).cpu().numpy()
    assert rel(g, case["st"]["g_adj"]) < 1e-12


def test_adjoint_state_and_gradients_match_oracle(case):
    gpu = case["gpu"]
    # the forward solution itself first (direct solve on the oracle side)
    assert rel(case["u"].cpu().numpy(), case["u_o"]) < 1e-9
    g = gpu.adjoint_rhs(case["r"])
    gpu.transpose()
    try:
        nu, rep, status = gpu.solve(g, tol=TIGHT, restart=60)
    finally:
        gpu.transpose()
    assert status == 0, rep
    assert rel(nu.cpu().numpy(), case["st"]["nu"]) < 1e-9
    mu = gpu.adjoint_recover(case["r"], nu)
    assert rel(mu.cpu().numpy(), case["st"]["mu"]) < 1e-9
    dk, df = gpu.gradient(case["x"], case["u"], mu, nu)
    assert rel(dk.cpu().numpy(), case["gk"]) < 1e-8
    assert rel(df.cpu().numpy(), case["gf"]) < 1e-8


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_adjoint_driver_in_every_solve_mode(case, mode):
    dk, df, rep = case["gpu"].adjoint(case["r"], case["x"], case["u"], tol=TIGHT, restart=60, mode=mode)
    assert rep["converged"] == 1
    assert rel(dk.cpu().numpy(), case["gk"]) < 1e-8
    assert rel(df.cpu().numpy(), case["gf"]) < 1e-8


def test_adjoint_with_face_blocks(case):
    """The face-block preconditioner kept through the transpose ((S_ff^-1)^T for S^T):
    the same gradients as the oracle adjoint."""
    gpu = case["gpu"]
    gpu.condense(keep_factors=True, store_df64=True, store_fp32=True, precond="face_schur")
    try:
        x, rep, st = gpu.solve(gpu.rhs(), tol=TIGHT, restart=60, mode=2)
        assert st == 0, rep
        u, _ = gpu.recover(x)
        dk, df, rep = gpu.adjoint(case["r"], x, u, tol=TIGHT, restart=60, mode=2)
        assert rep["converged"] == 1
        assert rel(dk.cpu().numpy(), case["gk"]) < 1e-8
        assert rel(df.cpu().numpy(), case["gf"]) < 1e-8
    finally:
        gpu.condense(keep_factors=True, store_df64=True, store_fp32=True)


# ------------------------------------------------------------- without oracle
def _J_problem(n=4, m=4, p=2, beta=(1.0, 0.5), seed=1):
    from paper_2302_10917_gb300 import Problem
    kappa = torch.from_numpy(wl.grf_kappa(n, seed)).cuda()
    pr = Problem(n, m, p, beta=beta, kappa=kappa.cpu().numpy())
    xy = pr.quad_points()
    f = wl.sin_sin_source(xy, 1.0, beta).contiguous()
    kobs = torch.from_numpy(wl.grf_kappa(n, seed + 1000)).cuda()
    from paper_2302_10917_gb300 import solve_u
    with torch.no_grad():
        u_obs = solve_u(pr, kobs, f, tol=TIGHT).clone()
    return pr, kappa, f, u_obs


def test_gradient_matches_central_differences_on_20_directions():
    """J = 1/2 |u - u_obs|^2 through the GPU path; (J(k + h d) - J(k - h d)) / 2h
    along 20 seeded directions d against dJ/dkappa . d (h = 1e-4 relative,
    truncation ~1e-8, solve error ~1e-13 / h)."""
    _need_gpu()
    from paper_2302_10917_gb300 import solve_u
    pr, kappa, f, u_obs = _J_problem()
    k = kappa.clone().requires_grad_(True)
    ff = f.clone().requires_grad_(True)
    J = 0.5 * ((solve_u(pr, k, ff, tol=TIGHT) - u_obs) ** 2).sum()
    J.backward()
    J = J.detach()
    gk, gf = k.grad.clone(), ff.grad.clone()
    g = np.random.default_rng([wl.MASTER_SEED, 97])

    def J_at(kk, fv):
        with torch.no_grad():
            return float(0.5 * ((solve_u(pr, kk, fv, tol=TIGHT) - u_obs) ** 2).sum())
    for i in range(20):
        d = torch.from_numpy(g.standard_normal(kappa.shape[0])).cuda()
        h = 1e-4
        kd = kappa * h * d / d.abs().max()
        fd = (J_at(kappa + kd, f) - J_at(kappa - kd, f)) / (2 * h)
        ad = float((gk * kappa * d / d.abs().max()).sum())
        assert abs(ad - fd) <= 1e-6 * max(abs(fd), 1e-3 * float(J)), (i, ad, fd)
    # J is quadratic in f: the central difference along f is exact up to rounding
    for i in range(3):
        d = torch.from_numpy(g.standard_normal(tuple(f.shape))).cuda()
        fd = (J_at(kappa, f + d) - J_at(kappa, f - d)) / 2.0
        ad = float((gf * d).sum())
        assert abs(ad - fd) <= 1e-8 * max(abs(fd), float(J)), (i, ad, fd)
    pr.close()


def test_autograd_gradcheck_tiny():
    _need_gpu()
    from paper_2302_10917_gb300 import Problem, solve_u
    pr = Problem(1, 1, 1, beta=(0.6, -0.2), kappa=[1.0, 1.5])
    xy = pr.quad_points()
    f = (1.0 + xy[..., 0] * xy[..., 1]).contiguous().requires_grad_(True)
    k = torch.tensor([0.9, 1.3], dtype=torch.float64, device="cuda", requires_grad=True)
    fn = lambda kk, fv: solve_u(pr, kk, fv, tol=1e-14)
    assert torch.autograd.gradcheck(fn, (k, f), eps=1e-6, atol=1e-7, rtol=1e-5)
    pr.close()


def test_set_kappa_equals_a_fresh_context():
    _need_gpu()
    from paper_2302_10917_gb300 import Problem
    n, m, p, beta = 3, 4, 2, (1.0, 0.5)
    k1, k2 = wl.grf_kappa(n, 3), wl.grf_kappa(n, 4)
    a, b = Problem(n, m, p, beta=beta, kappa=k1), Problem(n, m, p, beta=beta, kappa=k2)
    f = torch.from_numpy(np.random.default_rng(5).standard_normal((2 * n * n, a.info["n_qp"])))
    for pr in (a, b):
        pr.set_source(f)
    a.set_kappa(torch.from_numpy(k2))
    a.condense()
    b.condense()
    assert torch.equal(a.schur(), b.schur()) and torch.equal(a.rhs(), b.rhs())
    v = torch.ones(a.info["N_tr"], dtype=torch.float64, device="cuda")
    assert torch.equal(a.apply(v, precond=True), b.apply(v, precond=True))
    a.close()
    b.close()


def test_adjoint_error_statuses():
    _need_gpu()
    from paper_2302_10917_gb300 import HDG_ERR_ARG, HDG_ERR_STATE, HDGError, Problem
    pr = Problem(2, 2, 2, beta=(1.0, 0.0), kappa=1.0)
    N, Q = pr.info["N"], pr.info["Q"]
    with pytest.raises(HDGError) as ei:
        pr.transpose()                       # before hdg_condense
    assert ei.value.status == HDG_ERR_STATE
    pr.set_source(torch.zeros(N, pr.info["n_qp"], dtype=torch.float64))
    pr.condense(keep_factors=False)
    r = torch.zeros(N, Q, dtype=torch.float64, device="cuda")
    with pytest.raises(HDGError) as ei:
        pr.adjoint_rhs(r)                    # factors not kept
    assert ei.value.status == HDG_ERR_STATE
    bad = torch.ones(N, dtype=torch.float64)
    bad[3] = -1.0
    with pytest.raises(HDGError) as ei:
        pr.set_kappa(bad)
    assert ei.value.status == HDG_ERR_ARG and "negative" in str(ei.value)
    bad[3] = float("nan")
    with pytest.raises(HDGError) as ei:
        pr.set_kappa(bad)
    assert ei.value.status == HDG_ERR_ARG
    pr.set_kappa(torch.ones(N, dtype=torch.float64))
    with pytest.raises(HDGError) as ei:
        pr.apply(torch.ones(pr.info["N_tr"], dtype=torch.float64))   # blocks stale after set_kappa
    assert ei.value.status == HDG_ERR_STATE
    pr.close()
