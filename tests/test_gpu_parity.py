"""GPU path (C ABI, sm_103a) against the FP64 CPU oracle, element by element.

Inputs are seeded and shared: the same per-element kappa, the same source
values at the published quadrature points, the same Dirichlet data and the
same trace vectors go to both sides. Tolerances (FP64 everywhere):
  Schur blocks, right-hand side, operator apply: 1e-12 relative (max norm);
  back-solve from the same trace: 1e-11 relative;
  GMRES to a 1e-10 residual against the oracle's direct solve: 1e-8 relative.
"""
import math

import numpy as np
import pytest
import torch

from oracle.hdg import HDGProblem
from oracle.problems import polynomial, random_polynomial
from paper_2302_10917_gb300 import BASIS_DF64, BASIS_FIX, BASIS_FP64
from paper_2302_10917_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

B1 = (50.0 * math.cos(0.3), 50.0 * math.sin(0.3))
CASES = [
    # id, n, m, p, beta, kappa mode
    ("smoke_n4_m2_p2", 4, 2, 2, (1.0, 1.0), "const"),        # the small workload
    ("m4p2", 3, 4, 2, (0.8, -0.3), "rand"),
    ("m8p3", 2, 8, 3, B1, "rand"),              # the large workload's element (Q = 325: 21 LU panels)
    ("n1", 1, 1, 1, (0.3, 0.2), "rand"),         # two elements, one interior edge
    ("m1p3", 5, 1, 3, (1.0, -2.0), "rand"),      # standard HDG (m = 1)
    ("p4diff", 2, 2, 4, (0.0, 0.0), "rand"),     # p = 4, pure diffusion
    ("m16p1", 1, 16, 1, (2.0, 1.0), "rand"),     # largest m
]


def _lib_problem(n, m, p, beta, kappa):
    from paper_2302_10917_gb300 import Problem
    return Problem(n, m, p, beta=beta, kappa=kappa)


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.fixture(scope="module", params=CASES, ids=[c[0] for c in CASES])
def case(request):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    cid, n, m, p, beta, kmode = request.param
    N = 2 * n * n
    kappa = 1.0 if kmode == "const" else wl.random_kappa(N, seed=n * 100 + m * 10 + p)
    ora = HDGProblem(n, m, p, beta=beta, kappa=kappa)
    gpu = _lib_problem(n, m, p, beta, kappa)
    pts, _ = ora.quad_points()
    bpts, _ = ora.bnd_quad_points()
    g = np.random.default_rng([wl.MASTER_SEED, n, m, p])
    f_qp = g.standard_normal(pts.shape[:2])
    gD = g.standard_normal(bpts.shape[:2])
    S_el, g_ora, ghat = ora.condense(f_qp, gD)
    gpu.set_source(torch.from_numpy(f_qp), torch.from_numpy(gD))
    gpu.condense(store_fp32=True, keep_factors=True, store_df64=True)
    torch.cuda.synchronize()
    yield dict(ora=ora, gpu=gpu, f=f_qp, gD=gD, S_el=S_el, g=g_ora, ghat=ghat, n=n, m=m, p=p, rng=g)
    gpu.close()


def test_quadrature_points_match(case):
    ora, gpu = case["ora"], case["gpu"]
    pts, _ = ora.quad_points()
    bpts, _ = ora.bnd_quad_points()
    assert np.abs(gpu.quad_points().cpu().numpy() - pts).max() < 1e-14
    assert np.abs(gpu.bnd_quad_points().cpu().numpy() - bpts).max() < 1e-14


def test_schur_blocks_match_every_element(case):
    S_gpu = case["gpu"].schur().cpu().numpy()
    S_ora = case["S_el"]
    assert S_gpu.shape == S_ora.shape
    for e in range(S_ora.shape[0]):
        assert rel(S_gpu[e], S_ora[e]) < 1e-12, e


def test_split_fp32_panel_updates_keep_fp64_parity(case):
    """HDG_SPLIT_UPDATE: the LU's panel products on the FP32 pipe, everything else FP64."""
    ora = case["ora"]
    gpu2 = _lib_problem(case["n"], case["m"], case["p"], tuple(ora.beta), ora.kappa)
    gpu2.set_source(torch.from_numpy(case["f"]), torch.from_numpy(case["gD"]))
    gpu2.condense(keep_factors=True, split_update=True)
    S_gpu = gpu2.schur().cpu().numpy()
    for e in range(S_gpu.shape[0]):
        assert rel(S_gpu[e], case["S_el"][e]) < 1e-12, e
    assert rel(gpu2.rhs().cpu().numpy(), case["g"]) < 1e-12
    x = np.linalg.solve(ora.assemble_S(case["S_el"]), case["g"])
    u_o, q_o = ora.recover(x, case["f"], case["ghat"])
    u_g, q_g = gpu2.recover(torch.from_numpy(x))
    assert rel(u_g.cpu().numpy(), u_o) < 1e-11 and rel(q_g.cpu().numpy(), q_o) < 1e-11
    gpu2.close()


def test_tensor_core_updates_keep_fp64_parity(case):
    """HDG_TC_UPDATE: 32-column FP64 panels, trailing updates as exact 8-bit slice products on
    the tensor cores: Schur blocks, right-hand side and back-solve at the FP64 bounds."""
    ora = case["ora"]
    gpu2 = _lib_problem(case["n"], case["m"], case["p"], tuple(ora.beta), ora.kappa)
    gpu2.set_source(torch.from_numpy(case["f"]), torch.from_numpy(case["gD"]))
    gpu2.condense(keep_factors=True, tc_update=True)
    S_gpu = gpu2.schur().cpu().numpy()
    for e in range(S_gpu.shape[0]):
        assert rel(S_gpu[e], case["S_el"][e]) < 1e-12, e
    assert rel(gpu2.rhs().cpu().numpy(), case["g"]) < 1e-12
    x = np.linalg.solve(ora.assemble_S(case["S_el"]), case["g"])
    u_o, q_o = ora.recover(x, case["f"], case["ghat"])
    u_g, q_g = gpu2.recover(torch.from_numpy(x))
    assert rel(u_g.cpu().numpy(), u_o) < 1e-11 and rel(q_g.cpu().numpy(), q_o) < 1e-11
    # without kept factors the back-solve condenses again with the same kernel
    gpu2.condense(keep_factors=False, tc_update=True)
    u_g, q_g = gpu2.recover(torch.from_numpy(x))
    assert rel(u_g.cpu().numpy(), u_o) < 1e-11 and rel(q_g.cpu().numpy(), q_o) < 1e-11
    gpu2.close()


def test_condensed_rhs_matches(case):
    assert rel(case["gpu"].rhs().cpu().numpy(), case["g"]) < 1e-12


def test_apply_matches_on_random_and_structured_vectors(case):
    ora, gpu, S_el = case["ora"], case["gpu"], case["S_el"]
    N_tr = ora.mesh.N_tr
    Df = ora.face_D()
    vecs = [case["rng"].standard_normal(N_tr), np.ones(N_tr), np.zeros(N_tr)]
    e0 = np.zeros(N_tr)
    e0[N_tr // 2] = 1.0
    vecs.append(e0)
    for x in vecs:
        y_ora = ora.apply_S(S_el, x)
        y_gpu = gpu.apply(torch.from_numpy(x)).cpu().numpy()
        if np.abs(y_ora).max() == 0.0:
            assert np.abs(y_gpu).max() == 0.0
            continue
        assert rel(y_gpu, y_ora) < 1e-12
        z_ora = ora.apply_Dinv(y_ora, Df)
        z_gpu = gpu.apply(torch.from_numpy(x), precond=True).cpu().numpy()
        assert rel(z_gpu, z_ora) < 1e-12


def test_apply_matches_literal_four_step_algorithm(case):
    ora, gpu = case["ora"], case["gpu"]
    if ora.mesh.N > 32 or ora.mesh.Q > 100:
        pytest.skip("the literal four-step oracle is kept to small cases")
    x = case["rng"].standard_normal(ora.mesh.N_tr)
    assert rel(gpu.apply(torch.from_numpy(x)).cpu().numpy(), ora.apply_four_step(x)) < 1e-12
    assert rel(gpu.apply(torch.from_numpy(x), precond=True).cpu().numpy(),
               ora.apply_four_step(x, precondition=True)) < 1e-11


def test_fp32_preconditioned_apply(case):
    ora, gpu, S_el = case["ora"], case["gpu"], case["S_el"]
    x = case["rng"].standard_normal(ora.mesh.N_tr)
    z_ora = ora.apply_Dinv(ora.apply_S(S_el, x))
    z32 = gpu.apply(torch.from_numpy(x).float(), precond=True, prec=32).double().cpu().numpy()
    # FP32 blocks and FP32 accumulation over n_t terms: a few units of 2^-24 times the row sum
    assert rel(z32, z_ora) < 5e-5


def test_fp32_blocks_on_fp64_vectors_apply(case):
    """prec = 33: the FP32 blocks on FP64 vectors, the Arnoldi operator of mode 1 with the
    FP64 Krylov basis (the mixed-precision form): FP32 products and sums, FP64 in and out."""
    ora, gpu, S_el = case["ora"], case["gpu"], case["S_el"]
    x = case["rng"].standard_normal(ora.mesh.N_tr)
    z_ora = ora.apply_Dinv(ora.apply_S(S_el, x))
    z33 = gpu.apply(torch.from_numpy(x), precond=True, prec=33).cpu().numpy()
    assert rel(z33, z_ora) < 5e-5


def test_split_fp32_preconditioned_apply(case):
    """Blocks stored as FP32 hi/lo pairs, products on the FP32 pipe: FP64-level agreement."""
    ora, gpu, S_el = case["ora"], case["gpu"], case["S_el"]
    x = case["rng"].standard_normal(ora.mesh.N_tr)
    z_ora = ora.apply_Dinv(ora.apply_S(S_el, x))
    z_df = gpu.apply(torch.from_numpy(x), precond=True, prec=48).cpu().numpy()
    assert rel(z_df, z_ora) < 1e-12


def test_recover_from_same_trace(case):
    ora, gpu = case["ora"], case["gpu"]
    x = np.linalg.solve(ora.assemble_S(case["S_el"]), case["g"])
    u_o, q_o = ora.recover(x, case["f"], case["ghat"])
    u_g, q_g = gpu.recover(torch.from_numpy(x))
    assert rel(u_g.cpu().numpy(), u_o) < 1e-11
    assert rel(q_g.cpu().numpy(), q_o) < 1e-11


def test_gmres_solution_matches_direct_solve(case):
    """The all-FP64 solve (FP64 blocks, FP64 Krylov basis and orthogonalisation, the
    default options) against the oracle's direct solve of the assembled S."""
    ora, gpu = case["ora"], case["gpu"]
    S = ora.assemble_S(case["S_el"])
    x_dir = np.linalg.solve(S, case["g"])
    g_gpu = gpu.rhs()
    x_gpu, rep, st = gpu.solve(g_gpu, tol=1e-10, restart=30, maxit=5000)
    assert st == 0 and rep["converged"] == 1 and rep["rel_residual"] <= 1e-10
    x_gpu = x_gpu.cpu().numpy()
    # the reported residual is the true one
    assert abs(np.linalg.norm(case["g"] - S @ x_gpu) / np.linalg.norm(case["g"]) - rep["rel_residual"]) < 1e-12
    assert rel(x_gpu, x_dir) < 1e-8
    u_g, q_g = gpu.recover(torch.from_numpy(x_gpu))
    u_o, q_o = ora.recover(x_dir, case["f"], case["ghat"])
    assert rel(u_g.cpu().numpy(), u_o) < 1e-8
    assert rel(q_g.cpu().numpy(), q_o) < 1e-7


@pytest.mark.parametrize("basis", [BASIS_FP64, BASIS_DF64, BASIS_FIX])
def test_gmres_split_fp32_apply_mode(case, basis):
    """mode 2: GMRES with the split-FP32 preconditioned apply; the FP64 residual decides."""
    ora, gpu = case["ora"], case["gpu"]
    S = ora.assemble_S(case["S_el"])
    x_dir = np.linalg.solve(S, case["g"])
    x_gpu, rep, st = gpu.solve(gpu.rhs(), tol=1e-10, restart=30, maxit=5000, mode=2, basis=basis)
    assert st == 0 and rep["converged"] == 1 and rep["rel_residual"] <= 1e-10
    x_gpu = x_gpu.cpu().numpy()
    assert np.linalg.norm(case["g"] - S @ x_gpu) / np.linalg.norm(case["g"]) <= 1.01e-10
    assert rel(x_gpu, x_dir) < 1e-8


@pytest.mark.parametrize("basis", [BASIS_FP64, BASIS_DF64, BASIS_FIX])
def test_gmres_fp32_iterative_refinement_mode(case, basis):
    """mode 1: FP32 blocks inside FP64 iterative refinement still reach the FP64 residual
    (with BASIS_FP64: the mixed-precision form with FP64 orthogonalisation)."""
    ora, gpu = case["ora"], case["gpu"]
    S = ora.assemble_S(case["S_el"])
    x_dir = np.linalg.solve(S, case["g"])
    x_gpu, rep, st = gpu.solve(gpu.rhs(), tol=1e-10, restart=30, maxit=20000, mode=1, basis=basis)
    assert st == 0 and rep["converged"] == 1 and rep["rel_residual"] <= 1e-10 and rep["outer"] >= 1
    x_gpu = x_gpu.cpu().numpy()
    assert np.linalg.norm(case["g"] - S @ x_gpu) / np.linalg.norm(case["g"]) <= 1.01e-10
    assert rel(x_gpu, x_dir) < 1e-8


@pytest.mark.parametrize("basis", [BASIS_FP64, BASIS_DF64, BASIS_FIX])
@pytest.mark.parametrize("orth", [1, 2, 3])
def test_gmres_single_projection_variants(case, orth, basis):
    """orth = 1 (one projection, norm from Pythagoras), orth = 2 (a second projection
    where the first removed more than half of the new vector) and orth = 3 (a second
    projection where the first cancelled more than six digits): same solution, same residual."""
    ora, gpu = case["ora"], case["gpu"]
    S = ora.assemble_S(case["S_el"])
    x_dir = np.linalg.solve(S, case["g"])
    for mode in (0, 2):
        x_gpu, rep, st = gpu.solve(gpu.rhs(), tol=1e-10, restart=30, maxit=5000, mode=mode, orth=orth, basis=basis)
        assert st == 0 and rep["converged"] == 1 and rep["rel_residual"] <= 1e-10, (mode, rep)
        x_gpu = x_gpu.cpu().numpy()
        assert abs(np.linalg.norm(case["g"] - S @ x_gpu) / np.linalg.norm(case["g"]) - rep["rel_residual"]) < 1e-12
        assert rel(x_gpu, x_dir) < 1e-8


@pytest.mark.parametrize("augment", [1, 3])
@pytest.mark.parametrize("mode,basis", [(0, BASIS_FP64), (1, BASIS_FP64), (2, BASIS_DF64)])
def test_gmres_with_augmented_restarts(case, mode, basis, augment):
    """Augmented restarts (LGMRES): the last steps of each cycle run on the corrections of the
    previous cycles; the solution still matches the direct solve and the reported residual is
    the true one (restart 10 forces many cycles)."""
    ora, gpu = case["ora"], case["gpu"]
    S = ora.assemble_S(case["S_el"])
    x_dir = np.linalg.solve(S, case["g"])
    x_gpu, rep, st = gpu.solve(gpu.rhs(), tol=1e-10, restart=10, maxit=20000, mode=mode, orth=3, basis=basis,
                               augment=augment)
    assert st == 0 and rep["converged"] == 1 and rep["rel_residual"] <= 1e-10, rep
    x_gpu = x_gpu.cpu().numpy()
    assert abs(np.linalg.norm(case["g"] - S @ x_gpu) / np.linalg.norm(case["g"]) - rep["rel_residual"]) < 1e-12
    assert rel(x_gpu, x_dir) < 1e-8
    x2, rep2, _ = gpu.solve(gpu.rhs(), tol=1e-10, restart=10, maxit=20000, mode=mode, orth=3, basis=basis,
                            augment=augment)
    assert torch.equal(torch.from_numpy(x_gpu).cuda(), x2) and rep == rep2


@pytest.mark.parametrize("basis", [BASIS_FP64, BASIS_DF64, BASIS_FIX])
def test_solve_is_bitwise_reproducible(case, basis):
    gpu = case["gpu"]
    g = gpu.rhs()
    x1, r1, _ = gpu.solve(g, tol=1e-10, restart=20, maxit=3000, basis=basis)
    x2, r2, _ = gpu.solve(g, tol=1e-10, restart=20, maxit=3000, basis=basis)
    assert torch.equal(x1, x2) and r1 == r2


@pytest.mark.parametrize("n,m,p", [(2, 4, 2), (3, 2, 3), (1, 8, 1), (2, 1, 2)])
def test_polynomial_exactness_on_gpu(n, m, p):
    """u in P_p globally is reproduced exactly (Sec. 3.1 consistency) by the whole GPU path."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    kap, beta = 0.7, (0.9, -0.4)
    u, gr, f = polynomial(random_polynomial(p, seed=5 + p), kap, beta)
    gpu = _lib_problem(n, m, p, beta, kap)
    xy = gpu.quad_points().cpu().numpy()
    bxy = gpu.bnd_quad_points().cpu().numpy()
    gpu.set_source(torch.from_numpy(f(xy[..., 0], xy[..., 1])), torch.from_numpy(u(bxy[..., 0], bxy[..., 1])))
    gpu.condense()
    x, rep, st = gpu.solve(gpu.rhs(), tol=1e-13, restart=40, maxit=4000)
    assert st == 0
    uh, qh = gpu.recover(x)
    ora = HDGProblem(n, m, p)
    ref = ora.mesh.lattice_ref()
    err_u = err_q = 0.0
    for e in range(ora.mesh.N):
        v = ora.mesh.vertices(e)
        X = v[0] + np.outer(ref[:, 0], v[1] - v[0]) + np.outer(ref[:, 1], v[2] - v[0])
        err_u = max(err_u, np.abs(uh[e].cpu().numpy() - u(X[:, 0], X[:, 1])).max())
        gx, gy = gr(X[:, 0], X[:, 1])
        err_q = max(err_q, np.abs(qh[e, 0].cpu().numpy() + gx).max(), np.abs(qh[e, 1].cpu().numpy() + gy).max())
    assert err_u < 1e-10 and err_q < 1e-9
    gpu.close()


def test_error_statuses():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2302_10917_gb300 import (HDG_ERR_ARG, HDG_ERR_NOCONV, HDG_ERR_SINGULAR, HDG_ERR_STATE, HDGError,
                                        Problem)
    gpu = Problem(3, 2, 2, beta=(1.0, 0.0), kappa=1.0)
    x = torch.zeros(gpu.info["N_tr"], dtype=torch.float64, device="cuda")
    with pytest.raises(HDGError) as ei:
        gpu.apply(x)
    assert ei.value.status == HDG_ERR_STATE
    xy = gpu.quad_points()
    gpu.set_source(wl.sin_sin_source(xy, 1.0, (1.0, 0.0)))
    gpu.condense()
    with pytest.raises(HDGError) as ei:
        gpu.apply(x, prec=16)
    assert ei.value.status == HDG_ERR_ARG
    with pytest.raises(HDGError) as ei:
        gpu.apply(x.float(), prec=32, precond=True)     # FP32 blocks were not stored
    assert ei.value.status == HDG_ERR_ARG
    xs, rep, st = gpu.solve(gpu.rhs(), tol=1e-14, restart=2, maxit=3)
    assert st == HDG_ERR_NOCONV and rep["converged"] == 0 and rep["iterations"] == 3
    assert torch.isfinite(xs).all()
    gpu.close()
    # a zero local matrix (kappa = 0 and beta = 0 on one element) is reported with its index
    kap = np.ones(18)
    kap[7] = 0.0
    bad = Problem(3, 2, 2, beta=(0.0, 0.0), kappa=kap)
    bad.set_source(torch.zeros(18, bad.info["n_qp"], dtype=torch.float64))
    with pytest.raises(HDGError) as ei:
        bad.condense()
    assert ei.value.status == HDG_ERR_SINGULAR and "element 7" in str(ei.value)
    bad.close()


def test_levels_beyond_shared_memory_are_refused():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2302_10917_gb300 import HDG_ERR_ARG, HDGError, Problem
    with pytest.raises(HDGError) as ei:
        Problem(1, 16, 3, beta=(1.0, 0.0), kappa=1.0)
    assert ei.value.status == HDG_ERR_ARG and "shared memory" in str(ei.value)
    pr = Problem(1, 16, 2, beta=(1.0, 0.0), kappa=1.0)       # the largest m at p = 2 fits, also with 64 sources
    pr.set_source(torch.zeros(64, pr.info["N"], pr.info["n_qp"], dtype=torch.float64))
    pr.condense()
    pr.close()
