"""Face-block preconditioner with the diagonal blocks of S (HDG_PRECOND_FACE_SCHUR).

Reference: the block diagonal of the oracle's assembled S (one block per
interior face, global edge orientation), inverted densely, applied to S x.
The preconditioned apply (FP64, split-FP32, FP32 blocks), the GMRES solution
in every mode and with several right-hand sides, uniform and level meshes;
after hdg_transpose the transposed face blocks S_ff^T precondition S^T.
"""
import math

import numpy as np
import pytest
import torch

from oracle.hdg import HDGProblem
from oracle.levels import LevelHDGProblem
from oracle.precond import face_block_inverse
from paper_2302_10917_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


B1 = (50.0 * math.cos(0.3), 50.0 * math.sin(0.3))
CASES = [
    # id, n, m (or None: levels), p, beta, kappa
    ("u_m2p2", 3, 2, 2, (0.8, -0.3), "random"),
    ("u_m8p3", 2, 8, 3, B1, 1.0),
    ("lv_p2", 3, None, 2, (1.0, 0.0), 1e-2),
]


@pytest.fixture(scope="module", params=CASES, ids=[c[0] for c in CASES])
def case(request):
    _need_gpu()
    from paper_2302_10917_gb300 import Problem
    cid, n, m, p, beta, kap = request.param
    N = 2 * n * n
    kappa = wl.random_kappa(N, seed=n + p) if kap == "random" else kap
    g = np.random.default_rng([wl.MASTER_SEED, 81, n, p])
    if m is None:
        lev = g.integers(0, 4, size=N)
        ora = LevelHDGProblem(n, lev, p, beta=beta, kappa=kappa)
        gpu = Problem(n, 1, p, beta=beta, kappa=kappa, levels=lev)
        f = g.standard_normal(ora.qoff[-1])
        gD = g.standard_normal(ora.boff[-1])
        eoff = ora.eoff
        S_el, g_o, gh = ora.condense(f, gD)
    else:
        ora = HDGProblem(n, m, p, beta=beta, kappa=kappa)
        gpu = Problem(n, m, p, beta=beta, kappa=kappa)
        pts, _ = ora.quad_points()
        bpts, _ = ora.bnd_quad_points()
        f = g.standard_normal(pts.shape[:2])
        gD = g.standard_normal(bpts.shape[:2])
        P1 = ora.mesh.P1
        eoff = np.arange(ora.mesh.n_int_edges + 1) * P1
        S_el, g_o, gh = ora.condense(f, gD)
    S = ora.assemble_S(S_el)
    gpu.set_source(torch.from_numpy(f), torch.from_numpy(gD))
    gpu.condense(keep_factors=True, store_fp32=True, store_df64=True, precond="face_schur")
    yield dict(ora=ora, gpu=gpu, S=S, Pinv=face_block_inverse(S, eoff), g=g_o, f=f, gh=gh, rng=g, m=m)
    gpu.close()


@pytest.mark.parametrize("prec", [64, 48, 32])
def test_preconditioned_apply_is_the_inverse_face_block_times_S(case, prec):
    gpu = case["gpu"]
    x = case["rng"].standard_normal(case["S"].shape[0])
    y = gpu.apply(torch.from_numpy(x), precond=True, prec=prec).double().cpu().numpy()
    ref = case["Pinv"] @ (case["S"] @ x)
    assert rel(y, ref) < (2e-6 if prec == 32 else 1e-11)
    # the plain apply is unchanged
    assert rel(gpu.apply(torch.from_numpy(x)).cpu().numpy(), case["S"] @ x) < 1e-12


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_solve_with_face_blocks(case, mode):
    gpu = case["gpu"]
    x_dir = np.linalg.solve(case["S"], case["g"])
    x, rep, st = gpu.solve(gpu.rhs(), tol=1e-13, restart=60, mode=mode)
    assert st == 0, rep
    assert rel(x.cpu().numpy(), x_dir) < 1e-9


def test_several_rhs_with_face_blocks(case):
    gpu = case["gpu"]
    X = torch.from_numpy(case["rng"].standard_normal((3, case["S"].shape[0]))).cuda()
    Y = gpu.apply(X, precond=True)
    for r in range(3):
        assert rel(Y[r].cpu().numpy(), case["Pinv"] @ (case["S"] @ X[r].cpu().numpy())) < 1e-11
    G = torch.stack([gpu.rhs(), 2.0 * gpu.rhs(), gpu.apply(X[0])])
    x, rep, st = gpu.solve(G, tol=1e-12, restart=60, mode=2)
    assert st == 0, rep
    for r in range(3):
        assert rel(x[r].cpu().numpy(), np.linalg.solve(case["S"], G[r].cpu().numpy())) < 1e-8


def test_transposed_operator_with_transposed_face_blocks(case):
    if case["m"] is None:
        pytest.skip("level meshes have no transpose")
    gpu = case["gpu"]
    St = case["S"].T
    eoff = np.arange(St.shape[0] // case["ora"].mesh.P1 + 1) * case["ora"].mesh.P1
    PinvT = face_block_inverse(St, eoff)
    x = case["rng"].standard_normal(St.shape[0])
    gpu.transpose()
    try:
        for prec, tol in ((64, 1e-11), (48, 1e-11), (32, 2e-6)):
            y = gpu.apply(torch.from_numpy(x), precond=True, prec=prec).double().cpu().numpy()
            assert rel(y, PinvT @ (St @ x)) < tol, prec
        xs, rep, st = gpu.solve(torch.from_numpy(St @ x).cuda(), tol=1e-13, restart=60, mode=2)
        assert st == 0, rep
        assert rel(xs.cpu().numpy(), x) < 1e-8
    finally:
        gpu.transpose()
    y = gpu.apply(torch.from_numpy(x), precond=True).cpu().numpy()
    assert rel(y, case["Pinv"] @ (case["S"] @ x)) < 1e-11


def test_face_blocks_need_fewer_iterations_on_the_large_workload_element():
    """m = 8, p = 3, beta = 50 (cos 0.3, sin 0.3), kappa = 1 on an 8 x 8 macro grid: GMRES(80) to 1e-10."""
    _need_gpu()
    from paper_2302_10917_gb300 import Problem
    cfg = wl.CONFIGS["n128_m8_p3"]
    pr = Problem(8, cfg["m"], cfg["p"], beta=cfg["beta"], kappa=cfg["kappa"])
    try:
        pr.set_source(wl.sin_sin_source(pr.quad_points(), cfg["kappa"], cfg["beta"]))
        its = {}
        for pc in ("d", "face_schur"):
            pr.condense(keep_factors=True, store_df64=True, split_update=True, precond=pc)
            x, rep, st = pr.solve(pr.rhs(), tol=1e-10, restart=80, mode=2, orth=1)
            assert st == 0, rep
            its[pc] = rep["iterations"]
        assert its["face_schur"] < 0.5 * its["d"], its
    finally:
        pr.close()


def test_face_blocks_with_supg():
    """SUPG inside the macro-elements (Sec. 3.4): S_ff^-1 S x against the oracle's blocks;
    SUPG's consistency term conditions A_u less well, hence 2e-10 (see test_gpu_supg.py)."""
    _need_gpu()
    from paper_2302_10917_gb300 import Problem
    n, m, p, beta, kap = 2, 2, 2, (0.9, -0.5), 0.05
    ora = HDGProblem(n, m, p, beta=beta, kappa=kap, supg=True)
    gpu = Problem(n, m, p, beta=beta, kappa=kap, supg=True)
    try:
        g = np.random.default_rng([wl.MASTER_SEED, 82])
        pts, _ = ora.quad_points()
        f = g.standard_normal(pts.shape[:2])
        gpu.set_source(torch.from_numpy(f))
        gpu.condense(keep_factors=True, precond="face_schur")
        S_el, g_o, _ = ora.condense(f, None)
        S = ora.assemble_S(S_el)
        P1 = ora.mesh.P1
        Pinv = face_block_inverse(S, np.arange(ora.mesh.n_int_edges + 1) * P1)
        x = g.standard_normal(S.shape[0])
        y = gpu.apply(torch.from_numpy(x), precond=True).cpu().numpy()
        assert rel(y, Pinv @ (S @ x)) < 2e-10
        xs, rep, st = gpu.solve(gpu.rhs(), tol=1e-13, restart=40, mode=0)
        assert st == 0, rep
        assert rel(xs.cpu().numpy(), np.linalg.solve(S, g_o)) < 1e-8
    finally:
        gpu.close()
