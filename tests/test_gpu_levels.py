"""Level meshes on the GPU (Sec. 4.2): per-element refinement levels, faces at
the finer side's level, against the level-mesh oracle (oracle/levels.py).

The oracle integrates the coarse side's face couplings on the fine sub-edges;
the library condenses every element at its own level and lifts the blocks
with the face transfer T = Gh_r^-1 Pi^T Gh_R. Parity: Schur blocks, the
condensed right-hand side, the plain and preconditioned apply (FP64 to
1e-12; split-FP32 to 1e-12; FP32 to 1e-6), the solution and the back-solve
(GMRES to 1e-13 against the oracle's direct solve, 1e-9), several right-hand
sides, and polynomial exactness through non-conforming faces.
"""
import numpy as np
import pytest
import torch

from oracle.levels import LevelHDGProblem, band_levels
from oracle.problems import polynomial, random_polynomial
from paper_2302_10917_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def _levels(kind, n, p):
    g = np.random.default_rng([wl.MASTER_SEED, 71, n, p])
    if kind == "random":
        hi = 3 if p <= 2 else 2      # p = 3, 4: levels 0..2
        return g.integers(0, hi + 1, size=2 * n * n)
    if kind == "band":
        return band_levels(n, edges=(0.4, 0.6, 0.8), base=0)
    if kind == "level4":
        lev = np.ones(2 * n * n, dtype=np.int64)
        lev[:2] = 4
        return lev
    raise ValueError(kind)


CASES = [
    # id, n, p, levels, beta
    ("rand_p2", 2, 2, "random", (0.8, -0.3)),
    ("band_p2", 4, 2, "band", (1.0, 0.0)),
    ("rand_p3", 2, 3, "random", (0.5, 0.9)),
    ("lev4_p1", 2, 1, "level4", (0.3, 0.7)),
    ("rand_p4", 2, 4, "random", (0.4, -0.6)),
]


def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.fixture(scope="module", params=CASES, ids=[c[0] for c in CASES])
def case(request):
    _need_gpu()
    from paper_2302_10917_gb300 import Problem
    cid, n, p, kind, beta = request.param
    lev = _levels(kind, n, p)
    N = 2 * n * n
    kappa = wl.random_kappa(N, seed=13 * n + p)
    ora = LevelHDGProblem(n, lev, p, beta=beta, kappa=kappa)
    gpu = Problem(n, 1, p, beta=beta, kappa=kappa, levels=lev)
    g = np.random.default_rng([wl.MASTER_SEED, 72, n, p])
    f = g.standard_normal(ora.qoff[-1])
    gD = g.standard_normal(ora.boff[-1])
    gpu.set_source(torch.from_numpy(f), torch.from_numpy(gD))
    gpu.condense(keep_factors=True, store_fp32=True, store_df64=True)
    S_el, g_o, gh = ora.condense(f, gD)
    yield dict(ora=ora, gpu=gpu, f=f, gD=gD, S=S_el, g=g_o, gh=gh, rng=g, lev=lev)
    gpu.close()


def test_ragged_offsets_match_the_oracle(case):
    from paper_2302_10917_gb300 import (OFF_DIRICHLET_POINTS, OFF_DIRICHLET_TRACE, OFF_LATTICE, OFF_SCHUR,
                                        OFF_SOURCE, OFF_TRACE)
    ora, gpu = case["ora"], case["gpu"]
    assert gpu.info["levels"] == 1 and gpu.info["N_tr"] == ora.N_tr
    assert np.array_equal(gpu.offsets(OFF_SOURCE).numpy(), ora.qoff)
    assert np.array_equal(gpu.offsets(OFF_DIRICHLET_POINTS).numpy(), ora.boff)
    assert np.array_equal(gpu.offsets(OFF_LATTICE).numpy(), ora.uoff)
    assert np.array_equal(gpu.offsets(OFF_TRACE).numpy(), ora.eoff)
    assert np.array_equal(gpu.offsets(OFF_DIRICHLET_TRACE).numpy(), ora.goff)
    nt = np.array([ora.n_t(e) for e in range(ora.N)])
    assert np.array_equal(gpu.offsets(OFF_SCHUR).numpy(), np.concatenate([[0], np.cumsum(nt * nt)]))


def test_quadrature_points_match_the_oracle(case):
    ora, gpu = case["ora"], case["gpu"]
    assert np.abs(gpu.quad_points().cpu().numpy() - ora.quad_points()[0]).max() < 1e-15
    assert np.abs(gpu.bnd_quad_points().cpu().numpy() - ora.bnd_quad_points()[0]).max() < 1e-15


def test_schur_blocks_and_rhs_match_the_oracle(case):
    ora, gpu = case["ora"], case["gpu"]
    S = gpu.schur().cpu().numpy()
    from paper_2302_10917_gb300 import OFF_SCHUR
    off = gpu.offsets(OFF_SCHUR).numpy()
    for e in range(ora.N):
        nt = ora.n_t(e)
        Se = S[off[e]:off[e + 1]].reshape(nt, nt)
        assert rel(Se, case["S"][e]) < 1e-12, e
    assert rel(gpu.rhs().cpu().numpy(), case["g"]) < 1e-12
    # a sub-range of elements
    part = gpu.schur(3, 4).cpu().numpy()
    assert np.array_equal(part, S[off[3]:off[7]])


def test_tensor_core_elimination_on_level_meshes(case):
    """HDG_TC_UPDATE on every level bin: lifted Schur blocks, right-hand side and back-solve
    at the FP64 bounds."""
    from paper_2302_10917_gb300 import OFF_SCHUR, Problem
    ora = case["ora"]
    pr = Problem(ora.n, 1, ora.p, beta=tuple(ora.beta), kappa=ora.kappa, levels=case["lev"])
    try:
        pr.set_source(torch.from_numpy(case["f"]), torch.from_numpy(case["gD"]))
        pr.condense(keep_factors=True, tc_update=True)
        S = pr.schur().cpu().numpy()
        off = pr.offsets(OFF_SCHUR).numpy()
        for e in range(ora.N):
            nt = ora.n_t(e)
            assert rel(S[off[e]:off[e + 1]].reshape(nt, nt), case["S"][e]) < 1e-12, e
        assert rel(pr.rhs().cpu().numpy(), case["g"]) < 1e-12
        x_dir = np.linalg.solve(ora.assemble_S(case["S"]), case["g"])
        u, q = pr.recover(torch.from_numpy(x_dir))
        u_o, q_o = ora.recover(x_dir, case["f"], case["gh"])
        assert rel(u.cpu().numpy(), u_o) < 1e-11 and rel(q.cpu().numpy(), q_o) < 1e-11
    finally:
        pr.close()


@pytest.mark.parametrize("prec", [64, 48, 33, 32])
def test_apply_matches_the_oracle(case, prec):
    ora, gpu = case["ora"], case["gpu"]
    Sg = ora.assemble_S(case["S"])
    x = case["rng"].standard_normal(ora.N_tr)
    tol = 1e-6 if prec in (32, 33) else 1e-12
    yp = gpu.apply(torch.from_numpy(x), precond=True, prec=prec).double().cpu().numpy()
    assert rel(yp, ora.apply_Dinv(Sg @ x)) < tol
    if prec == 64:
        assert rel(gpu.apply(torch.from_numpy(x)).cpu().numpy(), Sg @ x) < 1e-12


@pytest.mark.parametrize("basis", [0, 1, 2])
@pytest.mark.parametrize("mode", [0, 1, 2])
def test_solve_and_recover_match_the_oracle(case, mode, basis):
    """Every operator precision with the FP64 (basis 0), split-FP32 (1) and fixed-point (2)
    Krylov basis, and augmented restarts with the FP64 basis."""
    ora, gpu = case["ora"], case["gpu"]
    x_dir = np.linalg.solve(ora.assemble_S(case["S"]), case["g"])
    x, rep, st = gpu.solve(gpu.rhs(), tol=1e-13, restart=12 if basis == 0 else 60, mode=mode, maxit=20000,
                           basis=basis, augment=2 if basis == 0 else 0)
    assert st == 0, rep
    assert rel(x.cpu().numpy(), x_dir) < 1e-9
    u, q = gpu.recover(x)
    u_o, q_o = ora.recover(x_dir, case["f"], case["gh"])
    assert rel(u.cpu().numpy(), u_o) < 1e-9
    assert rel(q.cpu().numpy(), q_o) < 1e-9


def test_several_right_hand_sides(case):
    from paper_2302_10917_gb300 import Problem
    ora, lev = case["ora"], case["lev"]
    rng = np.random.default_rng([wl.MASTER_SEED, 73, ora.n, ora.p])
    nrhs = 3
    f = rng.standard_normal((nrhs, ora.qoff[-1]))
    gD = rng.standard_normal((nrhs, ora.boff[-1]))
    gpu = Problem(ora.n, 1, ora.p, beta=tuple(ora.beta), kappa=ora.kappa, levels=lev)
    try:
        gpu.set_source(torch.from_numpy(f), torch.from_numpy(gD))
        gpu.condense(keep_factors=False, store_df64=True, split_update=True)
        g = gpu.rhs()
        x, rep, st = gpu.solve(g, tol=1e-13, restart=60, mode=2)
        assert st == 0, rep
        u, q = gpu.recover(x)
        Sg = ora.assemble_S(case["S"])
        for r in range(nrhs):
            _, g_o, gh = ora.condense(f[r], gD[r])
            assert rel(g[r].cpu().numpy(), g_o) < 1e-11
            x_dir = np.linalg.solve(Sg, g_o)
            assert rel(x[r].cpu().numpy(), x_dir) < 1e-9
            u_o, q_o = ora.recover(x_dir, f[r], gh)
            assert rel(u[r].cpu().numpy(), u_o) < 1e-9 and rel(q[r].cpu().numpy(), q_o) < 1e-9
        # the multi-column apply equals column-by-column applies
        X = torch.from_numpy(rng.standard_normal((nrhs, ora.N_tr))).cuda()
        Y = gpu.apply(X, precond=True)
        for r in range(nrhs):
            assert rel(Y[r].cpu().numpy(), gpu.apply(X[r], precond=True).cpu().numpy()) < 1e-14
    finally:
        gpu.close()


@pytest.mark.parametrize("n,p,kind", [(2, 2, "random"), (3, 3, "band"), (2, 1, "level4")])
def test_polynomial_exactness_through_nonconforming_faces(n, p, kind):
    _need_gpu()
    from paper_2302_10917_gb300 import Problem
    lev = _levels(kind, n, p)
    kap, beta = 0.7, (0.9, -0.4)
    u, _, f = polynomial(random_polynomial(p, seed=31 + p), kap, beta)
    ora = LevelHDGProblem(n, lev, p, beta=beta, kappa=kap)
    gpu = Problem(n, 1, p, beta=beta, kappa=kap, levels=lev)
    try:
        xy = gpu.quad_points().cpu().numpy()
        bxy = gpu.bnd_quad_points().cpu().numpy()
        gpu.set_source(torch.from_numpy(f(xy[:, 0], xy[:, 1])), torch.from_numpy(u(bxy[:, 0], bxy[:, 1])))
        gpu.condense()
        x, rep, st = gpu.solve(gpu.rhs(), tol=1e-14, restart=80, mode=0, maxit=40000)
        assert st == 0, rep
        uu, _ = gpu.recover(x)
        uu = uu.cpu().numpy()
        for e in range(ora.N):
            X = ora.lattice_points(e)
            assert np.abs(uu[ora.uoff[e]:ora.uoff[e + 1]] - u(X[:, 0], X[:, 1])).max() < 1e-10
    finally:
        gpu.close()


def test_uniform_levels_equal_the_uniform_context():
    _need_gpu()
    from paper_2302_10917_gb300 import Problem
    n, r, p, beta = 3, 2, 2, (0.6, 0.2)
    a = Problem(n, 2 ** r, p, beta=beta, kappa=0.8)
    b = Problem(n, 1, p, beta=beta, kappa=0.8, levels=np.full(2 * n * n, r))
    try:
        f = torch.from_numpy(np.random.default_rng(4).standard_normal((2 * n * n, a.info["n_qp"])))
        a.set_source(f)
        b.set_source(f.reshape(-1))
        a.condense()
        b.condense()
        assert rel(b.schur().cpu().numpy(), a.schur().reshape(-1).cpu().numpy()) < 1e-13
        assert rel(b.rhs().cpu().numpy(), a.rhs().cpu().numpy()) < 1e-13
        v = torch.ones(a.info["N_tr"], dtype=torch.float64, device="cuda")
        assert rel(b.apply(v, precond=True).cpu().numpy(), a.apply(v, precond=True).cpu().numpy()) < 1e-13
    finally:
        a.close()
        b.close()


def test_level_mesh_errors():
    _need_gpu()
    from paper_2302_10917_gb300 import HDG_ERR_ARG, HDG_ERR_SINGULAR, HDGError, Problem
    with pytest.raises(HDGError) as ei:
        Problem(2, 1, 2, levels=np.full(8, 5))
    assert ei.value.status == HDG_ERR_ARG
    with pytest.raises(HDGError) as ei:
        Problem(2, 1, 3, levels=np.full(8, 4))          # level 4 at p = 3 exceeds shared memory
    assert ei.value.status == HDG_ERR_ARG
    # a zero local matrix (kappa = 0, beta = 0) on element 5 of level 2 is reported with its element id
    kap = np.ones(8)
    kap[5] = 0.0
    bad = Problem(2, 1, 2, beta=(0.0, 0.0), kappa=kap, levels=np.arange(8) % 3)
    try:
        bad.set_source(torch.zeros(bad.info["n_qp_total"], dtype=torch.float64))
        with pytest.raises(HDGError) as ei:
            bad.condense()
        assert ei.value.status == HDG_ERR_SINGULAR and "element 5" in str(ei.value)
    finally:
        bad.close()
    pr = Problem(2, 1, 2, levels=np.arange(8) % 3)
    try:
        pr.set_source(torch.zeros(pr.info["n_qp_total"], dtype=torch.float64))
        pr.condense()
        for call in (lambda: pr.transpose(), lambda: pr.set_kappa(torch.ones(8, dtype=torch.float64))):
            with pytest.raises(HDGError) as ei:
                call()
            assert ei.value.status == HDG_ERR_ARG and "level mesh" in str(ei.value)
    finally:
        pr.close()


def test_band_levels_n32_against_the_oracle_direct_solution():
    """n = 32 banded-level mesh (2 048 elements, 28 336 trace unknowns): the condensed
    right-hand side and the solution at 600 sampled trace dofs against the oracle's sparse
    direct solve (tests/golden/levels_band_n32.json, written by make_levels_band_n32.py),
    with the D^-1 preconditioner (FP64 operator) and with the face blocks of S (split-FP32)."""
    _need_gpu()
    import json
    import os
    from paper_2302_10917_gb300 import Problem
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "levels_band_n32.json")))
    n = gold["n"]
    pr = Problem(n, 1, gold["p"], beta=tuple(gold["beta"]), kappa=gold["kappa"], levels=wl.band_levels(n))
    try:
        assert pr.info["N_tr"] == gold["N_tr"]
        f = wl.gaussian_bumps(pr.quad_points(), 1, seed=gold["seed"], width=gold["width"])[0].contiguous()
        pr.set_source(f)
        dofs = torch.tensor(gold["dofs"], device="cuda")
        xg, gg = np.array(gold["x"]), np.array(gold["g"])
        for pc, mode, restart in (("d", 0, 128), ("face_schur", 2, 80)):
            pr.condense(keep_factors=True, store_df64=True, split_update=(mode == 2), precond=pc)
            g = pr.rhs()
            assert abs(float(g.norm()) - gold["g_norm"]) <= 1e-12 * gold["g_norm"]
            assert np.abs(g[dofs].cpu().numpy() - gg).max() <= 1e-12 * np.abs(gg).max()
            x, rep, st = pr.solve(g, tol=1e-13, restart=restart, mode=mode, maxit=60000)
            assert st == 0, (pc, rep)
            assert np.abs(x[dofs].cpu().numpy() - xg).max() <= 1e-9 * gold["x_absmax"], pc
            assert abs(float(x.norm()) - gold["x_norm"]) <= 1e-9 * gold["x_norm"]
    finally:
        pr.close()


@pytest.mark.parametrize("n,lev,p,supg", [
    (1, [0, 3], 2, False),            # one macro square, its two elements three levels apart
    (2, [0] * 8, 2, False),           # every element of level 0: standard HDG with level-mesh layouts
    (2, [1, 2, 2, 1, 0, 1, 2, 0], 2, True),   # SUPG inside macro-elements of different levels
    (2, [2, 0, 1, 1, 0, 2, 1, 0], 3, True),
])
def test_edge_cases_and_supg(n, lev, p, supg):
    _need_gpu()
    from paper_2302_10917_gb300 import Problem
    lev = np.array(lev)
    beta, kappa = (0.9, -0.5), (0.05 if supg else 0.8)
    ora = LevelHDGProblem(n, lev, p, beta=beta, kappa=kappa, supg=supg)
    gpu = Problem(n, 1, p, beta=beta, kappa=kappa, levels=lev, supg=supg)
    try:
        g = np.random.default_rng([wl.MASTER_SEED, 74, n, p, int(supg)])
        f = g.standard_normal(ora.qoff[-1])
        gD = g.standard_normal(ora.boff[-1])
        gpu.set_source(torch.from_numpy(f), torch.from_numpy(gD))
        gpu.condense(keep_factors=True)
        S_el, g_o, gh = ora.condense(f, gD)
        from paper_2302_10917_gb300 import OFF_SCHUR
        S = gpu.schur().cpu().numpy()
        off = gpu.offsets(OFF_SCHUR).numpy()
        # SUPG's consistency term makes A_u less well conditioned (see test_gpu_supg.py)
        tol = 2e-10 if supg else 1e-12
        for e in range(ora.N):
            assert rel(S[off[e]:off[e + 1]], S_el[e].reshape(-1)) < tol, e
        assert rel(gpu.rhs().cpu().numpy(), g_o) < tol
        x_dir = np.linalg.solve(ora.assemble_S(S_el), g_o)
        x, rep, st = gpu.solve(gpu.rhs(), tol=1e-13, restart=60, mode=0, maxit=40000)
        assert st == 0, rep
        assert rel(x.cpu().numpy(), x_dir) < 1e-8
        u, q = gpu.recover(x)
        u_o, q_o = ora.recover(x_dir, f, gh)
        assert rel(u.cpu().numpy(), u_o) < 1e-8 and rel(q.cpu().numpy(), q_o) < 1e-8
    finally:
        gpu.close()


def test_batched_columns_finishing_in_different_cycles():
    """Lockstep GMRES whose columns converge in different restart cycles (a zero column, a
    smooth and a rough source): the Arnoldi operator then runs on the remaining columns
    only; every column equals its own single-column solve."""
    _need_gpu()
    from paper_2302_10917_gb300 import Problem
    n, p = 3, 2
    lev = band_levels(n, edges=(0.4, 0.6, 0.8), base=0)
    pr = Problem(n, 1, p, beta=(1.0, 0.3), kappa=0.05, levels=lev)
    try:
        xy = pr.quad_points()
        rough = torch.from_numpy(np.random.default_rng([wl.MASTER_SEED, 75]).standard_normal(xy.shape[0])).cuda()
        f = torch.stack([torch.sin(3.0 * xy[:, 0]) * xy[:, 1], torch.zeros_like(rough), rough, 0.5 * rough])
        pr.set_source(f)
        pr.condense(keep_factors=True, store_df64=True, split_update=True)
        g = pr.rhs()
        x, rep, st = pr.solve(g, tol=1e-12, restart=10, mode=2, maxit=20000)
        assert st == 0, rep
        assert torch.count_nonzero(x[1]) == 0
        for r in (0, 2, 3):
            xr, rr, sr = pr.solve(g[r].contiguous(), tol=1e-12, restart=10, mode=2, maxit=20000)
            assert sr == 0, rr
            assert rel(x[r].cpu().numpy(), xr.cpu().numpy()) < 1e-9, r
        assert rel(x[3].cpu().numpy(), 0.5 * x[2].cpu().numpy()) < 1e-9
    finally:
        pr.close()


def test_autotune_on_a_level_mesh(case):
    """hdg_autotune picks the apply's element-side rows per CTA (and the Krylov launch
    shapes); the tuned solve still matches the oracle."""
    ora, gpu = case["ora"], case["gpu"]
    rep = gpu.autotune(mode=2, restart=60)
    assert rep["apply_threads"] in (128, 256, 512) and rep["apply_edges_per_block"] == 0
    x_dir = np.linalg.solve(ora.assemble_S(case["S"]), case["g"])
    x, r, st = gpu.solve(gpu.rhs(), tol=1e-13, restart=60, mode=2, maxit=20000)
    assert st == 0, r
    assert rel(x.cpu().numpy(), x_dir) < 1e-9
