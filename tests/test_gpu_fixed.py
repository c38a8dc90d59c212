"""Fixed-point trace apply (HDG_STORE_FIX64, hdg_apply prec 56, solve mode 3)
against the oracle (Sec. 3.3.2, steps 1-4, with the D^-1 preconditioner of
Sec. 6.1) and against the properties that exact integer products give it:
power-of-two scale invariance and sign symmetry bit for bit, exact zeros,
non-finite inputs reported in the same rows as the FP64 apply."""
import math

import numpy as np
import pytest
import torch

from oracle.hdg import HDGProblem
from paper_2302_10917_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

B1 = (50.0 * math.cos(0.3), 50.0 * math.sin(0.3))
CASES = [
    # id, n, m, p, beta, kappa mode, preconditioner
    ("smoke_n4_m2_p2", 4, 2, 2, (1.0, 1.0), "const", "d"),
    ("m4p2", 3, 4, 2, (0.8, -0.3), "rand", "d"),
    ("m8p3", 2, 8, 3, B1, "rand", "d"),             # the large workload's element
    ("m8p3_face", 2, 8, 3, B1, "rand", "face_schur"),
    ("n1", 1, 1, 1, (0.3, 0.2), "rand", "d"),        # two elements, one interior edge
    ("m1p3", 5, 1, 3, (1.0, -2.0), "rand", "d"),
    ("p4diff", 2, 2, 4, (0.0, 0.0), "rand", "d"),
    ("m16p1", 1, 16, 1, (2.0, 1.0), "rand", "d"),
]


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.fixture(scope="module", params=CASES, ids=[c[0] for c in CASES])
def case(request):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2302_10917_gb300 import Problem
    cid, n, m, p, beta, kmode, pc = request.param
    N = 2 * n * n
    kappa = 1.0 if kmode == "const" else wl.random_kappa(N, seed=n * 100 + m * 10 + p)
    ora = HDGProblem(n, m, p, beta=beta, kappa=kappa)
    gpu = Problem(n, m, p, beta=beta, kappa=kappa)
    pts, _ = ora.quad_points()
    bpts, _ = ora.bnd_quad_points()
    g = np.random.default_rng([wl.MASTER_SEED, n, m, p, 56])
    f_qp = g.standard_normal(pts.shape[:2])
    gD = g.standard_normal(bpts.shape[:2])
    S_el, g_ora, ghat = ora.condense(f_qp, gD)
    gpu.set_source(torch.from_numpy(f_qp), torch.from_numpy(gD))
    gpu.condense(keep_factors=True, store_fix=True, precond=pc)
    torch.cuda.synchronize()
    yield dict(ora=ora, gpu=gpu, S_el=S_el, g=g_ora, rng=g, pc=pc)
    gpu.close()


def _apply(gpu, x, prec):
    return gpu.apply(torch.from_numpy(np.ascontiguousarray(x)), precond=True, prec=prec).cpu().numpy()


def test_fixed_apply_matches_oracle(case):
    ora, gpu, S_el = case["ora"], case["gpu"], case["S_el"]
    if case["pc"] != "d":
        pytest.skip("the oracle's preconditioner is D^-1")
    N_tr = ora.mesh.N_tr
    e0 = np.zeros(N_tr)
    e0[N_tr // 2] = 1.0
    for x in (case["rng"].standard_normal(N_tr), np.ones(N_tr), e0):
        z_ora = ora.apply_Dinv(ora.apply_S(S_el, x))
        assert rel(_apply(gpu, x, 56), z_ora) < 1e-12


def test_fixed_apply_matches_fp64_apply(case):
    """Against the FP64 FMA apply on the same stored rows: both within a few units of
    2^-53 of the row scale, so far below FP64's own n_t-term error bound."""
    gpu = case["gpu"]
    N_tr = case["ora"].mesh.N_tr
    rng = case["rng"]
    for x in (rng.standard_normal(N_tr), rng.uniform(0.5, 1.5, N_tr),
              rng.standard_normal(N_tr) * np.exp(rng.uniform(-20, 20, N_tr))):
        assert rel(_apply(gpu, x, 56), _apply(gpu, x, 64)) < 5e-14


def test_fixed_apply_is_exact_under_power_of_two_scaling_and_negation(case):
    gpu = case["gpu"]
    x = case["rng"].standard_normal(case["ora"].mesh.N_tr)
    y = _apply(gpu, x, 56)
    for k in (-300, -40, 40, 300):
        yk = _apply(gpu, np.ldexp(x, k), 56)
        np.testing.assert_array_equal(yk, np.ldexp(y, k))
    np.testing.assert_array_equal(_apply(gpu, -x, 56), -y)


def test_fixed_apply_zero_vector_gives_exact_zeros(case):
    y = _apply(case["gpu"], np.zeros(case["ora"].mesh.N_tr), 56)
    assert np.all(y == 0.0)


def test_fixed_apply_reports_non_finite_inputs_in_the_fp64_rows(case):
    gpu = case["gpu"]
    N_tr = case["ora"].mesh.N_tr
    x = case["rng"].standard_normal(N_tr)
    x[N_tr // 3] = np.nan
    y56, y64 = _apply(gpu, x, 56), _apply(gpu, x, 64)
    np.testing.assert_array_equal(np.isfinite(y56), np.isfinite(y64))
    fin = np.isfinite(y64)
    if fin.any():      # (with one interior edge every row sees the non-finite entry)
        assert rel(y56[fin], y64[fin]) < 5e-14


def test_fixed_apply_follows_transpose(case):
    gpu = case["gpu"]
    x = case["rng"].standard_normal(case["ora"].mesh.N_tr)
    gpu.transpose()
    try:
        assert rel(_apply(gpu, x, 56), _apply(gpu, x, 64)) < 5e-14
    finally:
        gpu.transpose()
    assert rel(_apply(gpu, x, 56), _apply(gpu, x, 64)) < 5e-14


def test_fixed_operator_solve_matches_direct_solve(case):
    """Mode 3 (fixed-point Arnoldi operator, FP64 basis, FP64 true residual) against the
    oracle's direct solve, with the reported residual the true one; bitwise reproducible."""
    ora, gpu = case["ora"], case["gpu"]
    S = ora.assemble_S(case["S_el"])
    x_dir = np.linalg.solve(S, case["g"])
    g_gpu = gpu.rhs()
    x3, rep3, st = gpu.solve(g_gpu, tol=1e-10, restart=30, maxit=5000, mode=3, orth=3)
    assert st == 0 and rep3["converged"] == 1 and rep3["rel_residual"] <= 1e-10
    xn = x3.cpu().numpy()
    assert abs(np.linalg.norm(case["g"] - S @ xn) / np.linalg.norm(case["g"]) - rep3["rel_residual"]) < 1e-12
    assert rel(xn, x_dir) < 1e-8
    x3b, rep3b, _ = gpu.solve(g_gpu, tol=1e-10, restart=30, maxit=5000, mode=3, orth=3)
    assert torch.equal(x3, x3b) and rep3 == rep3b
    _, rep0, _ = gpu.solve(g_gpu, tol=1e-10, restart=30, maxit=5000, mode=0, orth=3)
    assert abs(rep3["iterations"] - rep0["iterations"]) <= max(2, rep0["iterations"] // 10)


@pytest.mark.parametrize("orth", [0, 1, 3])
def test_fixed_point_basis_solve_matches_direct_solve(case, orth):
    """The fixed-point Krylov basis (chunks of 56-bit integers, products exact in integers)
    with the fixed-point and the FP64 operators, every orthogonalisation: against the oracle's
    direct solve, the true residual reported, bitwise reproducible, and (with the second
    projections) the iteration count of the FP64 basis within 20 % (the count of a
    restarted GMRES follows rounding)."""
    from paper_2302_10917_gb300 import BASIS_FIX
    ora, gpu = case["ora"], case["gpu"]
    S = ora.assemble_S(case["S_el"])
    x_dir = np.linalg.solve(S, case["g"])
    g_gpu = gpu.rhs()
    for mode in (3, 0):
        x2, rep2, st = gpu.solve(g_gpu, tol=1e-10, restart=30, maxit=5000, mode=mode, orth=orth, basis=BASIS_FIX)
        assert st == 0 and rep2["converged"] == 1 and rep2["rel_residual"] <= 1e-10
        xn = x2.cpu().numpy()
        assert abs(np.linalg.norm(case["g"] - S @ xn) / np.linalg.norm(case["g"]) - rep2["rel_residual"]) < 1e-12
        assert rel(xn, x_dir) < 1e-8
        x2b, rep2b, _ = gpu.solve(g_gpu, tol=1e-10, restart=30, maxit=5000, mode=mode, orth=orth, basis=BASIS_FIX)
        assert torch.equal(x2, x2b) and rep2 == rep2b
        if orth != 1:   # (the single projection's Pythagorean norm makes the count follow the rounding)
            _, rep0, _ = gpu.solve(g_gpu, tol=1e-10, restart=30, maxit=5000, mode=mode, orth=orth)
            assert abs(rep2["iterations"] - rep0["iterations"]) <= max(6, rep0["iterations"] // 5)


def test_fixed_point_basis_is_scale_invariant(case):
    """Power-of-two scaling of the right-hand side scales the fixed-point basis solve's
    iterate exactly (every chunk scale and coefficient scale moves by the same power)."""
    from paper_2302_10917_gb300 import BASIS_FIX
    gpu = case["gpu"]
    g = gpu.rhs()
    x1, r1, _ = gpu.solve(g, tol=1e-10, restart=30, maxit=5000, mode=3, orth=1, basis=BASIS_FIX)
    x2, r2, _ = gpu.solve(g * 2.0 ** 37, tol=1e-10, restart=30, maxit=5000, mode=3, orth=1, basis=BASIS_FIX)
    assert r1["iterations"] == r2["iterations"]
    assert torch.equal(x2, x1 * 2.0 ** 37)


def test_fixed_point_argument_errors():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2302_10917_gb300 import HDG_ERR_ARG, HDGError, Problem
    gpu = Problem(3, 2, 2, beta=(1.0, 0.0), kappa=1.0)
    gpu.set_source(wl.sin_sin_source(gpu.quad_points(), 1.0, (1.0, 0.0)))
    gpu.condense()
    x = torch.zeros(gpu.info["N_tr"], dtype=torch.float64, device="cuda")
    with pytest.raises(HDGError) as ei:
        gpu.apply(x, prec=56, precond=True)              # fixed-point blocks were not stored
    assert ei.value.status == HDG_ERR_ARG
    _, _, st = gpu.solve(gpu.rhs(), mode=3, check=False)
    assert st == HDG_ERR_ARG
    gpu.condense(store_fix=True)
    with pytest.raises(HDGError) as ei:
        gpu.apply(x, prec=56, precond=False)             # the fixed-point rows are the preconditioned ones
    assert ei.value.status == HDG_ERR_ARG
    g2 = torch.stack([gpu.rhs(), gpu.rhs()])
    _, _, st = gpu.solve(g2, mode=3, check=False)        # one right-hand side only
    assert st == HDG_ERR_ARG
    _, _, st = gpu.solve(gpu.rhs(), mode=3, basis=1, check=False)   # FP64 vectors only
    assert st == HDG_ERR_ARG
    _, _, st = gpu.solve(g2, basis=2, check=False)                  # the fixed-point basis: one column
    assert st == HDG_ERR_ARG
    _, _, st = gpu.solve(gpu.rhs(), basis=2, augment=1, restart=10, check=False)   # and no augmentation
    assert st == HDG_ERR_ARG
    gpu.close()
    lv = Problem(4, 1, 1, beta=(1.0, 0.0), kappa=1.0, levels=np.zeros(32, dtype=np.int32))
    lv.set_source(torch.zeros(lv.info["n_qp_total"], dtype=torch.float64))
    with pytest.raises(HDGError) as ei:
        lv.condense(store_fix=True)                      # uniform meshes only
    assert ei.value.status == HDG_ERR_ARG
    lv.close()
