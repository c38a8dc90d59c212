"""The precision forms of the whole path against the FP64 oracle.

The large workload's element (m = 8, p = 3, beta = 50 (cos 0.3, sin 0.3),
kappa = 1, sin-sin source) on a small macro mesh. The oracle condenses every
element from the literal 3Q x 3Q system of Eq. (D) and solves the assembled
trace system (Eq. global_problem) directly; each GPU form condenses, solves to
a 1e-10 true residual and back-solves:
  fp64     FP64 elimination, blocks, operator, Krylov basis and orthogonalisation;
  fp64_tc_fixed      the benchmark's step: FP64 panels with the trailing updates
           on the tensor cores (exact slices), the operator's products exact in
           integers (56-bit fixed-point rows), FP64 basis;
  fp64_tc_fixed_basis  as fp64_tc_fixed, with the fixed-point Krylov basis;
  fp32_ir  FP64 elimination, the preconditioned blocks stored and applied in
           FP32 inside FP64 residual replacement, FP64 basis;
  df64     split-FP32 elimination, blocks, operator and basis.
Bound: 1e-8 relative (max norm) for the trace, u and q (a 1e-10 residual times
the small meshes' condition numbers). The measured errors are printed (-s).
"""
import math

import numpy as np
import pytest
import torch

from oracle.hdg import HDGProblem
from oracle.problems import sin_sin

pytestmark = pytest.mark.gpu

FORMS = {"fp64": (0, 0, False), "fp64_tc_fixed": (3, 0, "tc"), "fp64_tc_fixed_basis": (3, 2, "tc"),
         "fp32_ir": (1, 0, False), "df64": (2, 1, True)}


def rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


@pytest.fixture(scope="module")
def oracle_solution():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    n, m, p = 4, 8, 3
    beta, kap = (50.0 * math.cos(0.3), 50.0 * math.sin(0.3)), 1.0
    ora = HDGProblem(n, m, p, beta=beta, kappa=kap)
    _, _, fexact = sin_sin(kap, beta)
    pts, _ = ora.quad_points()
    f_qp = fexact(pts[..., 0], pts[..., 1])
    S_el, g, ghat = ora.condense(f_qp, None)
    x = np.linalg.solve(ora.assemble_S(S_el), g)
    u, q = ora.recover(x, f_qp, ghat)
    return dict(n=n, m=m, p=p, beta=beta, kappa=kap, f=f_qp, x=x, u=u, q=q)


@pytest.mark.parametrize("form", list(FORMS))
def test_form_matches_the_oracle(oracle_solution, form):
    from paper_2302_10917_gb300 import Problem
    o = oracle_solution
    mode, basis, split = FORMS[form]
    pr = Problem(o["n"], o["m"], o["p"], beta=o["beta"], kappa=o["kappa"])
    try:
        pr.set_source(torch.from_numpy(o["f"]))
        pr.condense(keep_factors=True, store_fp32=(mode == 1), store_df64=(mode == 2), store_fix=(mode == 3),
                    split_update=split is True, tc_update=split == "tc")
        x, rep, st = pr.solve(pr.rhs(), tol=1e-10, restart=80, maxit=20000, mode=mode, orth=2, basis=basis)
        assert st == 0 and rep["converged"] == 1, rep
        u, q = pr.recover(x)
        ex, eu, eq = rel(x.cpu().numpy(), o["x"]), rel(u.cpu().numpy(), o["u"]), rel(q.cpu().numpy(), o["q"])
        print(f"\n{form}: iterations {rep['iterations']}, trace {ex:.2e}, u {eu:.2e}, q {eq:.2e}")
        assert ex < 1e-8 and eu < 1e-8 and eq < 1e-8, (ex, eu, eq)
    finally:
        pr.close()
