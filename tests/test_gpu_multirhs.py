"""Several right-hand sides on one condensation: per-source load columns of
the bordered system, the multi-RHS trace apply (every block streamed once
for all columns), the lockstep batched GMRES and the per-source back-solve,
each column against the oracle's single-source computation. Tolerances as
in the single-source parity tests: 1e-12 (right-hand sides, FP64 and
split-FP32 applies), 5e-5 (FP32 apply), 1e-8 (solutions at a 1e-10 residual),
1e-11 (back-solve from the same trace)."""
import math

import numpy as np
import pytest
import torch

from oracle.hdg import HDGProblem
from paper_2302_10917_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

B1 = (50.0 * math.cos(0.3), 50.0 * math.sin(0.3))
CASES = [("m2p2r5", 3, 2, 2, (0.8, -0.3), 5), ("m8p3r3", 2, 8, 3, B1, 3), ("m4p2r13", 2, 4, 2, (1.0, 0.5), 13)]


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.fixture(scope="module", params=CASES, ids=[c[0] for c in CASES])
def mcase(request):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2302_10917_gb300 import Problem
    cid, n, m, p, beta, nrhs = request.param
    kappa = wl.random_kappa(2 * n * n, seed=5 * n + m + nrhs)
    ora = HDGProblem(n, m, p, beta=beta, kappa=kappa)
    pts, _ = ora.quad_points()
    bpts, _ = ora.bnd_quad_points()
    g = np.random.default_rng([wl.MASTER_SEED, 151, n, m, p, nrhs])
    f = g.standard_normal((nrhs,) + pts.shape[:2])
    gD = g.standard_normal((nrhs,) + bpts.shape[:2])
    f[1] = 0.0          # one source with no volume load (its column is the Dirichlet lift only)
    cond = [ora.condense(f[r], gD[r]) for r in range(nrhs)]
    S_el = cond[0][0]
    pr = Problem(n, m, p, beta=beta, kappa=kappa)
    pr.set_source(torch.from_numpy(f), torch.from_numpy(gD))
    pr.condense(keep_factors=True, store_fp32=True, store_df64=True)
    torch.cuda.synchronize()
    yield dict(ora=ora, pr=pr, f=f, gD=gD, cond=cond, S=ora.assemble_S(S_el), S_el=S_el, nrhs=nrhs, rng=g)
    pr.close()


def test_schur_blocks_unchanged_by_extra_sources(mcase):
    S = mcase["pr"].schur().cpu().numpy()
    for e in range(S.shape[0]):
        assert rel(S[e], mcase["S_el"][e]) < 1e-12


def test_right_hand_sides_per_source(mcase):
    g = mcase["pr"].rhs().cpu().numpy()
    assert g.shape == (mcase["nrhs"], mcase["ora"].mesh.N_tr)
    for r in range(mcase["nrhs"]):
        assert rel(g[r], mcase["cond"][r][1]) < 1e-12, r


@pytest.mark.parametrize("k", [1, 2, 7, 33, 64])
def test_multi_rhs_apply_matches_oracle(mcase, k):
    ora, pr, S = mcase["ora"], mcase["pr"], mcase["S"]
    X = mcase["rng"].standard_normal((k, ora.mesh.N_tr))
    Xt = torch.from_numpy(X).cuda()
    ref = X @ S.T
    ref_p = np.stack([ora.apply_Dinv(v) for v in ref])
    y = pr.apply(Xt if k > 1 else Xt[0], precond=False, prec=64).reshape(k, -1).cpu().numpy()
    assert rel(y, ref) < 1e-12
    yp = pr.apply(Xt if k > 1 else Xt[0], precond=True, prec=64).reshape(k, -1).cpu().numpy()
    assert rel(yp, ref_p) < 1e-12
    y48 = pr.apply(Xt if k > 1 else Xt[0], precond=True, prec=48).reshape(k, -1).cpu().numpy()
    assert rel(y48, ref_p) < 1e-12
    y32 = pr.apply((Xt if k > 1 else Xt[0]).float(), precond=True, prec=32).reshape(k, -1).cpu().numpy()
    assert rel(y32, ref_p) < 5e-5


@pytest.mark.parametrize("mode,orth,basis,augment", [(2, 1, 1, 0), (0, 0, 0, 0), (1, 1, 0, 0), (2, 2, 0, 0),
                                                      (1, 1, 1, 0), (0, 2, 1, 0), (0, 3, 0, 2), (2, 3, 1, 3)])
def test_batched_solve_and_recover_match_oracle(mcase, mode, orth, basis, augment):
    """Lockstep batched GMRES on every column; basis 0: FP64 Krylov basis, 1: split-FP32;
    augment > 0: augmented restarts (LGMRES)."""
    ora, pr, S, nrhs = mcase["ora"], mcase["pr"], mcase["S"], mcase["nrhs"]
    g = pr.rhs()
    x, rep, st = pr.solve(g, tol=1e-10, restart=30 if augment == 0 else 8, mode=mode, orth=orth, basis=basis,
                          augment=augment)
    assert st == 0 and rep["converged"] == 1 and rep["rel_residual"] <= 1e-10
    xs = x.cpu().numpy()
    for r in range(nrhs):
        x_ref = np.linalg.solve(S, mcase["cond"][r][1])
        assert rel(xs[r], x_ref) < 1e-8, r
    u, q = pr.recover(x)
    u, q = u.cpu().numpy(), q.cpu().numpy()
    for r in range(nrhs):
        u_o, q_o = ora.recover(xs[r], mcase["f"][r], mcase["cond"][r][2])
        assert rel(u[r], u_o) < 1e-11 and rel(q[r], q_o) < 1e-11, r


def test_zero_right_hand_side_column():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2302_10917_gb300 import Problem
    pr = Problem(2, 2, 2, beta=(1.0, 0.0), kappa=1.0)
    f = torch.zeros(3, pr.info["N"], pr.info["n_qp"], dtype=torch.float64)
    f[0] = 1.0
    f[2] = -2.0
    pr.set_source(f)
    pr.condense()
    g = pr.rhs()
    assert torch.count_nonzero(g[1]) == 0
    x, rep, st = pr.solve(g, tol=1e-12, restart=20)
    assert st == 0 and torch.count_nonzero(x[1]) == 0
    assert torch.allclose(x[2], -2.0 * x[0], rtol=1e-9, atol=1e-14)
    pr.close()


def test_source_count_limits():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2302_10917_gb300 import HDG_ERR_ARG, HDGError, Problem
    pr = Problem(1, 1, 1, beta=(1.0, 0.0), kappa=1.0)
    with pytest.raises(HDGError) as ei:
        pr.set_source(torch.zeros(65, pr.info["N"], pr.info["n_qp"], dtype=torch.float64))
    assert ei.value.status == HDG_ERR_ARG
    pr.set_source(torch.zeros(2, pr.info["N"], pr.info["n_qp"], dtype=torch.float64))
    pr.condense()
    with pytest.raises(HDGError):
        pr.recover(torch.zeros(pr.info["N_tr"], dtype=torch.float64))   # one trace for two sources
    pr.close()
