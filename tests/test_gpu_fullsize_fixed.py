"""The large workload (n = 128, m = 8, p = 3, 32,768 macro-elements, 1,222,400
trace unknowns) in the configuration bench.py times: condensation with the
trailing updates on the tensor cores, the preconditioned blocks also as
fixed-point rows, GMRES(80) with the fixed-point operator (mode 3), orth 3,
autotuned launch shapes.

Sampled outputs against the oracle one by one (Schur blocks of sampled
elements; rows of the preconditioned operator D_f^-1 (S x)|_f of sampled faces
from the oracle's own blocks of the two adjacent elements and its own D_f,
Sec. 3.3.2 and Sec. 6.1), and the solve by properties that hold at any size
(the reported residual is the true one; closeness to the manufactured solution).
"""
import math

import numpy as np
import pytest
import torch

from oracle.hdg import HDGProblem
from paper_2302_10917_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

CFG = wl.CONFIGS["n128_m8_p3"]


@pytest.fixture(scope="module")
def big():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2302_10917_gb300 import Problem
    gpu = Problem(CFG["n"], CFG["m"], CFG["p"], beta=CFG["beta"], kappa=CFG["kappa"])
    gpu.set_source(wl.sin_sin_source(gpu.quad_points(), CFG["kappa"], CFG["beta"]))
    gpu.condense(keep_factors=True, tc_update=True, store_fix=True)
    ora = HDGProblem(CFG["n"], CFG["m"], CFG["p"], beta=CFG["beta"], kappa=CFG["kappa"])
    yield gpu, ora
    gpu.close()


def _sample(N, k, seed):
    return np.random.default_rng([wl.MASTER_SEED, seed]).choice(N, size=k, replace=False)


def _adjacent(msh, f):
    n = msh.n
    if f < n * n:
        j, i = divmod(f, n)
        cands = [2 * (j * n + i), 2 * (j * n + i) + 1]
    elif f < n * n + n * (n - 1):
        r = f - n * n
        j, i = 1 + r // n, r % n
        cands = [2 * ((j - 1) * n + i) + 1, 2 * (j * n + i)]
    else:
        r = f - n * n - n * (n - 1)
        j, i = r // (n - 1), 1 + r % (n - 1)
        cands = [2 * (j * n + i - 1), 2 * (j * n + i) + 1]
    for e in cands:     # consistency with the oracle's own edge tables
        assert any(kind == "int" and idx == f for kind, idx, _ in msh.element_edges(e))
    return cands


def test_sampled_schur_blocks_of_the_tensor_core_condensation(big):
    gpu, ora = big
    N = ora.mesh.N
    for e in sorted(set(_sample(N, 10, 11).tolist() + [0, N - 1])):
        S_o, _ = ora.condense_element(int(e))
        S_g = gpu.schur(int(e), 1)[0].cpu().numpy()
        assert np.abs(S_g - S_o).max() / np.abs(S_o).max() < 1e-12, e


def test_sampled_rows_of_the_fixed_point_operator(big):
    """hdg_apply prec 56 (the benchmark's Arnoldi operator) on sampled faces against
    D_f^-1 (S_e1 x_e1 + S_e2 x_e2)|_f from the oracle."""
    gpu, ora = big
    msh = ora.mesh
    P1 = msh.P1
    x = wl.random_vector(msh.N_tr, seed=17)
    z = gpu.apply(torch.from_numpy(x), precond=True, prec=56).cpu().numpy()
    scale = np.abs(z).max()
    zero_bnd = np.zeros((msh.n_bnd_edges, P1))
    for f in _sample(msh.n_int_edges, 5, 12).tolist() + [0, msh.n_int_edges - 1]:
        out = np.zeros(msh.N_tr)
        Df = np.zeros((P1, P1))
        for e in _adjacent(msh, f):
            S_e, _ = ora.condense_element(e)
            ora.scatter(e, S_e @ ora.element_trace(e, x, zero_bnd), out)
            _, _, _, D = ora.local_blocks(e)
            for k, (kind, idx, flip) in enumerate(msh.element_edges(e)):
                if kind == "int" and idx == f:
                    blk = D[k * P1:(k + 1) * P1, k * P1:(k + 1) * P1]
                    Df += blk[::-1, ::-1] if flip else blk
        sl = slice(f * P1, (f + 1) * P1)
        zf = np.linalg.solve(Df, out[sl])
        assert np.abs(z[sl] - zf).max() / scale < 1e-12, f


def test_benchmark_solve_reports_the_true_residual_and_is_accurate(big):
    gpu, ora = big
    gpu.autotune(mode=3, restart=80)
    g = gpu.rhs()
    x, rep, st = gpu.solve(g, tol=1e-10, restart=80, mode=3, orth=3, maxit=60000)
    assert st == 0 and rep["converged"] == 1 and rep["rel_residual"] <= 1e-10
    r = g - gpu.apply(x)               # the FP64 operator, checked row by row against the oracle elsewhere
    assert abs(float(r.norm() / g.norm()) - rep["rel_residual"]) < 1e-13
    u, _ = gpu.recover(x)
    msh = ora.mesh
    ref = msh.lattice_ref()
    e = np.arange(msh.N)
    sq, t = e // 2, e % 2
    j, i = sq // msh.n, sq % msh.n
    h = 1.0 / msh.n
    x0, x1, y0, y1 = i * h, (i + 1) * h, j * h, (j + 1) * h
    v0 = np.where(t[:, None] == 0, np.stack([x1, y0], 1), np.stack([x0, y1], 1))
    v1 = np.where(t[:, None] == 0, np.stack([x1, y1], 1), np.stack([x0, y0], 1))
    v2 = np.where(t[:, None] == 0, np.stack([x0, y0], 1), np.stack([x1, y1], 1))
    X = v0[:, None, :] + ref[None, :, 0:1] * (v1 - v0)[:, None, :] + ref[None, :, 1:2] * (v2 - v0)[:, None, :]
    u_ex = np.sin(math.pi * X[..., 0]) * np.sin(math.pi * X[..., 1])
    assert np.abs(u.cpu().numpy() - u_ex).max() < 1e-6
