"""The banded-level many-source workload at full size, through the calls
bench.py times: n = 128 (32,768 macro-elements), p = 2, levels by band of x
(r = 1 below x = 0.7, 2, 3, r = 4 from x = 0.9 on; 462,020 trace unknowns,
384 elements with a face finer than themselves), kappa = 1e-2, beta = (1, 0),
64 Gaussian-bump sources (width 0.05, seeded centres), g_D = 0; split-FP32
condensation, the face-block preconditioner with the diagonal blocks of S
(restarted GMRES with D^-1 of Sec. 6.1 stalls on this mesh), 64 right-hand
sides in lockstep GMRES (split-FP32 operator).

The oracle checks sampled outputs one by one: Schur blocks of sampled
elements of every level (conforming and non-conforming), the condensed
right-hand side on sampled faces from the oracle's own element right-hand
sides of the two sides, and the back-solve of sampled elements from the
GPU's trace solution; the solve itself by its reported residual.
"""
import numpy as np
import pytest
import torch

from oracle.levels import LevelHDGProblem
from paper_2302_10917_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

CFG = wl.CONFIGS["levels_n128_p2_64src"]
COLS = (0, 37, 63)          # sampled right-hand sides


@pytest.fixture(scope="module")
def big():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2302_10917_gb300 import Problem
    lev = wl.band_levels(CFG["n"])
    gpu = Problem(CFG["n"], 1, CFG["p"], beta=CFG["beta"], kappa=CFG["kappa"], levels=lev)
    f = wl.gaussian_bumps(gpu.quad_points(), CFG["nrhs"], seed=3, width=CFG["width"]).contiguous()
    gpu.set_source(f)
    gpu.condense(keep_factors=True, store_df64=True, split_update=True, precond="face_schur")
    ora = LevelHDGProblem(CFG["n"], lev, CFG["p"], beta=CFG["beta"], kappa=CFG["kappa"])
    fc = {r: f[r].cpu().numpy() for r in COLS}
    yield gpu, ora, lev, fc
    gpu.close()


def _sampled_elements(ora, lev):
    out = []
    for r in (1, 2, 3, 4):
        els = np.nonzero(lev == r)[0]
        out.append(int(els[len(els) // 2]))
    nonconf = [e for e in range(ora.N) if any(R != lev[e] for *_, R in ora.faces(e))]
    gaps = {}
    for e in nonconf:
        gap = max(R for *_, R in ora.faces(e)) - lev[e]
        gaps.setdefault((int(lev[e]), gap), e)
    out += sorted(gaps.values())
    return out


def test_sampled_schur_blocks(big):
    gpu, ora, lev, _ = big
    from paper_2302_10917_gb300 import OFF_SCHUR
    off = gpu.offsets(OFF_SCHUR)
    els = _sampled_elements(ora, lev)
    assert len(els) >= 6
    for e in els:
        S_o, _ = ora.condense_element(e)
        nt = S_o.shape[0]
        assert int(off[e + 1] - off[e]) == nt * nt
        S_g = gpu.schur(e, 1).cpu().numpy().reshape(nt, nt)
        assert np.abs(S_g - S_o).max() / np.abs(S_o).max() < 1e-11, e


def test_sampled_rhs_faces(big):
    gpu, ora, lev, fc = big
    g = gpu.rhs()
    assert g.shape == (CFG["nrhs"], ora.N_tr)
    # faces inside each band, and faces between bands (level jumps)
    faces, jumps = [], []
    for f in range(0, ora.n_int, 7):
        lv = {int(lev[e]) for e in _edge_elements(ora, f)}
        if len(lv) == 2 and len(jumps) < 3:
            jumps.append(f)
        elif len(lv) == 1 and int(ora.flevel[f]) not in [int(ora.flevel[h]) for h in faces]:
            faces.append(f)
    faces += jumps
    assert len(faces) == 7
    cache = {}
    for f in faces:
        for r in COLS:
            acc = np.zeros(int(ora.eoff[f + 1] - ora.eoff[f]))
            for e in _edge_elements(ora, f):
                key = (e, r)
                if key not in cache:
                    cache[key] = ora.condense_element(e, fc[r])[1]
                loc = _local_rows(ora, e, f)
                acc += cache[key][loc]
            got = g[r, ora.eoff[f]:ora.eoff[f + 1]].cpu().numpy()
            assert np.abs(got - acc).max() <= 1e-11 * max(np.abs(acc).max(), 1e-3 * float(g[r].abs().max())), (f, r)


def _edge_elements(ora, f):
    n = ora.n
    if f < n * n:
        j, i = divmod(f, n)
        return [2 * (j * n + i), 2 * (j * n + i) + 1]
    if f < n * n + n * (n - 1):
        rr = f - n * n
        j, i = 1 + rr // n, rr % n
        return [2 * ((j - 1) * n + i) + 1, 2 * (j * n + i)]
    rr = f - n * n - n * (n - 1)
    j, i = rr // (n - 1), 1 + rr % (n - 1)
    return [2 * (j * n + i - 1), 2 * (j * n + i) + 1]


def _local_rows(ora, e, f):
    """Element-local trace rows of face f in element e, ordered along the edge's orientation."""
    dmap = ora.element_dof_map(e)
    rows = {idx: loc for loc, (kind, idx) in enumerate(dmap) if kind == "int" and ora.eoff[f] <= idx < ora.eoff[f + 1]}
    return np.array([rows[i] for i in range(int(ora.eoff[f]), int(ora.eoff[f + 1]))])


def test_batched_solve_and_sampled_back_solve(big):
    gpu, ora, lev, fc = big
    g = gpu.rhs()
    x, rep, st = gpu.solve(g, tol=1e-10, restart=80, mode=2, orth=2, maxit=40000)
    assert st == 0 and rep["converged"] == 1 and rep["rel_residual"] <= 1e-10, rep
    # every column's residual with the FP64 operator, independently of the solver's own test
    res = (g - gpu.apply(x)).norm(dim=1) / g.norm(dim=1)
    assert float(res.max()) <= 1.05e-10
    u, q = gpu.recover(x)
    els = _sampled_elements(ora, lev)[:6]
    for r in COLS[:2]:
        xr = x[r].cpu().numpy()
        ur, qr = u[r].cpu().numpy(), q[r].cpu().numpy()
        for e in els:
            ue, qe = ora.recover_element(e, xr, fc[r])
            s = np.abs(ue).max()
            assert np.abs(ur[ora.uoff[e]:ora.uoff[e + 1]] - ue).max() <= 1e-9 * max(s, 1e-3 * np.abs(ur).max()), (r, e)
            assert np.abs(qr[2 * ora.uoff[e]:2 * ora.uoff[e + 1]] - qe.reshape(-1)).max() <= \
                1e-8 * max(np.abs(qe).max(), 1e-3 * np.abs(qr).max()), (r, e)
