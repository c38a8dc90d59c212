"""Writes levels_band_n32.json: the oracle's solution of the banded-level mesh at n = 32.

Inputs (seeded, from the workload generators): n = 32, p = 2, kappa = 1e-2,
beta = (1, 0), levels by band of the centroid's x (r = 1 below 0.7, 2, 3,
r = 4 from 0.9 on; faces at the finer side's level), one Gaussian-bump source
(width 0.05, centre seed 3), g_D = 0.

The oracle (oracle/levels.py) condenses every element by dense LU, assembles
S as a sparse matrix and solves S x = g directly (sparse LU); it also runs its
own GMRES(80) with the face preconditioner D^-1 (Sec. 6.1) and records the
iteration count. Stored: a seeded sample of 600 trace dofs with x and g
there, the norms of x and g, the iteration count, the direct solve's residual.

    python tests/golden/make_levels_band_n32.py      # a few minutes, CPU only
"""
import json
import os
import sys

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle.levels import LevelHDGProblem          # noqa: E402
from oracle.solver import gmres                    # noqa: E402
from paper_2302_10917_gb300 import workloads as wl  # noqa: E402  (input generators only)

N_SIDE, P, KAPPA, BETA, WIDTH, SEED = 32, 2, 1e-2, (1.0, 0.0), 0.05, 3


def main():
    import torch
    lev = wl.band_levels(N_SIDE)
    pr = LevelHDGProblem(N_SIDE, lev, P, beta=BETA, kappa=KAPPA)
    pts, _ = pr.quad_points()
    f = wl.gaussian_bumps(torch.from_numpy(pts), 1, seed=SEED, width=WIDTH)[0].numpy()
    S_el, g, _ = pr.condense(f, None)
    rows, cols, vals = [], [], []
    for e in range(pr.N):
        dm = pr.element_dof_map(e)
        idx = [(loc, i) for loc, (kind, i) in enumerate(dm) if kind == "int"]
        for la, ia in idx:
            for lb, ib in idx:
                rows.append(ia)
                cols.append(ib)
                vals.append(S_el[e][la, lb])
    S = sp.csr_matrix((vals, (rows, cols)), shape=(pr.N_tr, pr.N_tr))
    x = spla.spsolve(S.tocsc(), g)
    res = float(np.linalg.norm(g - S @ x) / np.linalg.norm(g))
    Df = pr.face_D()
    _, its, rel, ok = gmres(lambda v: S @ v, lambda y: pr.apply_Dinv(y, Df), g, tol=1e-10, restart=80,
                            maxit=20000)
    sample = np.sort(np.random.default_rng([wl.MASTER_SEED, 97]).choice(pr.N_tr, size=600, replace=False))
    out = {"n": N_SIDE, "p": P, "kappa": KAPPA, "beta": list(BETA), "width": WIDTH, "seed": SEED,
           "N_tr": int(pr.N_tr), "direct_rel_residual": res,
           "gmres80_iterations": int(its), "gmres80_rel_residual": float(rel), "gmres80_converged": bool(ok),
           "x_norm": float(np.linalg.norm(x)), "g_norm": float(np.linalg.norm(g)), "x_absmax": float(np.abs(x).max()),
           "dofs": sample.tolist(), "x": [float(v) for v in x[sample]], "g": [float(v) for v in g[sample]]}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "levels_band_n32.json")
    with open(path, "w") as fh:
        json.dump(out, fh, indent=0)
    print(path, "direct residual", res, "GMRES(80) iterations", its)


if __name__ == "__main__":
    main()
