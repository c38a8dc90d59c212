"""Small, self-contained run of the hot-path kernels for profiler captures.

    python -m paper_2302_10917_gb300.profcase --n 64 --m 8 --p 3 --applies 4
    python -m paper_2302_10917_gb300.profcase --n 128 --step --restart 80 --mode 2

Default: builds the n x n macro mesh with the manufactured source, condenses it
with a chunked workspace (factors not kept, a few GB on the device at most),
then runs `applies` FP64 preconditioned trace applies, then one
unpreconditioned FP64 apply, one split-FP32 (df64) apply and one FP32 apply,
and optionally `gmres-steps` Arnoldi steps. Prints the device time of each
phase.

--step: one step of the benchmark's pipeline with GMRES cut to one restart
cycle: set_source, condensation (factors kept, the blocks the mode needs,
split-FP32 panel updates), right-hand side, GMRES(restart) for `restart`
Arnoldi steps, back-solve. Its kernel mix is that of a full step with fewer
restart cycles.

--levels: the banded-level mesh (p = 2, kappa = 1e-2, beta = (1, 0), levels
r = 1 .. 4 by band of x) with `nrhs` Gaussian-bump sources: condensation
(factors not kept), then `applies` preconditioned applies of nrhs columns with
FP64, split-FP32 and FP32 blocks each.

    python -m paper_2302_10917_gb300.profcase --levels --n 64 --nrhs 1 --applies 3
"""
import argparse
import json
import math

import torch

from . import Problem
from . import workloads as wl


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=64)
    ap.add_argument("--m", type=int, default=8)
    ap.add_argument("--p", type=int, default=3)
    ap.add_argument("--applies", type=int, default=4)
    ap.add_argument("--gmres-steps", type=int, default=0,
                    help="also run this many GMRES(50) Arnoldi steps")
    ap.add_argument("--mode", type=int, default=2, help="GMRES Arnoldi operator (0 FP64, 1 FP32, 2 split FP32)")
    ap.add_argument("--lean", action="store_true", help="store only the blocks the chosen mode needs")
    ap.add_argument("--step", action="store_true", help="one benchmark step cut to one restart cycle")
    ap.add_argument("--restart", type=int, default=50)
    ap.add_argument("--split", action="store_true", help="split-FP32 condensation")
    ap.add_argument("--orth", type=int, default=1, help="0: CGS2, 1: single-projection Gram-Schmidt")
    ap.add_argument("--autotune", action="store_true", help="run the launch-shape autotuner before the solve")
    ap.add_argument("--bulk", type=int, default=0,
                    help="split-FP32 operator in the pipelined bulk-copy shape with this many warps per edge "
                         "(after --autotune); without --step also times it against the default shape")
    ap.add_argument("--levels", action="store_true", help="the banded-level mesh (see the module docstring)")
    ap.add_argument("--nrhs", type=int, default=1, help="columns of the level-mesh applies")
    a = ap.parse_args(argv)
    if a.levels:
        return _levels(a)
    beta = (50.0 * math.cos(0.3), 50.0 * math.sin(0.3))
    pr = Problem(a.n, a.m, a.p, beta=beta, kappa=1.0)
    xy = pr.quad_points()
    f = wl.sin_sin_source(xy, 1.0, beta)
    del xy
    if a.step:
        return _step(pr, f, a)
    pr.set_source(f)
    ev = lambda: torch.cuda.Event(enable_timing=True)
    t = [ev() for _ in range(7)]
    t[0].record()
    lean = a.lean
    pr.condense(store_fp32=not lean or a.mode == 1, keep_factors=False, store_df64=not lean or a.mode == 2,
                split_update=a.split)
    t[1].record()
    x = torch.from_numpy(wl.random_vector(pr.info["N_tr"], seed=5)).cuda()
    for _ in range(a.applies):
        y = pr.apply(x, precond=True)
    t[2].record()
    y = pr.apply(x, precond=False)
    t[3].record()
    y32 = pr.apply(x.float(), precond=True, prec=32) if (not lean or a.mode == 1) else y.float()
    t[4].record()
    ydf = pr.apply(x, precond=True, prec=48) if (not lean or a.mode == 2) else y
    t[5].record()
    torch.cuda.synchronize()
    gm = None
    if a.autotune:
        pr.autotune(mode=a.mode, restart=a.restart)
    bulk_ms = {}
    if a.bulk > 0:
        xs = torch.stack([x.float(), (x - x.float().double()).float()], dim=1).contiguous()
        for name, bulk in (("default", 0), ("bulk", a.bulk)):
            pr.set_apply_shape(2, bulk_warps=bulk)
            pr.apply(xs, precond=True, prec=49)
            e0, e1 = ev(), ev()
            e0.record()
            for _ in range(max(1, a.applies)):
                pr.apply(xs, precond=True, prec=49)
            e1.record()
            torch.cuda.synchronize()
            bulk_ms[name] = e0.elapsed_time(e1) / max(1, a.applies)
    if a.gmres_steps > 0:
        x0, rep, st = pr.solve(pr.rhs(), tol=1e-14, restart=a.restart, maxit=a.gmres_steps, mode=a.mode,
                               check=False, orth=a.orth)
        gm = rep
    out = {"info": pr.info, "gmres": gm, "condense_ms": t[0].elapsed_time(t[1]),
           "apply64_pc_ms": t[1].elapsed_time(t[2]) / max(1, a.applies), "apply64_ms": t[2].elapsed_time(t[3]),
           "apply32_ms": t[3].elapsed_time(t[4]), "apply_df_ms": t[4].elapsed_time(t[5]),
           "y_norm": float(y.norm()), "y32_norm": float(y32.norm()), "ydf_norm": float(ydf.norm()),
           "apply49_ms": bulk_ms}
    print(json.dumps(out))
    pr.close()


def _step(pr, f, a):
    ev = lambda: torch.cuda.Event(enable_timing=True)
    t = [ev() for _ in range(5)]
    torch.cuda.synchronize()
    t[0].record()
    pr.set_source(f)
    pr.condense(keep_factors=True, store_fp32=a.mode == 1, store_df64=a.mode == 2, split_update=True)
    t[1].record()
    g = pr.rhs()
    if a.autotune:
        pr.autotune(mode=a.mode, restart=a.restart)
    if a.bulk > 0:
        pr.set_apply_shape(2, bulk_warps=a.bulk)
    x, rep, st = pr.solve(g, tol=1e-14, restart=a.restart, maxit=a.restart, mode=a.mode, check=False, orth=a.orth)
    t[2].record()
    u, q = pr.recover(x)
    t[3].record()
    torch.cuda.synchronize()
    out = {"info": pr.info, "gmres": rep, "condense_ms": t[0].elapsed_time(t[1]),
           "gmres_ms": t[1].elapsed_time(t[2]), "recover_ms": t[2].elapsed_time(t[3]),
           "u_norm": float(u.norm()), "launches": pr.launches()}
    print(json.dumps(out))
    pr.close()



def _levels(a):
    cfg = wl.CONFIGS["levels_n128_p2_64src"]
    lev = wl.band_levels(a.n)
    pr = Problem(a.n, 1, cfg["p"], beta=cfg["beta"], kappa=cfg["kappa"], levels=lev)
    f = wl.gaussian_bumps(pr.quad_points(), a.nrhs, seed=3, width=cfg["width"]).contiguous()
    pr.set_source(f[0] if a.nrhs == 1 else f)
    ev = lambda: torch.cuda.Event(enable_timing=True)
    t = [ev() for _ in range(5)]
    t[0].record()
    pr.condense(store_fp32=True, keep_factors=False, store_df64=True, split_update=True)
    t[1].record()
    X = torch.randn(a.nrhs, pr.info["N_tr"], dtype=torch.float64, device=pr.device)
    X = X[0] if a.nrhs == 1 else X
    for _ in range(a.applies):
        pr.apply(X, precond=True, prec=64)
    t[2].record()
    for _ in range(a.applies):
        pr.apply(X, precond=True, prec=48)
    t[3].record()
    X32 = X.float()
    for _ in range(a.applies):
        pr.apply(X32, precond=True, prec=32)
    t[4].record()
    torch.cuda.synchronize()
    k = max(1, a.applies)
    print(json.dumps({"info": pr.info, "condense_ms": t[0].elapsed_time(t[1]),
                      "apply64_ms": t[1].elapsed_time(t[2]) / k, "apply_df_ms": t[2].elapsed_time(t[3]) / k,
                      "apply32_ms": t[3].elapsed_time(t[4]) / k}))
    pr.close()


if __name__ == "__main__":
    main()
