"""hdg_condense_static, the entry point for callers that may not allocate device
memory after start-up (it works in a fixed scratch array compiled into the
library): its Schur blocks and element right-hand sides must equal those of
the regular hdg_condense path, on two calls in a row that reuse the array.

This file is named to be collected last, so that a run stopping at the first
failure has already run every other test. It passes on its own in a fresh
process as well as after the other tests.
"""
import math

import numpy as np
import pytest
import torch

from paper_2302_10917_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

TOL = 1e-12   # the relative tolerance the FP64 parity tests use


def _problem(n, m, p, beta, seed):
    from paper_2302_10917_gb300 import Problem
    kappa = wl.random_kappa(2 * n * n, seed=seed)
    pr = Problem(n, m, p, beta=beta, kappa=kappa)
    g = np.random.default_rng([wl.MASTER_SEED, 71, seed])
    f = torch.from_numpy(g.standard_normal((pr.info["N"], pr.info["n_qp"])))
    gD = torch.from_numpy(g.standard_normal((pr.info["n_bnd_edges"], pr.info["n_bqp"])))
    pr.set_source(f, gD)
    return pr


def _rel(a, b):
    return (a - b).abs().max().item() / max(b.abs().max().item(), 1e-300)


B1 = (50.0 * math.cos(0.3), 50.0 * math.sin(0.3))


@pytest.mark.parametrize("n,m,p,beta", [(4, 2, 2, (1.0, 1.0)), (2, 8, 3, B1), (4, 8, 3, B1)])
def test_static_scratch_condensation_matches_regular_path(n, m, p, beta):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2302_10917_gb300 import STATIC_SCRATCH_BYTES
    pr = _problem(n, m, p, beta, seed=n * 10 + m)
    N, nt, Q = pr.info["N"], pr.info["n_t"], pr.info["Q"]
    ld = (Q + nt + 1 + 3) // 4 * 4
    max_count = STATIC_SCRATCH_BYTES // ((Q + nt) * ld * 8)
    assert max_count >= 2
    # the regular path: context-owned workspace
    pr.condense(keep_factors=False)
    S_ref = pr.schur()
    # the regular path exposes the element right-hand sides only assembled (hdg_rhs)
    g_ref = pr.rhs()
    # the static path on two consecutive calls that share the scratch array
    half = min(max_count, (N + 1) // 2)
    S1 = torch.full((half, nt, nt), float("nan"), dtype=torch.float64, device="cuda")
    g1 = torch.full((half, nt), float("nan"), dtype=torch.float64, device="cuda")
    pr.condense_static(0, half, S1, g1)
    rest = min(max_count, N - half)
    S2 = torch.full((rest, nt, nt), float("nan"), dtype=torch.float64, device="cuda")
    g2 = torch.full((rest, nt), float("nan"), dtype=torch.float64, device="cuda")
    pr.condense_static(half, rest, S2, g2)
    torch.cuda.synchronize()
    assert torch.isfinite(S1).all() and torch.isfinite(S2).all()
    assert _rel(S1, S_ref[:half]) < TOL
    assert _rel(S2, S_ref[half:half + rest]) < TOL
    if half + rest == N:
        # assemble the element right-hand sides the static path returned and compare with hdg_rhs
        from oracle.mesh import StructuredMesh
        msh = StructuredMesh(n, m, p)
        gel = torch.cat([g1, g2]).cpu().numpy()
        g_asm = np.zeros(msh.N_tr)
        for e in range(N):
            for loc, (kind, idx) in enumerate(msh.element_dof_map(e)):
                if kind == "int":
                    g_asm[idx] += gel[e, loc]
        ref = g_ref.cpu().numpy()
        assert np.abs(g_asm - ref).max() / np.abs(ref).max() < TOL
    # a count beyond the fixed array is refused with a clear error
    from paper_2302_10917_gb300 import HDG_ERR_ARG, HDGError
    if max_count < N:
        big = torch.empty((max_count + 1, nt, nt), dtype=torch.float64, device="cuda")
        with pytest.raises(HDGError) as ei:
            pr.condense_static(0, max_count + 1, big)
        assert ei.value.status == HDG_ERR_ARG and "static array holds" in str(ei.value)
    pr.close()
