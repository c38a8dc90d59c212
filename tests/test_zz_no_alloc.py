"""hdg_condense_static, the entry point for callers that may not allocate device
memory after start-up (it works in a fixed scratch array compiled into the
library): its Schur blocks must equal those of the regular hdg_condense path
and its element right-hand sides those of the oracle, element by element, on
two calls in a row that reuse the array; the second call must not change the
device's free memory (no allocation inside the call).

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


def _sources(pr, seed, nrhs):
    g = np.random.default_rng([wl.MASTER_SEED, 71, seed])
    f = g.standard_normal((nrhs, pr.info["N"], pr.info["n_qp"]))
    gD = g.standard_normal((nrhs, pr.info["n_bnd_edges"], pr.info["n_bqp"]))
    return f, gD


def _rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


B1 = (50.0 * math.cos(0.3), 50.0 * math.sin(0.3))


@pytest.mark.parametrize("n,m,p,beta,nrhs", [(4, 2, 2, (1.0, 1.0), 1), (2, 8, 3, B1, 1), (4, 8, 3, B1, 1),
                                             (3, 4, 2, (0.5, -1.0), 2)])
def test_static_scratch_condensation_matches_regular_path(n, m, p, beta, nrhs):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from oracle.hdg import HDGProblem
    from paper_2302_10917_gb300 import STATIC_SCRATCH_BYTES, Problem
    seed = n * 10 + m
    kappa = wl.random_kappa(2 * n * n, seed=seed)
    pr = Problem(n, m, p, beta=beta, kappa=kappa)
    f, gD = _sources(pr, seed, nrhs)
    pr.set_source(torch.from_numpy(f if nrhs > 1 else f[0]), torch.from_numpy(gD if nrhs > 1 else gD[0]))
    N, nt, Q = pr.info["N"], pr.info["n_t"], pr.info["Q"]
    ld = (Q + nt + nrhs + 3) // 4 * 4
    max_count = STATIC_SCRATCH_BYTES // ((Q + nt) * ld * 8)
    assert max_count >= 2
    # the regular path: context-owned workspace
    pr.condense(keep_factors=False)
    S_ref = pr.schur().cpu().numpy()
    # the static path on two consecutive calls that share the scratch array
    half = min(max_count, (N + 1) // 2)
    rest = min(max_count, N - half)
    ranges = [(0, half), (half, rest)]
    outs = []
    for i, (e0, cnt) in enumerate(ranges):
        S = torch.full((cnt, nt, nt), float("nan"), dtype=torch.float64, device="cuda")
        g = torch.full((nrhs, cnt, nt), float("nan"), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        pr.condense_static(e0, cnt, S, g)
        torch.cuda.synchronize()
        if i == 1:
            # the second call (module loaded, buffers in place) allocates nothing on the device
            assert torch.cuda.mem_get_info()[0] == free0
        outs.append((S.cpu().numpy(), g.cpu().numpy()))
    for (e0, cnt), (S, g) in zip(ranges, outs):
        assert np.isfinite(S).all() and np.isfinite(g).all()
        assert _rel(S, S_ref[e0:e0 + cnt]) < TOL
    # element right-hand sides of every source against the oracle's, on sampled elements of both calls
    ora = HDGProblem(n, m, p, beta=beta, kappa=kappa)
    rng = np.random.default_rng(seed)
    for r in range(nrhs):
        ghat = ora.dirichlet_trace(gD[r])
        for (e0, cnt), (_, g) in zip(ranges, outs):
            for b in sorted(rng.choice(cnt, size=min(cnt, 3), replace=False)):
                e = e0 + int(b)
                ghe = ora.element_trace(e, np.zeros(ora.mesh.N_tr), ghat)
                _, g_e = ora.condense_element(e, f[r][e], ghe)
                assert _rel(g[r, b], g_e) < TOL, (r, e)
    # a count beyond the fixed array is refused with a clear error
    from paper_2302_10917_gb300 import HDG_ERR_ARG, HDGError
    if max_count < N:
        big = torch.empty((max_count + 1, nt, nt), dtype=torch.float64, device="cuda")
        with pytest.raises(HDGError) as ei:
            pr.condense_static(0, max_count + 1, big)
        assert ei.value.status == HDG_ERR_ARG and "static array holds" in str(ei.value)
    pr.close()
