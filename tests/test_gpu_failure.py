"""Failure detection without a GPU fault.

The pipelined trace apply (bulk asynchronous copies into shared-memory slots,
consumer warps waiting on shared-memory barriers) bounds every wait. The
test hook of hdg_set_wait_hooks leaves one interior edge's copies unissued, so
the consumers of that slot wait for a copy that never comes: their bounded
wait gives up after the set number of cycles, the kernel records the failure
and returns, the entry point reports HDG_ERR_TIMEOUT, and the next call on the
same context, with the hook cleared, gives the same bits as before. Nothing
faults, traps or hangs: the wait's limit is what ends it.
"""
import time

import numpy as np
import pytest
import torch

from paper_2302_10917_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def _split(x):
    hi = x.astype(np.float32)
    lo = (x - hi.astype(np.float64)).astype(np.float32)
    return torch.from_numpy(np.stack([hi, lo], axis=1))


@pytest.fixture(scope="module")
def problem():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import math
    from paper_2302_10917_gb300 import Problem
    n, m, p = 8, 8, 3
    beta = (50.0 * math.cos(0.3), 50.0 * math.sin(0.3))
    pr = Problem(n, m, p, beta=beta, kappa=wl.random_kappa(2 * n * n, seed=5))
    pr.set_source(wl.sin_sin_source(pr.quad_points(), 1.0, beta).contiguous())
    pr.condense(keep_factors=True, store_df64=True, split_update=True)
    yield pr
    pr.close()


def test_bounded_wait_gives_up_and_the_context_stays_usable(problem):
    from paper_2302_10917_gb300 import BASIS_DF64, HDG_ERR_TIMEOUT, HDGError
    pr = problem
    try:
        pr.set_apply_shape(2, bulk_warps=1)
    except HDGError:
        pytest.skip("the pipelined apply does not fit this device")
    x = _split(wl.random_vector(pr.info["N_tr"], seed=4))
    try:
        y0 = pr.apply(x, precond=True, prec=49)
        torch.cuda.synchronize()
        # about 10 ms at 2 GHz per wait; the copies of interior edge 5 are never issued
        pr.set_wait_hooks(wait_cycles=20_000_000, skip_copy_edge=5)
        t0 = time.perf_counter()
        with pytest.raises(HDGError) as ei:
            pr.apply(x, precond=True, prec=49)
        assert ei.value.status == HDG_ERR_TIMEOUT
        assert time.perf_counter() - t0 < 10.0
        # a solve whose Arnoldi operator is the pipelined apply reports the timeout as well
        _, rep, st = pr.solve(pr.rhs(), tol=1e-10, restart=20, maxit=60, mode=2, basis=BASIS_DF64, check=False)
        assert st == HDG_ERR_TIMEOUT, rep
        # hook cleared, default limit: the same context gives the same bits as before
        pr.set_wait_hooks()
        assert torch.equal(pr.apply(x, precond=True, prec=49), y0)
        x_s, rep, st = pr.solve(pr.rhs(), tol=1e-10, restart=40, mode=2, basis=BASIS_DF64)
        assert st == 0 and rep["converged"] == 1
    finally:
        pr.set_wait_hooks()
        pr.set_apply_shape(2)


def test_wait_hooks_reject_bad_arguments(problem):
    from paper_2302_10917_gb300 import HDG_ERR_ARG, HDGError
    pr = problem
    for args in ((-1, -1), (0, -2), (0, pr.info["n_int_edges"])):
        with pytest.raises(HDGError) as ei:
            pr.set_wait_hooks(*args)
        assert ei.value.status == HDG_ERR_ARG, args
    pr.set_wait_hooks()
