"""The split-FP32 Arnoldi operator (hdg_apply prec = 49: split-FP32 blocks on
split-FP32 vectors, the kernel and launch shape hdg_solve's mode 2 uses) in
every launch shape: the one-thread-per-row apply (default and 1 edge per
block) and the pipelined apply (bulk asynchronous copies of each edge's two
row-blocks into shared-memory slots, consumed by 1, 2 or 3 warps per edge).

Reference: the oracle's D_f^-1 S x (Sec. 6.1) or, with face blocks, the
inverted diagonal face blocks of the oracle's assembled S times S x; on the
small meshes every edge, on a mesh with many edges per CTA (every slot
refilled many times) sampled edges from the oracle's blocks of the two adjacent
elements. Tolerance 1e-12 relative (max norm), as for the FP64-vector split
apply: split-FP32 arithmetic carries about 48 significant bits.
"""
import math

import numpy as np
import pytest
import scipy.linalg as sla
import torch

from oracle.hdg import HDGProblem
from oracle.precond import face_block_inverse
from paper_2302_10917_gb300 import BASIS_DF64
from paper_2302_10917_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

B1 = (50.0 * math.cos(0.3), 50.0 * math.sin(0.3))
CASES = [
    # id, n, m, p, beta: P1 = m p + 1 odd (row-blocks on 8-byte boundaries) and even
    ("m8p3", 3, 8, 3, B1),
    ("m4p2", 4, 4, 2, (0.8, -0.3)),
    ("m1p1", 5, 1, 1, (1.0, -2.0)),
    ("m2p4", 3, 2, 4, (0.0, 0.0)),
]
SHAPES = [("default", 0, 0), ("epb1", 1, 0), ("bulk1", 0, 1), ("bulk2", 0, 2), ("bulk3", 0, 3)]


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def split(x):
    hi = x.astype(np.float32)
    lo = (x - hi.astype(np.float64)).astype(np.float32)
    return torch.from_numpy(np.stack([hi, lo], axis=1))


def joined(y):
    y = y.cpu().numpy().astype(np.float64)
    return y[:, 0] + y[:, 1]


def _set_shape(gpu, epb, bulk):
    from paper_2302_10917_gb300 import HDGError
    try:
        gpu.set_apply_shape(2, edges_per_block=epb, bulk_warps=bulk)
    except HDGError:
        pytest.skip(f"shape ({epb}, {bulk}) does not fit this problem")


@pytest.fixture(scope="module", params=CASES, ids=[c[0] for c in CASES])
def case(request):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2302_10917_gb300 import Problem
    cid, n, m, p, beta = request.param
    kappa = wl.random_kappa(2 * n * n, seed=7 * n + m + p)
    ora = HDGProblem(n, m, p, beta=beta, kappa=kappa)
    gpu = Problem(n, m, p, beta=beta, kappa=kappa)
    g = np.random.default_rng([wl.MASTER_SEED, 171, n, m, p])
    pts, _ = ora.quad_points()
    bpts, _ = ora.bnd_quad_points()
    f = g.standard_normal(pts.shape[:2])
    gD = g.standard_normal(bpts.shape[:2])
    S_el, g_ora, _ = ora.condense(f, gD)
    gpu.set_source(torch.from_numpy(f), torch.from_numpy(gD))
    gpu.condense(keep_factors=True, store_df64=True)
    yield dict(ora=ora, gpu=gpu, S_el=S_el, g=g_ora, rng=g, f=f, gD=gD, n=n, m=m, p=p, beta=beta, kappa=kappa)
    gpu.close()


@pytest.mark.parametrize("shape", SHAPES, ids=[s[0] for s in SHAPES])
def test_split_operator_matches_oracle_in_every_shape(case, shape):
    ora, gpu = case["ora"], case["gpu"]
    _, epb, bulk = shape
    _set_shape(gpu, epb, bulk)
    try:
        for trial in range(2):
            x = case["rng"].standard_normal(ora.mesh.N_tr) * (1.0 if trial == 0 else 1e3)
            z_ora = ora.apply_Dinv(ora.apply_S(case["S_el"], x))
            y = gpu.apply(split(x), precond=True, prec=49)
            assert y.shape == (ora.mesh.N_tr, 2) and y.dtype == torch.float32
            assert rel(joined(y), z_ora) < 1e-12, (shape, trial)
    finally:
        gpu.set_apply_shape(2)


def test_pipelined_apply_gives_the_same_bits(case):
    """With one consumer warp per edge the pipelined apply walks each row in the
    one-thread-per-row apply's summation order: the same bits as every
    edges-per-block shape. Two or three warps per edge add their parts in a fixed
    order of their own: reproducible, and within rounding of the default."""
    ora, gpu = case["ora"], case["gpu"]
    x = split(case["rng"].standard_normal(ora.mesh.N_tr))
    gpu.set_apply_shape(2)
    y0 = gpu.apply(x, precond=True, prec=49)
    try:
        for epb, bulk in ((1, 0), (0, 1)):
            _set_shape(gpu, epb, bulk)
            assert torch.equal(gpu.apply(x, precond=True, prec=49), y0), (epb, bulk)
        for bulk in (2, 3):
            _set_shape(gpu, 0, bulk)
            y = gpu.apply(x, precond=True, prec=49)
            assert torch.equal(gpu.apply(x, precond=True, prec=49), y), bulk
            assert rel(joined(y), joined(y0)) < 1e-13, bulk
    finally:
        gpu.set_apply_shape(2)


def test_solve_with_the_pipelined_apply(case):
    ora, gpu = case["ora"], case["gpu"]
    _set_shape(gpu, 0, 2)
    try:
        x_dir = np.linalg.solve(ora.assemble_S(case["S_el"]), case["g"])
        x, rep, st = gpu.solve(gpu.rhs(), tol=1e-12, restart=40, mode=2, orth=1, basis=BASIS_DF64)
        assert st == 0 and rep["converged"] == 1, rep
        assert rel(x.cpu().numpy(), x_dir) < 1e-8
        x2, _, _ = gpu.solve(gpu.rhs(), tol=1e-12, restart=40, mode=2, orth=1, basis=BASIS_DF64)
        assert torch.equal(x, x2)
    finally:
        gpu.set_apply_shape(2)


def test_pipelined_apply_with_face_blocks_and_transposed():
    """The face-block preconditioner (no per-face scale in the kernel) and the
    transposed operator of the adjoint (transposed blocks, transposed face blocks)."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2302_10917_gb300 import Problem
    n, m, p, beta = 3, 8, 3, B1
    kappa = wl.random_kappa(2 * n * n, seed=5)
    ora = HDGProblem(n, m, p, beta=beta, kappa=kappa)
    gpu = Problem(n, m, p, beta=beta, kappa=kappa)
    try:
        g = np.random.default_rng([wl.MASTER_SEED, 172])
        pts, _ = ora.quad_points()
        f = g.standard_normal(pts.shape[:2])
        S_el, _, _ = ora.condense(f, None)
        S = ora.assemble_S(S_el)
        P1 = ora.mesh.P1
        gpu.set_source(torch.from_numpy(f))
        gpu.condense(keep_factors=True, store_df64=True, precond="face_schur")
        x = g.standard_normal(S.shape[0])
        eoff = np.arange(S.shape[0] // P1 + 1) * P1
        ref = face_block_inverse(S, eoff) @ (S @ x)
        refT = face_block_inverse(S.T, eoff) @ (S.T @ x)
        for bulk in (1, 2, 3):
            _set_shape(gpu, 0, bulk)
            assert rel(joined(gpu.apply(split(x), precond=True, prec=49)), ref) < 1e-12, bulk
            gpu.transpose()
            try:
                assert rel(joined(gpu.apply(split(x), precond=True, prec=49)), refT) < 1e-12, bulk
            finally:
                gpu.transpose()
    finally:
        gpu.close()


def _elements_of_edge(n, f):
    if f < n * n:
        j, i = divmod(f, n)
        return [2 * (j * n + i), 2 * (j * n + i) + 1]
    if f < n * n + n * (n - 1):
        r = f - n * n
        j, i = 1 + r // n, r % n
        return [2 * ((j - 1) * n + i) + 1, 2 * (j * n + i)]
    r = f - n * n - n * (n - 1)
    j, i = r // (n - 1), 1 + r % (n - 1)
    return [2 * (j * n + i - 1), 2 * (j * n + i) + 1]


def test_many_edges_per_cta_sampled_edges():
    """n = 64, m = 8, p = 3 (12,160 interior edges: 80 per CTA, so every slot is
    refilled many times): sampled edges, the first and
    the last, against the oracle's blocks of their two elements and D_f^-1."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2302_10917_gb300 import Problem
    n, m, p, beta, kap = 64, 8, 3, B1, 1.0
    gpu = Problem(n, m, p, beta=beta, kappa=kap)
    try:
        gpu.set_source(wl.sin_sin_source(gpu.quad_points(), kap, beta))
        gpu.condense(keep_factors=False, store_df64=True)
        ora = HDGProblem(n, m, p, beta=beta, kappa=kap)
        msh = ora.mesh
        x = wl.random_vector(msh.N_tr, seed=17)
        edges = sorted(set(np.random.default_rng([wl.MASTER_SEED, 173]).choice(msh.n_int_edges, 5, replace=False)
                           .tolist() + [0, msh.n_int_edges - 1]))
        zero_bnd = np.zeros((msh.n_bnd_edges, msh.P1))
        blocks, dblk = {}, {}
        ref = {}
        for f in edges:
            out = np.zeros(msh.N_tr)
            Df = np.zeros((msh.P1, msh.P1))
            for e in _elements_of_edge(n, f):
                if e not in blocks:
                    blocks[e] = ora.condense_element(e)[0]
                    dblk[e] = ora.local_blocks(e)[3]
                ora.scatter(e, blocks[e] @ ora.element_trace(e, x, zero_bnd), out)
                for k, (kind, idx, flip) in enumerate(msh.element_edges(e)):
                    if kind == "int" and idx == f:
                        b = dblk[e][k * msh.P1:(k + 1) * msh.P1, k * msh.P1:(k + 1) * msh.P1]
                        Df += b[::-1, ::-1] if flip else b
            sl = slice(f * msh.P1, (f + 1) * msh.P1)
            ref[f] = -sla.cho_solve(sla.cho_factor(-Df), out[sl])
        scale = max(np.abs(v).max() for v in ref.values())
        for bulk in (0, 1, 2, 3):
            if bulk:
                _set_shape(gpu, 0, bulk)
            y = joined(gpu.apply(split(x), precond=True, prec=49))
            for f in edges:
                got = y[f * msh.P1:(f + 1) * msh.P1]
                assert np.abs(got - ref[f]).max() / scale < 1e-12, (bulk, f)
    finally:
        gpu.close()


def test_shape_errors_and_autotune_report():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2302_10917_gb300 import HDG_ERR_ARG, HDGError, Problem
    gpu = Problem(3, 4, 2, beta=(1.0, 0.5), kappa=1.0)
    try:
        gpu.set_source(wl.sin_sin_source(gpu.quad_points(), 1.0, (1.0, 0.5)))
        gpu.condense(keep_factors=True, store_df64=True, store_fp32=True)
        for args in ((0, 0, 1), (1, 0, 2), (2, 1, 1), (3, 0, 1), (4, 0, 0), (2, -1, 0), (2, 0, -1), (2, 100, 0), (2, 0, 4)):
            with pytest.raises(HDGError) as ei:
                gpu.set_apply_shape(*args)
            assert ei.value.status == HDG_ERR_ARG, args
        x = split(np.ones(gpu.info["N_tr"]))
        with pytest.raises(HDGError):
            gpu.apply(x, precond=False, prec=49)
        # the pipelined shape is a candidate with the split-FP32 basis only
        assert gpu.autotune(mode=2, restart=20)["apply_bulk"] == 0
        for mode in (0, 1, 2):
            basis = BASIS_DF64 if mode == 2 else 0
            rep = gpu.autotune(mode=mode, restart=20, basis=basis)
            if mode == 2:
                assert rep["apply_bulk_ms"] > 0 and rep["apply_bulk"] in (0, 1, 2, 3)
                if rep["apply_bulk"]:
                    assert rep["apply_edges_per_block"] == 0 and 64 <= rep["apply_threads"] <= 512
                    assert rep["apply_threads"] % 32 == 0
            else:
                assert rep["apply_bulk"] == 0 and rep["apply_bulk_ms"] == 0
            x_s, r, st = gpu.solve(gpu.rhs(), tol=1e-10, restart=20, mode=mode, basis=basis)
            assert st == 0 and r["converged"] == 1
    finally:
        gpu.close()
    lv = Problem(2, 1, 2, beta=(1.0, 0.0), kappa=1.0, levels=np.array([0, 1, 1, 0, 2, 0, 1, 1]))
    try:
        with pytest.raises(HDGError):
            lv.set_apply_shape(2, bulk_warps=1)
    finally:
        lv.close()
