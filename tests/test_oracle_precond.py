"""Pins of the oracle's face-block preconditioner (oracle/precond.py), CPU only.

P = blockdiag(S_ff)^-1 with S_ff the diagonal face blocks of the condensed
operator S (Eq. global_problem). Facts that hold whatever S is, and facts of
the problem class, each chosen so that a plausible mistake fails one:
  * P is block diagonal over the faces and the diagonal face blocks of P S
    are identities, which together fix P (a transposed block or a missing
    inverse fails the second on an advective S, a face range off by one the
    first);
  * with a single interior face P S = I, and GMRES converges in one step;
  * at beta = 0, S is symmetric negative definite, so every S_ff is (a
    principal submatrix) and so is its inverse;
  * the face blocks of S^T are the S_ff^T (the adjoint's preconditioner);
  * preconditioned GMRES reaches the direct solution, uniform and level meshes.
"""
import numpy as np
import pytest

from oracle.hdg import HDGProblem
from oracle.levels import LevelHDGProblem
from oracle.precond import apply_face_blocks, face_block_inverse, face_blocks
from oracle.solver import gmres


def _uniform(n, m, p, beta, kappa=1.0, seed=3):
    pr = HDGProblem(n, m, p, beta=beta, kappa=kappa)
    pts, _ = pr.quad_points()
    f = np.random.default_rng(seed).standard_normal(pts.shape[:2])
    S_el, g, _ = pr.condense(f, None)
    eoff = np.arange(pr.mesh.n_int_edges + 1) * pr.mesh.P1
    return pr, pr.assemble_S(S_el), g, eoff


def _diag_blocks_identity(M, eoff):
    return max(np.abs(B - np.eye(B.shape[0])).max() for B in face_blocks(M, eoff))


def _off_block_max(P, eoff):
    """Largest entry of P outside its diagonal face blocks. Block-diagonal P with
    (P S)_ff = I for every face is exactly blockdiag(S_ff)^-1, so the two checks
    together pin P."""
    mask = np.ones(P.shape, dtype=bool)
    for f in range(len(eoff) - 1):
        mask[eoff[f]:eoff[f + 1], eoff[f]:eoff[f + 1]] = False
    return np.abs(P[mask]).max() if mask.any() else 0.0


@pytest.mark.parametrize("n,m,p,beta", [(3, 2, 2, (1.5, -0.5)), (2, 4, 3, (30.0, 10.0)), (3, 1, 2, (0.7, 0.2))])
def test_preconditioned_operator_has_identity_face_blocks(n, m, p, beta):
    _, S, _, eoff = _uniform(n, m, p, beta)
    P = face_block_inverse(S, eoff)
    assert _diag_blocks_identity(P @ S, eoff) < 1e-12
    assert _off_block_max(P, eoff) == 0.0
    # the off-diagonal face couplings survive (P is not the inverse of S)
    assert np.abs(P @ S - np.eye(S.shape[0])).max() > 1e-3
    # advection makes the blocks non-symmetric, so a transposed block would not pass
    assert max(np.abs(B - B.T).max() / np.abs(B).max() for B in face_blocks(S, eoff)) > 1e-3
    x = np.random.default_rng(5).standard_normal(S.shape[0])
    assert np.abs(apply_face_blocks(S, eoff, S @ x) - P @ (S @ x)).max() < 1e-12 * np.abs(P @ (S @ x)).max()


def test_single_interior_face_gives_the_identity():
    pr, S, g, eoff = _uniform(1, 4, 2, (0.8, 0.3))
    assert pr.mesh.n_int_edges == 1
    P = face_block_inverse(S, eoff)
    assert np.abs(P @ S - np.eye(S.shape[0])).max() < 1e-12
    x, its, rel, ok = gmres(lambda v: S @ v, lambda v: apply_face_blocks(S, eoff, v), g, tol=1e-12, restart=5)
    assert ok and its == 1


def test_pure_diffusion_blocks_symmetric_negative_definite():
    _, S, _, eoff = _uniform(3, 2, 3, (0.0, 0.0))
    for B in face_blocks(S, eoff):
        assert np.abs(B - B.T).max() < 1e-13 * np.abs(B).max()
        assert np.linalg.eigvalsh(B).max() < 0
        Bi = np.linalg.inv(B)
        assert np.abs(Bi - Bi.T).max() < 1e-12 * np.abs(Bi).max()


def test_transposed_operator_has_transposed_blocks():
    _, S, _, eoff = _uniform(3, 2, 2, (1.0, -2.0))
    for B, Bt in zip(face_blocks(S, eoff), face_blocks(S.T, eoff)):
        assert np.array_equal(Bt, B.T)
    P, Pt = face_block_inverse(S, eoff), face_block_inverse(S.T, eoff)
    assert np.abs(Pt - P.T).max() < 1e-12 * np.abs(P).max()


@pytest.mark.parametrize("n,m,p,kappa,beta", [(6, 2, 2, 1.0, (1.0, 0.5)), (6, 2, 2, 1e-2, (1.0, 0.0)),
                                              (5, 4, 2, 1.0, (0.3, 0.2))])
def test_gmres_with_face_blocks_reaches_the_direct_solution(n, m, p, kappa, beta):
    """Also a regression record for these seeded problems: fewer GMRES(20)
    iterations than with D^-1 (129 vs 208, 69 vs 90, 125 vs 269 when written)."""
    pr, S, g, eoff = _uniform(n, m, p, beta, kappa=kappa, seed=1)
    x_dir = np.linalg.solve(S, g)
    x, its_f, rel, ok = gmres(lambda v: S @ v, lambda v: apply_face_blocks(S, eoff, v), g, tol=1e-10, restart=20)
    assert ok and rel <= 1e-10
    assert np.abs(x - x_dir).max() < 1e-7 * np.abs(x_dir).max()
    Df = pr.face_D()
    _, its_d, _, ok_d = gmres(lambda v: S @ v, lambda v: pr.apply_Dinv(v, Df), g, tol=1e-10, restart=20)
    assert ok_d and its_f < its_d


def test_level_mesh_face_blocks():
    """Ragged faces (sizes 2^R_f p + 1 by the finer side's level)."""
    lev = np.array([0, 2, 1, 1, 0, 2, 2, 0, 1, 0, 2, 1, 1, 0, 0, 2, 1, 2])
    pr = LevelHDGProblem(3, lev, 2, beta=(1.0, 0.4), kappa=0.5)
    f = np.random.default_rng(9).standard_normal(pr.qoff[-1])
    S_el, g, _ = pr.condense(f, None)
    S = pr.assemble_S(S_el)
    sizes = np.diff(pr.eoff)
    assert len(set(sizes.tolist())) > 1
    P = face_block_inverse(S, pr.eoff)
    assert _diag_blocks_identity(P @ S, pr.eoff) < 1e-11
    assert _off_block_max(P, pr.eoff) == 0.0
    x, its, rel, ok = gmres(lambda v: S @ v, lambda v: apply_face_blocks(S, pr.eoff, v), g, tol=1e-11, restart=30)
    assert ok
    x_dir = np.linalg.solve(S, g)
    assert np.abs(x - x_dir).max() < 1e-8 * np.abs(x_dir).max()
