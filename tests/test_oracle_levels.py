"""Pins of the level-mesh oracle (oracle/levels.py): macro-elements of uneven
refinement level with faces at the finer side's level (Sec. 4.2).

Each test targets a mistake the non-conforming coupling could plausibly
contain: a fine sub-edge integrated against the wrong coarse sub-triangle, a
face block at the wrong level or offset, a flipped face orientation, a wrong
prefix-sum offset in the ragged layouts.
"""
import numpy as np
import pytest

from oracle.basis import line_lagrange
from oracle.hdg import HDGProblem
from oracle.levels import LevelHDGProblem, band_levels
from oracle.problems import polynomial, random_polynomial
from oracle.quadrature import gauss_legendre

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def random_levels(n, seed, lo=0, hi=3):
    return np.random.default_rng([0x230210917, 61, n, seed]).integers(lo, hi + 1, size=2 * n * n)


def trace_mass_1d(m, p):
    """C0 P_p mass matrix on [0, 1] with m equal sub-intervals."""
    x, w = gauss_legendre(p + 2)
    psi = line_lagrange(p, x)
    G = np.zeros((m * p + 1, m * p + 1))
    for s in range(m):
        c = s * p + np.arange(p + 1)
        G[np.ix_(c, c)] += np.einsum("q,qa,qb->ab", w / m, psi, psi)
    return G


def prolongation_1d(mc, mf, p):
    """Values of the level-mc C0 P_p nodal basis at the level-mf nodes (mf a multiple of mc)."""
    Pi = np.zeros((mf * p + 1, mc * p + 1))
    for j in range(mf * p + 1):
        t = j / (mf * p)
        s = min(int(t * mc), mc - 1)                 # coarse sub-interval holding t
        loc = t * mc - s
        Pi[j, s * p + np.arange(p + 1)] = line_lagrange(p, np.array([loc]))[0]
    return Pi


@pytest.mark.parametrize("r,p", [(1, 2), (0, 3), (2, 1)])
def test_uniform_levels_reduce_to_the_uniform_oracle(r, p):
    n, beta, kap = 2, (0.8, -0.3), 0.6
    lv = LevelHDGProblem(n, np.full(2 * n * n, r), p, beta=beta, kappa=kap)
    un = HDGProblem(n, 2 ** r, p, beta=beta, kappa=kap)
    rng = np.random.default_rng(5)
    pts, _ = un.quad_points()
    bpts, _ = un.bnd_quad_points()
    f = rng.standard_normal(pts.shape[:2])
    gD = rng.standard_normal(bpts.shape[:2])
    S1, g1, _ = lv.condense(f.reshape(-1), gD.reshape(-1))
    S0, g0, gh0 = un.condense(f, gD)
    assert lv.N_tr == un.mesh.N_tr
    assert max(np.abs(S1[e] - S0[e]).max() for e in range(un.mesh.N)) < 1e-13 * np.abs(S0).max()
    assert np.abs(g1 - g0).max() < 1e-12 * np.abs(g0).max()
    x = np.linalg.solve(un.assemble_S(S0), g0)
    u1, q1 = lv.recover(x, f.reshape(-1), lv.dirichlet_trace(gD.reshape(-1)))
    u0, q0 = un.recover(x, f, gh0)
    assert np.abs(u1 - u0.reshape(-1)).max() < 1e-12 * np.abs(u0).max()
    assert np.abs(q1 - q0.reshape(-1)).max() < 1e-12 * np.abs(q0).max()


@pytest.mark.parametrize("n,p,levels", [
    (2, 1, "random"), (2, 2, "random"), (2, 3, "random"), (3, 2, "band"), (2, 2, "jump3")])
def test_polynomial_exactness_on_nonconforming_meshes(n, p, levels):
    """u in P_p globally: u, q = -grad u and u^ = u|_F are reproduced to roundoff,
    through faces whose two sides differ by up to three levels."""
    if levels == "random":
        lev = random_levels(n, seed=p)
    elif levels == "band":
        lev = band_levels(n, edges=(0.4, 0.6, 0.8), base=0)
    else:
        lev = np.zeros(2 * n * n, dtype=int)
        lev[::3] = 3
    kap, beta = 0.7, (0.9, -0.4)
    pr = LevelHDGProblem(n, lev, p, beta=beta, kappa=kap)
    assert any(pr.flevel[f] != min(lev[e] for e in range(pr.N)) for f in range(pr.n_int))
    u, gr, f = polynomial(random_polynomial(p, seed=21 + p), kap, beta)
    pts, _ = pr.quad_points()
    bpts, _ = pr.bnd_quad_points()
    fq = f(pts[:, 0], pts[:, 1])
    gq = u(bpts[:, 0], bpts[:, 1])
    S_el, g, gh = pr.condense(fq, gq)
    x = np.linalg.solve(pr.assemble_S(S_el), g)
    uu, qq = pr.recover(x, fq, gh)
    eu, eq = pr.l2_errors(uu, qq, u, gr)
    assert eu < 1e-12 and eq < 1e-11
    for e in range(pr.N):
        X = pr.lattice_points(e)
        assert np.abs(uu[pr.uoff[e]:pr.uoff[e + 1]] - u(X[:, 0], X[:, 1])).max() < 1e-12
    # the trace at the nodes of every interior face, along the edge's orientation
    for e in range(pr.N):
        v = pr.skel.vertices(e)
        for k, (kind, idx, flip, R) in enumerate(pr.faces(e)):
            if kind != "int":
                continue
            a0, a1 = v[(k + 1) % 3], v[(k + 2) % 3]
            if flip:
                a0, a1 = a1, a0
            t = np.arange(2 ** R * p + 1) / (2 ** R * p)
            P = a0[None, :] + np.outer(t, a1 - a0)
            assert np.abs(x[pr.eoff[idx]:pr.eoff[idx + 1]] - u(P[:, 0], P[:, 1])).max() < 1e-12


def test_unreduced_equals_condensed_with_levels():
    n, p = 2, 2
    pr = LevelHDGProblem(n, random_levels(n, seed=9), p, beta=(0.5, 0.9), kappa=np.linspace(0.3, 1.2, 8))
    rng = np.random.default_rng(3)
    fq = rng.standard_normal(pr.qoff[-1])
    gq = rng.standard_normal(pr.boff[-1])
    S_el, g, gh = pr.condense(fq, gq)
    x = np.linalg.solve(pr.assemble_S(S_el), g)
    u, q = pr.recover(x, fq, gh)
    x2, u2, q2 = pr.solve_unreduced(fq, gq)
    assert np.abs(x - x2).max() < 1e-10 * np.abs(x2).max()
    assert np.abs(u - u2).max() < 1e-10 * np.abs(u2).max()
    assert np.abs(q - q2).max() < 1e-10 * np.abs(q2).max()
    # element-wise apply against the assembled operator
    v = rng.standard_normal(pr.N_tr)
    assert np.abs(pr.apply_S(S_el, v) - pr.assemble_S(S_el) @ v).max() < 1e-12 * np.abs(pr.assemble_S(S_el)).max()


def test_coarse_side_face_coupling_is_the_fine_mass_projection():
    """On a face finer than its element, <psi_fine, phi> = <psi_coarse, phi> T with
    T = G_c^-1 Pi^T G_f (the coarse basis restricted to the edge lies in the
    coarse trace space, Pi its fine nodal values); G is L times the fine 1D mass."""
    n, p = 2, 2
    lev = np.zeros(8, dtype=int)
    lev[1] = 2                       # element 1 fine: faces of its neighbours refined to level 2
    pr = LevelHDGProblem(n, lev, p)
    checked = 0
    for e in range(pr.N):
        if lev[e] != 0:
            continue
        em = pr.element_matrices(e)
        emc = pr.sub[0].element_matrices(e)     # the same element with faces at its own level
        for k, (_, _, _, R) in enumerate(pr.faces(e)):
            o0, o1 = em["offs"][k], em["offs"][k + 1]
            L = em["lengths"][k]
            assert np.abs(em["G"][o0:o1, o0:o1] - L * trace_mass_1d(2 ** R, p)).max() < 1e-15
            if R == 0:
                continue
            Gc = trace_mass_1d(1, p)
            Gf = trace_mass_1d(2 ** R, p)
            T = np.linalg.solve(Gc, prolongation_1d(1, 2 ** R, p).T @ Gf)
            Fc = emc["F"][:, k * (p + 1):(k + 1) * (p + 1)]
            assert np.abs(em["F"][:, o0:o1] - Fc @ T).max() < 1e-14
            checked += 1
    assert checked == 2           # the diagonal and the horizontal neighbour of element 1


def test_face_D_is_minus_tau_sum_times_fine_trace_mass():
    n, p = 2, 2
    pr = LevelHDGProblem(n, random_levels(n, seed=4), p, beta=(0.9, 0.3), kappa=np.linspace(0.5, 2.0, 8))
    Df = pr.face_D()
    for f in range(pr.n_int):
        sides = [e for e in range(pr.N) for kind, idx, _, _ in pr.faces(e) if kind == "int" and idx == f]
        assert len(sides) == 2
        e0 = sides[0]
        k0 = [k for k, fc in enumerate(pr.faces(e0)) if fc[0] == "int" and fc[1] == f][0]
        L = pr.element_matrices(e0)["lengths"][k0]
        ref = -(pr.tau[sides[0]] + pr.tau[sides[1]]) * L * trace_mass_1d(2 ** pr.flevel[f], p)
        assert np.abs(Df[f] - ref).max() < 1e-13 * np.abs(ref).max()


def test_pure_diffusion_operator_symmetric_negative_definite_with_levels():
    pr = LevelHDGProblem(2, random_levels(2, seed=7), 2, kappa=0.9)
    S_el, _, _ = pr.condense()
    S = pr.assemble_S(S_el)
    assert np.abs(S - S.T).max() < 1e-12 * np.abs(S).max()
    assert np.linalg.eigvalsh(0.5 * (S + S.T)).max() < 0.0


def test_local_conservation_with_levels():
    """w = 1 in Eq. (pde): <flux^ . n, 1>_dK = (f, 1)_K on every macro-element,
    coarse ones with refined faces included."""
    pr = LevelHDGProblem(2, random_levels(2, seed=2), 2, beta=(0.8, -0.3), kappa=0.5)
    rng = np.random.default_rng(8)
    pts, wts = pr.quad_points()
    fq = rng.standard_normal(pts.shape[0])
    S_el, g, gh = pr.condense(fq, None)
    x = np.linalg.solve(pr.assemble_S(S_el), g)
    u, q = pr.recover(x, fq, gh)
    for e in range(pr.N):
        em = pr.element_matrices(e)
        kap, tau = pr.kappa[e], pr.tau[e]
        ue = u[pr.uoff[e]:pr.uoff[e + 1]]
        qe = q[2 * pr.uoff[e]:2 * pr.uoff[e + 1]].reshape(2, -1)
        one = np.ones(ue.size)
        xe = pr.element_trace(e, x, gh)
        flux = (one @ (kap * (em["Ex"] @ qe[0] + em["Ey"] @ qe[1]) + tau * em["E"] @ ue)
                + one @ ((em["F"] * em["bn"][None, :] - tau * em["F"]) @ xe))
        sl = slice(pr.qoff[e], pr.qoff[e + 1])
        assert abs(flux - np.dot(wts[sl], fq[sl])) < 1e-12 * max(1.0, abs(flux))


def test_ragged_offsets():
    n, p = 3, 2
    lev = random_levels(n, seed=11)
    pr = LevelHDGProblem(n, lev, p)
    m = 2 ** lev
    assert np.array_equal(np.diff(pr.qoff), m * m * (p + 2) ** 2)
    assert np.array_equal(np.diff(pr.uoff), (m * p + 1) * (m * p + 2) // 2)
    assert np.array_equal(np.diff(pr.eoff), 2 ** pr.flevel * p + 1)
    assert sum(pr.n_t(e) for e in range(pr.N)) == 2 * (pr.eoff[-1]) + (pr.goff[-1])
    for e in range(pr.N):
        for kind, idx, _, R in pr.faces(e):
            assert R >= lev[e]
            if kind == "bnd":
                assert R == lev[e]


def test_band_levels_of_the_many_source_workload():
    """n = 128, r = 4 for centroid x >= 0.9, 3 in [0.8, 0.9), 2 in [0.7, 0.8), 1 elsewhere."""
    lev = band_levels(128)
    assert [int((lev == r).sum()) for r in (1, 2, 3, 4)] == [22912, 3328, 3200, 3328]


def test_band_levels_of_the_workload_generator_agree():
    from paper_2302_10917_gb300 import workloads as wl
    for n in (3, 10, 128):
        assert np.array_equal(wl.band_levels(n), band_levels(n))
    assert np.array_equal(wl.band_levels(5, (0.4, 0.6, 0.8), 0), band_levels(5, (0.4, 0.6, 0.8), 0))


def test_element_condensation_and_recovery_equal_the_global_route():
    pr = LevelHDGProblem(2, random_levels(2, seed=12), 2, beta=(0.7, 0.2), kappa=0.6)
    rng = np.random.default_rng(17)
    fq = rng.standard_normal(pr.qoff[-1])
    gq = rng.standard_normal(pr.boff[-1])
    S_el, g, gh = pr.condense(fq, gq)
    x = np.linalg.solve(pr.assemble_S(S_el), g)
    u, q = pr.recover(x, fq, gh)
    for e in (0, 3, 7):
        ue, qe = pr.recover_element(e, x, fq, gh)
        assert np.abs(ue - u[pr.uoff[e]:pr.uoff[e + 1]]).max() < 1e-13 * np.abs(u).max()
        assert np.abs(qe.reshape(-1) - q[2 * pr.uoff[e]:2 * pr.uoff[e + 1]]).max() < 1e-13 * np.abs(q).max()


@pytest.mark.parametrize("p", [1, 2])
def test_convergence_rate_on_a_nonconforming_band_mesh(p):
    """u = sin(pi x) sin(pi y) on band meshes (level 0 left of x = 0.5, level 1 right of it,
    non-conforming faces along the band edge) refined n = 2, 4, 8: the L2 errors of u and
    q = -grad u fall at order p + 1 (Sec. 4.1's rate, here through non-conforming faces)."""
    import math
    from oracle.problems import sin_sin
    errs = []
    for n in (2, 4, 8):
        pr = LevelHDGProblem(n, band_levels(n, edges=(0.5,), base=0), p, beta=(1.0, 1.0), kappa=1.0)
        u, gr, f = sin_sin(1.0, (1.0, 1.0))
        pts, _ = pr.quad_points()
        fq = f(pts[:, 0], pts[:, 1])
        S_el, g, gh = pr.condense(fq, None)
        x = np.linalg.solve(pr.assemble_S(S_el), g)
        uu, qq = pr.recover(x, fq, gh)
        errs.append(pr.l2_errors(uu, qq, u, gr))
    for k in (0, 1):
        assert math.log2(errs[1][k] / errs[2][k]) > p + 1 - 0.15, (k, errs)
