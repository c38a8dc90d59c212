"""Pins of the CPU oracle against facts the paper and the mathematics fix.

Each test targets a mistake the oracle could plausibly contain (a wrong
quadrature weight, a dropped boundary term, a flipped normal or sign, a
mis-numbered trace dof) and would fail if that mistake were made.
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import counting
from oracle.basis import line_lagrange, tri_lagrange
from oracle.hdg import HDGProblem
from oracle.mesh import StructuredMesh
from oracle.problems import polynomial, random_polynomial, sin_sin, tanh_layer
from oracle.quadrature import gauss_legendre, triangle_rule
from oracle.solver import gmres

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ------------------------------------------------------------------ quadrature
@pytest.mark.parametrize("n", [1, 2, 3, 5, 8])
def test_gauss_legendre_exact_for_monomials(n):
    x, w = gauss_legendre(n)
    assert np.all(np.diff(x) > 0) and x[0] > 0 and x[-1] < 1
    for k in range(2 * n):
        assert abs(np.dot(w, x ** k) - 1.0 / (k + 1)) < 1e-15
    # degree 2n is not integrated exactly (the rule is Gauss, not more)
    assert abs(np.dot(w, x ** (2 * n)) - 1.0 / (2 * n + 1)) > 1e-12


@pytest.mark.parametrize("ng", [1, 3, 5])
def test_triangle_rule_closed_form(ng):
    xi, eta, w = triangle_rule(ng)
    for a in range(2 * ng - 1):
        for b in range(2 * ng - 1 - a):
            exact = math.factorial(a) * math.factorial(b) / math.factorial(a + b + 2)
            assert abs(np.sum(w * xi ** a * eta ** b) - exact) < 1e-15


# ------------------------------------------------------------------- the bases
@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_triangle_lagrange_kronecker_and_unity(p):
    alphas = [(p - b - c, b, c) for c in range(p + 1) for b in range(p + 1 - c)]
    lam = np.array(alphas, dtype=float) / p
    dlam = np.array([[-1.0, -1.0], [1.0, 0.0], [0.0, 1.0]])
    phi, grad = tri_lagrange(alphas, p, lam, dlam)
    assert np.allclose(phi, np.eye(len(alphas)), atol=1e-14)
    rng = np.random.default_rng(3)
    r = rng.dirichlet([1, 1, 1], size=20)
    phi, grad = tri_lagrange(alphas, p, r, dlam)
    assert np.allclose(phi.sum(axis=1), 1.0, atol=1e-14)
    assert np.allclose(grad.sum(axis=1), 0.0, atol=1e-12)
    # the basis reproduces x = lambda_1 exactly (its gradient is (1, 0))
    xs = lam[:, 1]
    assert np.allclose(phi @ xs, r[:, 1], atol=1e-14)
    assert np.allclose(np.einsum("qbk,b->qk", grad, xs), [1.0, 0.0], atol=1e-12)


def test_line_lagrange_nodes():
    for p in (1, 2, 3):
        assert np.allclose(line_lagrange(p, np.arange(p + 1) / p), np.eye(p + 1), atol=1e-15)


# ------------------------------------------------------------- mesh and counts
def test_mesh_counts_and_workload_sizes():
    for (n, m, p, N_tr) in [(4, 2, 2, 200), (128, 8, 3, 1222400), (256, 8, 3, 4902400),
                            (256, 4, 2, 1764864)]:
        msh = StructuredMesh(n, m, p)
        assert msh.N == 2 * n * n
        assert msh.Q == math.comb(m * p + 2, 2)
        assert msh.n_int_edges == counting.interior_faces(2, n)
        assert msh.N_tr == N_tr


def test_trace_numbering_is_a_bijection_and_two_sided():
    msh = StructuredMesh(3, 2, 2)
    seen = np.zeros(msh.N_tr, dtype=int)
    bseen = np.zeros(msh.n_bnd_edges * msh.P1, dtype=int)
    for e in range(msh.N):
        for kind, idx in msh.element_dof_map(e):
            (seen if kind == "int" else bseen)[idx] += 1
    assert np.all(seen == 2)          # every interior dof has two element sides
    assert np.all(bseen == 1)


def test_edge_orientation_matches_geometry():
    """The dof map's flip flags agree with where the dofs physically are."""
    msh = StructuredMesh(3, 2, 1)
    ref = msh.lattice_ref()
    P = msh.P
    edge_nodes = {0: [msh.node(P - t, t) for t in range(P + 1)],
                  1: [msh.node(0, P - t) for t in range(P + 1)],
                  2: [msh.node(t, 0) for t in range(P + 1)]}
    pos = {}
    for e in range(msh.N):
        v = msh.vertices(e)
        X = v[0] + np.outer(ref[:, 0], v[1] - v[0]) + np.outer(ref[:, 1], v[2] - v[0])
        dmap = msh.element_dof_map(e)
        for k in range(3):
            for s_loc in range(P + 1):
                kind, idx = dmap[k * (P + 1) + s_loc]
                xk = X[edge_nodes[k][s_loc]]
                key = (kind, idx)
                if key in pos:
                    assert np.allclose(pos[key], xk, atol=1e-14)
                pos[key] = xk


@pytest.mark.parametrize("entry", json.load(open(os.path.join(GOLDEN, "paper_counts.json")))
                         ["table9_dof_global"]["rows"])
def test_table9_global_dofs(entry):
    d, p, m = 3, 2, entry["m"]
    n = round((entry["N_elm"] / (math.factorial(d) * m ** d)) ** (1.0 / d))
    assert counting.n_macro(d, n) * m ** d == entry["N_elm"]
    assert counting.dof_global(d, n, m, p) == entry["dof_global"]


@pytest.mark.parametrize("entry", json.load(open(os.path.join(GOLDEN, "paper_counts.json")))
                         ["table7_dof_local"]["rows"])
def test_table7_local_dofs(entry):
    d, p, m = 3, 2, entry["m"]
    n_macro = entry["N_elm"] // m ** d
    assert n_macro * (d + 1) * counting.q_nodes(d, m, p) == entry["dof_local"]


def test_sec43_local_dofs():
    g = json.load(open(os.path.join(GOLDEN, "paper_counts.json")))["sec43_dof_local"]
    n_macro = g["N_elm"] // g["m"] ** 3
    assert n_macro * 4 * counting.q_nodes(3, g["m"], g["p"]) == g["dof_local"]


# ------------------------------------------------------------ element matrices
def _rand_problem(n=2, m=2, p=2, beta=(0.8, -0.3), seed=0):
    rng = np.random.default_rng(seed)
    kap = rng.uniform(0.5, 2.0, size=2 * n * n)
    return HDGProblem(n, m, p, beta=beta, kappa=kap), rng


@pytest.mark.parametrize("m,p", [(1, 1), (2, 2), (4, 1), (2, 3)])
def test_mass_and_integration_by_parts(m, p):
    pr = HDGProblem(2, m, p)
    for e in (0, 3):
        em = pr.element_matrices(e)
        area = 0.5 / pr.n ** 2
        assert abs(em["M"].sum() - area) < 1e-15
        # (phi_j, d phi_i) + (d phi_j, phi_i) = <phi_i phi_j n>, i.e. Dx + Dx^T = Ex
        assert np.abs(em["Dx"] + em["Dx"].T - em["Ex"]).max() < 1e-13
        assert np.abs(em["Dy"] + em["Dy"].T - em["Ey"]).max() < 1e-13
        # perimeter = sum of the boundary mass, with sum of the lengths
        assert abs(em["E"].sum() - em["lengths"].sum()) < 1e-14
        # the divergence theorem on a closed boundary: sum over dK of n |F| = 0
        assert np.abs(em["Ex"].sum()) < 1e-14 and np.abs(em["Ey"].sum()) < 1e-14


def test_trace_mass_matches_1d_formula():
    for p, loc in [(1, np.array([[2.0, 1.0], [1.0, 2.0]]) / 6.0),
                   (2, np.array([[4.0, 2.0, -1.0], [2.0, 16.0, 2.0], [-1.0, 2.0, 4.0]]) / 30.0)]:
        m = 3
        pr = HDGProblem(2, m, p)
        em = pr.element_matrices(1)
        P1 = m * p + 1
        for k in range(3):
            h = em["lengths"][k] / m
            ref = np.zeros((P1, P1))
            for s in range(m):
                c = s * p + np.arange(p + 1)
                ref[np.ix_(c, c)] += h * loc
            assert np.abs(em["G"][k * P1:(k + 1) * P1, k * P1:(k + 1) * P1] - ref).max() < 1e-15


# ------------------------------------------------------------ discrete problem
@pytest.mark.parametrize("n,m,p", [(2, 1, 1), (2, 2, 2), (1, 4, 2), (2, 2, 3), (1, 8, 1)])
def test_polynomial_exactness(n, m, p):
    """u in P_p globally => the discrete solution equals u, -grad u, u|_E (roundoff)."""
    kap, beta = 0.7, (0.9, -0.4)
    pr = HDGProblem(n, m, p, beta=beta, kappa=kap)
    u, gr, f = polynomial(random_polynomial(p, seed=11 + p), kap, beta)
    pts, _ = pr.quad_points()
    bpts, _ = pr.bnd_quad_points()
    fq = f(pts[..., 0], pts[..., 1])
    gq = u(bpts[..., 0], bpts[..., 1])
    S_el, g, gh = pr.condense(fq, gq)
    x = np.linalg.solve(pr.assemble_S(S_el), g)
    uu, qq = pr.recover(x, fq, gh)
    eu, eq = pr.l2_errors(uu, qq, u, gr)
    assert eu < 1e-12 and eq < 1e-11
    # the trace equals u at its nodes
    msh = pr.mesh
    for e in range(msh.N):
        v = msh.vertices(e)
        ref = msh.lattice_ref()
        X = v[0] + np.outer(ref[:, 0], v[1] - v[0]) + np.outer(ref[:, 1], v[2] - v[0])
        assert np.abs(uu[e] - u(X[:, 0], X[:, 1])).max() < 1e-12


def test_convergence_rate_sin_sin():
    """Sec. 4.1: L2 error of u converges at order p + 1 (m = 2)."""
    kap, beta = 1.0, (1.0, 1.0)
    u, gr, f = sin_sin(kap, beta)
    for p in (1, 2):
        errs = []
        for n in (2, 4, 8):
            pr = HDGProblem(n, 2, p, beta=beta, kappa=kap)
            pts, _ = pr.quad_points()
            fq = f(pts[..., 0], pts[..., 1])
            S_el, g, gh = pr.condense(fq, None)
            x = np.linalg.solve(pr.assemble_S(S_el), g)
            uu, qq = pr.recover(x, fq, gh)
            errs.append(pr.l2_errors(uu, qq, u, gr))
        errs = np.array(errs)
        rate_u = np.log2(errs[-2, 0] / errs[-1, 0])
        rate_q = np.log2(errs[-2, 1] / errs[-1, 1])
        assert rate_u > p + 1 - 0.15
        assert rate_q > p + 1 - 0.5


def test_convergence_rate_tanh_layer():
    """Sec. 4.1 benchmark Eq. (C24a), kappa = 0.4, a = (1, 1), m = 2, p = 1."""
    kap, beta = 0.4, (1.0, 1.0)
    u, gr, f = tanh_layer(kap, beta)
    errs = []
    for n in (2, 4, 8):
        pr = HDGProblem(n, 2, 1, beta=beta, kappa=kap)
        pts, _ = pr.quad_points()
        bpts, _ = pr.bnd_quad_points()
        fq = f(pts[..., 0], pts[..., 1])
        gq = u(bpts[..., 0], bpts[..., 1])
        S_el, g, gh = pr.condense(fq, gq)
        x = np.linalg.solve(pr.assemble_S(S_el), g)
        uu, qq = pr.recover(x, fq, gh)
        errs.append(pr.l2_errors(uu, qq, u, gr)[0])
    assert np.log2(errs[-2] / errs[-1]) > 2 - 0.2


def test_assembled_equals_four_step_apply():
    pr, rng = _rand_problem()
    S_el, _, _ = pr.condense()
    S = pr.assemble_S(S_el)
    for col in range(0, pr.mesh.N_tr, 7):
        x = np.zeros(pr.mesh.N_tr)
        x[col] = 1.0
        assert np.abs(S[:, col] - pr.apply_four_step(x)).max() < 1e-13 * np.abs(S).max()
    x = rng.standard_normal(pr.mesh.N_tr)
    assert np.abs(pr.apply_S(S_el, x) - S @ x).max() < 1e-13 * np.abs(S @ x).max()
    Df = pr.face_D()
    z = pr.apply_Dinv(S @ x, Df)
    assert np.abs(z - pr.apply_four_step(x, precondition=True)).max() < 1e-12 * np.abs(z).max()


def test_face_D_is_minus_tau_sum_times_trace_mass():
    """D_f = -(tau+ + tau-) G_F on interior faces (beta.n cancels across the face)."""
    pr, _ = _rand_problem(beta=(2.0, 1.0))
    Df = pr.face_D()
    msh = pr.mesh
    tsum = np.zeros(msh.n_int_edges)
    for e in range(msh.N):
        for kind, idx, flip in msh.element_edges(e):
            if kind == "int":
                tsum[idx] += pr.tau[e]
    for f in range(msh.n_int_edges):
        ev = np.linalg.eigvalsh(-Df[f])
        assert ev.min() > 0
        assert np.allclose(Df[f], Df[f].T, atol=1e-15)
    # the sum of all entries of G_F is the edge length
    h = 1.0 / msh.n
    for f in range(msh.n_int_edges):
        L = h * math.sqrt(2.0) if f < msh.n * msh.n else h
        assert abs(-Df[f].sum() / tsum[f] - L) < 1e-13


def test_unreduced_equals_condensed():
    pr, rng = _rand_problem()
    pts, _ = pr.quad_points()
    bpts, _ = pr.bnd_quad_points()
    fq = rng.standard_normal(pts.shape[:2])
    gq = rng.standard_normal(bpts.shape[:2])
    S_el, g, gh = pr.condense(fq, gq)
    x = np.linalg.solve(pr.assemble_S(S_el), g)
    u, q = pr.recover(x, fq, gh)
    vt, ut, qt = pr.solve_unreduced(fq, gq)
    assert np.abs(vt - x).max() < 1e-12 * np.abs(x).max()
    assert np.abs(ut - u).max() < 1e-12 * np.abs(u).max()
    assert np.abs(qt - q).max() < 1e-11 * np.abs(q).max()


def test_gmres_equals_direct_solve():
    pr, rng = _rand_problem(n=3)
    pts, _ = pr.quad_points()
    fq = rng.standard_normal(pts.shape[:2])
    S_el, g, _ = pr.condense(fq, None)
    S = pr.assemble_S(S_el)
    Df = pr.face_D()
    xd = np.linalg.solve(S, g)
    x, it, rel, ok = gmres(lambda v: S @ v, lambda v: pr.apply_Dinv(v, Df), g,
                           tol=1e-13, restart=15)
    assert ok and rel <= 1e-13
    assert np.abs(x - xd).max() < 1e-10 * np.abs(xd).max()
    # non-convergence is reported, not hidden
    x, it, rel, ok = gmres(lambda v: S @ v, lambda v: pr.apply_Dinv(v, Df), g,
                           tol=1e-13, restart=5, maxit=5)
    assert not ok and it == 5 and rel > 1e-13


def test_pure_diffusion_trace_operator_symmetric_negative_definite():
    pr, _ = _rand_problem(n=3, beta=(0.0, 0.0))
    S_el, _, _ = pr.condense()
    S = pr.assemble_S(S_el)
    assert np.abs(S - S.T).max() < 1e-13 * np.abs(S).max()
    assert np.linalg.eigvalsh(S).max() < 0


def test_advection_breaks_symmetry():
    pr, _ = _rand_problem(n=2, beta=(1.5, 0.5))
    S_el, _, _ = pr.condense()
    S = pr.assemble_S(S_el)
    assert np.abs(S - S.T).max() > 1e-3 * np.abs(S).max()


def test_local_conservation():
    """With w = 1 in Eq. (pde): <flux^ . n, 1>_dK = (f, 1)_K on every macro-element."""
    pr, rng = _rand_problem()
    pts, wts = pr.quad_points()
    fq = rng.standard_normal(pts.shape[:2])
    S_el, g, gh = pr.condense(fq, None)
    x = np.linalg.solve(pr.assemble_S(S_el), g)
    u, q = pr.recover(x, fq, gh)
    for e in range(pr.mesh.N):
        em = pr.element_matrices(e)
        kap, tau = pr.kappa[e], pr.tau[e]
        xe = pr.element_trace(e, x, gh)
        one = np.ones(pr.mesh.Q)
        flux = (one @ (kap * (em["Ex"] @ q[e, 0] + em["Ey"] @ q[e, 1]) + tau * em["E"] @ u[e])
                + one @ ((em["F"] * em["bn"][None, :] - tau * em["F"]) @ xe))
        assert abs(flux - np.dot(wts[e], fq[e])) < 1e-12 * max(1.0, abs(flux))


def test_dirichlet_projection_reproduces_polynomials_and_is_l2_projection():
    pr = HDGProblem(2, 2, 2)
    bpts, bw = pr.bnd_quad_points()
    g = 1.0 + bpts[..., 0] ** 2 - 0.5 * bpts[..., 1]
    gh = pr.dirichlet_trace(g)
    msh = pr.mesh
    for b in range(msh.n_bnd_edges):
        a0, a1 = msh.boundary_edge_endpoints(b)
        for s in range(msh.P1):
            xy = a0 + s / msh.P * (a1 - a0)
            assert abs(gh[b, s] - (1.0 + xy[0] ** 2 - 0.5 * xy[1])) < 1e-13
    # non-polynomial data: the residual is orthogonal to the trace space
    gs = np.sin(3.0 * bpts[..., 0] + 2.0 * bpts[..., 1])
    gh = pr.dirichlet_trace(gs)
    from oracle.quadrature import gauss_legendre as gl
    x, _ = gl(pr.ng_edge)
    psi = line_lagrange(msh.p, x)
    for b in range(msh.n_bnd_edges):
        for s in range(msh.m):
            cols = s * msh.p + np.arange(msh.p + 1)
            sl = slice(s * x.size, (s + 1) * x.size)
            resid = gs[b, sl] - psi @ gh[b, cols]
            # orthogonality is global on the edge: accumulate per dof
        tot = np.zeros(msh.P1)
        for s in range(msh.m):
            cols = s * msh.p + np.arange(msh.p + 1)
            sl = slice(s * x.size, (s + 1) * x.size)
            tot[cols] += psi.T @ (bw[b, sl] * (gs[b, sl] - psi @ gh[b, cols]))
        assert np.abs(tot).max() < 1e-15


# --------------------------------------------------------------------- adjoint
def _adjoint_case(seed, beta=(0.7, -0.4)):
    from oracle.adjoint import forward
    rng = np.random.default_rng(seed)
    n, m, p = 2, 2, 2
    N = 2 * n * n
    kap = rng.uniform(0.5, 2.0, N)
    pr = HDGProblem(n, m, p, beta=beta, kappa=kap)
    pts, _ = pr.quad_points()
    bpts, _ = pr.bnd_quad_points()
    f = rng.standard_normal(pts.shape[:2])
    gD = rng.standard_normal(bpts.shape[:2])
    u_obs = rng.standard_normal((N, pr.mesh.Q))
    J = lambda u: 0.5 * np.sum((u - u_obs) ** 2)

    def J_of(kappa, ff):
        return J(forward(HDGProblem(n, m, p, beta=beta, kappa=kappa), ff, gD)[2])
    return pr, kap, f, gD, u_obs, J_of


@pytest.mark.parametrize("beta", [(0.7, -0.4), (0.0, 0.0)])
def test_adjoint_kappa_gradient_matches_central_differences(beta):
    """Brute force: every component of dJ/dkappa against a central difference
    of J (h = 1e-5; the truncation error is O(h^2) ~ 1e-10 relative)."""
    from oracle.adjoint import forward, gradient
    pr, kap, f, gD, u_obs, J_of = _adjoint_case(3, beta)
    _, _, u, _ = forward(pr, f, gD)
    gk, _, _ = gradient(pr, f, u - u_obs, gD)
    h = 1e-5
    for e in range(len(kap)):
        d = np.zeros_like(kap)
        d[e] = h
        fd = (J_of(kap + d, f) - J_of(kap - d, f)) / (2 * h)
        assert abs(gk[e] - fd) <= 1e-7 * max(abs(fd), 1e-3), (e, gk[e], fd)


def test_adjoint_source_gradient_matches_differences():
    """J is quadratic in f, so a central difference along any direction is exact
    up to rounding: dJ/df . d must match it to ~1e-9."""
    from oracle.adjoint import forward, gradient
    pr, kap, f, gD, u_obs, J_of = _adjoint_case(5)
    _, _, u, _ = forward(pr, f, gD)
    _, gf, _ = gradient(pr, f, u - u_obs, gD)
    rng = np.random.default_rng(11)
    for _ in range(3):
        d = rng.standard_normal(f.shape)
        h = 1e-3
        fd = (J_of(kap, f + h * d) - J_of(kap, f - h * d)) / (2 * h)
        assert abs(np.sum(gf * d) - fd) <= 1e-9 * max(abs(fd), 1.0)


def test_adjoint_blocks_affine_in_kappa():
    """The element blocks are affine in kappa_e (tau_e = kappa_e / tau_len + |beta|):
    K(k0 + 2) - K(k0) = 2 (K(k0 + 1) - K(k0)) entry by entry."""
    pr = HDGProblem(2, 2, 2, beta=(1.0, 0.5), kappa=1.3, tau_len=0.7)
    for e in (0, 5):
        k0 = pr.kappa[e]
        b0, b1, b2 = pr.blocks_at(e, k0), pr.blocks_at(e, k0 + 1), pr.blocks_at(e, k0 + 2)
        for X0, X1, X2 in zip(b0, b1, b2):
            assert np.abs((X2 - X0) - 2 * (X1 - X0)).max() <= 1e-12 * max(np.abs(X1).max(), 1.0)
        # and blocks_at restores the problem's own diffusivity
        assert pr.kappa[e] == k0


# ------------------------------------------------------------------------ SUPG
def test_supg_tau_closed_form():
    """Sec. 3.4 (read with "- 1/Pe"): tau_s = h/(2|a|) (coth Pe - 1/Pe)."""
    from oracle.hdg import supg_tau
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 40
    h, a = 0.1, 2.0
    for kap in (1e-6, 0.05, 0.3, 10.0, 1e3):
        pe = mpmath.mpf(a) * h / (2 * mpmath.mpf(kap))
        exact = float(mpmath.mpf(h) / (2 * a) * (mpmath.coth(pe) - 1 / pe))
        assert abs(supg_tau(h, a, kap) - exact) <= 1e-12 * exact
    assert supg_tau(h, a, 0.0) == h / (2 * a)          # pure advection limit
    assert supg_tau(h, 0.0, 1.0) == 0.0                # no advection, no stabilisation
    # the small-Pe series agrees with the direct formula at the switch (Pe = 0.1)
    kap = a * h / (2 * 0.1)
    lo, hi = supg_tau(h, a, kap * (1 + 1e-14)), supg_tau(h, a, kap * (1 - 1e-14))
    assert abs(hi - lo) < 1e-11 * hi


def test_laplacian_of_basis_reproduces_quadratics():
    """Lap of the P_p interpolant of x^2 + y^2 is 4 on every sub-triangle (p >= 2)."""
    from oracle.basis import tri_lagrange_laplacian
    rng = np.random.default_rng(3)
    for p in (2, 3):
        msh = StructuredMesh(1, 2, p)
        pr = HDGProblem(1, 2, p)
        v = msh.vertices(0)
        for tri in msh.sub_triangles():
            alphas, nodes = msh.sub_nodes(tri)
            A, B, C, Js, Jinv, dlam = pr._sub_triangle_data(v, tri)
            lam_nodes = np.array([[a[0] / p, a[1] / p, a[2] / p] for a in alphas])
            X = A[None, :] + np.outer(lam_nodes[:, 1], B - A) + np.outer(lam_nodes[:, 2], C - A)
            coef = X[:, 0] ** 2 + X[:, 1] ** 2
            lam = rng.dirichlet(np.ones(3), size=5)
            L = tri_lagrange_laplacian(alphas, p, lam, dlam)
            assert np.abs(L @ coef - 4.0).max() < 1e-10


@pytest.mark.parametrize("n,m,p", [(2, 2, 1), (2, 2, 2), (1, 4, 3)])
def test_supg_keeps_polynomial_exactness(n, m, p):
    """The SUPG residual a.grad u - kappa Lap u - f vanishes for the exact solution, so
    u in P_p is still reproduced to roundoff with SUPG on (a dropped Laplacian term or a
    wrong sign of a SUPG term breaks this for p >= 2)."""
    kap, beta = 0.05, (0.9, -0.4)
    pr = HDGProblem(n, m, p, beta=beta, kappa=kap, supg=True)
    u, gr, f = polynomial(random_polynomial(p, seed=21 + p), kap, beta)
    pts, _ = pr.quad_points()
    bpts, _ = pr.bnd_quad_points()
    fq = f(pts[..., 0], pts[..., 1])
    gq = u(bpts[..., 0], bpts[..., 1])
    S_el, g, gh = pr.condense(fq, gq)
    x = np.linalg.solve(pr.assemble_S(S_el), g)
    uu, qq = pr.recover(x, fq, gh)
    eu, eq = pr.l2_errors(uu, qq, u, gr)
    assert eu < 1e-11 and eq < 1e-10
    # and the SUPG terms are active: the condensed operator differs from the plain one
    S0, _, _ = HDGProblem(n, m, p, beta=beta, kappa=kap).condense(fq, gq)
    assert np.abs(np.stack(S_el) - np.stack(S0)).max() > 1e-6 * np.abs(np.stack(S0)).max()


def test_supg_vanishes_for_small_peclet():
    """tau_s ~ h Pe / (6 |a|) as Pe -> 0, so the SUPG terms relative to diffusion scale like
    |a| h^2 / kappa: at kappa = 1e6 the SUPG and plain solutions agree to ~1e-8."""
    kap, beta = 1e6, (1.0, 0.5)
    u, gr, f = sin_sin(kap, beta)
    sols = []
    for supg in (False, True):
        pr = HDGProblem(2, 2, 2, beta=beta, kappa=kap, supg=supg)
        pts, _ = pr.quad_points()
        fq = f(pts[..., 0], pts[..., 1])
        S_el, g, gh = pr.condense(fq)
        sols.append(np.linalg.solve(pr.assemble_S(S_el), g))
    assert np.abs(sols[1] - sols[0]).max() < 1e-6 * np.abs(sols[0]).max()
