"""Macro-element HDG for -kappa Lap u + beta . grad u = f on the unit square (oracle).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Model problem: Eq. (C21) with constant divergence-free a = beta, written in
first-order form Eq. (C22) with q = -grad u. Discrete problem: Eq. (weak_form)
of Sec. 3.2 with the LDG-H flux of Sec. 3.1,
    flux^ = beta u^ + kappa q + tau (u - u^) n,
on the macro-element spaces of Sec. 3.2.

Element matrices (rows = test function, columns = trial function; unknowns
ordered (q_x, q_y, u); phi_i the C0 lattice basis of the macro-element, psi_t
the trace basis of its three edges):
    M_ij  = (phi_j, phi_i)_K              Dx_ij = (phi_j, d_x phi_i)_K
    E_ij  = <phi_j, phi_i>_dK             Ex_ij = <phi_j n_x, phi_i>_dK
    F_it  = <psi_t, phi_i>_dK             Fx_it = <psi_t n_x, phi_i>_dK
    Fa_it = <(beta.n) psi_t, phi_i>_dK    G_st  = <psi_t, psi_s>_dK,  Ga likewise
From A(U, V), B(v^, V), C(U, mu), D(v^, mu) of Eq. (weak_form):
    A = [[M, 0, -Dx], [0, M, -Dy],
         [kappa (Ex - Dx), kappa (Ey - Dy), -(beta_x Dx + beta_y Dy) + tau E]]
    B = [[Fx], [Fy], [Fa - tau F]]
    C = [kappa Fx^T, kappa Fy^T, tau F^T]
    D = Ga - tau G
    R = [0; 0; (f, phi_i)_K]
Dirichlet data enter through u^ = v^ + g^ (Sec. 3.1): g^ is the L2 projection
of g_D onto M(F) on boundary edges (Sec. 2.3), so the element right-hand side
is R - B g^_e (reading of the Dirichlet terms in l(V)).

Static condensation, Eqs. (global_problem)/(local_problem):
    S = sum_e L_e^T (D_e - C_e A_e^-1 B_e) L_e,
    g = sum_e L_e^T (-C_e A_e^-1 R_e - (D_e - C_e A_e^-1 B_e) g^_e)   (unknown rows)
    A_e U_e = R_e - B_e (v^_e + g^_e).
The stabilisation tau is not given a value in the paper; the reading used is
tau_e = kappa_e / tau_len + |beta| on every edge of the element.

SUPG (Sec. 3.4, optional): every sub-triangle T of the macro-element adds
tau_s (beta . grad w, beta . grad u - kappa Lap u)_T to the u-equation and
tau_s (f, beta . grad w)_T to its load, with tau_s = h / (2 |beta|)
(coth Pe - 1 / Pe), Pe = |beta| h / (2 kappa_e), h the sub-triangle diameter.
Readings: the terms act on u (the printed form adds them to B), the printed
"+ 1/Pe" is "- 1/Pe", and Pe and h are the sub-triangle's.
"""
import numpy as np
import scipy.linalg as sla

from .basis import line_lagrange, tri_lagrange, tri_lagrange_laplacian
from .mesh import StructuredMesh
from .quadrature import gauss_legendre, triangle_rule


def supg_tau(h, abs_a, kappa):
    """SUPG parameter (Sec. 3.4, read with "- 1/Pe"): h / (2 |a|) (coth Pe - 1 / Pe),
    Pe = |a| h / (2 kappa); h / (2 |a|) for kappa = 0; 0 without advection."""
    if abs_a <= 0.0:
        return 0.0
    if kappa <= 0.0:
        return h / (2.0 * abs_a)
    pe = abs_a * h / (2.0 * kappa)
    if pe < 0.1:
        # Laurent series of coth x - 1/x (Bernoulli numbers): x/3 - x^3/45 + 2x^5/945 - x^7/4725 + 2x^9/93555
        x2 = pe * pe
        xi = pe * (1.0 / 3.0 + x2 * (-1.0 / 45.0 + x2 * (2.0 / 945.0 + x2 * (-1.0 / 4725.0 + x2 * 2.0 / 93555.0))))
    else:
        xi = 1.0 / np.tanh(pe) - 1.0 / pe
    return h / (2.0 * abs_a) * xi


class HDGProblem:
    """One discrete macro-element HDG problem on the structured unit-square mesh."""

    def __init__(self, n, m, p, beta=(0.0, 0.0), kappa=1.0, tau_len=1.0, supg=False):
        self.mesh = StructuredMesh(n, m, p)
        msh = self.mesh
        self.n, self.m, self.p = n, m, p
        self.beta = np.asarray(beta, dtype=np.float64)
        self.kappa = np.broadcast_to(np.asarray(kappa, dtype=np.float64), (msh.N,)).copy()
        self.tau_len = float(tau_len)
        self.tau = self.kappa / tau_len + np.hypot(self.beta[0], self.beta[1])
        self.ng = p + 2              # source rule: exact to degree 2p + 2
        self.ng_edge = p + 2         # boundary-data rule per sub-edge
        self.supg = bool(supg)
        self._cache = {}

    # ------------------------------------------------------------- quadrature
    def quad_points(self):
        """Physical source quadrature points [N, n_qp, 2] and weights [N, n_qp]."""
        msh = self.mesh
        pw = [self.element_quad_points(e) for e in range(msh.N)]
        return np.stack([a for a, _ in pw]), np.stack([b for _, b in pw])

    def element_quad_points(self, e):
        """Source points [n_qp, 2] and weights [n_qp] of macro-element e (published order)."""
        msh = self.mesh
        xi_q, eta_q, w_q = triangle_rule(self.ng)
        nq = xi_q.size
        subs = msh.sub_triangles()
        pts = np.empty((len(subs) * nq, 2))
        wts = np.empty(len(subs) * nq)
        v = msh.vertices(e)
        for s, tri in enumerate(subs):
            A, B, C = [v[0] + (v[1] - v[0]) * (t[0] / msh.m) + (v[2] - v[0]) * (t[1] / msh.m)
                       for t in tri]
            area = 0.5 * abs((B - A)[0] * (C - A)[1] - (B - A)[1] * (C - A)[0])
            sl = slice(s * nq, (s + 1) * nq)
            pts[sl, :] = A[None, :] + np.outer(xi_q, B - A) + np.outer(eta_q, C - A)
            wts[sl] = w_q * 2.0 * area
        return pts, wts

    def bnd_quad_points(self):
        """Dirichlet-data points [4 n, m * ng_edge, 2] and weights (sub-edge major)."""
        msh = self.mesh
        x, w = gauss_legendre(self.ng_edge)
        pts = np.empty((msh.n_bnd_edges, msh.m * x.size, 2))
        wts = np.empty((msh.n_bnd_edges, msh.m * x.size))
        for b in range(msh.n_bnd_edges):
            a0, a1 = msh.boundary_edge_endpoints(b)
            L = np.linalg.norm(a1 - a0)
            for s in range(msh.m):
                th = (s + x) / msh.m
                sl = slice(s * x.size, (s + 1) * x.size)
                pts[b, sl, :] = a0[None, :] + np.outer(th, a1 - a0)
                wts[b, sl] = w * L / msh.m
        return pts, wts

    # -------------------------------------------------------- element matrices
    def _sub_triangle_data(self, v, tri):
        """Physical vertices and barycentric gradients of one sub-triangle."""
        m = self.m
        A, B, C = [v[0] + (v[1] - v[0]) * (t[0] / m) + (v[2] - v[0]) * (t[1] / m) for t in tri]
        Js = np.column_stack([B - A, C - A])
        Jinv = np.linalg.inv(Js)
        dlam = np.array([-(Jinv[0] + Jinv[1]), Jinv[0], Jinv[1]])
        return A, B, C, Js, Jinv, dlam

    def element_matrices(self, e):
        """Geometric element matrices of macro-element e (independent of kappa, tau)."""
        if e in self._cache:
            return self._cache[e]
        msh = self.mesh
        p, m, P, Q, P1 = msh.p, msh.m, msh.P, msh.Q, msh.P1
        n_t = msh.n_t
        v = msh.vertices(e)
        xi_q, eta_q, w_q = triangle_rule(self.ng)
        lam_q = np.column_stack([1.0 - xi_q - eta_q, xi_q, eta_q])
        subs = msh.sub_triangles()

        M = np.zeros((Q, Q))
        Dx = np.zeros((Q, Q))
        Dy = np.zeros((Q, Q))
        Phi = np.zeros((len(subs) * xi_q.size, Q))      # basis at source points
        # SUPG (Sec. 3.4): (a.grad phi_i, a.grad phi_j) and (a.grad phi_i, Lap phi_j) per
        # sub-triangle, and a.grad phi at the source points
        Kbb = np.zeros((Q, Q))
        KbL = np.zeros((Q, Q))
        PhiB = np.zeros((len(subs) * xi_q.size, Q))
        hsub = 0.0
        for s, tri in enumerate(subs):
            alphas, nodes = msh.sub_nodes(tri)
            nodes = np.array(nodes)
            A, B, C, Js, Jinv, dlam = self._sub_triangle_data(v, tri)
            wq = w_q * abs(np.linalg.det(Js))
            phi, grad = tri_lagrange(alphas, p, lam_q, dlam)
            ix = np.ix_(nodes, nodes)
            np.add.at(M, ix, np.einsum("q,qa,qb->ab", wq, phi, phi))
            np.add.at(Dx, ix, np.einsum("q,qa,qb->ab", wq, grad[:, :, 0], phi))
            np.add.at(Dy, ix, np.einsum("q,qa,qb->ab", wq, grad[:, :, 1], phi))
            Phi[s * xi_q.size:(s + 1) * xi_q.size, nodes] = phi
            bgrad = self.beta[0] * grad[:, :, 0] + self.beta[1] * grad[:, :, 1]
            lap = tri_lagrange_laplacian(alphas, p, lam_q, dlam)
            np.add.at(Kbb, ix, np.einsum("q,qa,qb->ab", wq, bgrad, bgrad))
            np.add.at(KbL, ix, np.einsum("q,qa,qb->ab", wq, bgrad, lap))
            PhiB[s * xi_q.size:(s + 1) * xi_q.size, nodes] = bgrad
            hsub = max(hsub, np.linalg.norm(B - A), np.linalg.norm(C - A), np.linalg.norm(C - B))

        # boundary terms, edge k from v_{k+1} to v_{k+2}
        xg, wg = gauss_legendre(self.ng)
        E = np.zeros((Q, Q))
        Ex = np.zeros((Q, Q))
        Ey = np.zeros((Q, Q))
        F = np.zeros((Q, n_t))
        G = np.zeros((n_t, n_t))
        normals = np.zeros((3, 2))
        lengths = np.zeros(3)
        for k in range(3):
            a0, a1 = v[(k + 1) % 3], v[(k + 2) % 3]
            L = np.linalg.norm(a1 - a0)
            tvec = (a1 - a0) / L
            nvec = np.array([tvec[1], -tvec[0]])         # outward for CCW vertices
            normals[k], lengths[k] = nvec, L
            for s in range(m):
                th = (s + xg) / m
                xq = a0[None, :] + np.outer(th, a1 - a0)
                wq = wg * L / m
                mid = a0 + (s + 0.5) / m * (a1 - a0)
                # the (unique) sub-triangle that contains this boundary sub-edge
                found = None
                for tri in subs:
                    A, B, C, Js, Jinv, dlam = self._sub_triangle_data(v, tri)
                    lm = Jinv @ (mid - A)
                    bary = np.array([1.0 - lm[0] - lm[1], lm[0], lm[1]])
                    if bary.min() > -1e-12:
                        found = (tri, A, Jinv, dlam)
                        break
                tri, A, Jinv, dlam = found
                alphas, nodes = msh.sub_nodes(tri)
                nodes = np.array(nodes)
                lmq = (xq - A[None, :]) @ Jinv.T
                lam = np.column_stack([1.0 - lmq[:, 0] - lmq[:, 1], lmq[:, 0], lmq[:, 1]])
                phi, _ = tri_lagrange(alphas, p, lam, dlam)
                psi = line_lagrange(p, xg)               # local sub-edge parameter = xg
                cols = k * P1 + s * p + np.arange(p + 1)
                ix = np.ix_(nodes, nodes)
                Eloc = np.einsum("q,qa,qb->ab", wq, phi, phi)
                np.add.at(E, ix, Eloc)
                np.add.at(Ex, ix, nvec[0] * Eloc)
                np.add.at(Ey, ix, nvec[1] * Eloc)
                np.add.at(F, np.ix_(nodes, cols), np.einsum("q,qa,qt->at", wq, phi, psi))
                np.add.at(G, np.ix_(cols, cols), np.einsum("q,qs,qt->st", wq, psi, psi))
        nx = np.repeat(normals[:, 0], P1)
        ny = np.repeat(normals[:, 1], P1)
        out = dict(M=M, Dx=Dx, Dy=Dy, E=E, Ex=Ex, Ey=Ey, F=F, Fx=F * nx[None, :], Kbb=Kbb, KbL=KbL, PhiB=PhiB,
                   hsub=hsub,
                   Fy=F * ny[None, :], G=G, Phi=Phi, normals=normals, lengths=lengths,
                   bn=self.beta[0] * nx + self.beta[1] * ny)
        self._cache[e] = out
        return out

    def local_blocks(self, e):
        """A_e, B_e, C_e, D_e of Eq. (D) for macro-element e."""
        em = self.element_matrices(e)
        Q = self.mesh.Q
        kap, tau = self.kappa[e], self.tau[e]
        bx, by = self.beta
        M, Dx, Dy = em["M"], em["Dx"], em["Dy"]
        A = np.zeros((3 * Q, 3 * Q))
        A[0:Q, 0:Q] = M
        A[Q:2 * Q, Q:2 * Q] = M
        A[0:Q, 2 * Q:] = -Dx
        A[Q:2 * Q, 2 * Q:] = -Dy
        A[2 * Q:, 0:Q] = kap * (em["Ex"] - Dx)
        A[2 * Q:, Q:2 * Q] = kap * (em["Ey"] - Dy)
        A[2 * Q:, 2 * Q:] = -(bx * Dx + by * Dy) + tau * em["E"]
        Fa = em["F"] * em["bn"][None, :]
        B = np.vstack([em["Fx"], em["Fy"], Fa - tau * em["F"]])
        C = np.hstack([kap * em["Fx"].T, kap * em["Fy"].T, tau * em["F"].T])
        Ga = em["G"] * em["bn"][None, :]       # G is block diagonal per edge
        D = Ga - tau * em["G"]
        if self.supg:
            ts = self.supg_tau(e)
            A[2 * Q:, 2 * Q:] += ts * (em["Kbb"] - kap * em["KbL"])
        return A, B, C, D

    def supg_tau(self, e):
        """tau_s of Sec. 3.4 for macro-element e: h / (2 |a|) (coth Pe - 1 / Pe), Pe = |a| h /
        (2 kappa_e), h the sub-triangle diameter (the printed "+ 1/Pe" read as "- 1/Pe")."""
        h = self.element_matrices(e)["hsub"]
        return supg_tau(h, float(np.hypot(self.beta[0], self.beta[1])), float(self.kappa[e]))

    def blocks_at(self, e, kappa_e):
        """A_e, B_e, C_e, D_e evaluated with diffusivity kappa_e (tau_e follows kappa_e)."""
        k0, t0 = self.kappa[e], self.tau[e]
        self.kappa[e] = kappa_e
        self.tau[e] = kappa_e / self.tau_len + np.hypot(self.beta[0], self.beta[1])
        try:
            return self.local_blocks(e)
        finally:
            self.kappa[e], self.tau[e] = k0, t0

    def load_vector(self, e, f_vals):
        """R_e = [0; 0; (f, phi_i)_K] from f at the published source points of e."""
        em = self.element_matrices(e)
        Q = self.mesh.Q
        key = ("qw", e)
        if key not in self._cache:
            self._cache[key] = self.element_quad_points(e)[1]
        w = self._cache[key]
        R = np.zeros(3 * Q)
        R[2 * Q:] = em["Phi"].T @ (w * f_vals)
        if self.supg:
            R[2 * Q:] += self.supg_tau(e) * (em["PhiB"].T @ (w * f_vals))
        return R

    # ---------------------------------------------------------- Dirichlet data
    def dirichlet_trace(self, gD_vals):
        """L2 projection of g_D onto M(F) on every boundary edge: [4 n, P + 1]."""
        msh = self.mesh
        p, m, P1 = msh.p, msh.m, msh.P1
        x, w = gauss_legendre(self.ng_edge)
        psi = line_lagrange(p, x)
        out = np.zeros((msh.n_bnd_edges, P1))
        for b in range(msh.n_bnd_edges):
            a0, a1 = msh.boundary_edge_endpoints(b)
            L = np.linalg.norm(a1 - a0)
            G = np.zeros((P1, P1))
            rhs = np.zeros(P1)
            for s in range(m):
                cols = s * p + np.arange(p + 1)
                wq = w * L / m
                G[np.ix_(cols, cols)] += np.einsum("q,qs,qt->st", wq, psi, psi)
                rhs[cols] += psi.T @ (wq * gD_vals[b, s * x.size:(s + 1) * x.size])
            out[b] = np.linalg.solve(G, rhs)
        return out

    def element_trace(self, e, v_hat, g_hat):
        """Element-local trace vector (n_t): unknowns from v_hat, boundary from g_hat."""
        out = np.empty(self.mesh.n_t)
        gflat = g_hat.reshape(-1)
        for loc, (kind, idx) in enumerate(self.mesh.element_dof_map(e)):
            out[loc] = v_hat[idx] if kind == "int" else gflat[idx]
        return out

    def scatter(self, e, vec_loc, out):
        """out += L_e^T vec_loc on the unknown (interior) rows."""
        for loc, (kind, idx) in enumerate(self.mesh.element_dof_map(e)):
            if kind == "int":
                out[idx] += vec_loc[loc]

    # ----------------------------------------------------- static condensation
    def condense_element(self, e, f_vals=None, g_hat_e=None):
        """S_e = D_e - C_e A_e^-1 B_e and g_e (Eq. global_problem), by dense LU of A_e."""
        A, B, C, D = self.local_blocks(e)
        lu = sla.lu_factor(A)
        S = D - C @ sla.lu_solve(lu, B)
        g = np.zeros(self.mesh.n_t)
        if f_vals is not None:
            g -= C @ sla.lu_solve(lu, self.load_vector(e, f_vals))
        if g_hat_e is not None:
            g -= S @ g_hat_e
        return S, g

    def condense(self, f_qp=None, gD_qp=None):
        """All S_e, the assembled right-hand side g and the Dirichlet trace g^."""
        msh = self.mesh
        g_hat = (self.dirichlet_trace(gD_qp) if gD_qp is not None
                 else np.zeros((msh.n_bnd_edges, msh.P1)))
        S_el = np.empty((msh.N, msh.n_t, msh.n_t))
        g = np.zeros(msh.N_tr)
        for e in range(msh.N):
            ghe = self.element_trace(e, np.zeros(msh.N_tr), g_hat)
            S_el[e], g_e = self.condense_element(e, None if f_qp is None else f_qp[e], ghe)
            self.scatter(e, g_e, g)
        return S_el, g, g_hat

    def assemble_S(self, S_el):
        """Dense global trace operator sum_e L_e^T S_e L_e on the unknowns (tiny meshes)."""
        msh = self.mesh
        S = np.zeros((msh.N_tr, msh.N_tr))
        for e in range(msh.N):
            rows = [(loc, idx) for loc, (kind, idx) in enumerate(msh.element_dof_map(e))
                    if kind == "int"]
            for la, ia in rows:
                for lb, ib in rows:
                    S[ia, ib] += S_el[e][la, lb]
        return S

    def apply_S(self, S_el, x):
        """y = sum_e L_e^T S_e L_e x, element by element."""
        msh = self.mesh
        y = np.zeros(msh.N_tr)
        zero_bnd = np.zeros((msh.n_bnd_edges, msh.P1))
        for e in range(msh.N):
            xe = self.element_trace(e, x, zero_bnd)
            self.scatter(e, S_el[e] @ xe, y)
        return y

    # --------------------------------------------- four-step apply, Sec. 3.3.2
    def face_D(self):
        """D_f (summed over the two sides) for every interior edge: [n_int, P1, P1]."""
        msh = self.mesh
        P1 = msh.P1
        Df = np.zeros((msh.n_int_edges, P1, P1))
        for e in range(msh.N):
            _, _, _, D = self.local_blocks(e)
            for k, (kind, idx, flip) in enumerate(msh.element_edges(e)):
                if kind != "int":
                    continue
                blk = D[k * P1:(k + 1) * P1, k * P1:(k + 1) * P1]
                if flip:
                    blk = blk[::-1, ::-1]
                Df[idx] += blk
        return Df

    def apply_four_step(self, x, precondition=False):
        """The paper's matrix-free apply: steps 1-3 per element, step 4 per face.

        Step 1: x_e = B_e u^_e; step 2: y_e = A_e^-1 x_e; step 3: v^_e = C_e y_e;
        step 4: w^_f = D_f u^_f - v^_f1 - v^_f2, or, preconditioned (Sec. 6.1),
        w^_f = u^_f - D_f^-1 (v^_f1 + v^_f2).
        """
        msh = self.mesh
        P1 = msh.P1
        zero_bnd = np.zeros((msh.n_bnd_edges, P1))
        vsum = np.zeros(msh.N_tr)
        for e in range(msh.N):
            A, B, C, _ = self.local_blocks(e)
            ue = self.element_trace(e, x, zero_bnd)
            xe = B @ ue                                   # step 1
            ye = np.linalg.solve(A, xe)                   # step 2
            ve = C @ ye                                   # step 3
            self.scatter(e, ve, vsum)
        Df = self.face_D()
        w = np.empty(msh.N_tr)
        for f in range(msh.n_int_edges):                  # step 4
            sl = slice(f * P1, (f + 1) * P1)
            if precondition:
                w[sl] = x[sl] - np.linalg.solve(Df[f], vsum[sl])
            else:
                w[sl] = Df[f] @ x[sl] - vsum[sl]
        return w

    def apply_Dinv(self, y, Df=None):
        """z_f = D_f^-1 y_f through the Cholesky factor of -D_f (Sec. 6.1)."""
        msh = self.mesh
        P1 = msh.P1
        if Df is None:
            Df = self.face_D()
        z = np.empty_like(y)
        for f in range(msh.n_int_edges):
            sl = slice(f * P1, (f + 1) * P1)
            c = sla.cho_factor(-Df[f])
            z[sl] = -sla.cho_solve(c, y[sl])
        return z

    # -------------------------------------------------------------- recovery
    def recover(self, v_hat, f_qp=None, g_hat=None):
        """Local problem Eq. (local_matrix_problem): u [N, Q], q [N, 2, Q]."""
        msh = self.mesh
        Q = msh.Q
        if g_hat is None:
            g_hat = np.zeros((msh.n_bnd_edges, msh.P1))
        u = np.empty((msh.N, Q))
        q = np.empty((msh.N, 2, Q))
        for e in range(msh.N):
            A, B, _, _ = self.local_blocks(e)
            R = self.load_vector(e, f_qp[e]) if f_qp is not None else np.zeros(3 * Q)
            ue = self.element_trace(e, v_hat, g_hat)
            U = np.linalg.solve(A, R - B @ ue)
            q[e, 0], q[e, 1], u[e] = U[0:Q], U[Q:2 * Q], U[2 * Q:]
        return u, q

    # ------------------------------------------------ full unreduced system
    def solve_unreduced(self, f_qp=None, gD_qp=None):
        """Assemble [[A, B], [C, D]] of Eq. (D) globally and solve it directly."""
        msh = self.mesh
        Q3 = 3 * msh.Q
        nz = msh.N * Q3
        ntot = nz + msh.N_tr
        K = np.zeros((ntot, ntot))
        rhs = np.zeros(ntot)
        g_hat = (self.dirichlet_trace(gD_qp) if gD_qp is not None
                 else np.zeros((msh.n_bnd_edges, msh.P1)))
        for e in range(msh.N):
            A, B, C, D = self.local_blocks(e)
            r0 = e * Q3
            K[r0:r0 + Q3, r0:r0 + Q3] = A
            R = self.load_vector(e, f_qp[e]) if f_qp is not None else np.zeros(Q3)
            ghe = self.element_trace(e, np.zeros(msh.N_tr), g_hat)
            rhs[r0:r0 + Q3] = R - B @ ghe
            dmap = msh.element_dof_map(e)
            for la, (ka, ia) in enumerate(dmap):
                if ka != "int":
                    continue
                K[r0:r0 + Q3, nz + ia] += B[:, la]
                K[nz + ia, r0:r0 + Q3] += C[la, :]
                for lb, (kb, ib) in enumerate(dmap):
                    if kb == "int":
                        K[nz + ia, nz + ib] += D[la, lb]
                    else:
                        rhs[nz + ia] -= D[la, lb] * ghe[lb]
        sol = np.linalg.solve(K, rhs)
        U = sol[:nz].reshape(msh.N, Q3)
        Qn = msh.Q
        return sol[nz:], U[:, 2 * Qn:], np.stack([U[:, :Qn], U[:, Qn:2 * Qn]], axis=1)

    # ---------------------------------------------------------------- errors
    def l2_errors(self, u, q, u_exact, grad_u_exact, ng=None):
        """L2 errors of u and q = -grad u on every sub-triangle (rule exact to 2p + 6)."""
        msh = self.mesh
        p = msh.p
        ng = ng or (p + 4)
        xi_q, eta_q, w_q = triangle_rule(ng)
        lam_q = np.column_stack([1.0 - xi_q - eta_q, xi_q, eta_q])
        eu = eq = 0.0
        for e in range(msh.N):
            v = msh.vertices(e)
            for tri in msh.sub_triangles():
                alphas, nodes = msh.sub_nodes(tri)
                A, B, C, Js, Jinv, dlam = self._sub_triangle_data(v, tri)
                phi, _ = tri_lagrange(alphas, p, lam_q, dlam)
                xq = A[None, :] + np.outer(xi_q, B - A) + np.outer(eta_q, C - A)
                wq = w_q * abs(np.linalg.det(Js))
                uh = phi @ u[e][nodes]
                qxh = phi @ q[e][0][nodes]
                qyh = phi @ q[e][1][nodes]
                gx, gy = grad_u_exact(xq[:, 0], xq[:, 1])
                eu += np.sum(wq * (uh - u_exact(xq[:, 0], xq[:, 1])) ** 2)
                eq += np.sum(wq * ((qxh + gx) ** 2 + (qyh + gy) ** 2))
        return np.sqrt(eu), np.sqrt(eq)
