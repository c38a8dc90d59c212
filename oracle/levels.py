"""Macro-elements of uneven refinement level with non-conforming faces (oracle).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Sec. 4.2 (local adaptive refinement): every macro-element K carries its own
level r_K, i.e. m_K = 2^r_K sub-edges per macro-edge and the C0 lattice of
that level inside. The trace space of a macro-face F is refined to its finer
side, level R_F = max(r+, r-), so that it holds the trace of either side
exactly (continuity across the face is kept in the normal direction); a
boundary face has the level of its element. On the coarse side the face
integrals <psi, phi> pair a fine trace function with a coarse volume function;
they are integrated on the fine sub-edges, on each of which both are
polynomials.

Everything else is the discrete problem of oracle/hdg.py, element by element:
A_e from the element's own level, B_e, C_e, D_e from its face levels
(Eq. weak_form with the LDG-H flux). The element volume matrices come from the
uniform-level oracle of the element's level; the face matrices are built here.

Layouts (the library's level-mesh layout, restated):
  trace dofs: interior edge f carries 2^R_f p + 1 dofs along its orientation;
    global dof = eoff[f] + s, eoff the prefix sum over edges in edge-id order.
  Dirichlet trace: boundary edge b carries 2^r_b p + 1 values at goff[b].
  source points: element e's m_e^2 (p + 2)^2 points (uniform-level order) at qoff[e].
  Dirichlet-data points: boundary edge b's 2^r_b (p + 2) points at boff[b].
  u: element e's Q_e lattice values at uoff[e]; q: [2][Q_e] at 2 uoff[e].
"""
import numpy as np
import scipy.linalg as sla

from .basis import line_lagrange, tri_lagrange
from .hdg import HDGProblem
from .mesh import StructuredMesh
from .quadrature import gauss_legendre, triangle_rule

MAX_LEVEL = 4


class LevelHDGProblem:
    """Discrete macro-element HDG problem with per-element refinement levels."""

    def __init__(self, n, levels, p, beta=(0.0, 0.0), kappa=1.0, tau_len=1.0, supg=False):
        N = 2 * n * n
        levels = np.asarray(levels, dtype=np.int64).reshape(-1)
        if levels.shape[0] != N or levels.min() < 0 or levels.max() > MAX_LEVEL:
            raise ValueError("levels: N entries in 0 .. %d" % MAX_LEVEL)
        self.n, self.p, self.N, self.levels = n, p, N, levels
        self.beta = np.asarray(beta, dtype=np.float64)
        self.kappa = np.broadcast_to(np.asarray(kappa, dtype=np.float64), (N,)).copy()
        self.tau_len = float(tau_len)
        self.tau = self.kappa / tau_len + np.hypot(self.beta[0], self.beta[1])
        self.supg = bool(supg)
        self.ng = p + 2
        # one uniform-level problem per level present (volume matrices, sources, Dirichlet rule)
        self.sub = {int(r): HDGProblem(n, 2 ** int(r), p, beta=beta, kappa=self.kappa, tau_len=tau_len,
                                       supg=supg) for r in np.unique(levels)}
        self.skel = StructuredMesh(n, 1, p)          # edge numbering (independent of the level)
        sk = self.skel
        self.n_int, self.n_bnd = sk.n_int_edges, sk.n_bnd_edges
        self.flevel = np.zeros(self.n_int, dtype=np.int64)
        self.blevel = np.zeros(self.n_bnd, dtype=np.int64)
        for e in range(N):
            for kind, idx, _ in sk.element_edges(e):
                if kind == "int":
                    self.flevel[idx] = max(self.flevel[idx], levels[e])
                else:
                    self.blevel[idx] = levels[e]
        cum = lambda a: np.concatenate([[0], np.cumsum(a)]).astype(np.int64)
        self.eoff = cum(2 ** self.flevel * p + 1)
        self.goff = cum(2 ** self.blevel * p + 1)
        self.N_tr = int(self.eoff[-1])
        me = 2 ** levels
        self.Qe = (me * p + 1) * (me * p + 2) // 2
        self.uoff = cum(self.Qe)
        self.qoff = cum(me * me * self.ng * self.ng)
        self.boff = cum(2 ** self.blevel * self.ng)
        self._cache = {}

    # ----------------------------------------------------------- face levels
    def faces(self, e):
        """[(kind, index, flip, R)] for local edges 0, 1, 2 of element e."""
        out = []
        for kind, idx, flip in self.skel.element_edges(e):
            R = self.flevel[idx] if kind == "int" else self.blevel[idx]
            out.append((kind, idx, flip, int(R)))
        return out

    def n_t(self, e):
        return sum(2 ** R * self.p + 1 for *_, R in self.faces(e))

    def element_dof_map(self, e):
        """(kind, global index) of every element-local trace dof of e."""
        out = []
        for kind, idx, flip, R in self.faces(e):
            PR = 2 ** R * self.p
            base = self.eoff[idx] if kind == "int" else self.goff[idx]
            for s_loc in range(PR + 1):
                out.append((kind, int(base + (PR - s_loc if flip else s_loc))))
        return out

    # ------------------------------------------------------------ quadrature
    def quad_points(self):
        """Source points [sum n_qp, 2] and weights, element e's at qoff[e]."""
        pts = np.empty((self.qoff[-1], 2))
        wts = np.empty(self.qoff[-1])
        for r, sub in self.sub.items():
            sp, sw = sub.quad_points()
            for e in np.nonzero(self.levels == r)[0]:
                pts[self.qoff[e]:self.qoff[e + 1]] = sp[e]
                wts[self.qoff[e]:self.qoff[e + 1]] = sw[e]
        return pts, wts

    def bnd_quad_points(self):
        """Dirichlet-data points [sum n_bqp, 2] and weights, boundary edge b's at boff[b]."""
        pts = np.empty((self.boff[-1], 2))
        wts = np.empty(self.boff[-1])
        for b in range(self.n_bnd):
            sp, sw = self.sub[int(self.blevel[b])].bnd_quad_points()
            pts[self.boff[b]:self.boff[b + 1]] = sp[b]
            wts[self.boff[b]:self.boff[b + 1]] = sw[b]
        return pts, wts

    # ------------------------------------------------------ element matrices
    def element_matrices(self, e):
        """Volume matrices of e's own level; F, G, normals per face at the face levels."""
        key = ("em", e)
        if key in self._cache:
            return self._cache[key]
        r = int(self.levels[e])
        sub = self.sub[r]
        msh = sub.mesh
        p, m, Q = self.p, msh.m, msh.Q
        em = dict(sub.element_matrices(e))
        faces = self.faces(e)
        sizes = [2 ** R * p + 1 for *_, R in faces]
        offs = np.concatenate([[0], np.cumsum(sizes)])
        nt = int(offs[-1])
        v = msh.vertices(e)
        xg, wg = gauss_legendre(sub.ng)
        psi = line_lagrange(p, xg)
        subs = msh.sub_triangles()
        F = np.zeros((Q, nt))
        G = np.zeros((nt, nt))
        for k, (_, _, _, R) in enumerate(faces):
            a0, a1 = v[(k + 1) % 3], v[(k + 2) % 3]
            L = np.linalg.norm(a1 - a0)
            mf = 2 ** R
            for s in range(mf):
                xq = a0[None, :] + np.outer((s + xg) / mf, a1 - a0)
                wq = wg * L / mf
                mid = a0 + (s + 0.5) / mf * (a1 - a0)
                # the sub-triangle of the element's own lattice that holds this fine sub-edge
                for tri in subs:
                    A, B, C, Js, Jinv, dlam = sub._sub_triangle_data(v, tri)
                    lm = Jinv @ (mid - A)
                    if min(1.0 - lm[0] - lm[1], lm[0], lm[1]) > -1e-12:
                        break
                else:
                    raise RuntimeError("no sub-triangle holds the sub-edge")
                alphas, nodes = msh.sub_nodes(tri)
                lmq = (xq - A[None, :]) @ Jinv.T
                lam = np.column_stack([1.0 - lmq[:, 0] - lmq[:, 1], lmq[:, 0], lmq[:, 1]])
                phi, _ = tri_lagrange(alphas, p, lam, dlam)
                cols = offs[k] + s * p + np.arange(p + 1)
                np.add.at(F, np.ix_(np.array(nodes), cols), np.einsum("q,qa,qt->at", wq, phi, psi))
                G[np.ix_(cols, cols)] += np.einsum("q,qs,qt->st", wq, psi, psi)
        nrm = em["normals"]
        nx = np.concatenate([np.full(sizes[k], nrm[k, 0]) for k in range(3)])
        ny = np.concatenate([np.full(sizes[k], nrm[k, 1]) for k in range(3)])
        em.update(F=F, Fx=F * nx[None, :], Fy=F * ny[None, :], G=G, sizes=sizes, offs=offs,
                  bn=self.beta[0] * nx + self.beta[1] * ny)
        self._cache[key] = em
        return em

    def local_blocks(self, e):
        """A_e, B_e, C_e, D_e of Eq. (D) with the face levels of e."""
        em = self.element_matrices(e)
        Q = em["M"].shape[0]
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
        if self.supg:
            A[2 * Q:, 2 * Q:] += self.sub[int(self.levels[e])].supg_tau(e) * (em["Kbb"] - kap * em["KbL"])
        B = np.vstack([em["Fx"], em["Fy"], em["F"] * em["bn"][None, :] - tau * em["F"]])
        C = np.hstack([kap * em["Fx"].T, kap * em["Fy"].T, tau * em["F"].T])
        D = em["G"] * em["bn"][None, :] - tau * em["G"]
        return A, B, C, D

    def load_vector(self, e, f_flat):
        """R_e from f at e's source points (flat layout)."""
        return self.sub[int(self.levels[e])].load_vector(e, f_flat[self.qoff[e]:self.qoff[e + 1]])

    # ------------------------------------------------------- Dirichlet data
    def dirichlet_trace(self, gD_flat):
        """L2 projection of g_D onto M(F) on every boundary edge (flat, goff layout)."""
        p = self.p
        x, w = gauss_legendre(self.ng)
        psi = line_lagrange(p, x)
        out = np.zeros(self.goff[-1])
        for b in range(self.n_bnd):
            mb = 2 ** int(self.blevel[b])
            a0, a1 = self.skel.boundary_edge_endpoints(b)
            L = np.linalg.norm(a1 - a0)
            nb = mb * p + 1
            G = np.zeros((nb, nb))
            rhs = np.zeros(nb)
            vals = gD_flat[self.boff[b]:self.boff[b + 1]]
            for s in range(mb):
                cols = s * p + np.arange(p + 1)
                wq = w * L / mb
                G[np.ix_(cols, cols)] += np.einsum("q,qs,qt->st", wq, psi, psi)
                rhs[cols] += psi.T @ (wq * vals[s * x.size:(s + 1) * x.size])
            out[self.goff[b]:self.goff[b + 1]] = np.linalg.solve(G, rhs)
        return out

    def element_trace(self, e, v_hat, g_hat):
        return np.array([v_hat[i] if kind == "int" else g_hat[i] for kind, i in self.element_dof_map(e)])

    def scatter(self, e, vec_loc, out):
        for loc, (kind, i) in enumerate(self.element_dof_map(e)):
            if kind == "int":
                out[i] += vec_loc[loc]

    # -------------------------------------------------- static condensation
    def condense_element(self, e, f_flat=None, g_hat=None):
        """S_e = D_e - C_e A_e^-1 B_e and g_e = -C_e A_e^-1 R_e - S_e g^_e (dense LU of A_e)."""
        A, B, C, D = self.local_blocks(e)
        lu = sla.lu_factor(A)
        S = D - C @ sla.lu_solve(lu, B)
        ge = np.zeros(S.shape[0])
        if g_hat is not None:
            ge -= S @ self.element_trace(e, np.zeros(self.N_tr), g_hat)
        if f_flat is not None:
            ge -= C @ sla.lu_solve(lu, self.load_vector(e, f_flat))
        return S, ge

    def condense(self, f_flat=None, gD_flat=None):
        """S_e (list), the assembled right-hand side g and the Dirichlet trace g^."""
        g_hat = self.dirichlet_trace(gD_flat) if gD_flat is not None else np.zeros(self.goff[-1])
        S_el, g = [], np.zeros(self.N_tr)
        for e in range(self.N):
            S, ge = self.condense_element(e, f_flat, g_hat)
            S_el.append(S)
            self.scatter(e, ge, g)
        return S_el, g, g_hat

    def recover_element(self, e, v_hat, f_flat=None, g_hat=None):
        """(u_e, q_e) of Eq. (local_matrix_problem) for one element: u [Q_e], q [2, Q_e]."""
        A, B, _, _ = self.local_blocks(e)
        Q = self.Qe[e]
        if g_hat is None:
            g_hat = np.zeros(self.goff[-1])
        R = self.load_vector(e, f_flat) if f_flat is not None else np.zeros(3 * Q)
        U = np.linalg.solve(A, R - B @ self.element_trace(e, v_hat, g_hat))
        return U[2 * Q:], U[:2 * Q].reshape(2, Q)

    def assemble_S(self, S_el):
        S = np.zeros((self.N_tr, self.N_tr))
        for e in range(self.N):
            rows = [(loc, i) for loc, (kind, i) in enumerate(self.element_dof_map(e)) if kind == "int"]
            for la, ia in rows:
                for lb, ib in rows:
                    S[ia, ib] += S_el[e][la, lb]
        return S

    def apply_S(self, S_el, x):
        y = np.zeros(self.N_tr)
        zb = np.zeros(self.goff[-1])
        for e in range(self.N):
            self.scatter(e, S_el[e] @ self.element_trace(e, x, zb), y)
        return y

    def face_D(self):
        """D_f summed over the two sides of every interior edge (list of arrays)."""
        Df = [np.zeros((self.eoff[f + 1] - self.eoff[f],) * 2) for f in range(self.n_int)]
        for e in range(self.N):
            _, _, _, D = self.local_blocks(e)
            offs = self.element_matrices(e)["offs"]
            for k, (kind, idx, flip, _) in enumerate(self.faces(e)):
                if kind != "int":
                    continue
                blk = D[offs[k]:offs[k + 1], offs[k]:offs[k + 1]]
                Df[idx] += blk[::-1, ::-1] if flip else blk
        return Df

    def apply_Dinv(self, y, Df=None):
        """z_f = D_f^-1 y_f through the Cholesky factor of -D_f (Sec. 6.1)."""
        Df = Df if Df is not None else self.face_D()
        z = np.empty_like(y)
        for f in range(self.n_int):
            sl = slice(self.eoff[f], self.eoff[f + 1])
            z[sl] = -sla.cho_solve(sla.cho_factor(-Df[f]), y[sl])
        return z

    # --------------------------------------------------------------- recovery
    def recover(self, v_hat, f_flat=None, g_hat=None):
        """Eq. (local_matrix_problem) per element: u (uoff layout), q ([2][Q_e] at 2 uoff[e])."""
        if g_hat is None:
            g_hat = np.zeros(self.goff[-1])
        u = np.empty(self.uoff[-1])
        q = np.empty(2 * self.uoff[-1])
        for e in range(self.N):
            A, B, _, _ = self.local_blocks(e)
            Q = self.Qe[e]
            R = self.load_vector(e, f_flat) if f_flat is not None else np.zeros(3 * Q)
            U = np.linalg.solve(A, R - B @ self.element_trace(e, v_hat, g_hat))
            u[self.uoff[e]:self.uoff[e + 1]] = U[2 * Q:]
            q[2 * self.uoff[e]:2 * self.uoff[e + 1]] = U[:2 * Q]
        return u, q

    def solve_unreduced(self, f_flat=None, gD_flat=None):
        """The global [[A, B], [C, D]] system of Eq. (D) assembled and solved directly."""
        g_hat = self.dirichlet_trace(gD_flat) if gD_flat is not None else np.zeros(self.goff[-1])
        off = np.concatenate([[0], np.cumsum(3 * self.Qe)])
        nz = int(off[-1])
        K = np.zeros((nz + self.N_tr, nz + self.N_tr))
        rhs = np.zeros(nz + self.N_tr)
        zero = np.zeros(self.N_tr)
        for e in range(self.N):
            A, B, C, D = self.local_blocks(e)
            sl = slice(off[e], off[e + 1])
            K[sl, sl] = A
            ghe = self.element_trace(e, zero, g_hat)
            R = self.load_vector(e, f_flat) if f_flat is not None else np.zeros(A.shape[0])
            rhs[sl] = R - B @ ghe
            dmap = self.element_dof_map(e)
            for la, (ka, ia) in enumerate(dmap):
                if ka != "int":
                    continue
                K[sl, nz + ia] += B[:, la]
                K[nz + ia, sl] += C[la, :]
                for lb, (kb, ib) in enumerate(dmap):
                    if kb == "int":
                        K[nz + ia, nz + ib] += D[la, lb]
                    else:
                        rhs[nz + ia] -= D[la, lb] * ghe[lb]
        sol = np.linalg.solve(K, rhs)
        u = np.empty(self.uoff[-1])
        q = np.empty(2 * self.uoff[-1])
        for e in range(self.N):
            Q = self.Qe[e]
            U = sol[off[e]:off[e + 1]]
            u[self.uoff[e]:self.uoff[e + 1]] = U[2 * Q:]
            q[2 * self.uoff[e]:2 * self.uoff[e + 1]] = U[:2 * Q]
        return sol[nz:], u, q

    # ------------------------------------------------------------------ errors
    def lattice_points(self, e):
        """Physical coordinates of element e's Q_e lattice nodes."""
        msh = self.sub[int(self.levels[e])].mesh
        v = msh.vertices(e)
        ref = msh.lattice_ref()
        return v[0] + np.outer(ref[:, 0], v[1] - v[0]) + np.outer(ref[:, 1], v[2] - v[0])

    def l2_errors(self, u, q, u_exact, grad_u_exact):
        """L2 errors of u and q = -grad u over all sub-triangles (rule exact to 2p + 6)."""
        p = self.p
        xi_q, eta_q, w_q = triangle_rule(p + 4)
        lam_q = np.column_stack([1.0 - xi_q - eta_q, xi_q, eta_q])
        eu = eq = 0.0
        for e in range(self.N):
            sub = self.sub[int(self.levels[e])]
            msh = sub.mesh
            v = msh.vertices(e)
            ue = u[self.uoff[e]:self.uoff[e + 1]]
            qe = q[2 * self.uoff[e]:2 * self.uoff[e + 1]].reshape(2, -1)
            for tri in msh.sub_triangles():
                alphas, nodes = msh.sub_nodes(tri)
                A, B, C, Js, Jinv, dlam = sub._sub_triangle_data(v, tri)
                phi, _ = tri_lagrange(alphas, p, lam_q, dlam)
                xq = A[None, :] + np.outer(xi_q, B - A) + np.outer(eta_q, C - A)
                wq = w_q * abs(np.linalg.det(Js))
                gx, gy = grad_u_exact(xq[:, 0], xq[:, 1])
                eu += np.sum(wq * (phi @ ue[nodes] - u_exact(xq[:, 0], xq[:, 1])) ** 2)
                eq += np.sum(wq * ((phi @ qe[0][nodes] + gx) ** 2 + (phi @ qe[1][nodes] + gy) ** 2))
        return np.sqrt(eu), np.sqrt(eq)


def band_levels(n, edges=(0.7, 0.8, 0.9), base=1):
    """Levels by band of the element centroid's x: base below edges[0], base + 1 in
    [edges[0], edges[1]), ... (the banded-level workload's rule)."""
    N = 2 * n * n
    out = np.empty(N, dtype=np.int64)
    sk = StructuredMesh(n, 1, 1)
    for e in range(N):
        cx = sk.vertices(e)[:, 0].mean()
        out[e] = base + sum(cx >= t for t in edges)
    return out
