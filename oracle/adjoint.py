"""Adjoint gradient of a functional of u (oracle, test infrastructure only).

Not in the paper: the gradient of J(u) with respect to the per-element
diffusivity kappa_e and the source values f at the quadrature points, for the
discrete problem of Eq. (D) (full local systems, q included).

With K(kappa) X = R(f) the block system of Eq. (D) (local unknowns U_e, trace
unknowns v^, Dirichlet trace g^ fixed), the adjoint state solves
K^T Lambda = dJ/dX = [(0, 0, r_e)_e ; 0], r_e = dJ/du_e, and
    dJ/dkappa_e = -Lambda_e^T (dK_e/dkappa_e) X_e,
    dJ/df_{e,q} = Lambda_{u,e} . (w_q phi(x_q)).
The element blocks are affine in kappa_e (tau_e = kappa_e / tau_len + |beta|),
so dK_e/dkappa_e = K_e(kappa_e + 1) - K_e(kappa_e) exactly. K^T is condensed
like K (Eq. global_problem with transposed blocks) and the trace system
S^T nu = -sum L^T B^T A^-T rho is solved densely (small meshes).
"""
import numpy as np

from .hdg import HDGProblem


def forward(pr: HDGProblem, f_qp, gD_qp=None):
    """Direct solve: trace X, full local vectors U_e (3Q), u [N, Q], g^."""
    S_el, g, g_hat = pr.condense(f_qp, gD_qp)
    X = np.linalg.solve(pr.assemble_S(S_el), g)
    msh = pr.mesh
    U = []
    for e in range(msh.N):
        A, B, _, _ = pr.local_blocks(e)
        R = pr.load_vector(e, f_qp[e])
        U.append(np.linalg.solve(A, R - B @ pr.element_trace(e, X, g_hat)))
    Q = msh.Q
    u = np.stack([Ue[2 * Q:] for Ue in U])
    return X, U, u, g_hat


def gradient(pr: HDGProblem, f_qp, r, gD_qp=None, return_state=False):
    """dJ/dkappa [N] and dJ/df [N, n_qp] for dJ/du = r [N, Q] (and u [N, Q]); with
    return_state also a dict of the adjoint right-hand side g_adj [N_tr], the
    trace adjoint nu [N_tr] and the u-part of Lambda [N, Q]."""
    assert not pr.supg, "the kappa-derivative below assumes blocks affine in kappa (no SUPG)"
    msh = pr.mesh
    Q, n_t = msh.Q, msh.n_t
    X, U, u, g_hat = forward(pr, f_qp, gD_qp)
    # adjoint condensation with transposed element blocks
    St = np.zeros((msh.N_tr, msh.N_tr))
    gadj = np.zeros(msh.N_tr)
    zero_bnd = np.zeros((msh.n_bnd_edges, msh.P1))
    trans = []
    for e in range(msh.N):
        A, B, C, D = pr.local_blocks(e)
        rho = np.zeros(3 * Q)
        rho[2 * Q:] = r[e]
        Se_T = D.T - B.T @ np.linalg.solve(A.T, C.T)
        ge = -B.T @ np.linalg.solve(A.T, rho)
        trans.append((A, C, rho))
        dmap = msh.element_dof_map(e)
        for la, (ka, ia) in enumerate(dmap):
            if ka != "int":
                continue
            gadj[ia] += ge[la]
            for lb, (kb, ib) in enumerate(dmap):
                if kb == "int":
                    St[ia, ib] += Se_T[la, lb]
    nu = np.linalg.solve(St, gadj)
    _, wts = pr.quad_points()
    gk = np.zeros(msh.N)
    gf = np.zeros((msh.N, wts.shape[1]))
    lam_u = np.zeros((msh.N, Q))
    for e in range(msh.N):
        A, C, rho = trans[e]
        nu_e = pr.element_trace(e, nu, zero_bnd)
        lam = np.linalg.solve(A.T, rho - C.T @ nu_e)
        lam_u[e] = lam[2 * Q:]
        x_e = pr.element_trace(e, X, g_hat)
        A0, B0, C0, D0 = pr.blocks_at(e, pr.kappa[e])
        A1, B1, C1, D1 = pr.blocks_at(e, pr.kappa[e] + 1.0)
        dA, dB, dC, dD = A1 - A0, B1 - B0, C1 - C0, D1 - D0
        gk[e] = -(lam @ (dA @ U[e] + dB @ x_e)) - nu_e @ (dC @ U[e] + dD @ x_e)
        em = pr.element_matrices(e)
        gf[e] = wts[e] * (em["Phi"] @ lam[2 * Q:])
    if return_state:
        return gk, gf, u, dict(g_adj=gadj, nu=nu, mu=lam_u)
    return gk, gf, u
