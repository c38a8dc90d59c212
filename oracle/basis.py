"""Lagrange bases used by the oracle (test infrastructure only).

Section 3.2 of the paper: W(K), V(K) are C0 piecewise P_p on the
sub-triangulation of a macro-element, M(F) is C0 piecewise P_p on the
sub-edges of a macro-edge. The nodal (Lagrange) basis on equispaced points is
the reading adopted for the unspecified basis.

P_p Lagrange basis on one triangle, in barycentric coordinates lambda_k, for
the node with multi-index alpha (|alpha| = p, node at alpha / p):
    phi_alpha = prod_k prod_{j < alpha_k} (p lambda_k - j) / (j + 1).
"""
import numpy as np


def tri_lagrange(alphas, p, lam, dlam):
    """Values and physical gradients of the P_p Lagrange basis on one triangle.

    alphas : list of multi-indices (a0, a1, a2), sum p
    lam    : (npts, 3) barycentric coordinates of the evaluation points
    dlam   : (3, 2) physical gradients of lambda_0..2 (constant on the triangle)
    returns phi (npts, nb), grad (npts, nb, 2)
    """
    npts = lam.shape[0]
    nb = len(alphas)
    phi = np.ones((npts, nb))
    grad = np.zeros((npts, nb, 2))
    for b, alpha in enumerate(alphas):
        # factor_k(lambda_k) = prod_{j < alpha_k} (p lambda_k - j) / (j + 1)
        fac = np.ones((npts, 3))
        dfac = np.zeros((npts, 3))
        for k in range(3):
            f = np.ones(npts)
            df = np.zeros(npts)
            for j in range(alpha[k]):
                g = (p * lam[:, k] - j) / (j + 1)
                dg = p / (j + 1)
                df = df * g + f * dg
                f = f * g
            fac[:, k] = f
            dfac[:, k] = df
        phi[:, b] = fac[:, 0] * fac[:, 1] * fac[:, 2]
        d0 = dfac[:, 0] * fac[:, 1] * fac[:, 2]
        d1 = fac[:, 0] * dfac[:, 1] * fac[:, 2]
        d2 = fac[:, 0] * fac[:, 1] * dfac[:, 2]
        grad[:, b, :] = (d0[:, None] * dlam[0][None, :] + d1[:, None] * dlam[1][None, :]
                         + d2[:, None] * dlam[2][None, :])
    return phi, grad


def tri_lagrange_laplacian(alphas, p, lam, dlam):
    """Physical Laplacian of the P_p Lagrange basis on one triangle at the points
    lam: Lap phi = sum_{k,l} (d^2 phi / d lambda_k d lambda_l) (grad lambda_k . grad lambda_l)
    (the lambda_k are affine). Returns (npts, nb)."""
    npts = lam.shape[0]
    G = dlam @ dlam.T                       # grad lambda_k . grad lambda_l
    out = np.zeros((npts, len(alphas)))
    for b, alpha in enumerate(alphas):
        f = np.ones((npts, 3))
        d1 = np.zeros((npts, 3))
        d2 = np.zeros((npts, 3))
        for k in range(3):
            v = np.ones(npts)
            dv = np.zeros(npts)
            ddv = np.zeros(npts)
            for j in range(alpha[k]):
                g = (p * lam[:, k] - j) / (j + 1)
                dg = p / (j + 1)
                ddv = ddv * g + 2.0 * dv * dg
                dv = dv * g + v * dg
                v = v * g
            f[:, k], d1[:, k], d2[:, k] = v, dv, ddv
        lap = np.zeros(npts)
        for k in range(3):
            for l in range(3):
                if k == l:
                    o = [t for t in range(3) if t != k]
                    h = d2[:, k] * f[:, o[0]] * f[:, o[1]]
                else:
                    o = 3 - k - l
                    h = d1[:, k] * d1[:, l] * f[:, o]
                lap += h * G[k, l]
        out[:, b] = lap
    return out


def line_lagrange(p, s):
    """P_p Lagrange basis on [0, 1] with nodes k / p, evaluated at points s."""
    s = np.asarray(s, dtype=np.float64)
    out = np.ones((s.size, p + 1))
    nodes = np.arange(p + 1) / p
    for k in range(p + 1):
        for j in range(p + 1):
            if j != k:
                out[:, k] *= (s - nodes[j]) / (nodes[k] - nodes[j])
    return out
