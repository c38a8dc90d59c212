"""Quadrature rules used by the oracle (test infrastructure only).

The paper only says that quadrature is part of element formation (Sec. 6.1);
it fixes no rule. The rules here are:

* Gauss-Legendre on [0, 1], nodes found by Newton's method on the three-term
  Legendre recurrence (no library tables);
* the collapsed (Duffy) product rule on the unit triangle
  {(xi, eta): xi, eta >= 0, xi + eta <= 1}: (xi, eta) = (u (1 - v), v), weight
  w_u w_v (1 - v). With ng points per direction it integrates every
  polynomial of total degree <= 2 ng - 2 exactly.

Point order inside one triangle: v-index major, u-index minor
(index = j * ng + i for u = x_i, v = x_j).
"""
import numpy as np


def gauss_legendre(n):
    """n-point Gauss-Legendre rule on [0, 1]: (nodes ascending, weights)."""
    if n < 1:
        raise ValueError("n must be >= 1")
    t_all = np.empty(n)
    w_all = np.empty(n)
    for i in range(n):
        # Chebyshev-like initial guess for the i-th largest root of P_n
        t = np.cos(np.pi * (i + 0.75) / (n + 0.5))
        for _ in range(200):
            p_prev, p = 1.0, t           # P_0, P_1
            for k in range(2, n + 1):
                p_prev, p = p, ((2 * k - 1) * t * p - (k - 1) * p_prev) / k
            # derivative of P_n from P_n and P_{n-1}
            dp = n * (t * p - p_prev) / (t * t - 1.0)
            dt = p / dp
            t -= dt
            if abs(dt) < 1e-17:
                break
        # recompute derivative at the converged root
        p_prev, p = 1.0, t
        for k in range(2, n + 1):
            p_prev, p = p, ((2 * k - 1) * t * p - (k - 1) * p_prev) / k
        dp = n * (t * p - p_prev) / (t * t - 1.0)
        t_all[i] = t
        w_all[i] = 2.0 / ((1.0 - t * t) * dp * dp)
    order = np.argsort(t_all)
    x = 0.5 * (1.0 + t_all[order])
    w = 0.5 * w_all[order]
    return x, w


def triangle_rule(ng):
    """Collapsed Gauss rule on the unit triangle: arrays xi, eta, w (sum w = 1/2)."""
    x, w = gauss_legendre(ng)
    xi = np.empty(ng * ng)
    eta = np.empty(ng * ng)
    wt = np.empty(ng * ng)
    for j in range(ng):
        for i in range(ng):
            k = j * ng + i
            xi[k] = x[i] * (1.0 - x[j])
            eta[k] = x[j]
            wt[k] = w[i] * w[j] * (1.0 - x[j])
    return xi, eta, wt
