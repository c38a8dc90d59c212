"""Restarted GMRES for the condensed trace system (oracle, test infrastructure only).

The paper solves Eq. (global_problem) with PETSc GMRES, left-preconditioned by
D^-1 (Sec. 6.1), and reports a "drop tolerance" only. The reading used here:
GMRES(k) from x0 = 0 on D^-1 S x = D^-1 g with modified Gram-Schmidt; the
stopping test is the TRUE relative residual ||g - S x||_2 / ||g||_2 <= tol,
evaluated at every restart and whenever the Arnoldi estimate of the
preconditioned residual has dropped by the requested factor.
"""
import numpy as np


def gmres(apply_S, apply_Dinv, g, tol=1e-10, restart=50, maxit=20000):
    """Returns (x, iterations, true relative residual, converged flag)."""
    n = g.size
    x = np.zeros(n)
    gnorm = np.linalg.norm(g)
    if gnorm == 0.0:
        return x, 0, 0.0, True
    bt_norm = np.linalg.norm(apply_Dinv(g))
    target = tol * bt_norm        # threshold for the Arnoldi estimate
    it = 0
    rel = 1.0
    while it < maxit:
        r = apply_Dinv(g - apply_S(x))
        beta = np.linalg.norm(r)
        V = np.zeros((restart + 1, n))
        H = np.zeros((restart + 1, restart))
        V[0] = r / beta
        k_used = 0
        for j in range(restart):
            w = apply_Dinv(apply_S(V[j]))
            for i in range(j + 1):                    # modified Gram-Schmidt
                H[i, j] = np.dot(w, V[i])
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            it += 1
            k_used = j + 1
            e1 = np.zeros(j + 2)
            e1[0] = beta
            y, *_ = np.linalg.lstsq(H[:j + 2, :j + 1], e1, rcond=None)
            est = np.linalg.norm(e1 - H[:j + 2, :j + 1] @ y)
            if H[j + 1, j] == 0.0 or est <= target or it >= maxit:
                break
            V[j + 1] = w / H[j + 1, j]
        e1 = np.zeros(k_used + 1)
        e1[0] = beta
        y, *_ = np.linalg.lstsq(H[:k_used + 1, :k_used], e1, rcond=None)
        x = x + V[:k_used].T @ y
        rel = np.linalg.norm(g - apply_S(x)) / gnorm
        if rel <= tol:
            return x, it, rel, True
        if est <= target:
            # the preconditioned estimate met its target but the true residual
            # did not: tighten the estimate's target and restart
            target *= 0.5 * tol / rel
    return x, it, rel, False
