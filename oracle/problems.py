"""Analytic solutions and their data for -kappa Lap u + beta . grad u = f (oracle).

Test infrastructure only. Each problem returns callables u(x, y),
grad u(x, y) -> (ux, uy) and f(x, y) = -kappa Lap u + beta . grad u, with
constant kappa and beta (Eq. C21 with a = beta constant).
"""
import numpy as np


def sin_sin(kappa, beta):
    """u = sin(pi x) sin(pi y): the manufactured solution of the workloads."""
    pi = np.pi

    def u(x, y):
        return np.sin(pi * x) * np.sin(pi * y)

    def grad(x, y):
        return (pi * np.cos(pi * x) * np.sin(pi * y), pi * np.sin(pi * x) * np.cos(pi * y))

    def f(x, y):
        ux, uy = grad(x, y)
        return 2.0 * kappa * pi * pi * u(x, y) + beta[0] * ux + beta[1] * uy

    return u, grad, f


def tanh_layer(kappa, beta):
    """Eq. (C24a): u = (1 + tanh((y - 2x + 0.4) / kappa)) / 2, f including beta . grad u."""
    def u(x, y):
        return 0.5 * (1.0 + np.tanh((y - 2.0 * x + 0.4) / kappa))

    def grad(x, y):
        s = 1.0 / np.cosh((y - 2.0 * x + 0.4) / kappa) ** 2
        return (-1.0 * s / kappa, 0.5 * s / kappa)

    def f(x, y):
        z = (y - 2.0 * x + 0.4) / kappa
        s = 1.0 / np.cosh(z) ** 2
        # Lap u = u_xx + u_yy with u_z'' = -s tanh(z) and (dz/dx)^2 + (dz/dy)^2 = 5 / kappa^2
        lap = 0.5 * (-2.0 * s * np.tanh(z)) * 5.0 / kappa ** 2
        ux, uy = grad(x, y)
        return -kappa * lap + beta[0] * ux + beta[1] * uy

    return u, grad, f


def polynomial(coeffs, kappa, beta):
    """u = sum_{a+b<=deg} c_ab x^a y^b with coeffs {(a, b): c_ab}."""
    def u(x, y):
        x = np.asarray(x, dtype=np.float64)
        out = np.zeros_like(x)
        for (a, b), c in coeffs.items():
            out = out + c * x ** a * np.asarray(y, dtype=np.float64) ** b
        return out

    def grad(x, y):
        x = np.asarray(x, dtype=np.float64)
        y = np.asarray(y, dtype=np.float64)
        ux = np.zeros_like(x)
        uy = np.zeros_like(x)
        for (a, b), c in coeffs.items():
            if a > 0:
                ux = ux + c * a * x ** (a - 1) * y ** b
            if b > 0:
                uy = uy + c * b * x ** a * y ** (b - 1)
        return ux, uy

    def f(x, y):
        x = np.asarray(x, dtype=np.float64)
        y = np.asarray(y, dtype=np.float64)
        lap = np.zeros_like(x)
        for (a, b), c in coeffs.items():
            if a > 1:
                lap = lap + c * a * (a - 1) * x ** (a - 2) * y ** b
            if b > 1:
                lap = lap + c * b * (b - 1) * x ** a * y ** (b - 2)
        ux, uy = grad(x, y)
        return -kappa * lap + beta[0] * ux + beta[1] * uy

    return u, grad, f


def random_polynomial(deg, seed):
    """Seeded coefficients of a total-degree-deg polynomial (all monomials present)."""
    rng = np.random.default_rng(seed)
    return {(a, b): float(rng.uniform(-1.0, 1.0))
            for a in range(deg + 1) for b in range(deg + 1 - a)}
