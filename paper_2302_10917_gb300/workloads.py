"""Seeded synthetic workloads (inputs only; none of the method's arithmetic).

The paper's benchmarks are analytic (Sec. 4.1) and its timing runs use 3D
adaptive meshes that are not available, so every workload is synthetic:
structured unit-square macro meshes with the manufactured solution
u = sin(pi x) sin(pi y) (source f = -kappa Lap u + beta . grad u, g_D = 0),
plus seeded random fields for parity tests.
"""
import math

import numpy as np
import torch

MASTER_SEED = 0x230210917

# Workloads (n macro squares per side, m sub-edges per macro-edge, degree p).
CONFIGS = {
    "smoke_n4_m2_p2": dict(n=4, m=2, p=2, beta=(1.0, 1.0), kappa=1.0),
    "n128_m8_p3": dict(n=128, m=8, p=3, beta=(50.0 * math.cos(0.3), 50.0 * math.sin(0.3)), kappa=1.0),
    "n256_m8_p3": dict(n=256, m=8, p=3, beta=(50.0 * math.cos(0.3), 50.0 * math.sin(0.3)), kappa=1.0),
    "n256_m4_p2_grf": dict(n=256, m=4, p=2, beta=(1.0, 0.5), kappa=1.0),
    # many right-hand sides on one level (uniform counterpart of the banded-level workload)
    "n128_m4_p2_64src": dict(n=128, m=4, p=2, beta=(1.0, 0.0), kappa=1e-2),
    # many right-hand sides on levels by band of x (band_levels: r = 1 .. 4, faces at the finer side)
    "levels_n128_p2_64src": dict(n=128, m=0, p=2, beta=(1.0, 0.0), kappa=1e-2, nrhs=64, width=0.05),
}


def band_levels(n, edges=(0.7, 0.8, 0.9), base=1):
    """Refinement level of every macro-triangle by band of its centroid's x: base below
    edges[0], base + 1 in [edges[0], edges[1]), ..., base + len(edges) from edges[-1] on
    (int8 [2 n^2], element order e = 2 (j n + i) + t)."""
    e = np.arange(2 * n * n)
    sq, t = e // 2, e % 2
    i = sq % n
    # centroid x: (2 x_{i+1} + x_i) / 3 for t = 0, (2 x_i + x_{i+1}) / 3 for t = 1
    cx = np.where(t == 0, (3 * i + 2) / (3.0 * n), (3 * i + 1) / (3.0 * n))
    lev = np.full(e.shape, base, dtype=np.int64)
    for th in edges:
        lev += (cx >= th)
    return lev.astype(np.int8)


def sin_sin_source(xy, kappa, beta):
    """f = 2 kappa pi^2 sin(pi x) sin(pi y) + beta . grad(sin(pi x) sin(pi y)) at points xy[..., 2]."""
    x, y = xy[..., 0], xy[..., 1]
    pi = math.pi
    sx, sy = torch.sin(pi * x), torch.sin(pi * y)
    cx, cy = torch.cos(pi * x), torch.cos(pi * y)
    return 2.0 * kappa * pi * pi * sx * sy + beta[0] * pi * cx * sy + beta[1] * pi * sx * cy


def sin_sin_exact(xy):
    return torch.sin(math.pi * xy[..., 0]) * torch.sin(math.pi * xy[..., 1])


def tanh_layer_exact(xy, kappa):
    """The interior-layer benchmark of Sec. 4.1: u = (1 + tanh((y - 2x + 0.4) / kappa)) / 2."""
    return 0.5 * (1.0 + torch.tanh((xy[..., 1] - 2.0 * xy[..., 0] + 0.4) / kappa))


def tanh_layer_source(xy, kappa, beta):
    """f = -kappa Lap u + beta . grad u for the interior layer (beta . grad u is kept: the
    layer is not parallel to beta = (1, 1))."""
    z = (xy[..., 1] - 2.0 * xy[..., 0] + 0.4) / kappa
    t = torch.tanh(z)
    s = 1.0 - t * t                      # sech^2
    lap = -s * t * 5.0 / (kappa * kappa)  # 0.5 * (-2 s t) * |grad z|^2, |grad z|^2 = 5 / kappa^2
    ux, uy = -s / kappa, 0.5 * s / kappa
    return -kappa * lap + beta[0] * ux + beta[1] * uy


def random_kappa(N, seed, lo=0.5, hi=2.0):
    """Per-element diffusivities, log-uniform in [lo, hi]."""
    g = np.random.default_rng([MASTER_SEED, 17, int(seed)])
    return np.exp(g.uniform(np.log(lo), np.log(hi), size=N))


def grf_kappa(n, seed, std=0.5, ell=0.1, features=1024):
    """kappa_e = exp(g(c_e)) at the centroids c_e of the n x n "/"-split mesh, with g a
    Gaussian random field of standard deviation std and squared-exponential
    correlation length ell, drawn as `features` random Fourier features
    g(x) = std sqrt(2 / F) sum_k cos(w_k . x + phi_k), w_k ~ N(0, I / ell^2),
    phi_k ~ U[0, 2 pi) (Rahimi and Recht, 2007)."""
    g = np.random.default_rng([MASTER_SEED, 43, int(seed)])
    w = g.standard_normal((features, 2)) / ell
    phi = g.uniform(0.0, 2.0 * np.pi, features)
    c = element_centroids(n)
    field = std * np.sqrt(2.0 / features) * np.cos(c @ w.T + phi[None, :]).sum(axis=1)
    return np.exp(field)


def element_centroids(n):
    """Centroids [2 n^2, 2] of the macro-triangles of the n x n "/"-split unit square,
    element order e = 2 (j n + i) + t."""
    h = 1.0 / n
    i, j = np.meshgrid(np.arange(n), np.arange(n), indexing="xy")
    i, j = i.ravel(), j.ravel()          # square index j n + i
    c = np.empty((2 * n * n, 2))
    # t = 0: (x_{i+1}, y_j), (x_{i+1}, y_{j+1}), (x_i, y_j); t = 1: (x_i, y_{j+1}), (x_i, y_j), (x_{i+1}, y_{j+1})
    c[0::2, 0] = (i + 2.0 / 3.0) * h
    c[0::2, 1] = (j + 1.0 / 3.0) * h
    c[1::2, 0] = (i + 1.0 / 3.0) * h
    c[1::2, 1] = (j + 2.0 / 3.0) * h
    return c


def gaussian_bumps(xy, count, seed, width=0.05):
    """count sources f_k(x) = exp(-|x - c_k|^2 / (2 width^2)) with seeded centres
    c_k ~ U[0, 1]^2, evaluated at points xy[..., 2]: [count, *xy.shape[:-1]]."""
    c = torch.from_numpy(bump_centres(count, seed)).to(xy.device, xy.dtype)
    d2 = ((xy.unsqueeze(0) - c.view(count, *([1] * (xy.dim() - 1)), 2)) ** 2).sum(-1)
    return torch.exp(-d2 / (2.0 * width * width))


def bump_centres(count, seed):
    """The seeded centres c_k ~ U[0, 1]^2 of gaussian_bumps: [count, 2]."""
    g = np.random.default_rng([MASTER_SEED, 59, int(seed)])
    return g.uniform(0.0, 1.0, (count, 2))


def random_vector(n, seed):
    g = np.random.default_rng([MASTER_SEED, 29, int(seed)])
    return g.standard_normal(n)


def random_directions(count, shape, seed):
    """count seeded standard-normal directions of the given shape: [count, *shape]
    (the perturbation directions of the finite-difference gradient checks)."""
    g = np.random.default_rng([MASTER_SEED, 67, int(seed)])
    return g.standard_normal((count, *shape))
