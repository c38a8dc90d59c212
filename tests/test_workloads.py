"""Pins of the seeded synthetic inputs (paper_2302_10917_gb300/workloads.py), CPU only.

The generators feed the oracle and the CUDA path alike, so a mistake in them
would pass every parity test and still change what is measured. Each input
is checked against something independent of its own formula:
  * the manufactured sources f = -kappa Lap u + beta . grad u against
    central differences of the exact solutions (Sec. 4.1's interior layer
    and u = sin(pi x) sin(pi y));
  * the element centroids of the random field and of the level bands
    against the oracle mesh's own vertices;
  * the Gaussian bumps' peak and width at their centres;
  * the diffusivities' range and the random field's spread.
"""
import math

import numpy as np
import pytest
import torch

from oracle.mesh import StructuredMesh
from paper_2302_10917_gb300 import workloads as wl


def _fd_source(u, xy, kappa, beta, h=1e-4):
    """-kappa Lap u + beta . grad u by second-order central differences."""
    ex = torch.tensor([h, 0.0], dtype=xy.dtype)
    ey = torch.tensor([0.0, h], dtype=xy.dtype)
    ux = (u(xy + ex) - u(xy - ex)) / (2 * h)
    uy = (u(xy + ey) - u(xy - ey)) / (2 * h)
    lap = (u(xy + ex) + u(xy - ex) + u(xy + ey) + u(xy - ey) - 4 * u(xy)) / (h * h)
    return -kappa * lap + beta[0] * ux + beta[1] * uy


def _points(k=200, seed=0):
    return torch.rand(k, 2, dtype=torch.float64, generator=torch.Generator().manual_seed(seed)) * 0.9 + 0.05


def test_sin_sin_source_matches_differences():
    xy = _points()
    for kappa, beta in ((1.0, (50 * math.cos(0.3), 50 * math.sin(0.3))), (1e-2, (1.0, 0.0)), (0.3, (0.0, 0.0))):
        f = wl.sin_sin_source(xy, kappa, beta)
        fd = _fd_source(wl.sin_sin_exact, xy, kappa, beta)
        assert (f - fd).abs().max() <= 1e-5 * max(1.0, float(f.abs().max())), (kappa, beta)


def test_tanh_layer_source_matches_differences():
    xy = _points()
    for kappa, beta in ((0.4, (1.0, 1.0)), (0.1, (1.0, 1.0)), (0.25, (0.3, -0.7))):
        f = wl.tanh_layer_source(xy, kappa, beta)
        fd = _fd_source(lambda p: wl.tanh_layer_exact(p, kappa), xy, kappa, beta, h=1e-4 * kappa)
        assert (f - fd).abs().max() <= 1e-5 * max(1.0, float(f.abs().max())), (kappa, beta)
    # the exact solution has the layer on y = 2 x - 0.4 and the range (0, 1)
    x = torch.tensor([[0.5, 0.6]], dtype=torch.float64)
    assert abs(float(wl.tanh_layer_exact(x, 0.05)) - 0.5) < 1e-15


@pytest.mark.parametrize("n", [1, 3, 8])
def test_element_centroids_match_the_mesh(n):
    msh = StructuredMesh(n, 1, 1)
    c = wl.element_centroids(n)
    assert c.shape == (2 * n * n, 2)
    for e in range(2 * n * n):
        v = np.asarray(msh.vertices(e), dtype=np.float64)
        assert np.abs(c[e] - v.mean(axis=0)).max() < 1e-15, e


def test_band_levels_follow_the_centroid_x():
    n = 20
    lev = wl.band_levels(n)
    cx = wl.element_centroids(n)[:, 0]
    expect = 1 + (cx >= 0.7).astype(int) + (cx >= 0.8).astype(int) + (cx >= 0.9).astype(int)
    # band edges fall between centroids here, so the x-only rule is unambiguous
    assert np.min(np.abs(cx[:, None] - np.array([0.7, 0.8, 0.9])[None, :])) > 1e-9
    assert np.array_equal(lev.astype(int), expect)


def test_gaussian_bumps_peak_and_width():
    c = wl.bump_centres(6, seed=3)
    assert c.shape == (6, 2) and (c >= 0).all() and (c < 1).all()
    w = 0.05
    pts = torch.from_numpy(np.concatenate([c, c + np.array([w, 0.0]), c + np.array([0.0, 2 * w])]))
    f = wl.gaussian_bumps(pts, 6, seed=3, width=w)          # [6 sources, 18 points]
    for k in range(6):
        assert abs(float(f[k, k]) - 1.0) < 1e-15
        assert abs(float(f[k, 6 + k]) - math.exp(-0.5)) < 1e-14
        assert abs(float(f[k, 12 + k]) - math.exp(-2.0)) < 1e-14
    assert np.array_equal(wl.bump_centres(6, seed=3), c) and not np.array_equal(wl.bump_centres(6, seed=4), c)


def test_random_kappa_range_and_log_uniform():
    k = wl.random_kappa(20000, seed=1)
    assert k.min() >= 0.5 and k.max() <= 2.0
    lk = np.log(k)
    assert abs(lk.mean()) < 0.02 and abs(lk.std() - np.log(4.0) / math.sqrt(12.0)) < 0.02
    assert np.array_equal(k, wl.random_kappa(20000, seed=1))


def test_random_field_spread_and_correlation():
    """log kappa of the random Fourier features has standard deviation about std and
    stays nearly constant across one element (h = 1/64 << correlation length 0.1)."""
    n = 64
    g = np.log(wl.grf_kappa(n, seed=7))
    assert 0.35 < g.std() < 0.65
    # the two triangles of a square sit h / 3 apart: their values differ far less than std
    assert np.abs(g[0::2] - g[1::2]).mean() < 0.1 * g.std()
    g2 = np.log(wl.grf_kappa(n, seed=8))
    assert abs(np.corrcoef(g, g2)[0, 1]) < 0.3
