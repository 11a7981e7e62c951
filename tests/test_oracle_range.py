"""Pins of the App. A fitting-range extension of f2 (oracle/fit.py:
x_max_tile, fit_f2_range) against geometry and the definition of the fit,
not against the oracle's own formulas."""
import json
import os

import numpy as np
import pytest

from oracle import fit

HERE = os.path.dirname(os.path.abspath(__file__))
COEFFS = json.load(open(os.path.join(HERE, "golden", "coeffs.json")))
EPS = 1.0 / 255.0
XE = -2.0 * np.log(EPS)  # the exp cut-off in quadric units, 11.08


def _max_quadric_over_touched_tiles(tile, s_min, rng, n=4000):
    """Brute force over splats of smallest scale s_min: random orientation,
    larger scale and centre; keep those whose eps support {Q <= XE} reaches
    the tile [0, tile]^2 (dense grid) and return the largest Q any of them
    takes on the tile (a convex Q peaks at a corner)."""
    g = np.linspace(0.0, tile, 129)
    P = np.stack(np.meshgrid(g, g), -1).reshape(-1, 2)
    corners = np.array([[0, 0], [tile, 0], [0, tile], [tile, tile]], float)
    best = 0.0
    for _ in range(n):
        th = rng.uniform(0, np.pi)
        s_big = s_min * np.exp(rng.uniform(0, 4))
        R = np.array([[np.cos(th), -np.sin(th)], [np.sin(th), np.cos(th)]])
        Si = R @ np.diag([1 / s_min ** 2, 1 / s_big ** 2]) @ R.T
        reach = np.sqrt(XE) * s_big
        c = rng.uniform(-reach, tile + reach, 2)
        d = P - c
        if np.min(np.einsum("ni,ij,nj->n", d, Si, d)) > XE:
            continue
        dc = corners - c
        best = max(best, float(np.max(np.einsum("ni,ij,nj->n", dc, Si, dc))))
    return best


@pytest.mark.parametrize("tile", [8, 16])
def test_x_max_is_the_largest_quadric_a_touched_tile_evaluates(tile):
    s_min = np.sqrt(0.3)
    X = fit.x_max_tile(tile)
    rng = np.random.default_rng(tile)
    got = _max_quadric_over_touched_tiles(tile, s_min, rng)
    assert got <= X * (1 + 1e-9)
    # the configuration App. A describes: small axis along the diagonal, the
    # support touching the corner (0, 0) from outside; measured geometrically
    u = np.array([1.0, 1.0]) / np.sqrt(2.0)
    Si = np.outer(u, u) / s_min ** 2 + np.outer([u[1], -u[0]], [u[1], -u[0]]) / 25.0
    c = -u * np.sqrt(XE / (u @ Si @ u))  # Q(corner) = XE exactly
    d = np.array([tile, tile], float) - c
    assert (0.0 - c) @ Si @ (0.0 - c) == pytest.approx(XE, rel=1e-12)
    assert d @ Si @ d == pytest.approx(X, rel=1e-12)
    assert got > 0.98 * X  # and random search comes within 2% of it


def _l1_uniform(c, lo, hi, n=400000):
    """mean |max(poly, 0) - exp(-x/2)| on a uniform midpoint grid of [lo, hi]."""
    x = lo + (np.arange(n) + 0.5) / n * (hi - lo)
    p = c[0] + c[1] * x + c[2] * x * x
    return float(np.mean(np.abs(np.maximum(p, 0.0) - np.exp(-0.5 * x))))


@pytest.mark.parametrize("tile", ["8", "16"])
def test_f2_range_fit_is_a_local_optimum_of_the_extended_l1(tile):
    c = np.array(COEFFS["poly2_range"][tile][:3])
    X = fit.x_max_tile(int(tile))
    r = np.sort(np.roots([c[2], c[1], c[0]]).real)
    # both roots real and the second one at the end of the range: the
    # parabola never rises above zero where a tile renderer evaluates it
    assert 0 < r[0] < XE and r[1] == pytest.approx(X, rel=1e-6)
    base = _l1_uniform(c, 0.0, X)
    for i, h in ((0, 1e-3), (1, 1e-4), (2, 1e-6 * c[2] / 1e-4)):
        for sgn in (-1, 1):
            cc = c.copy()
            cc[i] += sgn * h
            assert _l1_uniform(cc, 0.0, X) >= base - 1e-9, (i, sgn)


def test_f2_range_tile_dependence():
    """Smaller tiles leave room for curvature, so the fit on the kernel's own
    range improves; at 16 pixels it is almost f1 (App. A)."""
    l8 = _l1_uniform(COEFFS["poly2_range"]["8"], 0.0, XE)
    l16 = _l1_uniform(COEFFS["poly2_range"]["16"], 0.0, XE)
    f1 = _l1_uniform([0.773, -0.773 / 4.386, 0.0], 0.0, XE)
    tangent = COEFFS["l1_loss"]["poly2"]
    assert tangent < l8 < l16 < f1
    assert (f1 - l16) / f1 < 0.005
    for t in ("8", "16"):
        c = COEFFS["poly2_range"][t]
        x = np.linspace(0, np.sort(np.roots([c[2], c[1], c[0]]).real)[0], 1000)
        assert np.all(c[1] + 2 * c[2] * x < 0)  # decreasing up to its first root
