"""Pins of the oracle's kernel math against what the paper prints and what
mathematics fixes (Sec. 3, 3.1, 3.2, 3.3, App. B). CPU only."""
import json
import math
import os

import numpy as np
import pytest

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")))
EPS = 1.0 / 255.0

# f1 reading: the paper prints c0 ~ -0.176, c1 ~ 0.773 but every other number
# it gives (root 4.386, 28.45/255, 2.1 sigma, max opacity < 1, Eq. 4/5 real)
# needs c0 = 0.773 and c1 = -0.773 / 4.386.
F1 = (0.773, -0.773 / 4.386)


def _fitted():
    from oracle import fit
    return {1: fit.fit(1, steps=6000), 2: fit.fit(2, steps=6000), 3: fit.fit(3)}


@pytest.fixture(scope="module")
def fitted():
    return _fitted()


def _cfg(orc, kind, coeffs, cull="opacity"):
    return orc.make_config(kind=kind, coeffs=coeffs, cull=cull)


def test_eps_range_and_3dgs_sigma(orc):
    assert GOLD["eps"]["value"] == pytest.approx(EPS, rel=1e-15)
    cfg = _cfg(orc, "exp", (), "universal")
    xmax = orc.xcut(cfg, 1.0)
    assert round(xmax, 2) == GOLD["x_max"]["value"]
    assert round(math.sqrt(xmax), 1) == GOLD["sigma_3dgs"]["value"]


def test_f1_printed_labels_are_swapped(orc):
    """With the labels as printed, max(c1 x + c0, 0) grows with x (it cannot
    approximate a decaying exponential) and its root -c0/c1 = 0.228 contradicts
    the printed 4.386; swapped, the printed numbers agree."""
    c0, c1 = GOLD["f1_printed_c0"]["value"], GOLD["f1_printed_c1"]["value"]
    cfg = _cfg(orc, "poly1", (c0, c1))
    ks = [orc.kernel(cfg, x) for x in np.linspace(0.0, 11.0, 23)]
    assert ks[0] == 0.0 and all(b >= a for a, b in zip(ks, ks[1:])) and ks[-1] > 1.0
    assert -c0 / c1 == pytest.approx(0.228, abs=1e-3)
    # the swapped reading reproduces the other printed numbers
    assert F1[0] == pytest.approx(c1) and F1[1] == pytest.approx(c0, abs=5e-4)


def test_f1_closed_forms(orc):
    cfg = _cfg(orc, "poly1", F1, "universal")
    root = orc.universal_root(cfg)
    assert round(root, 3) == GOLD["f1_root"]["value"]
    assert round(255.0 * math.exp(-root / 2.0), 2) == GOLD["f1_root_exp_value_255"]["value"]
    assert round(math.sqrt(root), 1) == GOLD["f1_root_sigma"]["value"]
    assert orc.kernel(cfg, 0.0) == pytest.approx(F1[0]) and orc.kernel(cfg, 0.0) < 1.0
    # Eq. 5: universal threshold = -c0/c1, independent of opacity
    for o in (0.01, 0.5, 1.0):
        assert orc.xcut(cfg, o) == pytest.approx(-F1[0] / F1[1], rel=1e-14)


def test_f1_fit_reproduces_paper(fitted):
    c = fitted[1]
    assert c[0] == pytest.approx(0.773, abs=5e-3)
    assert c[1] == pytest.approx(-0.176, abs=5e-3)
    assert -c[0] / c[1] == pytest.approx(GOLD["f1_root"]["value"], abs=0.02)


def test_fit_beats_neighbours(fitted):
    """The fitter reaches an L1 minimum: nudging any coefficient raises the loss."""
    from oracle import fit
    for order in (1, 3):
        c = fitted[order]
        base = fit.l1_loss(c, order, n=1 << 14)
        for i in range(order + 1):
            for s in (-1, 1):
                cc = np.array(c)
                cc[i] += s * 0.01 * abs(c[i])
                assert fit.l1_loss(cc, order, n=1 << 14) > base


def test_f3_structure(fitted, orc):
    """Sec. 3.3: strictly monotone cubic with a single real root."""
    c = fitted[3]
    # derivative c1 + 2 c2 x + 3 c3 x^2 has no real zero
    assert (2 * c[2]) ** 2 - 4 * (3 * c[3]) * c[1] < 0
    r = np.roots(c[::-1])
    real = r[np.abs(r.imag) < 1e-9].real
    assert real.size == 1 and 7.0 < real[0] < 8.5
    cfg = _cfg(orc, "poly3", c, "universal")
    assert orc.universal_root(cfg) == pytest.approx(real[0], rel=1e-10)
    # Cardano's real branch: Delta0 < 0 => Delta1^2 - 4 Delta0^3 > 0 for every o
    D0 = c[2] ** 2 - 3 * c[3] * c[1]
    assert D0 < 0
    for o in np.linspace(EPS / c[0] * 1.001, 1.0, 50):
        D1 = 2 * c[2] ** 3 - 9 * c[3] * c[2] * c[1] + 27 * c[3] ** 2 * (c[0] - EPS / o)
        assert D1 * D1 - 4 * D0 ** 3 > 0


def test_f2_structure(fitted, orc):
    """Sec. 3.3 / Eq. 6: the plain parabola rises again; the cut kernel is
    non-negative below its first root and zero from there on. The L1 optimum
    of the cut kernel is tangent to the axis (double root)."""
    c = fitted[2]
    assert c[2] > 0 and c[1] < 0
    disc = c[1] ** 2 - 4 * c[0] * c[2]
    assert abs(disc) < 1e-9
    cfg = _cfg(orc, "poly2", c, "universal")
    x0 = orc.universal_root(cfg)
    assert x0 == pytest.approx(-c[1] / (2 * c[2]), rel=1e-6)
    xs = np.linspace(0.0, 3 * x0, 301)
    k = np.array([orc.kernel(cfg, x) for x in xs])
    assert np.all(k[xs < x0] >= 0) and np.all(k[xs >= x0] == 0)
    plain = np.polyval(c[::-1], xs)
    assert plain[-1] > plain[xs < x0].min() + 0.1  # rises again


def test_fit_losses_order(fitted):
    """Higher orders fit better (Fig. 1, Table 1 trend)."""
    from oracle import fit
    l = [fit.l1_loss(fitted[n], n) for n in (1, 2, 3)]
    assert l[0] > l[1] > l[2]


def _brute_xcut(k, o, xmax=400.0):
    """Largest x with o k(x) >= eps by dense scan + bisection (k decreasing
    on its support), using numpy kernel values only."""
    xs = np.linspace(0.0, xmax, 400001)
    ok = o * k(xs) >= EPS
    if not ok[0]:
        return -1.0
    i = np.nonzero(ok)[0][-1]
    lo, hi = xs[i], xs[min(i + 1, xs.size - 1)]
    for _ in range(80):
        mid = 0.5 * (lo + hi)
        if o * k(np.array([mid]))[0] >= EPS:
            lo = mid
        else:
            hi = mid
    return lo


@pytest.mark.parametrize("order", [0, 1, 2, 3])
def test_opacity_radii_match_brute_force(orc, fitted, order):
    """Eq. 3, Eq. 4, App. B: per-opacity thresholds equal the alpha = eps
    boundary found by brute force."""
    if order == 0:
        kind, c = "exp", ()
        k = lambda x: np.exp(-0.5 * x)
    else:
        kind = {1: "poly1", 2: "poly2", 3: "poly3"}[order]
        c = F1 if order == 1 else tuple(fitted[order])
        cc = np.array(c)
        if order == 2:
            x0 = -cc[1] / (2 * cc[2])
            k = lambda x: np.where(x < x0, np.polyval(cc[::-1], x), 0.0)
        else:
            k = lambda x: np.maximum(np.polyval(cc[::-1], x), 0.0)
    cfg = _cfg(orc, kind, c, "opacity")
    k0 = 1.0 if order == 0 else c[0]
    for o in (EPS / k0 * 1.01, 0.01, 0.1, 0.5, 0.99, 1.0):
        got = orc.xcut(cfg, o)
        want = _brute_xcut(k, o)
        assert got == pytest.approx(want, rel=1e-9, abs=1e-9), (o, got, want)
    # no support at all below eps / k(0)
    assert orc.xcut(cfg, EPS / k0 * 0.99) < 0


def test_quadratic_and_cardano_against_numpy_roots(orc):
    rng = np.random.default_rng(5)
    for _ in range(200):
        c = rng.normal(size=4)
        for order in (2, 3):
            got = orc.first_root(c, order, 0.0)
            r = np.roots(c[:order + 1][::-1])
            real = np.sort(r[np.abs(r.imag) < 1e-7 * np.maximum(1, np.abs(r))].real)
            pos = real[real > 0]
            if pos.size == 0:
                assert got == math.inf
            else:
                assert got == pytest.approx(pos[0], rel=1e-7, abs=1e-9)


def test_kernel_values_at_zero_and_support(orc, fitted):
    """k(0) = 1 for exp and c0 for the polynomials; zero from the
    closed-form support on (Sec. 3.1, Eq. 5, Eq. 6)."""
    assert orc.kernel(_cfg(orc, "exp", ()), 0.0) == 1.0
    for kind, c in (("poly1", F1), ("poly2", fitted[2]), ("poly3", fitted[3])):
        cfg = _cfg(orc, kind, c)
        assert orc.kernel(cfg, 0.0) == pytest.approx(c[0])
        x0 = orc.universal_root(cfg)
        for x in (x0, x0 * 1.0001, x0 + 1, 2 * x0, 50.0):
            assert orc.kernel(cfg, x) == 0.0
        assert orc.kernel(cfg, 0.999 * x0) > 0.0


def test_npu_component_count():
    """Sec. 5.1: n_c = binom(2(N+1), 2)."""
    for n, want in GOLD["npu_components"]["value"].items():
        assert math.comb(2 * (int(n) + 1), 2) == want
