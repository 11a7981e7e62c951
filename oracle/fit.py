"""Coefficient fit of Sec. 3.1 — TEST INFRASTRUCTURE (oracle side).

The paper fits the kernel coefficients c_i by gradient descent on an L1 loss
against g(x) = exp(-x/2), with x sampled uniformly on [0, -2 ln eps],
eps = 1/255 (Sec. 3.1: uniform area sampling of the projected ellipse makes
the quadric uniform). This module restates that procedure in float64 numpy:

* samples: the midpoint grid of n points on [0, -2 ln eps] (a stratified
  uniform sample, deterministic);
* loss: mean |k(x) - g(x)| with k the kernel as rendered — f_N = max(poly, 0)
  (Eq. 2) for orders 1 and 3; for order 2 the cut kernel f'_2 of Eq. 6;
* optimiser: Adam on the (sub)gradient, coefficients rescaled to the unit
  interval (u = x / x_max) so that one step size suits every order.

f'_2 reading: with the cut inside the loss, the L1 optimum sits on the
boundary where the parabola's discriminant is zero (a parabola tangent to the
axis at x0), so the fit is run directly over that family,
f'_2(x) = a (x0 - x)^2 for x < x0, i.e. c = (a x0^2, -2 a x0, a).

Parity: the paper prints c0 and c1 of f1 (with their labels swapped) and the
root 4.386; the f'_2 and f3 values are not printed (parity unpinned for them).
"""
from __future__ import annotations

import numpy as np

EPS = 1.0 / 255.0


def x_max(eps: float = EPS) -> float:
    """Upper end of the fitted range, -2 ln eps (Sec. 3.1)."""
    return -2.0 * np.log(eps)


def samples(n: int = 1 << 14, eps: float = EPS) -> np.ndarray:
    X = x_max(eps)
    return (np.arange(n, dtype=np.float64) + 0.5) / n * X


def _adam(grad_fn, p0, steps, lr0, lr1):
    p = np.array(p0, dtype=np.float64)
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    b1, b2 = 0.9, 0.999
    for t in range(1, steps + 1):
        g = grad_fn(p)
        m = b1 * m + (1 - b1) * g
        v = b2 * v + (1 - b2) * g * g
        lr = lr1 + 0.5 * (lr0 - lr1) * (1 + np.cos(np.pi * (t - 1) / steps))
        p -= lr * (m / (1 - b1 ** t)) / (np.sqrt(v / (1 - b2 ** t)) + 1e-12)
    return p


def l1_loss(c, order: int, n: int = 1 << 16, eps: float = EPS) -> float:
    """mean |k(x) - g(x)| on the sample grid for the kernel of this order."""
    x = samples(n, eps)
    g = np.exp(-0.5 * x)
    return float(np.mean(np.abs(kernel_values(c, order, x) - g)))


def kernel_values(c, order: int, x):
    c = np.asarray(c, dtype=np.float64)
    p = sum(c[i] * x ** i for i in range(order + 1))
    if order == 2:
        x0 = first_root_quadratic(c)
        return np.where(x < x0, p, 0.0)
    return np.maximum(p, 0.0)


def first_root_quadratic(c) -> float:
    """First positive root of c0 + c1 x + c2 x^2 (discriminant clamped at 0
    for the tangent fit)."""
    c0, c1, c2 = (float(v) for v in c[:3])
    disc = max(c1 * c1 - 4 * c0 * c2, 0.0)
    r = sorted([(-c1 - np.sqrt(disc)) / (2 * c2), (-c1 + np.sqrt(disc)) / (2 * c2)])
    r = [v for v in r if v > 0]
    return r[0] if r else np.inf


def fit(order: int, n: int = 1 << 14, steps: int = 20000, eps: float = EPS) -> np.ndarray:
    """Fit k of the given order (1, 2 = f'_2 tangent family, 3) to g by L1."""
    x = samples(n, eps)
    X = x_max(eps)
    u = x / X
    g = np.exp(-0.5 * x)
    if order in (1, 3):
        # initial guess: the L2 fit of poly to g on the same grid
        V = np.stack([u ** i for i in range(order + 1)], axis=1)
        d0 = np.linalg.lstsq(V, g, rcond=None)[0]

        def grad(d):
            p = V @ d
            f = np.maximum(p, 0.0)
            s = np.sign(f - g) * (p > 0)
            return V.T @ s / n

        d = _adam(grad, d0, steps, 5e-2, 1e-5)
        return np.array([d[i] / X ** i for i in range(order + 1)])
    if order == 2:
        # f'_2(x) = a (x0 - x)^2 on x < x0, in unit-interval variables
        def grad(p):
            a, z0 = p
            inside = u < z0
            w = np.where(inside, (z0 - u), 0.0)
            f = a * w * w
            s = np.sign(f - g)
            return np.array([np.sum(s * w * w), np.sum(s * 2 * a * w)]) / n

        a, z0 = _adam(grad, [1.0, 0.6], steps, 5e-2, 1e-5)
        A, x0 = a / X ** 2, z0 * X
        return np.array([A * x0 * x0, -2 * A * x0, A])
    raise ValueError("order must be 1, 2 or 3")


def x_max_tile(tile: float, eps: float = EPS, v: float = 0.3) -> float:
    """App. A: the largest quadric a tile-culled renderer evaluates. A splat
    with opacity 1 and smallest scale s_min = sqrt(v) (the floor the AA
    dilation v puts on every scale) that barely touches a tile corner with its
    eps cut-off, p_c = s_min sqrt(-2 ln eps) from its centre along the tile
    diagonal, is still evaluated at the opposite corner, sqrt(2) p_t further:
    x_max = ((p_c + sqrt(2) p_t) / s_min)^2."""
    s_min = np.sqrt(v)
    p_c = s_min * np.sqrt(-2.0 * np.log(eps))
    return float(((p_c + np.sqrt(2.0) * tile) / s_min) ** 2)


def range_samples(X: float, eps: float = EPS, n_core: int = 1 << 14, n_tail: int = 1 << 12):
    """Midpoints and weights (interval width / X) of a grid on [0, X]: dense
    on [0, -2 ln eps] where g is not negligible, coarse beyond. The weighted
    sum is the same mean over x uniform on [0, X] as the uniform sampling of
    Sec. 3.1, with fewer points where the integrand is flat."""
    xe = min(x_max(eps), X)
    a = (np.arange(n_core) + 0.5) / n_core * xe
    wa = np.full(n_core, xe / n_core)
    if X <= xe:
        return a, wa / X
    b = xe + (np.arange(n_tail) + 0.5) / n_tail * (X - xe)
    wb = np.full(n_tail, (X - xe) / n_tail)
    return np.concatenate([a, b]), np.concatenate([wa, wb]) / X


def fit_f2_range(tile: float, steps: int = 20000, eps: float = EPS, v: float = 0.3) -> np.ndarray:
    """App. A alternative to the cut of Eq. 6: f2(x) = max(c0 + c1 x + c2 x^2, 0)
    (Eq. 2) fitted by the Sec. 3.1 L1 procedure over [0, x_max_tile(tile)]
    instead of [0, -2 ln eps], so that the parabola does not rise above zero
    again anywhere a tile-culled renderer evaluates it.

    Reading: over [0, -2 ln eps] alone the L1 optimum has its two roots
    together (the tangent parabola of the Eq. 6 fit, root 6.37), so over the
    extended range the tail binds and the optimum puts the second root at
    x_max exactly: f2(x) = c0 (1 - x / r) (1 - x / x_max) on [0, x_max]. The
    fit is run over (c0, r) in that family (both well scaled), Adam on the
    L1 subgradient as in fit()."""
    X = x_max_tile(tile, eps, v)
    x, w = range_samples(X, eps)
    g = np.exp(-0.5 * x)
    xe = x_max(eps)

    def grad(p):
        c0, z = p  # z = r / (-2 ln eps)
        r = z * xe
        a = 1.0 - x / r
        b = 1.0 - x / X
        f = c0 * a * b
        s = np.sign(np.maximum(f, 0.0) - g) * (f > 0) * w
        return np.array([np.sum(s * a * b), np.sum(s * c0 * b * x / (r * r) * xe)])

    c0, z = _adam(grad, [0.773, 4.386 / xe], steps, 2e-2, 1e-6)
    r = z * xe
    return np.array([c0, -c0 * (1.0 / r + 1.0 / X), c0 / (r * X)])


def roots_quadratic(c):
    """Real roots of c0 + c1 x + c2 x^2, ascending (numpy)."""
    r = np.roots([c[2], c[1], c[0]]) if c[2] != 0 else np.array([-c[0] / c[1]])
    return np.sort(r[np.isreal(r)].real)


if __name__ == "__main__":
    for N in (1, 2, 3):
        c = fit(N)
        print(N, repr(c), l1_loss(c, N))
