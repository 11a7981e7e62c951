"""Pins of the oracle's projection, anti-aliasing, compositing, culling and
reverse pass against closed forms, library routines, quadrature, brute force
and finite differences. CPU only."""
import json
import math
import os

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

from paper_2603_18707_b300 import synth

EPS = 1.0 / 255.0
_CO = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "coeffs.json")))
F1 = tuple(_CO["poly1"][:2])
F2 = tuple(_CO["poly2"][:3])
F3 = tuple(_CO["poly3"])
KINDS = {"exp": (), "poly1": F1, "poly2": F2, "poly3": F3}


def _one_splat(mean, scale, quat=(1, 0, 0, 0), opacity=0.8, dc=(0.3, -0.2, 0.1)):
    return {"means": np.array([mean], float), "scales": np.array([scale], float),
            "quats": np.array([quat], float), "opacities": np.array([opacity], float),
            "sh": np.array([[dc]], float), "sh_degree": 0}


def _cam(orc, W=64, H=48, fov=60.0, pos=(0.0, 0.0, -3.0)):
    return orc.camera_from_dict(synth.look_at(pos, [0, 0, 0], W, H, fov))


def test_sh_basis_orthonormal(orc):
    """Real SH basis functions are orthonormal on the sphere (Gauss-Legendre
    in cos(theta) x uniform in phi, exact for these polynomial degrees)."""
    nt, nphi = 16, 32
    ct, wt = np.polynomial.legendre.leggauss(nt)
    phi = (np.arange(nphi) + 0.5) * 2 * np.pi / nphi
    G = np.zeros((16, 16))
    for c, w in zip(ct, wt):
        st = math.sqrt(1 - c * c)
        for p in phi:
            Y = orc.sh_basis(3, [st * math.cos(p), st * math.sin(p), c])
            G += w * (2 * np.pi / nphi) * np.outer(Y, Y)
    assert np.allclose(G, np.eye(16), atol=1e-12)


def _real_sh_from_scipy(degree, d):
    """Real SH built independently from scipy's complex Y_l^m (which carries
    the Condon-Shortley phase): m = 0 -> Y_l^0; m > 0 -> sqrt(2) Re Y_l^m;
    m < 0 -> sqrt(2) Im Y_l^|m|; bands in order m = -l .. l."""
    from scipy.special import sph_harm_y
    theta = math.acos(max(-1.0, min(1.0, d[2])))
    phi = math.atan2(d[1], d[0]) % (2 * math.pi)
    out = []
    for l in range(degree + 1):
        for m in range(-l, l + 1):
            y = complex(sph_harm_y(l, abs(m), theta, phi))
            out.append(y.real if m == 0 else math.sqrt(2) * (y.real if m > 0 else y.imag))
    return np.array(out)


def test_sh_basis_matches_scipy_real_harmonics(orc):
    """Order and sign of every basis function within each band, against
    real harmonics assembled from scipy's associated-Legendre based Y_l^m
    (orthonormality alone would accept a swapped order or a flipped sign)."""
    rng = np.random.default_rng(7)
    for _ in range(50):
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        assert orc.sh_basis(3, d) == pytest.approx(_real_sh_from_scipy(3, d), abs=1e-13)


def test_sh_basis_worked_directions(orc):
    """Hand values: along +z only the m = 0 functions survive,
    sqrt((2l+1)/(4 pi)); along +x band 1 is (0, 0, -sqrt(3/(4 pi))) and
    along +y it is (-sqrt(3/(4 pi)), 0, 0) (3DGS's -y, z, -x order)."""
    Yz = orc.sh_basis(3, [0.0, 0.0, 1.0])
    want = np.zeros(16)
    for l, k in ((0, 0), (1, 2), (2, 6), (3, 12)):
        want[k] = math.sqrt((2 * l + 1) / (4 * math.pi))
    assert Yz == pytest.approx(want, abs=1e-15)
    c1 = math.sqrt(3 / (4 * math.pi))
    assert orc.sh_basis(1, [1.0, 0.0, 0.0])[1:] == pytest.approx([0.0, 0.0, -c1], abs=1e-15)
    assert orc.sh_basis(1, [0.0, 1.0, 0.0])[1:] == pytest.approx([-c1, 0.0, 0.0], abs=1e-15)
    # band 2 at (x, y, z) = (1, 1, 0)/sqrt(2): xy term 0.5 sqrt(15/pi) / 2, (x^2 - y^2) term 0
    Y = orc.sh_basis(2, [1 / math.sqrt(2), 1 / math.sqrt(2), 0.0])
    assert Y[4] == pytest.approx(0.25 * math.sqrt(15 / math.pi), abs=1e-15)
    assert Y[8] == pytest.approx(0.0, abs=1e-15)


def test_projection_jacobian_clamped_outside_frustum(orc):
    """Means whose tx/tz or ty/tz lie beyond 1.3 tan(fov/2) (3DGS): Sigma'
    uses the pinhole Jacobian at the clamped point (tx, ty clamped to
    +-1.3 tan(fov/2) tz, same depth), taken here numerically from the plain
    pinhole map, while mu' stays the unclamped projection. The unclamped
    numerical Jacobian gives a different Sigma' (the branch is reached)."""
    cam = _cam(orc, 80, 60, fov=60.0)
    vm = np.array(cam.viewmat[:]).reshape(4, 4)
    R, tv = vm[:3, :3], vm[:3, 3]
    limx, limy = 1.3 * 0.5 * cam.width / cam.fx, 1.3 * 0.5 * cam.height / cam.fy
    rng = np.random.default_rng(5)
    h = 1e-6
    for ux, uy in ((2.0, 0.1), (-1.5, -0.2), (0.2, 1.4), (-0.1, -2.5), (1.9, -1.7)):
        tz = 2.5
        t = np.array([ux * tz, uy * tz, tz])
        mu = R.T @ (t - tv)
        s = np.exp(rng.normal(-2.5, 0.3, 3))
        q = rng.normal(size=4)
        out = orc.splats_to_numpy(orc.project(_one_splat(mu, s, q), cam,
                                              orc.make_config("exp", (), "universal")), 1)
        Rm = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
        Sig = Rm @ np.diag(s * s) @ Rm.T
        tc = np.array([np.clip(ux, -limx, limx) * tz, np.clip(uy, -limy, limy) * tz, tz])
        mc = R.T @ (tc - tv)

        def jac(p):
            return np.stack([(_pinhole(cam, p + h * e) - _pinhole(cam, p - h * e)) / (2 * h)
                             for e in np.eye(3)], axis=1)

        Jc, Ju = jac(mc), jac(mu)
        Sc, Su = Jc @ Sig @ Jc.T, Ju @ Sig @ Ju.T
        got = out["cov2d"][0]
        assert got == pytest.approx([Sc[0, 0], Sc[0, 1], Sc[1, 1]], rel=1e-6, abs=1e-9)
        assert not np.allclose(got, [Su[0, 0], Su[0, 1], Su[1, 1]], rtol=1e-3, atol=0)
        assert out["mean2d"][0] == pytest.approx(_pinhole(cam, mu), abs=1e-9)


def test_projection_on_axis_identity_rotation(orc):
    """Identity quaternion => Sigma = diag(s^2); on the optical axis
    J = diag(f/z) so Sigma' = diag((f s_x / z)^2, (f s_y / z)^2)."""
    cam = _cam(orc, 64, 64)
    sc = _one_splat([0, 0, 0], [0.05, 0.02, 0.04])
    s = orc.splats_to_numpy(orc.project(sc, cam, orc.make_config("exp", (), "universal")), 1)
    f, z = cam.fx, 3.0
    assert s["cov2d"][0] == pytest.approx([(f * 0.05 / z) ** 2, 0.0, (f * 0.02 / z) ** 2], abs=1e-12)
    assert s["mean2d"][0] == pytest.approx([32.0, 32.0], abs=1e-12)
    assert s["depth"][0] == pytest.approx(3.0)


def _pinhole(cam, p):
    vm = np.array(cam.viewmat[:]).reshape(4, 4)
    t = vm[:3, :3] @ p + vm[:3, 3]
    return np.array([cam.fx * t[0] / t[2] + cam.cx, cam.fy * t[1] / t[2] + cam.cy])


def test_projection_matches_numerical_jacobian(orc):
    """Sigma' = J W Sigma W^T J^T equals the covariance pushed through the
    numerical Jacobian of the pinhole map; Sigma from scipy's rotation."""
    rng = np.random.default_rng(3)
    cam = orc.camera_from_dict(synth.look_at([1.0, -0.5, -4.0], [0, 0, 0], 96, 64, 60.0))
    for _ in range(20):
        mu = rng.uniform(-0.6, 0.6, 3)
        s = np.exp(rng.normal(-2.5, 0.4, 3))
        q = rng.normal(size=4)
        sc = _one_splat(mu, s, q)
        out = orc.splats_to_numpy(orc.project(sc, cam, orc.make_config("exp", (), "universal")), 1)
        Rm = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
        Sig = Rm @ np.diag(s * s) @ Rm.T
        h = 1e-6
        Jn = np.stack([(_pinhole(cam, mu + h * e) - _pinhole(cam, mu - h * e)) / (2 * h)
                       for e in np.eye(3)], axis=1)
        Sp = Jn @ Sig @ Jn.T
        assert out["cov2d"][0] == pytest.approx([Sp[0, 0], Sp[0, 1], Sp[1, 1]], rel=1e-6, abs=1e-9)
        assert out["mean2d"][0] == pytest.approx(_pinhole(cam, mu), abs=1e-9)


def _quad_integral(kfun, S, extent):
    """Integral of k(d^T S^-1 d) over the plane by a fine midpoint grid."""
    n = 1500
    hx = math.sqrt(extent * S[0, 0])
    hy = math.sqrt(extent * S[1, 1])
    xs = (np.arange(n) + 0.5) / n * 2 * hx - hx
    ys = (np.arange(n) + 0.5) / n * 2 * hy - hy
    X, Y = np.meshgrid(xs, ys)
    Si = np.linalg.inv(S)
    Q = Si[0, 0] * X * X + 2 * Si[0, 1] * X * Y + Si[1, 1] * Y * Y
    return kfun(Q).sum() * (2 * hx / n) * (2 * hy / n)


@pytest.mark.parametrize("kind", ["exp", "poly1", "poly3"])
def test_aa_normaliser_kernel_invariant(orc, kind):
    """Eq. 7-9: N_Sigma = sqrt|Sigma| * int k(y^T y) dy for any kernel, so the
    AA factor sqrt(|Sigma'| / |Sigma' + v I|) is the same for every kernel
    and equals the oracle's rho. Closed forms of int k(y^T y) dy =
    pi int_0^inf k(s) ds: exp 2 pi; f1 pi c0^2 / (2 |c1|)."""
    c = np.array(KINDS[kind])
    if kind == "exp":
        kfun, extent, closed = (lambda Q: np.exp(-0.5 * Q)), 70.0, 2 * math.pi
    else:
        kfun = lambda Q: np.maximum(np.polyval(c[::-1], Q), 0.0)
        root = np.roots(c[::-1])
        root = root[np.abs(root.imag) < 1e-9].real.min()
        extent = root * 1.05
        closed = math.pi * F1[0] ** 2 / (2 * abs(F1[1])) if kind == "poly1" else None
    cam = _cam(orc, 64, 64)
    cfg = orc.make_config(kind, tuple(c), "universal", aa=True)
    rng = np.random.default_rng(11)
    for _ in range(3):
        sc = _one_splat(rng.uniform(-0.2, 0.2, 3), np.exp(rng.normal(-3.3, 0.4, 3)), rng.normal(size=4))
        s = orc.splats_to_numpy(orc.project(sc, cam, cfg), 1)
        a, b, cc = s["cov2d"][0]
        S0 = np.array([[a, b], [b, cc]])
        S1 = S0 + 0.3 * np.eye(2)
        N0 = _quad_integral(kfun, S0, extent)
        N1 = _quad_integral(kfun, S1, extent)
        assert N0 / N1 == pytest.approx(s["rho"][0], rel=2e-4)
        if closed is not None:
            assert N1 / math.sqrt(np.linalg.det(S1)) == pytest.approx(closed, rel=2e-4)


@pytest.mark.parametrize("kind", ["exp", "poly1", "poly2", "poly3"])
def test_single_splat_closed_form(orc, kind):
    """One axis-aligned splat on the optical axis: each pixel is
    min(0.99, o rho k(Q)) c with Q = dx^2/(sx^2+v) + dy^2/(sy^2+v), or the
    background where that alpha is below eps."""
    W = H = 40
    cam = _cam(orc, W, H)
    cfg = orc.make_config(kind, KINDS[kind], "opacity", aa=True)
    sc = _one_splat([0.0, 0.0, 0.0], [0.06, 0.03, 0.05], opacity=0.9, dc=(0.7, -0.4, 0.2))
    bg = np.array([0.1, 0.2, 0.3])
    img, T, _ = orc.render_untiled(sc, cam, cfg, bg)
    f = cam.fx
    sx2, sy2 = (f * 0.06 / 3) ** 2, (f * 0.03 / 3) ** 2
    rho = math.sqrt(sx2 * sy2 / ((sx2 + 0.3) * (sy2 + 0.3)))
    col = 0.5 + 0.5 / math.sqrt(math.pi) * np.array([0.7, -0.4, 0.2])
    col = np.maximum(col, 0)
    c = np.array(KINDS[kind])
    xs = np.arange(W) + 0.5 - W / 2
    ys = np.arange(H) + 0.5 - H / 2
    X, Y = np.meshgrid(xs, ys)
    Q = X * X / (sx2 + 0.3) + Y * Y / (sy2 + 0.3)
    if kind == "exp":
        k = np.exp(-0.5 * Q)
    elif kind == "poly2":
        x0 = -c[1] / (2 * c[2])
        k = np.where(Q < x0, np.polyval(c[::-1], Q), 0.0)
    else:
        k = np.maximum(np.polyval(c[::-1], Q), 0.0)
    a = np.minimum(0.99, 0.9 * rho * k)
    a = np.where(a < EPS, 0.0, a)
    want = a[..., None] * col + (1 - a)[..., None] * bg
    assert np.abs(img - want).max() < 1e-12
    assert np.abs(T - (1 - a)).max() < 1e-12


def test_front_to_back_order_and_stop(orc):
    """Stack of exp splats with alpha 0.95 at the centre pixel (AA off): T goes
    0.05, 0.0025, 1.25e-4, then 6.25e-6 < 1e-4 stops without adding the 4th.
    Colour = sum c_i alpha T_i over the first three in depth order."""
    W = H = 8
    cam = _cam(orc, W, H)
    cfg = orc.make_config("exp", (), "universal", aa=False)
    # put the splats exactly on the centre pixel's ray: tiny, at pixel centre (3.5+0.5)
    zs = [2.0, 1.0, 0.5, 1.5, 0.0]  # world z; depth = z + 3
    cols = [(0.9, 0.1, 0.1), (0.1, 0.9, 0.1), (0.1, 0.1, 0.9), (0.5, 0.5, 0.5), (0.2, 0.3, 0.4)]
    P = len(zs)
    # each mean on the ray through the centre (4.5, 4.5) of pixel (4, 4)
    sc = {"means": np.array([[0.5 * (z + 3) / cam.fx, 0.5 * (z + 3) / cam.fy, z] for z in zs]),
          "scales": np.full((P, 3), 1e-4),
          "quats": np.tile([1.0, 0, 0, 0], (P, 1)), "opacities": np.full(P, 0.95),
          "sh": np.array([[[(ci - 0.5) * 2 * math.sqrt(math.pi) for ci in c]] for c in cols]),
          "sh_degree": 0}
    img, T, nc = orc.render_untiled(sc, cam, cfg)
    a = 0.95  # Q = 0 at that pixel, k(0) = 1
    order = np.argsort(zs)
    Tacc, C = 1.0, np.zeros(3)
    n = 0
    for i in order:
        if Tacc * (1 - a) < 1e-4:
            break
        C += np.array(cols[i]) * a * Tacc
        Tacc *= (1 - a)
        n += 1
    assert n == 3
    assert img[4, 4] == pytest.approx(C, abs=1e-9)
    assert T[4, 4] == pytest.approx(Tacc, abs=1e-15)
    assert nc[4, 4] == n


def _scene_small(P=4096, seed=0):
    import oracle
    return oracle.activate(synth.scene_uniform(P, seed))


@pytest.fixture(scope="module")
def small_scene():
    return _scene_small()


@pytest.mark.parametrize("kind", ["exp", "poly1", "poly2", "poly3"])
@pytest.mark.parametrize("cull", ["universal", "opacity"])
def test_culling_changes_no_pixel(orc, small_scene, kind, cull):
    """Table 3 (identical quality for cull S/0/1): the tile-binned render with
    the paper's radii equals the untiled, unculled render bit for bit."""
    cam = orc.camera_from_dict(synth.camera_small())
    cfg = orc.make_config(kind, KINDS[kind], cull, aa=True)
    a, Ta, _ = orc.render_untiled(small_scene, cam, cfg)
    b, Tb, _, nev, _ = orc.render_tiled(small_scene, cam, cfg)
    assert np.array_equal(a, b) and np.array_equal(Ta, Tb)
    assert nev.sum() > 0


def test_circle_rect_also_exact(orc, small_scene):
    cam = orc.camera_from_dict(synth.camera_small())
    cfg = orc.make_config("poly1", F1, "opacity", rect_mode=orc.RECT_CIRCLE)
    a, *_ = orc.render_untiled(small_scene, cam, cfg)
    b, *_ = orc.render_tiled(small_scene, cam, cfg)
    assert np.array_equal(a, b)


def test_opacity_cull_shrinks_lists(orc, small_scene):
    """Tighter radii bin fewer splat-tile pairs: exp > f1 universal > f1 opacity."""
    cam = orc.camera_from_dict(synth.camera_small())
    tot = {}
    for kind, cull in (("exp", "universal"), ("poly1", "universal"), ("poly1", "opacity")):
        *_, llen = orc.render_tiled(small_scene, cam, orc.make_config(kind, KINDS[kind], cull))
        tot[(kind, cull)] = llen.sum()
    assert tot[("exp", "universal")] > tot[("poly1", "universal")] > tot[("poly1", "opacity")]


def test_exp_with_f1_cut_changes_pixels(orc, small_scene):
    """Fig. 3a negative control: the exponential rendered with f1's
    opacity-aware radius is culled too tightly and differs visibly; the
    3-sigma legacy radius is not pixel exact for exp either."""
    cam = orc.camera_from_dict(synth.camera_small())
    P = small_scene["means"].shape[0]
    cfg_e = orc.make_config("exp", (), "opacity")
    ref, *_ = orc.render_untiled(small_scene, cam, cfg_e)
    s_e = orc.project(small_scene, cam, cfg_e)
    s_f = orc.project(small_scene, cam, orc.make_config("poly1", F1, "opacity"))
    for i in range(P):
        s_e[i].visible = s_f[i].visible
        s_e[i].tiles = s_f[i].tiles
        for j in range(4):
            s_e[i].rect[j] = s_f[i].rect[j]
    bad, *_ = orc.render_tiled(small_scene, cam, cfg_e, s2d=s_e)
    assert np.abs(bad - ref).max() > 5e-3
    leg, *_ = orc.render_tiled(small_scene, cam, orc.make_config("exp", (), "legacy3"))
    assert np.abs(leg - ref).max() > 1e-4


def _fd_scene(P=14, seed=4):
    r = np.random.default_rng(seed)
    return {"means": r.uniform(-0.35, 0.35, (P, 3)), "scales": np.exp(r.normal(-2.2, 0.3, (P, 3))),
            "quats": r.normal(size=(P, 4)), "opacities": 1 / (1 + np.exp(-r.normal(0.5, 1.0, P))),
            "sh": np.concatenate([r.uniform(-1.5, 1.5, (P, 1, 3)), r.normal(0, 0.3, (P, 15, 3))], 1),
            "sh_degree": 3}


@pytest.mark.parametrize("kind,cull", [("poly1", "opacity"), ("exp", "universal"),
                                       ("poly2", "opacity"), ("poly3", "opacity")])
def test_backward_matches_finite_differences(orc, kind, cull):
    """Analytic reverse pass vs FP64 central differences of L = sum w * image,
    skipping entries where a skip / clamp / stop decision flips within +-h."""
    sc = _fd_scene()
    cam = orc.camera_from_dict(synth.look_at([0.3, -0.2, -2.5], [0, 0, 0], 28, 24, 60.0))
    cfg = orc.make_config(kind, KINDS[kind], cull, aa=True)
    bg = np.array([0.2, 0.4, 0.1])
    w = np.random.default_rng(9).normal(size=(24, 28, 3))
    g = orc.render_backward(sc, cam, cfg, w, bg)
    base_sig = orc.decisions(sc, cam, cfg)
    img0, _, _ = orc.render_untiled(sc, cam, cfg, bg)
    # rounding noise of a central difference of L: ~ eps_mach * sum |terms| / h
    noise = 100 * 2.2e-16 * np.abs(img0 * w).sum()
    checked = 0
    for name in ("means", "scales", "quats", "opacities", "sh"):
        arr = sc[name]
        gan = g[name]
        for idx in np.ndindex(arr.shape):
            h = 1e-6 * max(1.0, abs(arr[idx]))
            vals = []
            flip = False
            for sgn in (1, -1):
                sc2 = {k: (np.array(v, copy=True) if isinstance(v, np.ndarray) else v) for k, v in sc.items()}
                sc2[name][idx] += sgn * h
                if not np.array_equal(orc.decisions(sc2, cam, cfg), base_sig):
                    flip = True
                    break
                img, _, _ = orc.render_untiled(sc2, cam, cfg, bg)
                vals.append((img * w).sum())
            if flip:
                continue
            fd = (vals[0] - vals[1]) / (2 * h)
            assert abs(fd - gan[idx]) <= 1e-6 * abs(gan[idx]) + noise / h, (name, idx, fd, gan[idx])
            checked += 1
    assert checked > 600
