"""GPU parity of the forward path through the C ABI: preprocess records,
bit-exact binning, images against the FP64 oracle, batching, tile shapes,
edge cases, and sampled tiles of the 3M-splat 1080p scene."""
import numpy as np
import pytest
import torch

from gpu_helpers import (KIND_COEFFS, NEAR_MARGIN, TOL_FP32, expected_binning, n_eval_mismatches,
                         oracle_tile_list, parse_splat2d)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gs():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2603_18707_b300 import build
    build.build()
    import paper_2603_18707_b300 as pkg
    return pkg


def _gpu(gs, raw, cams, kind, cull, keep_keys=True, **over):
    from paper_2603_18707_b300 import api, render
    cfg = api.make_config(kind, cull, **over)
    sc = render.activate(raw)
    R = render.Rasterizer(cams, cfg, raw["means"].shape[0], keep_keys=keep_keys)
    R.forward(sc)
    torch.cuda.synchronize()
    return R


def _oracle_cfg(orc, kind, cull, tile=(16, 16)):
    return orc.make_config(kind, KIND_COEFFS[kind], cull, tile=tile)


def _compare(img_gpu, img_orc, margin, tol=TOL_FP32):
    """Max error over pixels whose decisions are not within NEAR_MARGIN of a
    threshold, and the count of such near-threshold pixels."""
    err = np.abs(img_gpu.astype(np.float64) - img_orc).max(axis=-1)
    near = margin < NEAR_MARGIN
    return float(err[~near].max(initial=0.0)), int(near.sum()), float(err.max(initial=0.0))


@pytest.fixture(scope="module")
def small(gs):
    from paper_2603_18707_b300 import synth
    return synth.scene_uniform(4096, 0)


def test_preprocess_parity(gs, orc, small):
    from paper_2603_18707_b300 import synth
    cam = synth.camera_small()
    for kind, cull in (("exp", "opacity"), ("poly1", "opacity"), ("poly3", "opacity"),
                       ("poly2", "universal")):
        R = _gpu(gs, small, [cam], kind, cull)
        g = parse_splat2d(R.splat2d.cpu().numpy(), R.P)
        o = orc.splats_to_numpy(orc.project(orc.activate(small), orc.camera_from_dict(cam),
                                            _oracle_cfg(orc, kind, cull)), R.P)
        vis_g = g["tiles"] > 0
        vis_o = (o["visible"] == 1) & (o["tiles"] > 0)
        # visibility differs at most for splats whose support grazes the image
        assert (vis_g != vis_o).sum() <= 3
        both = vis_g & vis_o
        assert both.sum() > 1000
        assert np.abs(g["mean2d"][both] - o["mean2d"][both]).max() < 2e-4
        assert np.abs(g["depth"][both] - o["depth"][both]).max() < 1e-5
        rel = np.abs(g["conic"][both] - o["conic"][both]) / (np.abs(o["conic"][both]).max(1, keepdims=True))
        assert rel.max() < 2e-4
        assert np.abs(g["opacity"][both] - o["opacity"][both]).max() < 2e-5
        assert np.abs(g["color"][both] - o["color"][both]).max() < 2e-5
        # support threshold: conservative (never smaller), within the stated margin
        xo, xg = o["xcut"][both], g["xcut"][both]
        assert np.all(xg >= xo * (1 - 1e-5))
        assert np.all(xg <= xo * 1.0012 + 2e-4)
        # tile rectangles contain the oracle's
        ro, rg = o["rect"][both], g["rect"][both]
        assert np.all(rg[:, :2] <= ro[:, :2]) and np.all(rg[:, 2:] >= ro[:, 2:])
        assert (rg != ro).any(axis=1).sum() <= max(3, both.sum() // 200)


@pytest.mark.parametrize("kind,cull", [("exp", "opacity"), ("poly1", "opacity"), ("poly1", "universal"),
                                       ("poly3", "opacity")])
def test_border_splats_never_dropped(gs, orc, kind, cull):
    """Large anisotropic splats scattered around the image border (most
    projected outside it, many reaching in): every record the FP64 oracle
    draws is drawn on the GPU, with a rectangle containing the oracle's
    (the FP32 support and rectangle are conservative)."""
    from paper_2603_18707_b300 import synth
    r = np.random.default_rng(11)
    P = 3000
    raw = synth.scene_uniform(P, 5)
    raw["means"] = np.stack([r.uniform(-2.8, 2.8, P), r.uniform(-2.8, 2.8, P), r.uniform(-0.6, 0.6, P)],
                            1).astype(np.float32)
    raw["log_scales"] = np.stack([r.normal(-2.4, 0.6, P), r.normal(-3.5, 0.6, P), r.normal(-3.0, 0.6, P)],
                                 1).astype(np.float32)
    raw["opacity_logits"] = r.normal(1.0, 2.0, P).astype(np.float32)
    cam = synth.camera_small()
    R = _gpu(gs, raw, [cam], kind, cull)
    g = parse_splat2d(R.splat2d.cpu().numpy(), R.P)
    o = orc.splats_to_numpy(orc.project(orc.activate(raw), orc.camera_from_dict(cam),
                                        _oracle_cfg(orc, kind, cull)), R.P)
    vis_g = g["tiles"] > 0
    vis_o = (o["visible"] == 1) & (o["tiles"] > 0)
    assert vis_o.sum() > 500 and (~vis_o).sum() > 500  # both sides of the border are exercised
    assert not (vis_o & ~vis_g).any()
    both = vis_g & vis_o
    ro, rg = o["rect"][both], g["rect"][both]
    assert np.all(rg[:, :2] <= ro[:, :2]) and np.all(rg[:, 2:] >= ro[:, 2:])


@pytest.mark.parametrize("case", ["small3cam", "clusters", "ties", "wide", "tall", "many_small"])
def test_binning_bit_exact(gs, case):
    """Sorted record ids, 64-bit (tile, depth) keys and per-tile ranges equal a
    CPU stable sort of keys built from the GPU's own rectangles and depths.
    "wide" / "tall": a frame of 512 tile columns / rows at 8x8 tiles, beyond
    the 384 of the thread-counter splits (the warp-ranking kernels, the
    look-back column split and the atomic tile counts run there), and of 256
    / 128 at the wider tiles."""
    from paper_2603_18707_b300 import synth
    if case == "many_small":
        # 12 cameras of 1000 splats: a compaction partition (8192 records)
        # spans up to 9 cameras; the last camera looks away and draws nothing
        raw = synth.scene_uniform(1000, 8)
        cams = [synth.look_at([3.0 * np.sin(a), 0.4, -3.0 * np.cos(a)], [0, 0, 0], 64 + 8 * k, 48 + 4 * k)
                for k, a in enumerate(np.linspace(0.0, 2.0, 11))]
        cams.append(synth.look_at([0.0, 0.0, -3.0], [0.0, 0.0, -6.0], 64, 64))
    elif case == "wide":
        raw = synth.scene_uniform(4096, 2)
        cams = [synth.camera_small(4096, 96), synth.camera_small(128, 128)]
    elif case == "tall":
        raw = synth.scene_uniform(4096, 3)
        cams = [synth.camera_small(96, 4096)]
    elif case == "small3cam":
        raw = synth.scene_uniform(4096, 0)
        cams = [synth.camera_small(128, 128), synth.camera_small(100, 75),
                synth.look_at([1.0, -0.5, -3.0], [0, 0, 0], 64, 200)]
    elif case == "clusters":
        raw = synth.scene_clusters(200_000, 3, sh_degree=1)
        cams = synth.orbit_cameras(2, 640, 360)
    else:
        raw = synth.scene_uniform(6000, 5)
        raw["means"][:, 2] = np.round(raw["means"][:, 2] * 4) / 4  # many exact depth ties
        raw["means"][:3000] = raw["means"][3000:]                   # duplicated splats
        cams = [synth.camera_small(96, 96)]
    for tile in ((16, 16), (8, 8), (32, 8)):
        R = _gpu(gs, raw, cams, "poly1", "opacity", tile=tile)
        g = parse_splat2d(R.splat2d.cpu().numpy(), R.ncam * R.P)
        I, keys, ranges = expected_binning(g, cams, tile[0], tile[1], R.P)
        n_vis, n_over = R.n_records()
        assert n_over == I.size and n_vis == int((g["tiles"] > 0).sum())
        if case == "many_small":
            assert not (g["tiles"][-R.P:] > 0).any()  # the camera looking away draws nothing
        assert np.array_equal(R.vals[:n_over].cpu().numpy().astype(np.int64), I)
        assert np.array_equal(R.keys64[:n_over].cpu().numpy().view(np.uint64), keys)
        assert np.array_equal(R.ranges.cpu().numpy().astype(np.int64), ranges)


@pytest.mark.parametrize("kind", ["exp", "poly1", "poly2", "poly3"])
@pytest.mark.parametrize("cull", ["universal", "opacity"])
@pytest.mark.parametrize("ppt", [1, 4])
def test_image_matches_oracle(gs, orc, small, kind, cull, ppt):
    """Config-1 scene (4096 splats, 128^2): GPU image vs the untiled, unculled
    FP64 oracle within 2e-4 per channel outside threshold flips."""
    from paper_2603_18707_b300 import synth
    cam = synth.camera_small()
    R = _gpu(gs, small, [cam], kind, cull, px_per_thread=ppt)
    img = R.images()[0].cpu().numpy()
    T = R.per_camera(R.final_T)[0].cpu().numpy()
    oc = orc.camera_from_dict(cam)
    cfg = _oracle_cfg(orc, kind, cull)
    sc = orc.activate(small)
    ref, Tref, _ = orc.render_untiled(sc, oc, cfg)
    *_, margin = orc.render_tiled(sc, oc, orc.make_config(kind, KIND_COEFFS[kind], "universal"),
                                  with_margin=True)
    worst, n_near, _ = _compare(img, ref, margin)
    assert worst < TOL_FP32, (worst, n_near)
    assert n_near < 0.01 * img.shape[0] * img.shape[1]
    far = margin >= NEAR_MARGIN
    assert np.abs(T - Tref)[far].max() < TOL_FP32


@pytest.mark.parametrize("kind", ["exp", "poly1", "poly2", "poly3"])
@pytest.mark.parametrize("mode", ["fp32", "fp16x2", "persistent"])
def test_image_without_last_contributor_is_identical(gs, orc, small, kind, mode):
    """The blend that keeps neither the last contributor nor the evaluation
    count (an image-only render) takes the same decisions: its image and final
    T equal, bit for bit, those of the blend that keeps both (which the other
    tests hold to the oracle), and its image is within 2e-4 of the oracle."""
    from paper_2603_18707_b300 import api, render, synth
    cam = synth.camera_small()
    over = {"fp16x2": 1, "px_per_thread": 4} if mode == "fp16x2" else {"px_per_thread": 4}
    cfg = api.make_config(kind, "opacity", **over)
    sc = render.activate(small)
    out = {}
    for keep in (True, False):
        R = render.Rasterizer([cam], cfg, small["means"].shape[0], persistent=mode == "persistent", last=keep)
        R.forward(sc, n_eval=keep)
        torch.cuda.synchronize()
        out[keep] = (R.out.clone(), R.final_T.clone())
    assert torch.equal(out[True][0], out[False][0])
    assert torch.equal(out[True][1], out[False][1])
    if mode == "fp32":
        ref, _, _ = orc.render_untiled(orc.activate(small), orc.camera_from_dict(cam),
                                       _oracle_cfg(orc, kind, "opacity"))
        *_, margin = orc.render_tiled(orc.activate(small), orc.camera_from_dict(cam),
                                      orc.make_config(kind, KIND_COEFFS[kind], "universal"), with_margin=True)
        worst, _, _ = _compare(out[False][0].cpu().numpy().reshape(ref.shape), ref, margin)
        assert worst < TOL_FP32


@pytest.mark.parametrize("tile", [8, 16])
@pytest.mark.parametrize("cull", ["universal", "opacity"])
def test_f2_range_coefficients_match_oracle(gs, orc, small, tile, cull):
    """App. A: f2 fitted over [0, x_max(tile)] renders through the quadratic
    kernel (its second root lies past x_max, so the cut of Eq. 6 and
    max(poly, 0) agree wherever the tile renderer evaluates it); GPU image vs
    the untiled FP64 oracle with the same coefficients, at that tile size."""
    from gpu_helpers import COEFFS
    from paper_2603_18707_b300 import synth
    c = tuple(COEFFS["poly2_range"][str(tile)][:3])
    cam = synth.camera_small()
    R = _gpu(gs, small, [cam], "poly2", cull, tile=(tile, tile), coeffs=c)
    img = R.images()[0].cpu().numpy()
    oc = orc.camera_from_dict(cam)
    sc = orc.activate(small)
    ref, _, _ = orc.render_untiled(sc, oc, orc.make_config("poly2", c, cull, tile=(tile, tile)))
    *_, margin = orc.render_tiled(sc, oc, orc.make_config("poly2", c, "universal", tile=(tile, tile)),
                                  with_margin=True)
    worst, n_near, _ = _compare(img, ref, margin)
    assert worst < TOL_FP32, (worst, n_near)
    assert n_near < 0.01 * img.shape[0] * img.shape[1]


@pytest.mark.parametrize("kind", ["exp", "poly1", "poly2", "poly3"])
@pytest.mark.parametrize("cull", ["universal", "opacity"])
@pytest.mark.parametrize("tc", [1, 2])
def test_tensor_core_quadric_matches_oracle(gs, orc, small, kind, cull, tc):
    """The tensor-core variants (Q of every pixel-splat pair with split TF32
    weights; 1: warp-level mma.sync, 2: tcgen05.mma into TMEM) against the
    untiled FP64 oracle, same tolerance as the FP32 path outside threshold
    flips; the blend's device error word stays clear."""
    from paper_2603_18707_b300 import api, synth
    cam = synth.camera_small()
    R = _gpu(gs, small, [cam], kind, cull, tensor_alpha=tc)
    st = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    api.gs_render_status_async(st)
    assert int(st.item()) == 0
    img = R.images()[0].cpu().numpy()
    oc = orc.camera_from_dict(cam)
    sc = orc.activate(small)
    ref, _, _ = orc.render_untiled(sc, oc, _oracle_cfg(orc, kind, cull))
    *_, margin = orc.render_tiled(sc, oc, orc.make_config(kind, KIND_COEFFS[kind], "universal"),
                                  with_margin=True)
    worst, n_near, _ = _compare(img, ref, margin)
    assert worst < TOL_FP32, (worst, n_near)
    assert n_near < 0.01 * img.shape[0] * img.shape[1]


@pytest.mark.parametrize("tc", [1, 2])
def test_tensor_core_quadric_full_size_tiles(gs, orc, tc):
    """3M-splat 1080p scene (splats of every size, far-off centres): sampled
    tiles of the tensor-core variants against the oracle's tile render."""
    from paper_2603_18707_b300 import synth
    raw = synth.scene_clusters(3_000_000, 0, sh_degree=3)
    cam = synth.orbit_cameras(16, 1920, 1080)[0]
    R = _gpu(gs, raw, [cam], "poly1", "opacity", keep_keys=False, tensor_alpha=tc)
    img = R.images()[0].cpu().numpy()
    tx, ty = (1920 + 15) // 16, (1080 + 15) // 16
    rng = np.random.default_rng(7)
    tiles = sorted(set(rng.integers(0, tx * ty, 16).tolist()) | {tx * ty - 1})
    ref, _, _, _, _, margin = orc.render_tiled(orc.activate(raw), orc.camera_from_dict(cam),
                                               _oracle_cfg(orc, "poly1", "opacity"), tiles=tiles,
                                               with_margin=True)
    mask = np.zeros((1080, 1920), bool)
    for t in tiles:
        y, x = (t // tx) * 16, (t % tx) * 16
        mask[y:y + 16, x:x + 16] = True
    err = np.abs(img.astype(np.float64) - ref).max(-1)
    near = margin < NEAR_MARGIN
    assert err[mask & ~near].max() < TOL_FP32
    assert (mask & near).sum() < 0.02 * mask.sum()


def test_poly1_vs_exp_psnr_reported(gs, small):
    """Sec. 4.1 trend on the config-1 scene: f3 is closer to exp than f1."""
    from paper_2603_18707_b300 import synth
    cam = synth.camera_small()
    ims = {k: _gpu(gs, small, [cam], k, "opacity").images()[0].cpu().numpy() for k in
           ("exp", "poly1", "poly3")}
    psnr = {k: -10 * np.log10(np.mean((ims[k] - ims["exp"]) ** 2)) for k in ("poly1", "poly3")}
    assert psnr["poly3"] > psnr["poly1"] > 20


def test_batched_cameras_equal_single(gs, small):
    from paper_2603_18707_b300 import synth
    cams = [synth.camera_small(128, 128), synth.camera_small(100, 75),
            synth.look_at([1.0, -0.5, -3.0], [0, 0, 0], 64, 200)]
    R = _gpu(gs, small, cams, "poly1", "opacity")
    many = [im.cpu().numpy().copy() for im in R.images()]
    for i, cam in enumerate(cams):
        one = _gpu(gs, small, [cam], "poly1", "opacity").images()[0].cpu().numpy()
        assert np.array_equal(one, many[i])


def test_tile_shapes_and_pixels_per_thread(gs, orc, small):
    """On a ragged 100x75 frame: pixels per thread do not change a pixel's
    arithmetic (bit-identical images for 1, 2, 4 at a given tile shape); the
    tile shape only moves the origin of the per-tile coefficients (FP32
    rounding differences), and every combination matches the oracle."""
    from paper_2603_18707_b300 import synth
    cam = synth.camera_small(100, 75)
    sc = orc.activate(small)
    oc = orc.camera_from_dict(cam)
    ref, _, _ = orc.render_untiled(sc, oc, _oracle_cfg(orc, "poly1", "opacity"))
    *_, margin = orc.render_tiled(sc, oc, _oracle_cfg(orc, "poly1", "universal"), with_margin=True)
    for tile, ppts in (((16, 16), (1, 2, 4)), ((8, 8), (1, 2, 4)), ((32, 8), (1, 4)), ((8, 16), (1, 2)),
                       ((32, 16), (2, 4)), ((16, 32), (2, 4))):
        imgs = [_gpu(gs, small, [cam], "poly1", "opacity", tile=tile, px_per_thread=p).images()[0]
                .cpu().numpy() for p in ppts]
        for im in imgs[1:]:
            assert np.array_equal(im, imgs[0]), tile
        worst, _, _ = _compare(imgs[0], ref, margin)
        assert worst < TOL_FP32, tile


@pytest.mark.parametrize("kind", ["exp", "poly1", "poly2", "poly3"])
@pytest.mark.parametrize("cull", ["universal", "opacity"])
def test_packed_pixel_pairs_equal_scalar_update(gs, small, kind, cull):
    """Two and four pixels per thread update pixel pairs with packed FP32x2
    FMAs (signs of the colours, and for f1 / exp of beta and the exponent,
    flipped so that no operand is negated); one pixel per thread takes the
    scalar update. Every rounding step is the same, so images and final T
    are equal bit for bit, for every kernel and cut."""
    from paper_2603_18707_b300 import synth
    cam = synth.camera_small(100, 75)
    out = []
    for p in (1, 2, 4):
        R = _gpu(gs, small, [cam], kind, cull, px_per_thread=p)
        out.append((R.images()[0].cpu().numpy(), R.per_camera(R.final_T)[0].cpu().numpy()))
    for img, T in out[1:]:
        assert np.array_equal(img, out[0][0])
        assert np.array_equal(T, out[0][1])


@pytest.mark.parametrize("kind,cull", [("poly1", "opacity"), ("exp", "opacity"), ("poly3", "universal")])
def test_n_eval_matches_oracle_count(gs, orc, small, kind, cull):
    """The per-pixel evaluation count (the numerator of Gsplat-evals/s): the
    list position where the pixel stops, or the list length. It equals the
    oracle's tile-binned count on every pixel away from threshold flips,
    once the GPU's conservative extra entries are accounted for (the pixel
    stops on the same splat)."""
    from paper_2603_18707_b300 import synth
    cam = synth.camera_small()
    R = _gpu(gs, small, [cam], kind, cull)
    nev_g = R.per_camera(R.n_eval)[0].cpu().numpy().astype(np.int64)
    vals, rg = R.vals.cpu().numpy().astype(np.int64), R.ranges.cpu().numpy().reshape(-1, 2)
    sc, oc, cfg = orc.activate(small), orc.camera_from_dict(cam), _oracle_cfg(orc, kind, cull)
    s2d = orc.project(sc, oc, cfg)
    o = orc.splats_to_numpy(s2d, R.P)
    _, _, _, nev_o, llen, margin = orc.render_tiled(sc, oc, cfg, s2d=s2d, with_margin=True)
    tiles_x = 8
    bad, total_g, total_o = 0, 0, 0
    for t in range(64):
        ys, xs = slice((t // tiles_x) * 16, (t // tiles_x) * 16 + 16), slice((t % tiles_x) * 16,
                                                                            (t % tiles_x) * 16 + 16)
        G = vals[rg[t, 0]:rg[t, 1]]
        O = oracle_tile_list(o, t, tiles_x)
        assert O.size == llen[t]
        assert set(O.tolist()) <= set(G.tolist())  # conservative lists
        far = (margin[ys, xs] >= NEAR_MARGIN).ravel()
        bad += n_eval_mismatches(nev_g[ys, xs].ravel(), nev_o[ys, xs].ravel(), far, O, G)
        total_g += int(nev_g[ys, xs].sum())
        total_o += int(nev_o[ys, xs].sum())
    assert bad == 0
    assert total_o <= total_g <= total_o * 1.01  # extras are below 1% of the evaluations


def test_edge_cases(gs, orc):
    from paper_2603_18707_b300 import synth
    cam = synth.camera_small(40, 24)
    bg = (0.25, 0.5, 0.75)
    from paper_2603_18707_b300 import api, render
    cfg = api.make_config("poly1", "opacity")
    # no splats at all
    empty = synth.scene_uniform(1, 0)
    empty = {k: (v[:0] if isinstance(v, np.ndarray) else v) for k, v in empty.items()}
    R = render.Rasterizer([cam], cfg, 0)
    R.forward(render.activate(empty), bg)
    assert np.allclose(R.images()[0].cpu().numpy(), np.array(bg), atol=0)
    # every splat behind the camera
    beh = synth.scene_uniform(500, 1)
    beh["means"][:, 2] = -10.0
    R = render.Rasterizer([cam], cfg, 500)
    R.forward(render.activate(beh), bg)
    assert np.allclose(R.images()[0].cpu().numpy(), np.array(bg), atol=0)
    assert R.n_records() == (0, 0)
    # every splat below the opacity threshold (culled whole)
    faint = synth.scene_uniform(500, 2)
    faint["opacity_logits"][:] = -8.0
    R = render.Rasterizer([cam], cfg, 500)
    R.forward(render.activate(faint), bg)
    assert np.allclose(R.images()[0].cpu().numpy(), np.array(bg), atol=0)
    # one large splat covering every tile: closed form via the oracle
    one = synth.scene_uniform(1, 3)
    one["means"][:] = 0.0
    one["log_scales"][:] = np.log(0.3)
    one["opacity_logits"][:] = 3.0
    R = render.Rasterizer([cam], cfg, 1)
    R.forward(render.activate(one), bg)
    ref, _, _ = orc.render_untiled(orc.activate(one), orc.camera_from_dict(cam),
                                   _oracle_cfg(orc, "poly1", "opacity"), bg)
    assert np.abs(R.images()[0].cpu().numpy() - ref).max() < TOL_FP32


def test_capacity_overflow_is_reported_and_recovered(gs, small):
    from paper_2603_18707_b300 import api, render, synth
    from paper_2603_18707_b300._lib import GS_ERR_CAPACITY
    cam = synth.camera_small()
    cfg = api.make_config("poly1", "opacity")
    sc = render.activate(small)
    R = render.Rasterizer([cam], cfg, 4096, capacity=1000)
    R.run_async(sc)
    assert api.gs_workspace_status(R.workspace) & GS_ERR_CAPACITY
    n_vis, n_over = R.n_records()
    assert n_over == 1000 and int(R.count[2].item()) > 1000
    R.forward(sc)
    ref = _gpu(gs, small, [cam], "poly1", "opacity").images()[0]
    assert torch.equal(R.images()[0], ref)
    assert api.gs_workspace_status(R.workspace) == 0


def test_deferred_capacity_check(gs, small):
    """forward(deferred=True) renders exactly what the synchronous pass
    renders, and a deferred pass that overflows the capacity is reported by
    the next call (CapacityOverflow, buffers grown); the repeated pass is
    exact again."""
    from paper_2603_18707_b300 import api, render, synth
    cam = synth.camera_small()
    cfg = api.make_config("poly1", "opacity")
    sc = render.activate(small)
    ref = _gpu(gs, small, [cam], "poly1", "opacity").images()[0].clone()
    R = render.Rasterizer([cam], cfg, 4096)
    R.forward(sc, deferred=True)  # not sized yet: synchronous
    assert R.sized and torch.equal(R.images()[0], ref)
    for _ in range(3):
        R.forward(sc, deferred=True)
    R.check_deferred()
    assert torch.equal(R.images()[0], ref) and R.overflows == 0
    need = R.n_records()[1]
    R._alloc(need // 2)
    R.forward(sc, deferred=True)  # overflows; not known yet
    with pytest.raises(render.CapacityOverflow):
        R.forward(sc, deferred=True)
    assert R.overflows == 1 and R.capacity >= need
    R.forward(sc, deferred=True)
    R.check_deferred()
    assert torch.equal(R.images()[0], ref)
    assert api.gs_workspace_status(R.workspace) == 0


def test_full_size_scene_sampled_tiles(gs, orc):
    """3M-splat cluster scene at 1920x1080 (SH degree 3), camera 0 of the
    orbit, in the launch configuration of the benchmark: 24 sampled tiles
    (including the ragged bottom row) against the FP64 tiled oracle."""
    from paper_2603_18707_b300 import synth
    raw = synth.scene_clusters(3_000_000, 0, sh_degree=3)
    cams = synth.orbit_cameras(16, 1920, 1080)
    R = _gpu(gs, raw, cams, "poly1", "opacity", keep_keys=False)
    img = R.images()[0].cpu().numpy()
    nev_g = R.per_camera(R.n_eval)[0].cpu().numpy().astype(np.int64)
    oc = orc.camera_from_dict(cams[0])
    cfg = _oracle_cfg(orc, "poly1", "opacity")
    tx, ty = (1920 + 15) // 16, (1080 + 15) // 16
    rng = np.random.default_rng(0)
    tiles = sorted(set(rng.integers(0, tx * ty, 20).tolist()) |
                   {0, tx - 1, (ty - 1) * tx, tx * ty - 1})
    sc = orc.activate(raw)
    s2d = orc.project(sc, oc, cfg)
    ref, _, _, nev, _, margin = orc.render_tiled(sc, oc, cfg, tiles=tiles, s2d=s2d, with_margin=True)
    mask = np.zeros((1080, 1920), bool)
    for t in tiles:
        y, x = (t // tx) * 16, (t % tx) * 16
        mask[y:y + 16, x:x + 16] = True
    err = np.abs(img.astype(np.float64) - ref).max(-1)
    near = margin < NEAR_MARGIN
    assert err[mask & ~near].max() < TOL_FP32
    assert (mask & near).sum() < 0.02 * mask.sum()
    # evaluation counts (camera 0's records are ids 0 .. P-1, its tiles 0 .. tx*ty-1)
    o = orc.splats_to_numpy(s2d, R.P)
    vals, rg = R.vals.cpu().numpy().astype(np.int64), R.ranges.cpu().numpy().reshape(-1, 2)
    bad = 0
    for t in tiles:
        y, x = (t // tx) * 16, (t % tx) * 16
        G, O = vals[rg[t, 0]:rg[t, 1]], oracle_tile_list(o, t, tx)
        assert set(O.tolist()) <= set(G.tolist())
        far = ~near[y:y + 16, x:x + 16].ravel()
        bad += n_eval_mismatches(nev_g[y:y + 16, x:x + 16].ravel(), nev[y:y + 16, x:x + 16].ravel(), far, O, G)
    assert bad == 0


@pytest.mark.parametrize("kind,cull", [("poly1", "opacity"), ("exp", "opacity"), ("poly3", "universal")])
def test_ellipse_binning_drops_only_unreached_tiles(gs, orc, kind, cull):
    """GS_RECT_ELLIPSE bins a splat only to the tiles of each row that its
    support ellipse reaches (the per-tile culling of StopThePop). Every list
    is an order-preserving subsequence of the AABB list, fewer overlaps are
    emitted, and the image is bit-identical (dropped tiles held only alpha <
    eps entries) and matches the oracle."""
    from paper_2603_18707_b300 import synth
    raw = synth.scene_clusters(300_000, 4, sh_degree=1)
    cams = [synth.orbit_cameras(3, 320, 240)[1], synth.camera_small(100, 75)]
    Ra = _gpu(gs, raw, cams, kind, cull, rect="aabb")
    Re = _gpu(gs, raw, cams, kind, cull, rect="ellipse")
    assert torch.equal(Ra.out, Re.out)
    na, ne = Ra.n_records()[1], Re.n_records()[1]
    assert ne < na
    va, ve = Ra.vals.cpu().numpy(), Re.vals.cpu().numpy()
    ra = Ra.ranges.cpu().numpy().reshape(-1, 2)
    re_ = Re.ranges.cpu().numpy().reshape(-1, 2)
    for t in range(ra.shape[0]):
        la = va[ra[t, 0]:ra[t, 1]]
        le = ve[re_[t, 0]:re_[t, 1]]
        it = iter(la.tolist())
        assert all(x in it for x in le.tolist()), t
    # keys are still sorted by (tile, depth)
    k = Re.keys64[:ne].cpu().numpy().view(np.uint64)
    assert np.all(k[1:] >= k[:-1])
    img = Re.images()[1].cpu().numpy()
    oc = orc.camera_from_dict(cams[1])
    sc = orc.activate(raw)
    *_, margin = orc.render_tiled(sc, oc, _oracle_cfg(orc, kind, "universal"), with_margin=True)
    ref_t, *_ = orc.render_tiled(sc, oc, _oracle_cfg(orc, kind, cull))
    worst, _, _ = _compare(img, ref_t, margin)
    assert worst < TOL_FP32


@pytest.mark.parametrize("shape", ["wide", "tall"])
def test_ellipse_binning_wide_and_tall_frames(gs, shape):
    """The ellipse mode on frames of 512 tile columns / rows at 8x8 tiles,
    where the binning runs its warp-ranking splits (the row split cuts each
    row's columns to the ellipse there too): the image equals the AABB
    binning's bit for bit, every list is an order-preserving subsequence of
    the AABB list, and the keys stay sorted by (tile, depth)."""
    from paper_2603_18707_b300 import synth
    raw = synth.scene_uniform(4096, 7)
    cams = [synth.camera_small(4096, 96)] if shape == "wide" else [synth.camera_small(96, 4096)]
    Ra = _gpu(gs, raw, cams, "poly1", "opacity", rect="aabb", tile=(8, 8))
    Re = _gpu(gs, raw, cams, "poly1", "opacity", rect="ellipse", tile=(8, 8))
    assert torch.equal(Ra.out, Re.out)
    na, ne = Ra.n_records()[1], Re.n_records()[1]
    assert 0 < ne < na
    va, ve = Ra.vals.cpu().numpy(), Re.vals.cpu().numpy()
    ra = Ra.ranges.cpu().numpy().reshape(-1, 2)
    re_ = Re.ranges.cpu().numpy().reshape(-1, 2)
    for t in np.nonzero(re_[:, 1] > re_[:, 0])[0]:
        it = iter(va[ra[t, 0]:ra[t, 1]].tolist())
        assert all(x in it for x in ve[re_[t, 0]:re_[t, 1]].tolist()), t
    k = Re.keys64[:ne].cpu().numpy().view(np.uint64)
    assert np.all(k[1:] >= k[:-1])
