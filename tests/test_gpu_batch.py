"""Batched multi-camera rendering: persistent launch, CUDA-graph replay,
mixed resolutions, staging depth, and the autotuner."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gs():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2603_18707_b300 import build
    build.build()
    from paper_2603_18707_b300 import api, render, synth
    return api, render, synth


def _mixed_small(synth):
    # the 4:3:2:1 resolution mix of the serving workload, scaled down 4x
    return [synth.look_at(_pos(c), [0, 0, 0], c["width"] // 4, c["height"] // 4)
            for c in synth.mixed_cameras(10)]


def _pos(c):
    vm = np.asarray(c["viewmat"])
    return -vm[:3, :3].T @ vm[:3, 3]


@pytest.fixture(scope="module")
def scene(gs):
    api, render, synth = gs
    raw = synth.scene_clusters(200_000, 2, sh_degree=3)
    return raw, render.activate(raw)


def test_persistent_launch_matches_per_tile_launch(gs, scene):
    api, render, synth = gs
    raw, sc = scene
    cams = _mixed_small(synth)
    for kind in ("poly1", "exp"):
        cfg = api.make_config(kind, "opacity")
        a = render.Rasterizer(cams, cfg, 200_000)
        b = render.Rasterizer(cams, cfg, 200_000, persistent=True)
        a.forward(sc)
        b.forward(sc)
        torch.cuda.synchronize()
        assert torch.equal(a.out, b.out) and torch.equal(a.last, b.last)
        assert torch.equal(a.n_eval, b.n_eval)


def test_mixed_batch_equals_single_cameras(gs, scene):
    api, render, synth = gs
    raw, sc = scene
    cams = _mixed_small(synth)
    cfg = api.make_config("poly1", "opacity")
    R = render.Rasterizer(cams, cfg, 200_000, persistent=True)
    R.forward(sc)
    imgs = [im.clone() for im in R.images()]
    for cam, im in zip(cams, imgs):
        one = render.Rasterizer([cam], cfg, 200_000)
        one.forward(sc)
        assert torch.equal(one.images()[0], im)


def test_sixty_four_cameras_the_batch_limit(gs, scene):
    """The largest camera batch (GS_MAX_CAMERAS = 64, ragged 200x120 frames):
    every image bit-identical to the same camera rendered alone; 65 cameras
    are rejected."""
    api, render, synth = gs
    raw, sc = scene
    from paper_2603_18707_b300 import _lib
    cams = synth.orbit_cameras(64, 200, 120)
    cfg = api.make_config("poly1", "opacity")
    R = render.Rasterizer(cams, cfg, 200_000)
    R.forward(sc)
    imgs = R.images()
    for k in (0, 17, 40, 63):
        one = render.Rasterizer([cams[k]], cfg, 200_000)
        one.forward(sc)
        assert torch.equal(one.images()[0], imgs[k]), k
    with pytest.raises((_lib.GsError, ValueError)):
        render.Rasterizer(synth.orbit_cameras(65, 200, 120), cfg, 200_000).forward(sc)


def test_graph_replay_matches_eager(gs, scene):
    api, render, synth = gs
    raw, sc = scene
    cams = _mixed_small(synth)
    cfg = api.make_config("poly1", "opacity")
    R = render.Rasterizer(cams, cfg, 200_000, persistent=True)
    static = {k: (v.clone() if torch.is_tensor(v) else v) for k, v in sc.items()}
    R.forward(static)
    eager = R.out.clone()
    graph = R.capture(static)
    R.out.zero_()
    graph.replay()
    torch.cuda.synchronize()
    assert torch.equal(R.out, eager)
    # new inputs written in place are picked up by the replay
    static["means"].add_(0.01)
    graph.replay()
    torch.cuda.synchronize()
    replayed = R.out.clone()
    ref = render.Rasterizer(cams, cfg, 200_000, capacity=R.capacity)
    ref.forward(static)
    assert torch.equal(replayed, ref.out)
    assert not torch.equal(replayed, eager)


def test_batch_depth_does_not_change_pixels(gs, scene):
    api, render, synth = gs
    raw, sc = scene
    cams = _mixed_small(synth)[:3]
    outs = []
    for b in (256, 100, 32):
        R = render.Rasterizer(cams, api.make_config("poly3", "opacity", batch=b), 200_000)
        R.forward(sc)
        outs.append(R.out.clone())
    assert torch.equal(outs[0], outs[1]) and torch.equal(outs[0], outs[2])


def test_autotuner_picks_a_measured_candidate_and_caches(gs, scene, tmp_path):
    api, render, synth = gs
    from paper_2603_18707_b300 import autotune
    raw, sc = scene
    cams = _mixed_small(synth)[:4]
    cache = str(tmp_path / "tune.json")
    r1 = autotune.autotune(cams, "poly1", "opacity", sc, 200_000, steps=2, cache=cache)
    assert tuple(r1["tile"]) in autotune.TILES and r1["px_per_thread"] in autotune.PPTS
    assert r1["batch"] in autotune.BATCHES
    assert r1["ms"] == min(v for v in r1["trials_ms"].values() if v is not None)
    assert len(r1["trials_ms"]) == len(autotune.TILES) * len(autotune.PPTS) + len(autotune.BATCHES) - 1
    r2 = autotune.autotune(cams, "poly1", "opacity", sc, 200_000, steps=2, cache=cache)
    assert r2 == r1
    R = render.Rasterizer(cams, api.make_config("poly1", "opacity", **autotune.config_overrides(r1)),
                          200_000)
    R.forward(sc)
    assert torch.isfinite(R.out).all()


def test_streamed_camera_groups_equal_single():
    """Cameras split into sets on their own streams (StreamedRasterizer):
    every image bit-identical to the one-stream render of all cameras (each
    camera's tile lists do not depend on the other cameras)."""
    import torch
    from paper_2603_18707_b300 import api, render, synth
    raw = synth.scene_clusters(200_000, 3, sh_degree=1)
    cams = synth.mixed_cameras(6)
    sc = render.activate(raw)
    one = render.Rasterizer(cams, api.make_config("poly1", "opacity"), 200_000)
    one.forward(sc)
    for groups, persistent in ((2, False), (3, False), (2, True)):
        st = render.StreamedRasterizer(cams, api.make_config("poly1", "opacity"), 200_000, groups=groups,
                                       persistent=persistent)
        st.forward(sc)
        st.run_async(sc)
        torch.cuda.synchronize()
        assert torch.equal(st.out, one.out)
        assert torch.equal(st.final_T, one.final_T)
        assert st.n_records() == one.n_records()
        g = st.capture(sc)
        st.out.zero_()
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(st.out, one.out)


def test_host_pipeline_frames_match_device_renders():
    """render.HostPipeline (overlapped upload / render / download): each
    step's host image equals the device render of that step's own input,
    with two different scenes alternating."""
    import torch
    from paper_2603_18707_b300 import api, render, synth
    cams = synth.mixed_cameras(3)
    scenes = [render.activate(synth.scene_clusters(100_000, s, sh_degree=2)) for s in (1, 2)]
    R = render.StreamedRasterizer(cams, api.make_config("poly1", "opacity"), 100_000, groups=2)
    want = []
    for sc in scenes:
        R.forward(sc)
        want.append(R.out.clone())
    hosts = [{k: sc[k].cpu().pin_memory() for k in render.HostPipeline.KEYS} for sc in scenes]
    for h in hosts:
        h["sh_degree"] = 2
    outs = [torch.empty_like(R.out, device="cpu").pin_memory() for _ in range(5)]
    pipe = render.HostPipeline(R)
    for k in range(5):
        pipe.step(hosts[k % 2], outs[k])
    pipe.finish()
    torch.cuda.synchronize()
    for k in range(5):
        assert torch.equal(outs[k], want[k % 2].cpu()), k


def test_set_cameras_and_serving_pipeline(gs):
    """New poses on an existing (streamed) rasterizer render exactly what a
    fresh rasterizer renders for them; HostPipeline.step_views delivers the
    same images to pinned host memory."""
    from paper_2603_18707_b300 import api, render, synth
    raw = synth.scene_clusters(200_000, 0, sh_degree=3)
    sc = render.activate(raw)
    cfg = api.make_config("poly1", "opacity")
    a = synth.orbit_cameras(4, 320, 240)
    b = synth.orbit_cameras(4, 320, 240, phase=0.3)
    R = render.StreamedRasterizer(a, cfg, 200_000, groups=2)
    R.forward(sc)
    R.set_cameras(b)
    R.forward(sc)
    ref = render.Rasterizer(b, cfg, 200_000)
    ref.forward(sc)
    torch.cuda.synchronize()
    assert torch.equal(R.out, ref.out)
    with pytest.raises(ValueError):
        R.set_cameras(synth.orbit_cameras(4, 321, 240))
    host = torch.empty_like(R.out, device="cpu").pin_memory()
    pipe = render.HostPipeline(R)
    pipe.step_views(sc, a, host)
    pipe.step_views(sc, b, host)
    pipe.finish()
    torch.cuda.synchronize()
    assert torch.equal(host, ref.out.cpu())


def _morton_np(means):
    """Z-order codes by the definition in gs.h, written independently with
    integer bit loops: 10 bits per axis over the box of the finite means."""
    m = np.asarray(means, np.float64)
    fin = np.isfinite(m)
    lo = np.where(fin, m, np.inf).min(0)
    hi = np.where(fin, m, -np.inf).max(0)
    lo32, hi32 = lo.astype(np.float32), hi.astype(np.float32)
    ext = (hi32 - lo32).astype(np.float32)
    sc = np.where(ext > 0, np.float32(1023.0) / np.where(ext > 0, ext, 1), 0).astype(np.float32)
    q = np.clip(np.nan_to_num((m.astype(np.float32) - lo32) * sc, nan=0.0, posinf=1023, neginf=0), 0, 1023)
    q = q.astype(np.int64)
    code = np.zeros(len(m), np.int64)
    for b in range(10):
        for k in range(3):
            code |= ((q[:, k] >> b) & 1) << (3 * b + k)
    return code


def test_spatial_order_is_a_stable_z_order_permutation(gs):
    """The permutation equals a stable argsort of the codes computed on the
    CPU (same FP32 scaling: (m - lo) * (1023 / (hi - lo)), no fused ops), so
    equal codes, including exact duplicates, stay in index order."""
    from paper_2603_18707_b300 import api
    r = np.random.default_rng(3)
    P = 200_000
    means = r.normal(0, 3, (P, 3)).astype(np.float32)
    means[:50] = means[50:100]          # exact duplicates: ties resolved by index
    means[150, 1] = np.nan               # a non-finite coordinate counts as the box's lower end
    means[151, 2] = np.inf               # and +inf as its upper end
    perm = api.gs_spatial_order(torch.tensor(means, device="cuda")).cpu().numpy()
    assert np.array_equal(np.sort(perm), np.arange(P))
    ref = np.argsort(_morton_np(means), kind="stable")
    assert np.array_equal(perm, ref)
    pos = np.argsort(perm)
    assert np.all(pos[:50] < pos[50:100])
    # degenerate inputs: one splat, and all means equal (every code 0: identity)
    one = api.gs_spatial_order(torch.zeros(1, 3, device="cuda")).cpu().numpy()
    assert one.tolist() == [0]
    same = api.gs_spatial_order(torch.ones(5000, 3, device="cuda")).cpu().numpy()
    assert np.array_equal(same, np.arange(5000))


def test_gather_rows_and_reordered_scene_renders_the_same(gs):
    from paper_2603_18707_b300 import api, render, synth
    raw = synth.scene_clusters(300_000, 2, sh_degree=3)
    sc = render.activate(raw)
    perm = api.gs_spatial_order(sc["means"])
    for k in ("means", "scales", "quats", "opacities", "sh"):
        got = api.gs_gather_rows(sc[k], perm)
        assert torch.equal(got, sc[k][perm.long()])
    sc2, perm2 = render.spatial_order(sc)
    assert torch.equal(perm2, perm)
    cams = synth.orbit_cameras(3, 640, 360)
    cfg = api.make_config("poly1", "opacity")

    def both(s1, s2, P):
        a = render.Rasterizer(cams, cfg, P)
        a.forward(s1)
        b = render.Rasterizer(cams, cfg, P)
        b.forward(s2)
        torch.cuda.synchronize()
        assert a.n_records() == b.n_records()
        return a.out, b.out

    # the cluster scene clips means to a box, so some splats coincide: only
    # pixels where coinciding splats meet (exactly equal depths, ordered by
    # index) may change
    x, y = both(sc, sc2, 300_000)
    d = (x - y).abs().amax(1)
    assert (d > 0).float().mean().item() < 1e-3 and d.max().item() < 5e-3
    # a scene without coinciding splats renders bit-identically in either order
    u = render.activate(synth.scene_uniform(100_000, 4))
    u["means"] = u["means"] * 4.0
    u2, _ = render.spatial_order(u)
    x, y = both(u, u2, 100_000)
    assert torch.equal(x, y)


def test_persistent_graph_mixed_batch_matches_oracle(gs, orc):
    """The serving launch against the FP64 oracle: cameras of all four
    resolutions of the mixed workload (one full 3840x2160 frame among them),
    the blend as one persistent launch, the whole pass replayed from a CUDA
    graph, with the launch shape the autotuner picks here and with the 32x16
    tiles / 4 pixels per thread it picks on the 6M-splat batch. Sampled tiles
    of every camera (the last, ragged tile included): pixels within 2e-4 of
    the oracle's tile render of the same tile shape outside threshold flips,
    and evaluation counts equal to the oracle's (same stopping splat)."""
    api, render, synth = gs
    from gpu_helpers import (KIND_COEFFS, NEAR_MARGIN, TOL_FP32, n_eval_mismatches,
                             oracle_tile_list)
    from paper_2603_18707_b300 import autotune
    P = 600_000
    raw = synth.scene_clusters(P, 4, sh_degree=3)
    sc = render.activate(raw)
    cams = synth.mixed_cameras(10)  # 4 x 640x360, 3 x 1280x720, 2 x 1920x1080, 1 x 3840x2160
    assert sorted({(c["width"], c["height"]) for c in cams}) == [(640, 360), (1280, 720), (1920, 1080),
                                                                   (3840, 2160)]
    tuned = autotune.autotune(cams, "poly1", "opacity", sc, P, persistent=True, steps=2, cache=None)
    shapes = [autotune.config_overrides(tuned), {"tile": (32, 16), "batch": 256, "px_per_thread": 4}]
    osc = orc.activate(raw)
    rng = np.random.default_rng(3)
    checked = n_near = n_px = 0
    for over in shapes:
        cfg = api.make_config("poly1", "opacity", **over)
        R = render.Rasterizer(cams, cfg, P, persistent=True)
        R.forward(sc)
        graph = R.capture(sc, n_eval=True)
        R.out.zero_()
        R.n_eval.zero_()
        graph.replay()
        torch.cuda.synchronize()
        imgs = [im.cpu().numpy() for im in R.images()]
        nevs = [n.cpu().numpy().astype(np.int64) for n in R.per_camera(R.n_eval)]
        vals, rg = R.vals.cpu().numpy().astype(np.int64), R.ranges.cpu().numpy().reshape(-1, 2)
        tw, th = over["tile"]
        ocfg = orc.make_config("poly1", KIND_COEFFS["poly1"], "opacity", tile=(tw, th))
        base = 0
        for c, (cam, img, nev_g) in enumerate(zip(cams, imgs, nevs)):
            W, H = cam["width"], cam["height"]
            tx, ty = -(-W // tw), -(-H // th)
            tiles = sorted(set(rng.integers(0, tx * ty, 5).tolist()) | {tx * ty - 1})
            oc = orc.camera_from_dict(cam)
            s2d = orc.project(osc, oc, ocfg)
            ref, _, _, nev_o, _ = orc.render_tiled(osc, oc, ocfg, tiles=tiles, s2d=s2d)
            # decision margins over the universal-cull lists, which contain every
            # entry the GPU's conservative rectangles can add
            ucfg = orc.make_config("poly1", KIND_COEFFS["poly1"], "universal", tile=(tw, th))
            *_, margin = orc.render_tiled(osc, oc, ucfg, tiles=tiles, with_margin=True)
            o = orc.splats_to_numpy(s2d, P)
            for t in tiles:
                y0, x0 = (t // tx) * th, (t % tx) * tw
                ys, xs = slice(y0, min(y0 + th, H)), slice(x0, min(x0 + tw, W))
                far = margin[ys, xs] >= NEAR_MARGIN
                err = np.abs(img[ys, xs].astype(np.float64) - ref[ys, xs]).max(-1)
                assert err[far].max(initial=0.0) < TOL_FP32, (c, t, over)
                n_near += int((~far).sum())
                n_px += far.size
                G = vals[rg[base + t, 0]:rg[base + t, 1]] - c * P
                O = oracle_tile_list(o, t, tx)
                assert set(O.tolist()) <= set(G.tolist())
                assert n_eval_mismatches(nev_g[ys, xs].ravel(), nev_o[ys, xs].ravel(), far.ravel(), O, G) == 0
                checked += 1
            base += tx * ty
        del graph, R
    assert checked >= 2 * 10 * 2
    assert n_near < 0.03 * n_px  # threshold flips are a small minority of the checked pixels
