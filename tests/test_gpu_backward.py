"""GPU reverse pass through the C ABI against the FP64 oracle's reverse pass
and its central finite differences; autograd chaining; sampled tiles of the
1M-splat 1024^2 differentiable-render workload."""
import numpy as np
import pytest
import torch

from gpu_helpers import KIND_COEFFS, NEAR_MARGIN

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gs():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2603_18707_b300 import build
    build.build()
    from paper_2603_18707_b300 import api, render, synth
    return api, render, synth


def _small_scene(P=48, seed=4):
    r = np.random.default_rng(seed)
    return {"means": r.uniform(-0.4, 0.4, (P, 3)).astype(np.float32),
            "log_scales": r.normal(-2.6, 0.4, (P, 3)).astype(np.float32),
            "quats": r.normal(size=(P, 4)).astype(np.float32),
            "opacity_logits": r.normal(0.5, 1.2, P).astype(np.float32),
            "sh": np.concatenate([r.uniform(-1.5, 1.5, (P, 1, 3)), r.normal(0, 0.3, (P, 15, 3))],
                                 1).astype(np.float32),
            "sh_degree": 3}


def _gpu_grads(api, render, raw, cams, kind, cull, w, bg, **over):
    cfg = api.make_config(kind, cull, **over)
    sc = render.activate(raw)
    R = render.Rasterizer(cams, cfg, raw["means"].shape[0])
    R.forward(sc, bg)
    g = {k: torch.zeros_like(sc[k]) for k in ("means", "scales", "quats", "opacities", "sh")}
    grad2d = torch.empty(api.gs_grad2d_bytes(R.ncam, R.P), dtype=torch.uint8, device="cuda")
    gout = torch.as_tensor(w.reshape(-1, 3), dtype=torch.float32, device="cuda").contiguous()
    api.gs_render_backward(R.cams, R.P, cfg, sc["means"], sc["scales"], sc["quats"],
                           sc["opacities"], sc["sh"], sc["sh_degree"], R.splat2d, R.vals,
                           R.ranges, bg, R.final_T, R.last, gout, grad2d, g["means"],
                           g["scales"], g["quats"], g["opacities"], g["sh"])
    torch.cuda.synchronize()
    return {k: v.cpu().numpy().astype(np.float64) for k, v in g.items()}, R


def _oracle_inputs(orc, raw):
    sc = orc.activate(raw)
    # the GPU path receives float32 activations: give the oracle the same values
    sc["scales"] = np.exp(raw["log_scales"].astype(np.float32)).astype(np.float64)
    sc["opacities"] = (1 / (1 + np.exp(-raw["opacity_logits"].astype(np.float32)))).astype(np.float64)
    return sc


def _masked_weights(orc, sc, oc, kind, shape, seed=9):
    w = np.random.default_rng(seed).normal(size=shape)
    *_, margin = orc.render_tiled(sc, oc, orc.make_config(kind, KIND_COEFFS[kind], "universal"),
                                  with_margin=True)
    w[margin < NEAR_MARGIN] = 0.0  # no gradient through pixels with threshold flips
    return w


def _check(gpu, ref, rel=1e-3, floor=1e-5, name=None):
    """Every gradient entry within 1e-3 of the oracle's, relative; entries
    near zero within 1e-5 of the tensor's largest (FP32 accumulation over
    many pixels leaves an absolute error of ~1e-7 of the largest, measured on
    the finite-difference sub-case, so 1e-5 is no relative bound for them but
    a tight absolute one). The worst relative error of the entries above the
    floor and the worst floor-relative error are reported."""
    import json
    import os
    stats = {}
    for k in ("means", "scales", "quats", "opacities", "sh"):
        a, b = gpu[k].reshape(-1), ref[k].reshape(-1)
        scale = np.abs(b).max()
        assert scale > 0, k
        err = np.abs(a - b)
        big = np.abs(b) > floor * scale / rel
        stats[k] = {"max_rel_above_floor": float((err[big] / np.abs(b[big])).max(initial=0.0)),
                    "max_abs_over_largest": float((err / scale).max())}
        assert np.all(err <= rel * np.abs(b) + floor * scale), (k, stats[k])
        assert np.linalg.norm(a - b) <= rel * np.linalg.norm(b), k
    rep = os.environ.get("GS_REPORT_DIR")
    if rep and name:
        os.makedirs(rep, exist_ok=True)
        with open(os.path.join(rep, "backward_vs_oracle.jsonl"), "a") as f:
            f.write(json.dumps({"case": name, **stats}) + "\n")


@pytest.mark.parametrize("kind,cull", [("poly1", "opacity"), ("exp", "universal"),
                                       ("exp", "opacity"), ("poly2", "opacity"),
                                       ("poly3", "opacity")])
def test_backward_matches_oracle_reverse_pass(gs, orc, kind, cull):
    api, render, synth = gs
    raw = _small_scene()
    cam = synth.look_at([0.3, -0.2, -2.5], [0, 0, 0], 56, 48, 60.0)
    oc = orc.camera_from_dict(cam)
    sc = _oracle_inputs(orc, raw)
    bg = (0.2, 0.4, 0.1)
    w = _masked_weights(orc, sc, oc, kind, (48, 56, 3))
    gpu, _ = _gpu_grads(api, render, raw, [cam], kind, cull, w, bg)
    ref = orc.render_backward(sc, oc, orc.make_config(kind, KIND_COEFFS[kind], cull), w, bg)
    _check(gpu, ref, name=f"{kind}-{cull}")


@pytest.mark.parametrize("tile", [(8, 8), (32, 8), (32, 16)])
def test_backward_tile_shapes(gs, orc, tile):
    """The reverse pass runs two pixels per thread on every tile shape up to
    512 pixels (256 threads for 32x16) and its gradients do not depend on
    the tiling: they match the oracle's tile-free reverse pass."""
    api, render, synth = gs
    raw = _small_scene()
    cam = synth.look_at([0.3, -0.2, -2.5], [0, 0, 0], 56, 48, 60.0)
    oc = orc.camera_from_dict(cam)
    sc = _oracle_inputs(orc, raw)
    bg = (0.2, 0.4, 0.1)
    w = _masked_weights(orc, sc, oc, "poly1", (48, 56, 3))
    gpu, _ = _gpu_grads(api, render, raw, [cam], "poly1", "opacity", w, bg, tile=tile)
    ref = orc.render_backward(sc, oc, orc.make_config("poly1", KIND_COEFFS["poly1"], "opacity"), w, bg)
    _check(gpu, ref, name=f"tile{tile[0]}x{tile[1]}")


def test_backward_matches_finite_differences(gs, orc):
    """GPU gradient vs FP64 central differences of the oracle's forward,
    on sampled entries where no skip / clamp / stop decision flips."""
    api, render, synth = gs
    raw = _small_scene(P=20, seed=7)
    cam = synth.look_at([0.3, -0.2, -2.5], [0, 0, 0], 40, 32, 60.0)
    oc = orc.camera_from_dict(cam)
    sc = _oracle_inputs(orc, raw)
    cfg = orc.make_config("poly1", KIND_COEFFS["poly1"], "opacity")
    bg = (0.1, 0.1, 0.1)
    w = _masked_weights(orc, sc, oc, "poly1", (32, 40, 3), seed=3)
    gpu, _ = _gpu_grads(api, render, raw, [cam], "poly1", "opacity", w, bg)
    base = orc.decisions(sc, oc, cfg)
    rng = np.random.default_rng(1)
    checked = 0
    for name in ("means", "scales", "quats", "opacities", "sh"):
        arr = sc[name]
        scale = np.abs(gpu[name]).max()
        flat = list(np.ndindex(arr.shape))
        for idx in [flat[i] for i in rng.choice(len(flat), min(25, len(flat)), replace=False)]:
            h = 1e-6 * max(1.0, abs(arr[idx]))
            vals = []
            for sgn in (1, -1):
                s2 = {k: (np.array(v, copy=True) if isinstance(v, np.ndarray) else v) for k, v in sc.items()}
                s2[name][idx] += sgn * h
                if not np.array_equal(orc.decisions(s2, oc, cfg), base):
                    break
                img, _, _ = orc.render_untiled(s2, oc, cfg, bg)
                vals.append((img * w).sum())
            if len(vals) < 2:
                continue
            fd = (vals[0] - vals[1]) / (2 * h)
            assert abs(gpu[name][idx] - fd) <= 1e-3 * abs(fd) + 1e-5 * scale, (name, idx, gpu[name][idx], fd)
            checked += 1
    assert checked >= 80


def test_autograd_function_chains_activations(gs):
    api, render, synth = gs
    from paper_2603_18707_b300 import autograd
    raw = _small_scene()
    cam = synth.look_at([0.3, -0.2, -2.5], [0, 0, 0], 56, 48, 60.0)
    t = {k: torch.tensor(raw[k], device="cuda", requires_grad=True)
         for k in ("means", "log_scales", "quats", "opacity_logits", "sh")}
    R = render.Rasterizer([cam], api.make_config("poly1", "opacity"), 48)
    w = torch.randn(48 * 56, 3, device="cuda", generator=torch.Generator("cuda").manual_seed(0))
    img = autograd.render(t["means"], t["log_scales"], t["quats"], t["opacity_logits"], t["sh"], 3, R)
    (img * w).sum().backward()
    gpu, _ = _gpu_grads(api, render, raw, [cam], "poly1", "opacity",
                        w.cpu().numpy().reshape(48, 56, 3), (0.0, 0.0, 0.0))
    s = np.exp(raw["log_scales"].astype(np.float64))
    o = 1 / (1 + np.exp(-raw["opacity_logits"].astype(np.float64)))
    assert np.allclose(t["means"].grad.cpu().numpy(), gpu["means"], rtol=1e-5, atol=1e-7)
    assert np.allclose(t["log_scales"].grad.cpu().numpy(), gpu["scales"] * s, rtol=1e-4, atol=1e-6)
    assert np.allclose(t["opacity_logits"].grad.cpu().numpy(), gpu["opacities"] * o * (1 - o),
                       rtol=1e-4, atol=1e-7)
    assert np.allclose(t["sh"].grad.cpu().numpy(), gpu["sh"], rtol=1e-5, atol=1e-7)


def test_autograd_deferred_check_matches_synchronous(gs):
    """The training-loop mode (capacity checked one call late) gives the
    gradients of the synchronous mode."""
    api, render, synth = gs
    from paper_2603_18707_b300 import autograd
    raw = _small_scene()
    cam = synth.look_at([0.3, -0.2, -2.5], [0, 0, 0], 56, 48, 60.0)
    R = render.Rasterizer([cam], api.make_config("poly1", "opacity"), 48)
    w = torch.randn(48 * 56, 3, device="cuda", generator=torch.Generator("cuda").manual_seed(1))
    grads = []
    for deferred in (False, True, True):
        t = {k: torch.tensor(raw[k], device="cuda", requires_grad=True)
             for k in ("means", "log_scales", "quats", "opacity_logits", "sh")}
        img = autograd.render(t["means"], t["log_scales"], t["quats"], t["opacity_logits"], t["sh"], 3, R,
                              deferred=deferred)
        (img * w).sum().backward()
        grads.append({k: v.grad.clone() for k, v in t.items()})
    R.check_deferred()
    for g in grads[1:]:
        for k in g:
            assert torch.allclose(g[k], grads[0][k], rtol=1e-5, atol=1e-8), k


def test_graphed_step_matches_eager_and_recaptures_on_overflow(gs):
    """autograd.GraphedStep replays give the eager step's gradients; a
    replay whose overlaps outgrow the buffers is reported by the next call
    (CapacityOverflow, buffers grown, graph recaptured) and the repeated
    step is right again."""
    api, render, synth = gs
    from paper_2603_18707_b300 import autograd
    raw = _small_scene()
    cam = synth.look_at([0.3, -0.2, -2.5], [0, 0, 0], 56, 48, 60.0)
    probe = render.Rasterizer([cam], api.make_config("poly1", "opacity"), 48)
    probe.forward(render.activate(raw))
    need = probe.n_records()[1]
    # an explicit capacity just above what the scene needs (kept, not shrunk)
    R = render.Rasterizer([cam], api.make_config("poly1", "opacity"), 48, capacity=need + 8)
    w = torch.randn(48 * 56, 3, device="cuda", generator=torch.Generator("cuda").manual_seed(2))
    t = {k: torch.tensor(raw[k], device="cuda", requires_grad=True)
         for k in ("means", "log_scales", "quats", "opacity_logits", "sh")}

    def fn():
        for v in t.values():
            v.grad = None
        img = autograd.render(t["means"], t["log_scales"], t["quats"], t["opacity_logits"], t["sh"], 3, R,
                              deferred=True)
        loss = (img * w).sum()
        loss.backward()
        return loss

    def eager():
        R2 = render.Rasterizer([cam], api.make_config("poly1", "opacity"), 48)
        t2 = {k: v.detach().clone().requires_grad_(True) for k, v in t.items()}
        img = autograd.render(t2["means"], t2["log_scales"], t2["quats"], t2["opacity_logits"], t2["sh"], 3, R2)
        (img * w).sum().backward()
        return {k: v.grad for k, v in t2.items()}

    def same(got, ref):
        # the two runs differ only in the order of the FP32 atomic additions
        for k in ref:
            d = (got[k] - ref[k]).abs().max().item()
            assert d <= 1e-4 * ref[k].abs().max().item(), (k, d)

    G = autograd.GraphedStep(fn, R)
    for _ in range(3):
        G()
    G.check()
    same({k: v.grad for k, v in t.items()}, eager())
    cap = R.capacity
    with torch.no_grad():
        t["log_scales"] += 1.5  # larger splats: many more overlaps than the buffers hold
    G()
    with pytest.raises(render.CapacityOverflow):
        G()
    assert R.overflows == 1 and R.capacity > cap
    G()
    G.check()
    same({k: v.grad for k, v in t.items()}, eager())


def test_differentiable_1M_scene_sampled_tiles(gs, orc):
    """1M-splat cluster scene at 1024x1024: L1 loss against the render of a
    perturbed copy. The full gradient is finite; with the loss restricted to
    four tiles the GPU gradient matches the FP64 oracle's reverse pass."""
    api, render, synth = gs
    from paper_2603_18707_b300 import autograd
    raw = synth.scene_clusters(1_000_000, 0, sh_degree=3)
    cam = synth.orbit_cameras(1, 1024, 1024)[0]
    Rt = render.Rasterizer([cam], api.make_config("poly1", "opacity"), 1_000_000)
    target = Rt.forward(render.activate(synth.perturbed(raw, 1))).clone()
    t = {k: torch.tensor(raw[k], device="cuda", requires_grad=True)
         for k in ("means", "log_scales", "quats", "opacity_logits", "sh")}
    R = render.Rasterizer([cam], api.make_config("poly1", "opacity"), 1_000_000)
    img = autograd.render(t["means"], t["log_scales"], t["quats"], t["opacity_logits"], t["sh"], 3, R)
    loss = (img - target).abs().mean()
    loss.backward()
    for v in t.values():
        assert torch.isfinite(v.grad).all()
    assert t["means"].grad.abs().sum() > 0
    # restricted loss: four tiles
    g = torch.sign(img.detach() - target).cpu().numpy().reshape(1024, 1024, 3)
    mask = np.zeros((1024, 1024, 1))
    for ty, tx in ((20, 20), (30, 33), (40, 25), (32, 32)):
        mask[ty * 16:(ty + 1) * 16, tx * 16:(tx + 1) * 16] = 1.0
    w = g * mask
    oc = orc.camera_from_dict(cam)
    sc = _oracle_inputs(orc, raw)
    cfg = orc.make_config("poly1", KIND_COEFFS["poly1"], "opacity")
    tiles = [ty * 64 + tx for ty, tx in ((20, 20), (30, 33), (40, 25), (32, 32))]
    *_, margin = orc.render_tiled(sc, oc, cfg, tiles=tiles, with_margin=True)
    w[margin < NEAR_MARGIN] = 0.0
    gpu, _ = _gpu_grads(api, render, raw, [cam], "poly1", "opacity", w, (0.0, 0.0, 0.0))
    ref = orc.render_backward(sc, oc, cfg, w, (0.0, 0.0, 0.0))
    _check(gpu, ref, name="1M-1024-sampled-tiles")


def test_backward_finite_differences_256_splats_64x64(gs, orc):
    """The finite-difference sub-case of the differentiable workload: 256
    splats (SH degree 3) at 64x64, f1 with opacity culling. GPU gradients
    against FP64 central differences of the oracle's forward, on 60 sampled
    entries of each parameter tensor where no skip / clamp / stop decision
    flips. Each entry whose gradient is not negligible (|fd| >= 1% of the
    tensor's largest) must agree within 1e-3 relative; the near-zero rest
    within 1e-5 of the largest (FP32 accumulation over many pixels leaves an
    absolute error of that order, which is no relative bound for a
    near-zero gradient)."""
    import json
    import os
    api, render, synth = gs
    raw = _small_scene(P=256, seed=11)
    cam = synth.look_at([0.3, -0.2, -2.5], [0, 0, 0], 64, 64, 60.0)
    oc = orc.camera_from_dict(cam)
    sc = _oracle_inputs(orc, raw)
    cfg = orc.make_config("poly1", KIND_COEFFS["poly1"], "opacity")
    bg = (0.1, 0.1, 0.1)
    w = _masked_weights(orc, sc, oc, "poly1", (64, 64, 3), seed=5)
    gpu, _ = _gpu_grads(api, render, raw, [cam], "poly1", "opacity", w, bg)
    base = orc.decisions(sc, oc, cfg)
    rng = np.random.default_rng(2)
    stats, checked = {}, 0
    for name in ("means", "scales", "quats", "opacities", "sh"):
        arr = sc[name]
        flat = list(np.ndindex(arr.shape))
        pairs = []
        for idx in [flat[i] for i in rng.choice(len(flat), min(60, len(flat)), replace=False)]:
            h = 1e-6 * max(1.0, abs(arr[idx]))
            vals = []
            for sgn in (1, -1):
                s2 = {k: (np.array(v, copy=True) if isinstance(v, np.ndarray) else v) for k, v in sc.items()}
                s2[name][idx] += sgn * h
                if not np.array_equal(orc.decisions(s2, oc, cfg), base):
                    break
                img, _, _ = orc.render_untiled(s2, oc, cfg, bg)
                vals.append((img * w).sum())
            if len(vals) == 2:
                pairs.append((gpu[name][idx], (vals[0] - vals[1]) / (2 * h)))
        g, fd = np.array(pairs).T
        big = np.abs(fd).max()
        sig = np.abs(fd) >= 0.01 * big
        rel = np.abs(g - fd)[sig] / np.abs(fd)[sig]
        small = np.abs(g - fd)[~sig] / big
        stats[name] = {"checked": int(g.size), "significant": int(sig.sum()),
                       "max_rel_significant": float(rel.max(initial=0.0)),
                       "max_abs_small_over_largest": float(small.max(initial=0.0))}
        assert sig.sum() >= 10, name
        assert rel.max() <= 1e-3, (name, stats[name])
        assert small.max(initial=0.0) <= 1e-5, (name, stats[name])
        checked += g.size
    rep = os.environ.get("GS_REPORT_DIR")
    if rep:
        os.makedirs(rep, exist_ok=True)
        with open(os.path.join(rep, "fd_256_64x64.json"), "w") as f:
            json.dump(stats, f, indent=1)
    assert checked >= 250
