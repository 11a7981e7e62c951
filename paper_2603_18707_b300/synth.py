"""Seeded synthetic scenes and cameras shaped like the paper's workloads.

The paper evaluates trained 3DGS scenes of 1.0M-5.3M splats at SH degree 3
(Sec. 4, App. D, Table 5). Those datasets are not available here; these
generators stand in for them. Every draw uses numpy's PCG64 with an explicit
seed, in the order listed in each function.

This module holds no rendering arithmetic: it returns raw parameters
(means, log-scales, unnormalised quaternions, opacity logits, SH
coefficients) and camera matrices. Both the CUDA renderer and the test
oracle consume its output, each applying activations on its own side.
"""
from __future__ import annotations

import math

import numpy as np

# DC coefficient range for which the 3DGS colour model (0.5 + Y00 * dc with
# Y00 = 1/(2 sqrt(pi))) maps to colours uniform in [0, 1].
_DC_HALF_RANGE = math.sqrt(math.pi)


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def scene_uniform(P: int = 4096, seed: int = 0) -> dict:
    """Small scene: means U[-1,1]^3, log-scales N(-4.5, 0.5) per axis,
    quaternions N(0, I4) (uniform rotations once normalised), opacity logits
    N(0, 1.5), SH degree 0 with colour uniform in [0, 1]."""
    r = _rng(seed)
    means = r.uniform(-1.0, 1.0, (P, 3))
    log_scales = r.normal(-4.5, 0.5, (P, 3))
    quats = r.normal(0.0, 1.0, (P, 4))
    logits = r.normal(0.0, 1.5, P)
    dc = r.uniform(-_DC_HALF_RANGE, _DC_HALF_RANGE, (P, 1, 3))
    return _pack(means, log_scales, quats, logits, dc, 0)


def _random_rotation(r: np.random.Generator) -> np.ndarray:
    q, rr = np.linalg.qr(r.normal(size=(3, 3)))
    q = q * np.sign(np.diag(rr))
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q


def scene_clusters(P: int, seed: int = 0, sh_degree: int = 3, n_clusters: int = 64) -> dict:
    """Paper-scale scene: 90% of the means from a mixture of anisotropic
    clusters (centres U[-8,8]^3, per-axis sigma log-uniform in [0.3, 2.0],
    random orientation, equal weights, clipped to [-10,10]^3), 10% on a
    spherical shell of radius U[40, 50]. Log-scales N(-4, 1) clipped to
    [-9, -1]; opacity logits N(1, 2) (bimodal opacities near 0 and 1); SH DC
    giving colours uniform in [0, 1], higher bands N(0, 0.1)."""
    r = _rng(seed)
    n_bg = P // 10
    n_cl = P - n_bg
    centres = r.uniform(-8.0, 8.0, (n_clusters, 3))
    sig = np.exp(r.uniform(np.log(0.3), np.log(2.0), (n_clusters, 3)))
    rots = np.stack([_random_rotation(r) for _ in range(n_clusters)])
    assign = r.integers(0, n_clusters, n_cl)
    z = r.normal(size=(n_cl, 3))
    local = z * sig[assign]
    pts = centres[assign] + np.einsum("nij,nj->ni", rots[assign], local)
    pts = np.clip(pts, -10.0, 10.0)
    d = r.normal(size=(n_bg, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    shell = d * r.uniform(40.0, 50.0, (n_bg, 1))
    means = np.concatenate([pts, shell], axis=0)
    log_scales = np.clip(r.normal(-4.0, 1.0, (P, 3)), -9.0, -1.0)
    quats = r.normal(0.0, 1.0, (P, 4))
    logits = r.normal(1.0, 2.0, P)
    K = (sh_degree + 1) ** 2
    sh = np.empty((P, K, 3))
    sh[:, 0, :] = r.uniform(-_DC_HALF_RANGE, _DC_HALF_RANGE, (P, 3))
    if K > 1:
        sh[:, 1:, :] = r.normal(0.0, 0.1, (P, K - 1, 3))
    return _pack(means, log_scales, quats, logits, sh, sh_degree)


def perturbed(scene: dict, seed: int = 1) -> dict:
    """Copy of a scene with seeded perturbations (target of the
    differentiable-render workload): means + N(0, 0.01), log-scales +
    N(0, 0.1), logits + N(0, 0.5), SH + N(0, 0.05)."""
    r = _rng(seed)
    P = scene["means"].shape[0]
    out = dict(scene)
    out["means"] = (scene["means"] + r.normal(0.0, 0.01, (P, 3))).astype(np.float32)
    out["log_scales"] = (scene["log_scales"] + r.normal(0.0, 0.1, (P, 3))).astype(np.float32)
    out["opacity_logits"] = (scene["opacity_logits"] + r.normal(0.0, 0.5, P)).astype(np.float32)
    out["sh"] = (scene["sh"] + r.normal(0.0, 0.05, scene["sh"].shape)).astype(np.float32)
    return out


def _pack(means, log_scales, quats, logits, sh, deg) -> dict:
    f = np.float32
    return {"means": np.ascontiguousarray(means, dtype=f),
            "log_scales": np.ascontiguousarray(log_scales, dtype=f),
            "quats": np.ascontiguousarray(quats, dtype=f),
            "opacity_logits": np.ascontiguousarray(logits, dtype=f),
            "sh": np.ascontiguousarray(sh, dtype=f),
            "sh_degree": int(deg)}


# --------------------------------------------------------------------------
# Cameras
# --------------------------------------------------------------------------

def look_at(pos, target, width: int, height: int, fovx_deg: float = 60.0, znear: float = 0.2) -> dict:
    """Pinhole camera at ``pos`` looking at ``target``. Camera axes: +z
    forward, +x right, +y down; world "up" is -y (so the default scene camera
    has an identity rotation). Principal point at the image centre, square
    pixels, fx = (W/2) / tan(fovx/2)."""
    pos = np.asarray(pos, dtype=np.float64)
    f = np.asarray(target, dtype=np.float64) - pos
    f /= np.linalg.norm(f)
    up = np.array([0.0, -1.0, 0.0])
    rgt = np.cross(f, up)
    if np.linalg.norm(rgt) < 1e-9:
        rgt = np.array([1.0, 0.0, 0.0])
    rgt /= np.linalg.norm(rgt)
    dwn = np.cross(f, rgt)
    R = np.stack([rgt, dwn, f])
    vm = np.eye(4)
    vm[:3, :3] = R
    vm[:3, 3] = -R @ pos
    fx = 0.5 * width / math.tan(math.radians(fovx_deg) / 2.0)
    return {"viewmat": vm, "fx": fx, "fy": fx, "cx": 0.5 * width, "cy": 0.5 * height,
            "width": int(width), "height": int(height), "znear": float(znear)}


def camera_small(width: int = 128, height: int = 128) -> dict:
    """Camera of the small scene: at z = -3 looking at the origin, fov 60 deg."""
    return look_at([0.0, 0.0, -3.0], [0.0, 0.0, 0.0], width, height, 60.0)


def orbit_cameras(n: int, width: int = 1920, height: int = 1080, radius: float = 18.0,
                  height_above: float = 2.0, fovx_deg: float = 60.0, phase: float = 0.0) -> list:
    """n cameras evenly spaced on a horizontal orbit around the origin, the
    k-th at angle 2 pi (k + phase) / n."""
    cams = []
    for k in range(n):
        a = 2.0 * math.pi * (k + phase) / n
        pos = [radius * math.sin(a), -height_above, -radius * math.cos(a)]
        cams.append(look_at(pos, [0.0, 0.0, 0.0], width, height, fovx_deg))
    return cams


def shard_orbit(n: int, rank: int, world: int, width: int = 1920, height: int = 1080) -> list:
    """Rank `rank` of `world`: n orbit cameras interleaved with the other
    ranks' (phase rank / world), so that the ranks together render the
    n * world views of one orbit and each rank as many as a single GPU."""
    return orbit_cameras(n, width, height, phase=rank / world)


def mixed_cameras(n: int = 64, radius: float = 18.0) -> list:
    """Batched-serving camera set: resolutions 640x360, 1280x720, 1920x1080
    and 3840x2160 in a 4:3:2:1 ratio (largest-remainder rounding), spread over
    an orbit with heights alternating in [-1, 5]."""
    ratio = [4, 3, 2, 1]
    res = [(640, 360), (1280, 720), (1920, 1080), (3840, 2160)]
    exact = [n * w / sum(ratio) for w in ratio]
    counts = [int(math.floor(e)) for e in exact]
    order = sorted(range(4), key=lambda i: -(exact[i] - counts[i]))
    for i in order[: n - sum(counts)]:
        counts[i] += 1
    cams = []
    k = 0
    for (w, h), c in zip(res, counts):
        for _ in range(c):
            a = 2.0 * math.pi * k / n
            hgt = -1.0 + 6.0 * ((k * 7) % n) / max(n - 1, 1)
            pos = [radius * math.sin(a), -hgt, -radius * math.cos(a)]
            cams.append(look_at(pos, [0.0, 0.0, 0.0], w, h, 60.0))
            k += 1
    return cams
