"""Shared helpers of the GPU parity tests (not a test module)."""
from __future__ import annotations

import json
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
COEFFS = json.load(open(os.path.join(HERE, "golden", "coeffs.json")))
KIND_COEFFS = {"exp": (), "poly1": tuple(COEFFS["poly1"][:2]), "poly2": tuple(COEFFS["poly2"][:3]),
               "poly3": tuple(COEFFS["poly3"])}
TOL_FP32 = 2e-4      # per-channel absolute tolerance of the FP32 path
NEAR_MARGIN = 1e-3   # relative distance of a skip / stop decision treated as a threshold flip


def a256(x: int) -> int:
    return (x + 255) // 256 * 256


def parse_splat2d(buf: np.ndarray, N: int) -> dict:
    """Views of the record buffer written by gs_preprocess (layout of
    gs_splat2d_bytes in include/gs.h)."""
    buf = np.ascontiguousarray(buf).view(np.uint8)
    o = 0
    rec = buf[o:o + 48 * N].view(np.float32).reshape(N, 3, 4)
    o += a256(48 * N)
    rect = buf[o:o + 8 * N].view(np.uint16).reshape(N, 4)
    o += a256(8 * N)
    tiles = buf[o:o + 4 * N].view(np.uint32)
    o += a256(4 * N)
    dkey = buf[o:o + 4 * N].view(np.uint32)
    return {"mean2d": rec[:, 0, :2], "opacity": rec[:, 0, 2], "depth": rec[:, 0, 3],
            "conic": rec[:, 1, :3], "xcut": rec[:, 1, 3], "color": rec[:, 2, :3], "rho": rec[:, 2, 3],
            "rect": rect.astype(np.int64), "tiles": tiles.astype(np.int64), "dkey": dkey}


def expected_binning(rec: dict, cams, tile_w: int, tile_h: int, P: int):
    """CPU recomputation of the binning from the GPU's own per-record tile
    rectangles and depth keys: every (record, covered tile) pair, stably
    ordered by (global tile id, depth bits, record index)."""
    tiles_x = [(c["width"] + tile_w - 1) // tile_w for c in cams]
    tiles_y = [(c["height"] + tile_h - 1) // tile_h for c in cams]
    base = np.concatenate([[0], np.cumsum([a * b for a, b in zip(tiles_x, tiles_y)])])
    T, D, I = [], [], []
    for n in np.nonzero(rec["tiles"] > 0)[0]:
        c = n // P
        x0, y0, x1, y1 = rec["rect"][n]
        ys, xs = np.meshgrid(np.arange(y0, y1 + 1), np.arange(x0, x1 + 1), indexing="ij")
        t = base[c] + ys.ravel() * tiles_x[c] + xs.ravel()
        T.append(t)
        D.append(np.full(t.size, rec["dkey"][n], dtype=np.uint64))
        I.append(np.full(t.size, n, dtype=np.int64))
    if not T:
        return np.zeros(0, np.int64), np.zeros(0, np.uint64), np.zeros(2 * int(base[-1]), np.int64)
    T, D, I = np.concatenate(T), np.concatenate(D), np.concatenate(I)
    order = np.lexsort((I, D, T))
    T, D, I = T[order], D[order], I[order]
    keys = (T.astype(np.uint64) << np.uint64(32)) | D
    ranges = np.zeros((int(base[-1]), 2), dtype=np.int64)
    if T.size:
        starts = np.r_[0, np.nonzero(np.diff(T))[0] + 1]
        ends = np.r_[starts[1:], T.size]
        ranges[T[starts], 0] = starts
        ranges[T[starts], 1] = ends
    return I, keys, ranges.ravel()


def oracle_tile_list(o: dict, tile: int, tiles_x: int) -> np.ndarray:
    """Splat ids of the oracle's list for one tile, from the oracle's own
    projection records (splats_to_numpy): drawn splats whose rectangle
    contains the tile, in (depth, index) order."""
    tx, ty = tile % tiles_x, tile // tiles_x
    r = o["rect"]
    m = ((o["visible"] == 1) & (o["tiles"] > 0) & (r[:, 0] <= tx) & (r[:, 2] >= tx)
         & (r[:, 1] <= ty) & (r[:, 3] >= ty))
    ids = np.nonzero(m)[0]
    return ids[np.lexsort((ids, o["depth"][ids]))]


def n_eval_mismatches(nev_gpu: np.ndarray, nev_orc: np.ndarray, far: np.ndarray, O: np.ndarray,
                      G: np.ndarray) -> int:
    """Pixels of one tile (flattened arrays) whose GPU evaluation count is
    not the oracle's. The GPU's FP32 rectangles are conservative, so its list
    G may hold entries the oracle's list O lacks (all below eps at every pixel
    centre); a pixel that stops on O[e - 1] must stop on that same splat in G,
    and one that never stops evaluates all of G. With e == len(O) the oracle
    either stopped on its last entry or never stopped: both are accepted.
    Only pixels away from threshold flips (far) are compared."""
    pos = {int(s): k for k, s in enumerate(G.tolist())}
    bad = 0
    for p in np.nonzero(far)[0]:
        e, g = int(nev_orc[p]), int(nev_gpu[p])
        if e < O.size:
            ok = g == pos.get(int(O[e - 1]), -2) + 1
        else:
            ok = g == G.size or (O.size > 0 and g == pos.get(int(O[-1]), -2) + 1)
        bad += not ok
    return bad
