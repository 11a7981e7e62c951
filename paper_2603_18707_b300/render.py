"""Frame-level driver: owns the device buffers of one camera set and runs
preprocess -> bin/sort -> blend on the current CUDA stream.

Buffer management only (torch allocates, the library computes). The overlap
capacity is sized on first use: a run whose overlap count exceeds the
capacity is detected from the device counters and repeated with a larger
buffer (outside any timed or captured region).
"""
from __future__ import annotations

import torch

from . import api
from ._lib import GS_ERR_CAPACITY

MAX_CAPACITY = (1 << 30) - 2  # the binning's counters hold 30 bits (< 2^30 - 1 overlaps)


class CapacityOverflow(RuntimeError):
    """A deferred pass had more tile overlaps than the buffers held; they
    have been grown, and the pass should be repeated."""


def activate(scene: dict, device="cuda") -> dict:
    """3DGS activations of raw parameters: scale = exp(log-scale), opacity =
    sigmoid(logit). Means, quaternions (normalised inside the library) and SH
    are passed through."""
    t = lambda a: torch.as_tensor(a, dtype=torch.float32, device=device).contiguous()
    return {"means": t(scene["means"]), "scales": torch.exp(t(scene["log_scales"])),
            "quats": t(scene["quats"]), "opacities": torch.sigmoid(t(scene["opacity_logits"])),
            "sh": t(scene["sh"]), "sh_degree": int(scene["sh_degree"])}


def spatial_order(scene: dict, keys=("means", "scales", "quats", "opacities", "sh", "log_scales",
                                      "opacity_logits")) -> tuple[dict, torch.Tensor]:
    """The scene's splats stored along a Z-order curve of their means (a
    one-time preparation when a scene is loaded; gs_spatial_order +
    gs_gather_rows on the GPU). Returns the reordered scene (device tensors,
    other entries passed through) and the permutation: new row k is old row
    perm[k]. Images are unchanged except where two splats meet in a tile at
    exactly equal depth."""
    dev = torch.device("cuda")
    means = torch.as_tensor(scene["means"], dtype=torch.float32, device=dev).contiguous()
    perm = api.gs_spatial_order(means)
    out = {}
    for k, v in scene.items():
        if k in keys:
            t = torch.as_tensor(v, device=dev).contiguous()
            out[k] = api.gs_gather_rows(t, perm)
        else:
            out[k] = v
    return out, perm


class Rasterizer:
    """Renders P splats into a fixed list of cameras (at most 64)."""

    def __init__(self, cams, cfg, P: int, capacity: int | None = None, device="cuda",
                 keep_keys: bool = False, persistent: bool = False, outputs: dict | None = None,
                 last: bool = True):
        """outputs: optional views (out [npix, 3], final_T, last, n_eval [npix])
        to render into instead of buffers of its own. last=False: the blend
        does not keep each pixel's last contributor (`self.last` is left
        unwritten), which only the reverse pass reads; the image and final T
        are the same and the blend does less work per entry."""
        self.cams = api.camera_array(cams)
        self.ncam = len(self.cams)
        self.cfg = cfg
        self.P = int(P)
        self.device = torch.device(device)
        self.total_tiles = api.gs_total_tiles(self.cams, cfg)
        self.sizes = [(c.height, c.width) for c in self.cams]
        self.npix = sum(h * w for h, w in self.sizes)
        u8 = dict(dtype=torch.uint8, device=self.device)
        i32 = dict(dtype=torch.int32, device=self.device)
        self.splat2d = torch.empty(api.gs_splat2d_bytes(self.ncam, self.P), **u8)
        self.ranges = torch.zeros(2 * self.total_tiles, **i32)
        self.count = torch.zeros(3, **i32)
        if outputs is not None:
            self.out, self.final_T = outputs["out"], outputs["final_T"]
            self.last, self.n_eval = outputs["last"], outputs["n_eval"]
        else:
            self.out = torch.empty(self.npix, 3, dtype=torch.float32, device=self.device)
            self.final_T = torch.empty(self.npix, dtype=torch.float32, device=self.device)
            self.last = torch.empty(self.npix, **i32)
            self.n_eval = torch.empty(self.npix, **i32)
        self.keep_keys = keep_keys
        self.keep_last = bool(last)
        self.work = (torch.zeros(api.gs_render_work_bytes(), **u8) if persistent else None)
        self.shrink = capacity is None  # an explicit capacity is kept as given
        self.capacity = 0
        self.sized = False  # a synchronous forward() has fitted the capacity
        self.overflows = 0  # deferred passes found to have exceeded the capacity
        self._pending = None
        self._status_dev = torch.zeros(4, **i32)
        self._status_host = torch.zeros(4, dtype=torch.int32).pin_memory() if self.device.type == "cuda" else None
        self._alloc(capacity if capacity else min(max(1 << 20, 8 * self.ncam * self.P), MAX_CAPACITY))

    def _alloc(self, capacity: int):
        self.capacity = int(capacity)
        ws = api.gs_bin_sort_workspace_bytes(self.cams, self.P, self.cfg, self.capacity)
        self.workspace = torch.empty(ws, dtype=torch.uint8, device=self.device)
        self.vals = torch.empty(max(self.capacity, 1), dtype=torch.int32, device=self.device)
        self.keys64 = (torch.empty(max(self.capacity, 1), dtype=torch.int64, device=self.device)
                       if self.keep_keys else None)

    def set_cameras(self, cams):
        """New poses (and intrinsics) for the same number of cameras at the
        same resolutions: the buffers stay valid. Cameras reach the kernels
        as launch parameters, so this costs no device copy."""
        arr = api.camera_array(cams)
        if len(arr) != self.ncam or any((a.width, a.height) != (b.width, b.height)
                                        for a, b in zip(arr, self.cams)):
            raise ValueError("set_cameras keeps the camera count and resolutions")
        self.cams = arr

    def preprocess(self, sc: dict):
        api.gs_preprocess(self.cams, self.P, sc["means"], sc["scales"], sc["quats"],
                          sc["opacities"], sc["sh"], sc["sh_degree"], self.cfg, self.splat2d)

    def bin_sort(self):
        api.gs_bin_sort(self.cams, self.P, self.cfg, self.splat2d, self.capacity, self.workspace,
                        self.vals, self.ranges, self.keys64, self.count)

    def blend(self, bg=(0.0, 0.0, 0.0), n_eval: bool = True):
        api.gs_render(self.cams, self.P, self.cfg, self.splat2d, self.vals, self.ranges, bg,
                      self.out, self.final_T, self.last if self.keep_last else None,
                      self.n_eval if n_eval else None,
                      self.work)

    def forward(self, sc: dict, bg=(0.0, 0.0, 0.0), n_eval: bool = True, deferred: bool = False):
        """One pass of the whole path; grows the overlap buffer when it was
        too small and shrinks it when it is far too large (the sort's grids
        and look-back state scale with the capacity), then reruns.

        deferred=True (once a synchronous pass has sized the buffers) runs the
        pass without waiting for the GPU: the device error word and the
        overlap count are copied to pinned host memory behind the pass and
        checked at the next deferred call, so a training loop never stalls
        the GPU on a read-back. A pass that overflowed the capacity (its
        image and gradients miss the overlaps beyond it) is found one call
        later: that call grows the buffers, counts it in `overflows` and
        raises CapacityOverflow, so the caller can repeat the step."""
        if deferred and self.sized:
            self.check_deferred()
            self.run_async(sc, bg, n_eval)
            api.gs_workspace_status_async(self.workspace, self._status_dev[0:1])
            self._status_dev[1:4].copy_(self.count)
            self._status_host.copy_(self._status_dev, non_blocking=True)
            if torch.cuda.is_current_stream_capturing():
                return self.out  # a graph's replays are checked by their owner (autograd.GraphedStep)
            ev = torch.cuda.Event()
            ev.record()
            self._pending = ev
            return self.out
        self._pending = None
        for _ in range(4):
            self.preprocess(sc)
            self.bin_sort()
            self.blend(bg, n_eval)
            err = api.gs_workspace_status(self.workspace)
            need = int(self.count[2].item() & 0xFFFFFFFF)
            if not err & GS_ERR_CAPACITY:
                if err:
                    raise RuntimeError(f"device error word {err}")
                if self.shrink and self.capacity > 2 * need + (1 << 16):
                    self._alloc(int(need * 1.15) + 4096)
                    continue
                self.sized = True
                return self.out
            if self.capacity >= MAX_CAPACITY:
                raise RuntimeError("more than 2^30 - 1 tile overlaps: split the camera batch")
            self._alloc(min(int(max(need, self.capacity) * 1.25) + 1024, MAX_CAPACITY))
        raise RuntimeError("overlap capacity could not be sized")

    def check_deferred(self, event=None):
        """Waits for the last deferred pass's status copy (normally long
        complete; `event`: one recorded after it, e.g. after a graph replay)
        and raises CapacityOverflow, after growing the buffers, if that pass
        exceeded the overlap capacity."""
        ev, self._pending = (event if event is not None else self._pending), None
        if ev is None:
            return
        ev.synchronize()
        err, need = int(self._status_host[0]), int(self._status_host[3]) & 0xFFFFFFFF
        if err & GS_ERR_CAPACITY:
            self.overflows += 1
            if self.capacity >= MAX_CAPACITY:
                raise RuntimeError("more than 2^30 - 1 tile overlaps: split the camera batch")
            self._alloc(min(int(max(need, self.capacity) * 1.25) + 1024, MAX_CAPACITY))
            raise CapacityOverflow(f"the previous pass needed {need} overlaps; capacity grown to {self.capacity}")
        if err:
            raise RuntimeError(f"device error word {err}")

    def run_async(self, sc: dict, bg=(0.0, 0.0, 0.0), n_eval: bool = False):
        """The same pass without any host synchronisation (for timing and
        graph capture, after forward() has sized the buffers)."""
        self.preprocess(sc)
        self.bin_sort()
        self.blend(bg, n_eval)
        return self.out

    def capture(self, sc: dict, bg=(0.0, 0.0, 0.0), n_eval: bool = False):
        """CUDA graph of one whole pass (every launch and memset of
        preprocess, bin/sort and blend) over the given, fixed input tensors.
        Call forward() first so that the buffers are sized; replay with
        graph.replay()."""
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            self.run_async(sc, bg, n_eval)  # warm-up on the capture stream
        torch.cuda.current_stream().wait_stream(side)
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            self.run_async(sc, bg, n_eval)
        return graph

    def images(self):
        out, o = [], 0
        for h, w in self.sizes:
            out.append(self.out[o:o + h * w].view(h, w, 3))
            o += h * w
        return out

    def per_camera(self, t):
        out, o = [], 0
        for h, w in self.sizes:
            out.append(t[o:o + h * w].view(h, w))
            o += h * w
        return out

    def n_records(self) -> tuple[int, int]:
        c = self.count.cpu().tolist()
        return c[0] & 0xFFFFFFFF, c[1] & 0xFFFFFFFF


class StreamedRasterizer:
    """The cameras split into `groups` consecutive sets, each with a
    Rasterizer of its own rendering into its slice of shared output buffers,
    and each set's pass (preprocess, bin/sort, blend) issued on a stream of
    its own: one set's latency-bound sort overlaps another's ALU-bound blend.
    persistent: each set's blend as one persistent launch; last: see Rasterizer.
    Same interface as Rasterizer; the work per pass is the same."""

    def __init__(self, cams, cfg, P: int, groups: int = 2, device="cuda", keep_keys: bool = False,
                 persistent: bool = False, last: bool = True):
        cams = list(cams)
        groups = max(1, min(int(groups), len(cams)))
        bounds = [round(k * len(cams) / groups) for k in range(groups + 1)]
        sets = [cams[bounds[k]:bounds[k + 1]] for k in range(groups)]
        self.cams = api.camera_array(cams)
        self.ncam = len(cams)
        self.cfg = cfg
        self.P = int(P)
        self.device = torch.device(device)
        self.sizes = [(c.height, c.width) for c in self.cams]
        self.npix = sum(h * w for h, w in self.sizes)
        i32 = dict(dtype=torch.int32, device=self.device)
        self.out = torch.empty(self.npix, 3, dtype=torch.float32, device=self.device)
        self.final_T = torch.empty(self.npix, dtype=torch.float32, device=self.device)
        self.last = torch.empty(self.npix, **i32)
        self.n_eval = torch.empty(self.npix, **i32)
        self.parts, o = [], 0
        for cs in sets:
            n = sum(c["height"] * c["width"] for c in cs)
            views = {"out": self.out[o:o + n], "final_T": self.final_T[o:o + n],
                     "last": self.last[o:o + n], "n_eval": self.n_eval[o:o + n]}
            self.parts.append(Rasterizer(cs, cfg, P, device=device, keep_keys=keep_keys, outputs=views,
                                         persistent=persistent, last=last))
            o += n
        self.streams = [torch.cuda.Stream(device=self.device) for _ in self.parts]
        self.bounds = bounds

    def set_cameras(self, cams):
        cams = list(cams)
        if len(cams) != self.ncam:
            raise ValueError("set_cameras keeps the camera count and resolutions")
        for k, r in enumerate(self.parts):
            r.set_cameras(cams[self.bounds[k]:self.bounds[k + 1]])
        self.cams = api.camera_array(cams)

    def preprocess(self, sc: dict):
        for r in self.parts:
            r.preprocess(sc)

    def bin_sort(self):
        for r in self.parts:
            r.bin_sort()

    def blend(self, bg=(0.0, 0.0, 0.0), n_eval: bool = True):
        for r in self.parts:
            r.blend(bg, n_eval)

    def forward(self, sc: dict, bg=(0.0, 0.0, 0.0), n_eval: bool = True, deferred: bool = False):
        for r in self.parts:
            r.forward(sc, bg, n_eval, deferred)
        return self.out

    def run_async(self, sc: dict, bg=(0.0, 0.0, 0.0), n_eval: bool = False):
        cur = torch.cuda.current_stream(self.device)
        for r, st in zip(self.parts, self.streams):
            st.wait_stream(cur)
            with torch.cuda.stream(st):
                r.run_async(sc, bg, n_eval)
        for st in self.streams:
            cur.wait_stream(st)
        return self.out

    def capture(self, sc: dict, bg=(0.0, 0.0, 0.0), n_eval: bool = False):
        side = torch.cuda.Stream(device=self.device)
        side.wait_stream(torch.cuda.current_stream(self.device))
        with torch.cuda.stream(side):
            self.run_async(sc, bg, n_eval)
        torch.cuda.current_stream(self.device).wait_stream(side)
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            self.run_async(sc, bg, n_eval)
        return graph

    def images(self):
        return Rasterizer.images(self)

    def per_camera(self, t):
        return Rasterizer.per_camera(self, t)

    def n_records(self) -> tuple[int, int]:
        recs = [r.n_records() for r in self.parts]
        return sum(a for a, _ in recs), sum(b for _, b in recs)


class HostPipeline:
    """Frames from pinned host inputs to pinned host images: step k's
    upload and step k-1's download run on copy streams of their own while
    the rasterizer renders, with two device copies of the inputs and of the
    image so that no step waits for a copy it does not need. Every step
    uploads its whole input and downloads its whole image."""

    KEYS = ("means", "scales", "quats", "opacities", "sh")

    def __init__(self, raster, upload_streams: int = 1):
        self.R = raster
        dev = raster.out.device
        # uploads may be split by rows over several copy streams (measured:
        # one stream already runs at the host link's rate)
        self.up = [torch.cuda.Stream(device=dev) for _ in range(max(1, int(upload_streams)))]
        self.h2d = self.up[0]
        self.d2h = torch.cuda.Stream(device=dev)
        self.dev_in = [None, None]
        self.dev_out = [torch.empty_like(raster.out) for _ in range(2)]
        self.ev_in_free = [torch.cuda.Event(), torch.cuda.Event()]
        self.ev_uploaded = [torch.cuda.Event(), torch.cuda.Event()]
        self.ev_rendered = [torch.cuda.Event(), torch.cuda.Event()]
        self.ev_out_free = [torch.cuda.Event(), torch.cuda.Event()]
        self.k = 0

    def step(self, host_in: dict, host_out: torch.Tensor):
        """Enqueues one frame: host_in (pinned tensors of the activated scene,
        plus sh_degree) -> host_out (pinned, the shape of raster.out)."""
        b = self.k & 1
        self.k += 1
        if self.dev_in[b] is None:
            self.dev_in[b] = {k: torch.empty_like(host_in[k], device=self.R.out.device) for k in self.KEYS}
            self.dev_in[b]["sh_degree"] = int(host_in["sh_degree"])
        cur = torch.cuda.current_stream(self.R.out.device)
        m = len(self.up)
        for i, st in enumerate(self.up):
            st.wait_event(self.ev_in_free[b])  # the render that read these inputs is done
            with torch.cuda.stream(st):
                for k in self.KEYS:
                    n = host_in[k].shape[0]
                    lo, hi = n * i // m, n * (i + 1) // m
                    self.dev_in[b][k][lo:hi].copy_(host_in[k][lo:hi], non_blocking=True)
        for st in self.up[1:]:
            self.h2d.wait_stream(st)
        self.ev_uploaded[b].record(self.h2d)
        cur.wait_event(self.ev_uploaded[b])
        cur.wait_event(self.ev_out_free[b])  # the download of this image buffer is done
        self.R.run_async(self.dev_in[b])
        self.dev_out[b].copy_(self.R.out, non_blocking=True)
        self.ev_in_free[b].record(cur)
        self.ev_rendered[b].record(cur)
        self.d2h.wait_event(self.ev_rendered[b])
        with torch.cuda.stream(self.d2h):
            host_out.copy_(self.dev_out[b], non_blocking=True)
            self.ev_out_free[b].record(self.d2h)

    def step_views(self, sc: dict, cams, host_out: torch.Tensor):
        """Enqueues one frame of a resident scene (serving): new camera
        poses (launch parameters, no copy) -> host_out (pinned). Step k's
        download runs on the copy stream while step k + 1 renders."""
        b = self.k & 1
        self.k += 1
        cur = torch.cuda.current_stream(self.R.out.device)
        cur.wait_event(self.ev_out_free[b])  # the download of this image buffer is done
        self.R.set_cameras(cams)
        self.R.run_async(sc)
        self.dev_out[b].copy_(self.R.out, non_blocking=True)
        self.ev_rendered[b].record(cur)
        self.d2h.wait_event(self.ev_rendered[b])
        with torch.cuda.stream(self.d2h):
            host_out.copy_(self.dev_out[b], non_blocking=True)
            self.ev_out_free[b].record(self.d2h)

    def finish(self):
        """Makes the current stream wait for every enqueued download."""
        torch.cuda.current_stream(self.R.out.device).wait_stream(self.d2h)
