"""torch.autograd.Function over the C ABI: forward = gs_preprocess +
gs_bin_sort + gs_render, backward = gs_render_backward.

The library consumes activated values (scales, opacities, any-norm
quaternions); `render` applies the 3DGS activations (exp of log-scales,
sigmoid of opacity logits) in torch so that autograd chains through them.
"""
from __future__ import annotations

import torch

from . import api
from .render import CapacityOverflow, Rasterizer


class RenderFunction(torch.autograd.Function):
    """Images of one Rasterizer's cameras, [sum H W, 3], differentiable in
    means, scales, quats, opacities and SH. The rasterizer keeps the forward
    state (records, sorted lists, final T, last contributor) that the backward
    reads: run backward before the next forward on the same rasterizer."""

    @staticmethod
    def forward(ctx, means, scales, quats, opacities, sh, rasterizer: Rasterizer, sh_degree: int, bg,
                deferred: bool = False):
        sc = {"means": means.contiguous(), "scales": scales.contiguous(),
              "quats": quats.contiguous(), "opacities": opacities.contiguous(),
              "sh": sh.contiguous(), "sh_degree": int(sh_degree)}
        out = rasterizer.forward(sc, bg, n_eval=False, deferred=deferred)
        ctx.rasterizer = rasterizer
        ctx.sh_degree = int(sh_degree)
        ctx.bg = tuple(float(v) for v in bg)
        ctx.save_for_backward(sc["means"], sc["scales"], sc["quats"], sc["opacities"], sc["sh"])
        return out.clone()

    @staticmethod
    def backward(ctx, grad_out):
        means, scales, quats, opacities, sh = ctx.saved_tensors
        R = ctx.rasterizer
        g = {k: torch.zeros_like(v) for k, v in
             (("means", means), ("scales", scales), ("quats", quats), ("opacities", opacities),
              ("sh", sh))}
        grad2d = torch.empty(api.gs_grad2d_bytes(R.ncam, R.P), dtype=torch.uint8,
                             device=means.device)
        api.gs_render_backward(R.cams, R.P, R.cfg, means, scales, quats, opacities, sh,
                               ctx.sh_degree, R.splat2d, R.vals, R.ranges, ctx.bg, R.final_T,
                               R.last, grad_out.contiguous(), grad2d, g["means"], g["scales"],
                               g["quats"], g["opacities"], g["sh"])
        return g["means"], g["scales"], g["quats"], g["opacities"], g["sh"], None, None, None, None


def render(means, log_scales, quats, opacity_logits, sh, sh_degree, rasterizer, bg=(0.0, 0.0, 0.0),
           deferred: bool = False):
    """Differentiable render from raw 3DGS parameters. deferred=True checks
    the overlap capacity one call late instead of waiting for the GPU
    (Rasterizer.forward): a training step then never stalls on a read-back,
    and the rare step that overflowed raises render.CapacityOverflow at the
    next call, with the buffers already grown."""
    return RenderFunction.apply(means, torch.exp(log_scales), quats, torch.sigmoid(opacity_logits),
                                sh, rasterizer, sh_degree, bg, deferred)


class GraphedStep:
    """A whole training step captured once as a CUDA graph and replayed.

    fn() runs one step on tensors that keep their storage: `render(...,
    deferred=True)` on `rasterizer`, a loss, backward (with the parameters'
    .grad set to None first, so that the capture allocates them), optionally
    an optimizer update; it returns what the caller wants to read (e.g. the
    loss). The step's host work (its ~40 launches, the autograd graph) is
    paid once at capture; a replay is one graph launch, so the GPU runs the
    steps back to back. The overlap capacity is checked one replay late from
    the status the graph copies to pinned host memory: a replay that
    overflowed raises render.CapacityOverflow at the next call, after the
    rasterizer's buffers have been grown and the graph captured again, so
    that the caller can repeat that step."""

    def __init__(self, fn, rasterizer, warmup: int = 3):
        self.fn, self.R, self.warmup = fn, rasterizer, int(warmup)
        self._event = None
        self._capture()

    def _capture(self):
        self.out = None
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            for _ in range(max(1, self.warmup)):
                while True:
                    try:
                        self.fn()
                        break
                    except CapacityOverflow:
                        continue
            self.R.check_deferred()
        torch.cuda.current_stream().wait_stream(side)
        torch.cuda.synchronize()
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            out = self.fn()
        # detached views of the static outputs: holding a loss with its
        # grad_fn would keep the captured autograd graph (and its saved
        # tensors) alive
        self.out = out.detach() if isinstance(out, torch.Tensor) else out

    def check(self):
        """Raises CapacityOverflow (graph recaptured) if the last replay
        exceeded the overlap capacity."""
        ev, self._event = self._event, None
        if ev is None:
            return
        try:
            self.R.check_deferred(ev)
        except CapacityOverflow:
            self.graph = None
            self._capture()
            raise

    def __call__(self):
        self.check()
        self.graph.replay()
        self._event = torch.cuda.Event()
        self._event.record()
        return self.out
