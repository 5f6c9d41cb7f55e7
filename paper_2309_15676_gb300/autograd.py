"""torch.autograd.Function over the library's render and path-replay adjoint.

forward renders with a fixed Philox key (problem, stream, iteration, spp); backward calls
the hand-written adjoint kernels, which recompute every path from that key instead of
storing vertices (path replay as checkpointing).
"""
from __future__ import annotations

import torch

from .api import STREAM_EVAL, Context


class RenderFn(torch.autograd.Function):
    @staticmethod
    def forward(fctx, tex: torch.Tensor, mctx: Context, pid: int, spp: int, stream: int, iteration: int):
        img = mctx.render(pid, tex.detach(), spp, stream, iteration)
        fctx.save_for_backward(tex)
        fctx.key = (mctx, pid, spp, stream, iteration)
        return img

    @staticmethod
    def backward(fctx, dimg: torch.Tensor):
        (tex,) = fctx.saved_tensors
        mctx, pid, spp, stream, iteration = fctx.key
        g = mctx.adjoint(pid, tex.detach(), dimg.contiguous(), spp, stream, iteration)
        return g, None, None, None, None, None


def render(mctx: Context, pid: int, tex: torch.Tensor, spp: int = 1, stream: int = STREAM_EVAL,
           iteration: int = 0) -> torch.Tensor:
    """Differentiable render of problem pid with texture tex (HWC, on the context's device)."""
    return RenderFn.apply(tex, mctx, pid, spp, stream, iteration)
