"""Differentiable sampling: the in-bin positions as a function of the weights.

``sample_positions(w, u, m)`` builds the structure of the weights and maps the
samples through it (Algorithm 2 and the in-bin position of Sec. 5 of the
paper); the bins are piecewise constant in w, the positions are not.  The
backward pass calls ``rtf_sample_backward``: with every sample's bin held
fixed, the position is x = (xi W - C_i) / w_i, whose gradient the library
accumulates per bin and turns into dL/dw with a reverse suffix scan.

Only argument marshalling happens here; the build, the sampling and the
gradient run in the CUDA library.
"""

from __future__ import annotations

import torch

from . import api


class SamplePositions(torch.autograd.Function):
    """forward(w, u, m) -> (pos, idx); only pos carries a gradient."""

    @staticmethod
    def forward(ctx, w: torch.Tensor, u: torch.Tensor, m: int):
        f = api.rtf_build(w.detach().contiguous(), m)
        idx, pos = api.rtf_sample(f, u)
        ctx.forest = f
        ctx.save_for_backward(w, u, idx, pos)
        ctx.mark_non_differentiable(idx)
        return pos, idx

    @staticmethod
    def backward(ctx, grad_pos, grad_idx):
        w, u, idx, pos = ctx.saved_tensors
        gw = None
        if ctx.needs_input_grad[0]:
            gw = api.rtf_sample_backward(ctx.forest, w.detach().contiguous(), u, None, idx, pos,
                                         grad_pos.contiguous().to(torch.float32))
        return gw, None, None


class SamplePositions2D(torch.autograd.Function):
    """forward(lum, u, m_row, m_col) -> (pos[count, 2], idx[count, 2]) for a
    piecewise constant map lum[rows, cols] (component-wise sampling, Sec. 5)."""

    @staticmethod
    def forward(ctx, lum: torch.Tensor, u: torch.Tensor, m_row: int, m_col: int):
        H, W = lum.shape
        sizes = [W] * H + [H]
        ms = [m_col] * H + [m_row]
        f = api.rtf_build_batched(lum.detach().contiguous().view(-1), sizes, ms, marginal=True)
        idx, pos = api.rtf_sample(f, u, mode=api.SAMPLE_2D)
        ctx.forest = f
        ctx.shape = (H, W)
        ctx.save_for_backward(lum, u, idx, pos)
        ctx.mark_non_differentiable(idx)
        return pos, idx

    @staticmethod
    def backward(ctx, grad_pos, grad_idx):
        lum, u, idx, pos = ctx.saved_tensors
        gl = None
        if ctx.needs_input_grad[0]:
            g = api.rtf_sample_backward(ctx.forest, lum.detach().contiguous().view(-1), u, None,
                                        idx, pos, grad_pos.contiguous().to(torch.float32),
                                        mode=api.SAMPLE_2D)
            gl = g.view(ctx.shape)
        return gl, None, None, None


def sample_positions(w: torch.Tensor, u: torch.Tensor, m: int):
    """In-bin positions (differentiable in w) and bins of uint32 samples `u`."""
    return SamplePositions.apply(w, u, m)


def sample_positions_2d(lum: torch.Tensor, u: torch.Tensor, m_row: int, m_col: int):
    """2-D positions (row, column; differentiable in lum) and (row, column) bins
    of (u1, u2) sample pairs."""
    return SamplePositions2D.apply(lum, u, m_row, m_col)
