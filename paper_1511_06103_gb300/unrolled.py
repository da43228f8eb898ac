"""Differentiable unrolled inference: K parallel proximal steps (Sec. 3.1,
Eq. method:update_natural) from q^0 = softmax(-U), as a torch autograd
function whose backward is the library's hand-written reverse pass.

The step eta is held constant in the gradient (it is not differentiated
through the curvature bound Lambda).  Marshalling only: the forward and the
backward each run entirely in the CUDA library.
"""
from __future__ import annotations

import torch

from . import binding

_handles: dict = {}


def _handle(conn: int, L: int, H: int, W: int, B: int, device: torch.device):
    stream = torch.cuda.current_stream(device).cuda_stream
    key = (conn, L, H, W, B, device.index, stream)
    h = _handles.get(key)
    if h is None:
        topo = binding.CRF_GRID8 if conn == 8 else binding.CRF_GRID4
        h = binding.CRF(topo, L, H, W, batch=B, stream=stream)
        h.owner = None
        _handles[key] = h
    return h


class UnrolledMeanField(torch.autograd.Function):
    """log q^K = UnrolledMeanField.apply(U, mu, w, H, W, conn, K, eta).

    U [B][H*W][L], mu [L][L], w [B][n_dirs][H][W] (n_dirs 2 for conn 4, 4 for
    conn 8), all float32 CUDA tensors.  Returns log q^K [B][H*W][L]."""

    @staticmethod
    def forward(ctx, U, mu, w, H: int, W: int, conn: int, K: int, eta: float):
        B, N, L = U.shape
        if N != H * W or tuple(mu.shape) != (L, L):
            raise ValueError("U must be [B][H*W][L] and mu [L][L]")
        U, mu, w = U.contiguous(), mu.contiguous(), w.contiguous()
        crf = _handle(conn, L, H, W, B, U.device)
        crf.set_unary(U)
        crf.set_pairwise(mu, w)
        ckpt = torch.empty(crf.checkpoint_floats(K), dtype=torch.float32, device=U.device)
        crf.unrolled_forward(K, eta, ckpt)
        out = torch.empty((B, N, L), dtype=torch.float32, device=U.device)
        crf.log_marginals(out)
        token = object()
        crf.owner = token
        ctx.save_for_backward(ckpt, mu, w)
        ctx.crf, ctx.token, ctx.K, ctx.eta = crf, token, K, eta
        return out

    @staticmethod
    def backward(ctx, g):
        ckpt, mu, w = ctx.saved_tensors
        crf = ctx.crf
        if crf.owner is not ctx.token:
            # the handle served another forward since: restore this one's pairwise terms
            crf.set_pairwise(mu, w)
            crf.owner = ctx.token
        dU, dmu, dw = crf.unrolled_backward(ctx.K, ctx.eta, ckpt, g.contiguous())
        return dU, dmu, dw, None, None, None, None, None


def unrolled_log_marginals(U, mu, w, H: int, W: int, conn: int, K: int, eta: float):
    return UnrolledMeanField.apply(U, mu, w, H, W, conn, K, eta)
