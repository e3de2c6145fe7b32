"""torch.autograd.Function around the C ABI: forward jets and the hand-written
backward (weight gradient through the jets' chain rule and v''').

    from paper_2409_14248_gb300.autograd import HRKAN
    net = HRKAN([2, 32, 32, 1], G=20)            # owns a C-ABI handle
    jets = net(W, x, mask)                        # [J, N], differentiable in W
    loss = residual(jets).pow(2).mean(); loss.backward()

Gradients flow to the weights only (the coordinates are data).  When the
layer-wise path keeps a tape (hrkan_tape_floats > 0) and it fits the handle's
HBM budget, the forward stores the layer jets for the backward; otherwise the
backward recomputes them.  Everything runs in libhrkan.so's kernels.
"""
from __future__ import annotations

import torch

from . import capi


class _Jets(torch.autograd.Function):
    @staticmethod
    def forward(ctx, W, x, net, mask):
        N = x.shape[1]
        J = bin(int(mask) & 0xFFF).count("1")
        jets = torch.empty((J, N), dtype=torch.float32, device=W.device)
        tape = None
        n_tape = capi.hrkan_tape_floats(net.handle, N, mask)
        if n_tape > 0 and (net.hbm_budget_bytes == 0 or 4 * n_tape <= net.hbm_budget_bytes):
            tape = torch.empty(n_tape, dtype=torch.float32, device=W.device)
        capi.hrkan_forward_jets(net.handle, W, x, N, mask, jets, tape)
        ctx.net, ctx.mask = net, mask
        ctx.save_for_backward(W, x, tape if tape is not None else torch.empty(0, device=W.device))
        ctx.has_tape = tape is not None
        return jets

    @staticmethod
    def backward(ctx, g):
        W, x, tape = ctx.saved_tensors
        dW = torch.empty_like(W)
        capi.hrkan_backward(ctx.net.handle, W, x, x.shape[1], ctx.mask, tape if ctx.has_tape else None,
                            g.contiguous(), dW)
        return dW, None, None, None


class HRKAN:
    """A network shape bound to a C-ABI handle; call it to get differentiable jets."""

    def __init__(self, widths, G, k=3, m=4, lo=-1.0, hi=1.0, prec=capi.HRKAN_FP32, hbm_budget_bytes=0, flags=0):
        self.cfg = capi.make_cfg(widths, G, k, m, lo, hi, prec=prec, hbm_budget_bytes=hbm_budget_bytes,
                                 flags=flags)
        self.hbm_budget_bytes = hbm_budget_bytes
        self.handle = capi.hrkan_init(self.cfg)
        self.n_params = capi.hrkan_param_count(self.cfg)

    def __call__(self, W, x, mask):
        if W.dtype != torch.float32 or x.dtype != torch.float32 or not W.is_cuda or not x.is_cuda:
            raise ValueError("W and x must be float32 CUDA tensors")
        return _Jets.apply(W.contiguous(), x.contiguous(), self, int(mask))

    def close(self):
        if self.handle is not None:
            capi.hrkan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
