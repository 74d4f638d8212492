"""torch.autograd.Function over the CUDA ELBO kernels.

``NegELBO.apply(loc, raw, eps, ctx)`` returns the negative Monte-Carlo ELBO
(Sec. 3.2) as a float64 scalar tensor; its backward calls the library's
hand-written backward kernel, which recomputes the profiles from (loc, raw,
eps) instead of keeping anything of size S*K*N from the forward.  Tensors are
CUDA float32: loc, raw [K, 5], eps [S, K, 5] standard normals.  The context's
kernels run on torch's current stream.
"""
from __future__ import annotations

import torch

from . import xrdvi


def _bind_stream(c: xrdvi.Context):
    s = torch.cuda.current_stream().cuda_stream
    if getattr(c, "_torch_stream", None) != s:
        c.set_stream(s)
        c._torch_stream = s


def _check(t, shape, name):
    if not (t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
        raise TypeError(f"{name} must be a contiguous CUDA float32 tensor")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")


class NegELBO(torch.autograd.Function):
    @staticmethod
    def forward(fctx, loc, raw, eps, c: xrdvi.Context):
        info = c.info
        K, S = info.K, info.S
        _check(loc, (K, 5), "loc")
        _check(raw, (K, 5), "raw")
        _check(eps, (S, K, 5), "eps")
        _bind_stream(c)
        elbo = torch.empty(1, dtype=torch.float64, device=loc.device)
        xrdvi.xrdvi_forward_dev(c.h, loc.data_ptr(), raw.data_ptr(), eps.data_ptr(), elbo.data_ptr())
        fctx.save_for_backward(loc, raw, eps)
        fctx.c = c
        return -elbo[0]

    @staticmethod
    def backward(fctx, gout):
        loc, raw, eps = fctx.saved_tensors
        c = fctx.c
        K = loc.shape[0]
        _bind_stream(c)
        grad = torch.empty(K * 10, dtype=torch.float32, device=loc.device)
        xrdvi.xrdvi_backward_dev(c.h, loc.data_ptr(), raw.data_ptr(), eps.data_ptr(), grad.data_ptr())
        g = grad.view(K, 10)
        scale = -gout.to(torch.float32)
        return g[:, :5] * scale, g[:, 5:] * scale, None, None


class PhaseSearch(torch.nn.Module):
    """Variational parameters of one problem as torch Parameters; ``forward``
    returns the negative ELBO for injected noise eps [S, K, 5]."""

    def __init__(self, inst, **cfg):
        super().__init__()
        self.ctx = xrdvi.Context.from_instance(inst, **cfg)
        loc, raw = self.ctx.params()
        self.loc = torch.nn.Parameter(torch.tensor(loc, device="cuda"))
        self.raw = torch.nn.Parameter(torch.tensor(raw, device="cuda"))

    def forward(self, eps):
        return NegELBO.apply(self.loc, self.raw, eps, self.ctx)
