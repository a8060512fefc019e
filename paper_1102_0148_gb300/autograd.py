"""Visibilities as a differentiable function of the per-antenna gains and
delays applied in the F-engine (Sec. 2.1 of the paper: a phase per stream
before accumulation).

    V = visibilities(gains, delays, samples, correlator)   # [P][C] complex128
    loss = (V - M).abs().pow(2).sum(); loss.backward()

The forward is the correlator itself (corrections in the F-engine, FP32 or
the handle's X-engine precision, FP64 accumulation).  The backward is the
library's corr_grad kernel: it recomputes the uncorrected visibilities from
the samples pass by pass and forms dL/dg and dL/dtau in closed form.  Only
argument marshalling happens here.
"""

import torch

from . import corr


class Visibilities(torch.autograd.Function):
    @staticmethod
    def forward(ctx, gains, delays, samples, correlator):
        c = correlator
        g = gains.detach().to(torch.complex64).contiguous()
        t = delays.detach().to(torch.float32).contiguous()
        if not (g.is_cuda and t.is_cuda and samples.is_cuda):
            raise ValueError("gains, delays and samples must be CUDA tensors")
        corr.corr_set_stream(c.h, torch.cuda.current_stream().cuda_stream)
        corr.corr_set_corrections(c.h, g, t)
        n = samples.numel() * 2 // c.N
        corr.corr_push(c.h, samples, n)
        V = torch.empty((c.P, c.C), dtype=torch.complex128, device=samples.device)
        corr.corr_dump(c.h, V, fp64=True)
        ctx.save_for_backward(g, t, samples)
        ctx.c = c
        ctx.n = n
        ctx.dtypes = (gains.dtype, delays.dtype)
        return V

    @staticmethod
    def backward(ctx, grad_V):
        g, t, samples = ctx.saved_tensors
        gV = grad_V.to(torch.complex128).contiguous()
        gg = torch.empty_like(g)
        gt = torch.empty_like(t)
        corr.corr_set_stream(ctx.c.h, torch.cuda.current_stream().cuda_stream)
        corr.corr_grad(ctx.c.h, samples, ctx.n, g, t, gV, True, gg, gt)
        return gg.to(ctx.dtypes[0]), gt.to(ctx.dtypes[1]), None, None


def visibilities(gains, delays, samples, correlator):
    """[P][C] complex128 visibilities of `samples` under per-antenna complex
    `gains` and `delays` (samples), differentiable in gains and delays."""
    return Visibilities.apply(gains, delays, samples, correlator)
