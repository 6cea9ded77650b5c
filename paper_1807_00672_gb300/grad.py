"""Differentiable rollout of the solver for PyTorch (a torch.autograd.Function
over the library's recorded steps and hand-written adjoint kernels).

``rollout(mesh, h0, hu0, hv0, z, n, n_steps, ...)`` advances the initial
state by ``n_steps`` CFL steps and returns the final (h, hu, hv) and the
depths at the gauge cells after every step; its backward gives the gradient
of any loss of those outputs with respect to h0, hu0, hv0, z and n. The time
steps are those of the forward run, held fixed (not differentiated).

CUDA tensors (on the mesh's device) are handed to the library's
device-pointer calls (swe_state_init_device, swe_copy_out_device,
swe_tape_gauges_device, swe_grad_device), ordered on the current torch
stream: nothing goes through host memory. CPU tensors go through the host
calls. Either way all stepping runs on the GPU.
"""
from __future__ import annotations

import numpy as np
import torch

from . import swe


def _np(t: torch.Tensor) -> np.ndarray:
    return t.detach().to("cpu", torch.float64).contiguous().numpy()


def _dev64(t: torch.Tensor, device) -> torch.Tensor:
    """float64, contiguous, on `device` (the library's arrays are FP64)."""
    return t.detach().to(device=device, dtype=torch.float64).contiguous()


def _ptr(t):
    return None if t is None else t.data_ptr()


class Rollout(torch.autograd.Function):
    @staticmethod
    def forward(ctx, h0, hu0, hv0, z, n, mesh, n_steps, checkpoint_every, gauges):
        ctx.like = h0
        ctx.on_device = h0.is_cuda
        G = int(gauges.shape[0])
        if ctx.on_device:
            dev = h0.device
            stream = torch.cuda.current_stream(dev)
            ins = [_dev64(t, dev) for t in (h0, hu0, hv0, z, n)]
            st = swe.State.from_device(mesh, *[t.data_ptr() for t in ins],
                                       stream=stream.cuda_stream)
            tape = swe.Tape(st, n_steps, checkpoint_every, gauges, host_gauges=False)
            outs = [torch.empty(mesh.T, dtype=torch.float64, device=dev) for _ in range(3)]
            st.copy_out_device(*[t.data_ptr() for t in outs], stream=stream.cuda_stream)
            gh = torch.empty((n_steps, G), dtype=torch.float64, device=dev)
            if G:
                tape.gauges_device(gh.data_ptr(), stream=stream.cuda_stream)
            st.close()
            res = outs + [gh]
        else:
            st = swe.State(mesh, _np(h0), _np(hu0), _np(hv0), _np(z), _np(n))
            tape = swe.Tape(st, n_steps, checkpoint_every, gauges)
            h, hu, hv = st.fields()
            st.close()
            res = [torch.from_numpy(a) for a in (h, hu, hv, tape.gauge_h)]
        ctx.tape = tape
        ctx.mesh = mesh
        return tuple(t.to(h0.device, h0.dtype) for t in res)

    @staticmethod
    def backward(ctx, gh, ghu, ghv, ggauge):
        tape, like = ctx.tape, ctx.like
        if ctx.on_device:
            dev = like.device
            stream = torch.cuda.current_stream(dev)
            seeds = [None if g is None else _dev64(g, dev) for g in (gh, ghu, ghv, ggauge)]
            outs = [torch.empty(ctx.mesh.T, dtype=torch.float64, device=dev) for _ in range(5)]
            tape.grad_device([_ptr(t) for t in seeds], [t.data_ptr() for t in outs],
                             stream=stream.cuda_stream)
            grads = [t.to(like.dtype) for t in outs]
        else:
            r = tape.grad(None if gh is None else _np(gh), None if ghu is None else _np(ghu),
                          None if ghv is None else _np(ghv),
                          None if ggauge is None else _np(ggauge))
            grads = [torch.from_numpy(r[k]).to(like.device, like.dtype)
                     for k in ("h", "hu", "hv", "z", "n")]
        return (*grads, None, None, None, None)


def rollout(mesh: swe.Mesh, h0, hu0, hv0, z, n, n_steps: int, checkpoint_every: int = 50,
            gauges=None):
    """(h, hu, hv) after n_steps steps and the gauge depths [n_steps, G]."""
    g = np.asarray(gauges if gauges is not None else [], dtype=np.int32)
    return Rollout.apply(h0, hu0, hv0, z, n, mesh, int(n_steps), int(checkpoint_every), g)
