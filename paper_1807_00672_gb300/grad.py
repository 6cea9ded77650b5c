"""Differentiable rollout of the solver for PyTorch (a torch.autograd.Function
over the library's recorded steps and hand-written adjoint kernels).

``rollout(mesh, h0, hu0, hv0, z, n, n_steps, ...)`` advances the initial
state by ``n_steps`` CFL steps and returns the final (h, hu, hv) and the
depths at the gauge cells after every step; its backward gives the gradient
of any loss of those outputs with respect to h0, hu0, hv0, z and n. The time
steps are those of the forward run, held fixed (not differentiated). Tensors
may live on any device; the library copies them through host memory at the
call boundary and does all the stepping on the GPU.
"""
from __future__ import annotations

import numpy as np
import torch

from . import swe


def _np(t: torch.Tensor) -> np.ndarray:
    return t.detach().to("cpu", torch.float64).contiguous().numpy()


class Rollout(torch.autograd.Function):
    @staticmethod
    def forward(ctx, h0, hu0, hv0, z, n, mesh, n_steps, checkpoint_every, gauges):
        st = swe.State(mesh, _np(h0), _np(hu0), _np(hv0), _np(z), _np(n))
        tape = swe.Tape(st, n_steps, checkpoint_every, gauges)
        h, hu, hv = st.fields()
        st.close()
        ctx.tape = tape
        ctx.like = h0
        out = [torch.from_numpy(a).to(h0.device, h0.dtype) for a in (h, hu, hv, tape.gauge_h)]
        return tuple(out)

    @staticmethod
    def backward(ctx, gh, ghu, ghv, ggauge):
        tape = ctx.tape
        r = tape.grad(None if gh is None else _np(gh), None if ghu is None else _np(ghu),
                      None if ghv is None else _np(ghv), None if ggauge is None else _np(ggauge))
        like = ctx.like
        cv = lambda a: torch.from_numpy(a).to(like.device, like.dtype)
        return cv(r["h"]), cv(r["hu"]), cv(r["hv"]), cv(r["z"]), cv(r["n"]), None, None, None, None


def rollout(mesh: swe.Mesh, h0, hu0, hv0, z, n, n_steps: int, checkpoint_every: int = 50,
            gauges=None):
    """(h, hu, hv) after n_steps steps and the gauge depths [n_steps, G]."""
    g = np.asarray(gauges if gauges is not None else [], dtype=np.int32)
    return Rollout.apply(h0, hu0, hv0, z, n, mesh, int(n_steps), int(checkpoint_every), g)
