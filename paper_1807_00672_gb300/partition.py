"""Domain decomposition of one mesh: sub-domains stepped by the library's
kernels, with a halo exchange and a global CFL time step between steps
(the paper's future work of several GPUs on one mesh, Sec. 5; the step is
that of Sec. 2.2).

The cut and the exchange lists come from ``swe.Partition``. One step of a
decomposed run is, for every sub-domain:

  1. one step of its local mesh (own cells and one ring of ghost cells),
     with the global time step;
  2. halo exchange: for every ordered pair (src, dst), src packs the cells
     dst holds as ghosts into a buffer, the buffer moves, dst unpacks it
     into its ghosts;
  3. global time step: every sub-domain's CFL step (over its own cells),
     then their minimum, set as every sub-domain's next step.

Two drivers share that schedule. ``LocalRun`` keeps every sub-domain in
this process on one GPU: a buffer moves by being the same device array on
both sides, and the minimum is one kernel over all the sub-domains' values.
``run_distributed`` keeps one sub-domain per rank of a torch.distributed
group: buffers move by point-to-point send/receive and the minimum and the
mass are all-reduced (NCCL between GPUs). Its sub-domain object only needs
``step``, ``pack``, ``unpack``, ``dt`` and ``set_dt`` on tensors of its own
device, so the same function drives GPU sub-domains under NCCL and host
ones under gloo.
"""
from __future__ import annotations

import contextlib

import numpy as np
import torch

from . import swe


class GpuSubdomain:
    """Part `part` of a Partition as a library mesh and state on the current
    GPU, with its exchange lists and buffers in device memory.

    fields: the whole mesh's initial (h, hu, hv, z, n) in caller order;
    every local cell, ghosts included, starts from its global values."""

    def __init__(self, plan: swe.Partition, part: int, fields, *, precision="f64", tile=0,
                 stream=None):
        self.part = part
        self.plan = plan
        loc = plan.local(part)
        self.cells = loc["cells"]
        self.ghost = loc["ghost"].astype(bool)
        self.device = torch.device("cuda", torch.cuda.current_device())
        # The library's kernels and every torch operation on this part's
        # buffers share one (non-default) stream: packs, unpacks, the time
        # step reductions and the steps are ordered by it.
        self.stream = stream if stream is not None else torch.cuda.Stream(device=self.device)
        if not self.stream.cuda_stream:
            raise ValueError("a sub-domain needs a non-default CUDA stream")
        self.mesh = swe.Mesh.part(loc["xy"], loc["tri"], loc["ghost"], precision=precision,
                                  tile=tile, stream=swe._vp(self.stream.cuda_stream))
        h0, hu0, hv0, z, n = (np.asarray(f, dtype=np.float64)[self.cells] for f in fields)
        self.state = swe.State(self.mesh, h0, hu0, hv0, z, n)
        # exchange lists: cells this part sends to each peer, and where each
        # peer's cells land here
        self.send, self.recv, self.buf = {}, {}, {}
        with torch.cuda.stream(self.stream):
            for q in range(plan.n_parts):
                if q == part:
                    continue
                a, _ = plan.exchange(part, q)
                _, b = plan.exchange(q, part)
                if a.size:
                    self.send[q] = torch.from_numpy(a).to(self.device)
                    self.buf[q] = torch.empty(3 * a.size, dtype=torch.float64, device=self.device)
                if b.size:
                    self.recv[q] = torch.from_numpy(b).to(self.device)
            self._dt = torch.empty(1, dtype=torch.float64, device=self.device)
        self.stream.synchronize()

    def stream_context(self):
        """Makes this part's stream torch's current one (for collectives)."""
        return torch.cuda.stream(self.stream)

    # --- the sub-domain interface of run_distributed ----------------------
    def step(self):
        self.state.run(1, sync=False)

    def pack(self, peer: int) -> torch.Tensor:
        ids = self.send[peer]
        self.state.halo_pack(ids.data_ptr(), ids.numel(), self.buf[peer].data_ptr())
        return self.buf[peer]

    def recv_buffer(self, peer: int) -> torch.Tensor:
        with torch.cuda.stream(self.stream):
            return torch.empty(3 * self.recv[peer].numel(), dtype=torch.float64,
                               device=self.device)

    def unpack(self, peer: int, buf: torch.Tensor):
        ids = self.recv[peer]
        self.state.halo_unpack(ids.data_ptr(), ids.numel(), buf.data_ptr())

    def dt(self) -> torch.Tensor:
        self.state.dt_device(self._dt.data_ptr())
        return self._dt

    def set_dt(self, dts: torch.Tensor):
        self.state.set_dt_min_device(dts.data_ptr(), dts.numel())

    # --- results ------------------------------------------------------------
    def owned_fields(self):
        """(global ids, h, hu, hv) of the cells this part owns."""
        h, hu, hv = self.state.fields()
        own = ~self.ghost
        return self.cells[own], h[own], hu[own], hv[own]

    def mass(self) -> float:
        """Sum of area * h over the owned cells (FP64)."""
        return self.state.mass

    def close(self):
        self.state.close()
        self.mesh.close()


class LocalRun:
    """Every sub-domain of a Partition in this process, on one GPU and one
    stream. ``run(k)`` takes k decomposed steps; ``fields()`` assembles the
    whole mesh's state from the owned cells."""

    def __init__(self, xy, tri, fields, n_parts: int, *, precision="f64", tile=0, stream=None):
        self.plan = swe.Partition(xy, tri, n_parts)
        self.n_tris = self.plan.n_tris
        dev = torch.device("cuda", torch.cuda.current_device())
        # one stream for every part: each part's work is ordered after the
        # packs of its peers and the reductions
        self.stream = stream if stream is not None else torch.cuda.Stream(device=dev)
        self.parts = [GpuSubdomain(self.plan, p, fields, precision=precision, tile=tile,
                                   stream=self.stream) for p in range(n_parts)]
        with torch.cuda.stream(self.stream):
            self._dts = torch.empty(n_parts, dtype=torch.float64, device=dev)
        self._global_dt()  # the first step already takes the global CFL step

    def _global_dt(self):
        for p, s in enumerate(self.parts):
            s.state.dt_device(self._dts[p:p + 1].data_ptr())
        for s in self.parts:
            s.set_dt(self._dts)

    def run(self, n_steps: int):
        for _ in range(int(n_steps)):
            for s in self.parts:
                s.step()
            # one GPU: the packed buffer of (src, dst) is unpacked in place
            for s in self.parts:
                for q in s.send:
                    self.parts[q].unpack(s.part, s.pack(q))
            self._global_dt()
        self.parts[0].state.sync()

    def fields(self):
        h, hu, hv = (np.full(self.n_tris, np.nan) for _ in range(3))
        for s in self.parts:
            ids, a, b, c = s.owned_fields()
            h[ids], hu[ids], hv[ids] = a, b, c
        return h, hu, hv

    def mass(self) -> float:
        return float(sum(s.mass() for s in self.parts))

    def close(self):
        for s in self.parts:
            s.close()
        self.plan.close()


def run_distributed(sub, n_steps: int, dist, group=None):
    """One sub-domain per rank: k decomposed steps of `sub` (GpuSubdomain
    under NCCL, or any object with the same step/pack/recv_buffer/unpack/
    dt/set_dt methods on tensors of its device). Halo buffers move by
    point-to-point send/receive, ordered by peer so that every pair's
    transfers match; the global time step is an all-reduce (min), taken
    once before the first step as well."""
    ctx = sub.stream_context() if hasattr(sub, "stream_context") else contextlib.nullcontext()
    with ctx:
        _run_distributed(sub, n_steps, dist, group)


def _run_distributed(sub, n_steps, dist, group):
    dt = sub.dt().clone()
    dist.all_reduce(dt, op=dist.ReduceOp.MIN, group=group)
    sub.set_dt(dt)
    for _ in range(int(n_steps)):
        sub.step()
        reqs, inbox = [], {}
        for q in sorted(set(sub.send) | set(sub.recv)):
            if q in sub.send:
                reqs.append(dist.isend(sub.pack(q), dst=q, group=group))
            if q in sub.recv:
                inbox[q] = sub.recv_buffer(q)
                reqs.append(dist.irecv(inbox[q], src=q, group=group))
        for r in reqs:
            r.wait()
        for q, buf in inbox.items():
            sub.unpack(q, buf)
        dt = sub.dt().clone()
        dist.all_reduce(dt, op=dist.ReduceOp.MIN, group=group)
        sub.set_dt(dt)


def global_mass(sub, dist, group=None) -> float:
    """FP64 all-reduce (sum) of the sub-domains' owned masses."""
    ctx = sub.stream_context() if hasattr(sub, "stream_context") else contextlib.nullcontext()
    with ctx:
        m = torch.tensor([float(sub.mass())], dtype=torch.float64, device=sub.dt().device)
        dist.all_reduce(m, op=dist.ReduceOp.SUM, group=group)
        return float(m.item())
