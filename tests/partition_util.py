"""A host sub-domain for the decomposition tests: one part of a partition
stepped by the FP64 oracle (test infrastructure), with the interface that
paper_1807_00672_gb300.partition.run_distributed drives (tensors on the
host, for gloo)."""
import numpy as np
import torch

import oracle


class OracleSubdomain:
    def __init__(self, plan, part, fields):
        self.part = part
        loc = plan.local(part)
        self.cells = loc["cells"]
        self.ghost = loc["ghost"].astype(bool)
        self.mesh = oracle.Mesh(loc["xy"], loc["tri"])
        h, hu, hv, z, n = (np.asarray(f, dtype=np.float64)[self.cells] for f in fields)
        self.state = oracle.State(self.mesh, h, hu, hv, z, n)
        self.send, self.recv = {}, {}
        for q in range(plan.n_parts):
            if q == part:
                continue
            a, _ = plan.exchange(part, q)
            _, b = plan.exchange(q, part)
            if a.size:
                self.send[q] = a
            if b.size:
                self.recv[q] = b
        self.next_dt = None
        self.dts = []

    def step(self):
        self.state.step(self.next_dt)
        self.dts.append(self.next_dt)

    def pack(self, peer):
        ids = self.send[peer]
        s = self.state
        return torch.from_numpy(np.stack([s.h[ids], s.hu[ids], s.hv[ids]], 1).ravel().copy())

    def recv_buffer(self, peer):
        return torch.empty(3 * self.recv[peer].size, dtype=torch.float64)

    def unpack(self, peer, buf):
        ids = self.recv[peer]
        b = buf.numpy().reshape(-1, 3)
        self.state.h[ids], self.state.hu[ids], self.state.hv[ids] = b[:, 0], b[:, 1], b[:, 2]

    def dt(self):
        return torch.tensor([self.state.cfl_dt()], dtype=torch.float64)

    def set_dt(self, dts):
        self.next_dt = float(dts.min())

    def owned(self):
        own = ~self.ghost
        s = self.state
        return self.cells[own], s.h[own], s.hu[own], s.hv[own]

    def mass(self):
        own = ~self.ghost
        area = self.mesh.cells()["area"]
        return float((area[own] * self.state.h[own]).sum())
