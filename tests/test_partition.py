"""Domain decomposition without a GPU: the partition plan (swe_partition_*,
host code of the library) against its definition, and decomposed runs
stepped by the FP64 oracle, in one process and over two gloo ranks, equal
to the whole mesh's run bit for bit."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
from paper_1807_00672_gb300 import build, inputs, swe
from paper_1807_00672_gb300.partition import global_mass, run_distributed

from partition_util import OracleSubdomain


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()


def neighbours(tri):
    """Cells sharing an edge, from a plain dictionary of node pairs."""
    seen, nb = {}, [set() for _ in range(tri.shape[0])]
    for c, t in enumerate(tri):
        for k in range(3):
            e = tuple(sorted((int(t[k]), int(t[(k + 1) % 3]))))
            if e in seen:
                nb[c].add(seen[e])
                nb[seen[e]].add(c)
            else:
                seen[e] = c
    return nb


@pytest.mark.parametrize("P", [1, 2, 3, 5])
def test_plan_matches_its_definition(P):
    case = inputs.random_flow_case(nx=37, ny=23, seed=41)
    xy, tri = case.mesh.xy, case.mesh.tri
    T = tri.shape[0]
    plan = swe.Partition(xy, tri, P)
    nb = neighbours(tri)
    owner = np.full(T, -1)
    locs = [plan.local(p) for p in range(P)]
    for p, loc in enumerate(locs):
        own = loc["cells"][loc["ghost"] == 0]
        assert np.all(owner[own] == -1)
        owner[own] = p
        assert abs(own.size - T / P) <= 1            # balanced ranges
        assert np.all(np.diff(loc["cells"]) > 0)     # ascending global order
        # ghosts: exactly the other parts' cells that touch an owned cell
        ring = set().union(*(nb[c] for c in own)) - set(own.tolist())
        assert set(loc["cells"][loc["ghost"] == 1].tolist()) == ring
        # the local triangles are the global ones, node order kept
        assert np.array_equal(loc["xy"][loc["tri"]], xy[tri[loc["cells"]]])
    assert np.all(owner >= 0)
    for a in range(P):
        for b in range(P):
            fa, tb = plan.exchange(a, b)
            if a == b:
                assert fa.size == 0
                continue
            ga, gb = locs[a]["cells"][fa], locs[b]["cells"][tb]
            assert np.array_equal(ga, gb) and np.all(np.diff(ga) > 0)
            assert np.all(owner[ga] == a) and np.all(locs[b]["ghost"][tb] == 1)
            want = [c for c in locs[b]["cells"][locs[b]["ghost"] == 1] if owner[c] == a]
            assert ga.tolist() == want
    plan.close()


def test_plan_rejects_bad_arguments():
    case = inputs.random_flow_case(nx=4, ny=3, seed=1)
    for P in (0, -1, case.mesh.n_tris + 1):
        with pytest.raises(swe.SweError) as e:
            swe.Partition(case.mesh.xy, case.mesh.tri, P)
        assert e.value.status == swe.SWE_EINVAL
    bad = case.mesh.tri.copy()
    bad[2, 1] = case.mesh.n_nodes
    with pytest.raises(swe.SweError) as e:
        swe.Partition(case.mesh.xy, bad, 2)
    assert e.value.status == swe.SWE_EMESH


def _fields(case):
    return (case.h, case.hu, case.hv, case.z, case.n)


def _local_decomposed_run(case, P, n_steps):
    """All parts in this process: step, exchange, global dt (min)."""
    plan = swe.Partition(case.mesh.xy, case.mesh.tri, P)
    subs = [OracleSubdomain(plan, p, _fields(case)) for p in range(P)]

    def global_dt():
        dts = [s.dt() for s in subs]
        for s in subs:
            s.set_dt(min(dts, key=float))
    global_dt()
    for _ in range(n_steps):
        for s in subs:
            s.step()
        for s in subs:
            for q in s.send:
                subs[q].unpack(s.part, s.pack(q))
        global_dt()
    T = case.mesh.n_tris
    out = [np.full(T, np.nan) for _ in range(3)]
    for s in subs:
        ids, a, b, c = s.owned()
        out[0][ids], out[1][ids], out[2][ids] = a, b, c
    return out, subs


@pytest.mark.parametrize("name,case", [
    ("random_flow", inputs.random_flow_case(nx=37, ny=23, seed=41)),
    ("humps", inputs.humps_case(nx=61, ny=33, lx=2_000.0, ly=1_000.0, seed=45)),
])
@pytest.mark.parametrize("P", [2, 3, 4])
def test_decomposed_oracle_run_equals_the_whole_mesh_bitwise(name, case, P):
    ref = oracle.state_from_case(case)
    dts = ref.run(30)
    got, subs = _local_decomposed_run(case, P, 30)
    assert np.array_equal(np.array(subs[0].dts), dts)
    for a, b in zip(got, (ref.h, ref.hu, ref.hv)):
        assert np.array_equal(a, b)
    assert sum(s.mass() for s in subs) == pytest.approx(ref.mass(), rel=1e-13)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, n_steps, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        build.build()
        case = inputs.random_flow_case(nx=37, ny=23, seed=41)
        plan = swe.Partition(case.mesh.xy, case.mesh.tri, world)
        sub = OracleSubdomain(plan, rank, _fields(case))
        run_distributed(sub, n_steps, dist)
        m = global_mass(sub, dist)
        ids, h, hu, hv = sub.owned()
        q.put((rank, ids, h, hu, hv, m, sub.dts))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_equal_the_whole_mesh_bitwise():
    """One sub-domain per rank: halos by send/receive, the time step by an
    all-reduce (min), the mass by an FP64 all-reduce (sum)."""
    n_steps = 25
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, n_steps, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = [q.get(timeout=180) for _ in procs]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    case = inputs.random_flow_case(nx=37, ny=23, seed=41)
    ref = oracle.state_from_case(case)
    dts = ref.run(n_steps)
    seen = np.zeros(case.mesh.n_tris, dtype=int)
    for rank, ids, h, hu, hv, m, rdts in got:
        seen[ids] += 1
        assert np.array_equal(np.array(rdts), dts)
        assert np.array_equal(h, ref.h[ids]) and np.array_equal(hu, ref.hu[ids])
        assert np.array_equal(hv, ref.hv[ids])
        assert m == pytest.approx(ref.mass(), rel=1e-13)
    assert np.all(seen == 1)


def test_as_many_parts_as_cells_and_one_part():
    """Degenerate cuts: one part (no ghost, local = whole mesh) and one cell
    per part (every neighbour a ghost); decomposed oracle runs still equal
    the whole mesh bitwise."""
    case = inputs.random_flow_case(nx=3, ny=2, lx=30.0, ly=20.0, seed=3)   # 12 cells
    T = case.mesh.n_tris
    one = swe.Partition(case.mesh.xy, case.mesh.tri, 1).local(0)
    assert one["ghost"].sum() == 0 and np.array_equal(one["cells"], np.arange(T))
    ref = oracle.state_from_case(case)
    dts = ref.run(15)
    got, subs = _local_decomposed_run(case, T, 15)
    assert all((~s.ghost).sum() == 1 for s in subs)
    assert np.array_equal(np.array(subs[0].dts), dts)
    for a, b in zip(got, (ref.h, ref.hu, ref.hv)):
        assert np.array_equal(a, b)
