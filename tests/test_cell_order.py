"""Internal cell orders (swe_cell_order, host only): caller order, Morton
order of the centroids and reverse Cuthill-McKee (RCM) order of the
edge-neighbour graph. Each is a permutation; Morton sorts the centroid
Z-order keys; RCM is a reversed breadth-first order whose matrix bandwidth
matches scipy's RCM."""
import numpy as np
import pytest

from paper_1807_00672_gb300 import build, inputs, swe

scipy_sparse = pytest.importorskip("scipy.sparse")
csgraph = pytest.importorskip("scipy.sparse.csgraph")


@pytest.fixture(scope="module", autouse=True)
def built():
    build.build()


def neighbour_pairs(tri):
    """Pairs of cells sharing an edge (each pair once)."""
    T = tri.shape[0]
    half = np.sort(np.stack([tri, np.roll(tri, -1, axis=1)], axis=2), axis=2).reshape(-1, 2)
    cell = np.repeat(np.arange(T), 3)
    key = half[:, 0].astype(np.int64) << 32 | half[:, 1]
    o = np.argsort(key, kind="stable")
    key, cell = key[o], cell[o]
    same = np.nonzero(key[1:] == key[:-1])[0]
    return np.stack([cell[same], cell[same + 1]], axis=1)


def bandwidth(perm, pairs):
    pos = np.empty(perm.size, dtype=np.int64)
    pos[perm] = np.arange(perm.size)
    return int(np.abs(pos[pairs[:, 0]] - pos[pairs[:, 1]]).max())


def two_islands():
    """Two grids that share no edge (two connected components), the second
    listed first in caller order."""
    a = inputs.random_flow_case(nx=9, ny=5, seed=3).mesh
    b = inputs.random_flow_case(nx=7, ny=6, seed=4).mesh
    xy = np.concatenate([b.xy + [1e4, 0.0], a.xy])
    tri = np.concatenate([b.tri, a.tri + b.xy.shape[0]])
    return xy, tri, b.tri.shape[0]


def meshes():
    out = []
    for c in (inputs.random_flow_case(nx=60, ny=15, seed=3), inputs.stoker_case(),
              inputs.humps_case(nx=41, ny=33, lx=2_000.0, ly=1_600.0, seed=5)):
        out.append((c.mesh.xy, c.mesh.tri))
    xy, tri, _ = two_islands()
    out.append((xy, tri))
    return out


@pytest.mark.parametrize("order", ["none", "morton", "rcm"])
def test_every_order_is_a_deterministic_permutation(order):
    for xy, tri in meshes():
        p = swe.cell_order(xy, tri, order)
        assert np.array_equal(np.sort(p), np.arange(tri.shape[0]))
        assert np.array_equal(p, swe.cell_order(xy, tri, order))
        if order == "none":
            assert np.array_equal(p, np.arange(tri.shape[0]))


def test_morton_order_sorts_the_centroid_keys():
    for xy, tri in meshes():
        c = xy[tri].mean(axis=1)
        lo = xy.min(axis=0)
        span = float((xy.max(axis=0) - lo).max())
        q = (1 << 22) - 1
        ix = np.clip(((c - lo) / span * q).astype(np.int64), 0, q)

        def spread(v):
            out = np.zeros_like(v)
            for bit in range(22):
                out |= ((v >> bit) & 1) << (2 * bit)
            return out

        key = spread(ix[:, 0]) | (spread(ix[:, 1]) << 1)
        p = swe.cell_order(xy, tri, "morton")
        assert np.all(np.diff(key[p]) >= 0)


def test_rcm_is_a_reversed_breadth_first_order():
    """Read backwards, the order visits every component from one start cell
    in breadth-first order: each cell's distance from its component's start
    never decreases along the order, and every cell but the start has a
    neighbour placed before it."""
    for xy, tri in meshes():
        T = tri.shape[0]
        pairs = neighbour_pairs(tri)
        nbr = [[] for _ in range(T)]
        for a, b in pairs:
            nbr[a].append(b)
            nbr[b].append(a)
        cm = swe.cell_order(xy, tri, "rcm")[::-1]
        pos = np.empty(T, dtype=np.int64)
        pos[cm] = np.arange(T)
        dist = np.full(T, -1)
        comp_start = []
        for j, c in enumerate(cm):
            before = [d for d in nbr[c] if pos[d] < j]
            if not before:  # the start of a new component
                assert all(dist[d] < 0 for d in nbr[c])
                comp_start.append(j)
                dist[c] = 0
                # breadth-first distances over the component
                frontier = [c]
                while frontier:
                    nxt = []
                    for u in frontier:
                        for v in nbr[u]:
                            if dist[v] < 0:
                                dist[v] = dist[u] + 1
                                nxt.append(v)
                    frontier = nxt
        assert np.all(dist >= 0)
        starts = comp_start + [T]
        for s, e in zip(starts[:-1], starts[1:]):  # components are contiguous
            d = dist[cm[s:e]]
            assert np.all(np.diff(d) >= 0)


def test_rcm_bandwidth_matches_scipy():
    for xy, tri in meshes():
        T = tri.shape[0]
        pairs = neighbour_pairs(tri)
        A = scipy_sparse.coo_matrix((np.ones(len(pairs)), (pairs[:, 0], pairs[:, 1])),
                                    shape=(T, T))
        A = (A + A.T).tocsr()
        ref = bandwidth(csgraph.reverse_cuthill_mckee(A, symmetric_mode=True), pairs)
        got = bandwidth(swe.cell_order(xy, tri, "rcm"), pairs)
        assert got <= 1.25 * ref + 2, (got, ref)


def test_rcm_narrows_a_wide_grid():
    """On a 60 x 15 grid numbered along its long side the caller order's
    bandwidth is about two rows of the long side; RCM sweeps across the short
    side instead."""
    c = inputs.random_flow_case(nx=60, ny=15, seed=3)
    pairs = neighbour_pairs(c.mesh.tri)
    caller = bandwidth(np.arange(c.mesh.tri.shape[0]), pairs)
    rcm = bandwidth(swe.cell_order(c.mesh.xy, c.mesh.tri, "rcm"), pairs)
    assert rcm * 3 < caller


def test_cell_order_rejects_bad_input():
    c = inputs.random_flow_case(nx=5, ny=4, seed=1)
    with pytest.raises(KeyError):
        swe.cell_order(c.mesh.xy, c.mesh.tri, "hilbert")
    perm = np.empty(c.mesh.tri.shape[0], dtype=np.int32)
    st = swe.lib().swe_cell_order(swe._p(np.ascontiguousarray(c.mesh.xy)), c.mesh.xy.shape[0],
                                  swe._p(np.ascontiguousarray(c.mesh.tri, dtype=np.int32)),
                                  c.mesh.tri.shape[0], 7, swe._p(perm))
    assert st == swe.SWE_EINVAL
    bad = c.mesh.tri.copy()
    bad[0, 1] = bad[0, 0]  # a degenerate triangle
    with pytest.raises(swe.SweError) as e:
        swe.cell_order(c.mesh.xy, bad, "rcm")
    assert e.value.status == swe.SWE_EMESH
