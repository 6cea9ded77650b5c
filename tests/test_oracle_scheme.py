"""Pins of the oracle's mesh, step and time loop against closed forms and invariants."""
import math
import os

import numpy as np
import pytest

import oracle
from paper_1807_00672_gb300 import inputs

from closed_forms import friction_decay, ritter_depth, stoker_depth, stoker_middle

HERE = os.path.dirname(os.path.abspath(__file__))


# --------------------------------------------------------------------------- mesh

def test_table2_grids_satisfy_euler_formula():
    """The paper's grids (Table 2) are simply connected triangulations:
    V - E + T = 1, and 2E - 3T counts the boundary edges (positive)."""
    rows = [list(map(int, l.split())) for l in open(os.path.join(HERE, "golden", "table2_grids.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 5
    for _, T, E, V in rows:
        assert V - E + T == 1
        assert 2 * E - 3 * T > 0


@pytest.mark.parametrize("nx,ny,jit", [(50, 25, 0.0), (37, 11, 0.3), (1, 1, 0.0), (64, 64, 0.3)])
def test_mesh_counts_and_geometry(nx, ny, jit):
    m = inputs.jittered_grid(nx, ny, 3.0 * nx, 2.0 * ny, jitter=jit, diagonal="shorter", seed=nx)
    om = oracle.Mesh(m.xy, m.tri)
    assert om.T == 2 * nx * ny and om.V == (nx + 1) * (ny + 1)
    assert om.V - om.E + om.T == 1
    assert 2 * om.E - 3 * om.T == om.Eb == 2 * (nx + ny)
    c = om.cells()
    e = om.edges()
    assert np.all(c["area"] > 0)
    assert c["area"].sum() == pytest.approx(3.0 * nx * 2.0 * ny, rel=1e-12)
    assert np.allclose(e["nx"] ** 2 + e["ny"] ** 2, 1.0, rtol=0, atol=1e-15)
    # closure: sum over the faces of s l n vanishes for every cell
    ce = c["cell_edge"]
    s = np.where(e["L"][ce] == np.arange(om.T)[:, None], 1.0, -1.0)
    sx = (s * e["len"][ce] * e["nx"][ce]).sum(1)
    sy = (s * e["len"][ce] * e["ny"][ce]).sum(1)
    assert np.abs(sx).max() <= 1e-12 * e["len"].max() and np.abs(sy).max() <= 1e-12 * e["len"].max()
    # normals point out of the left cell; perimeters add up
    cen = m.xy[c["tri"]].mean(1)
    tri = c["tri"]
    for i in range(0, om.T, max(1, om.T // 50)):
        for k in range(3):
            ed = ce[i, k]
            mid = 0.5 * (m.xy[tri[i, k]] + m.xy[tri[i, (k + 1) % 3]])
            d = (mid - cen[i]) @ np.array([e["nx"][ed], e["ny"][ed]])
            assert (d > 0) == (e["L"][ed] == i)
    assert np.allclose(c["perim"], e["len"][ce].sum(1), rtol=1e-15)
    # walls are exactly the boundary edges
    assert np.count_nonzero(e["R"] < 0) == om.Eb
    assert np.all(e["L"] < np.where(e["R"] < 0, np.iinfo(np.int32).max, e["R"]))


def test_clockwise_triangles_are_reoriented():
    m = inputs.jittered_grid(4, 3, 4.0, 3.0, seed=2)
    tri = m.tri.copy()
    tri[::3] = tri[::3, [0, 2, 1]]
    a = oracle.Mesh(m.xy, m.tri).cells()
    b = oracle.Mesh(m.xy, tri).cells()
    assert np.array_equal(a["area"], b["area"])


@pytest.mark.parametrize("bad", ["index", "degenerate", "nonmanifold"])
def test_invalid_meshes_are_rejected(bad):
    m = inputs.jittered_grid(3, 3, 3.0, 3.0)
    xy, tri = m.xy.copy(), m.tri.copy()
    if bad == "index":
        tri[4, 1] = m.n_nodes
    elif bad == "degenerate":
        tri[2, 2] = tri[2, 0]
    else:
        tri = np.concatenate([tri, tri[:1]])
    with pytest.raises(oracle.OracleError) as ei:
        oracle.Mesh(xy, tri)
    assert ei.value.status == oracle.E_MESH


# --------------------------------------------------------------------------- step

def test_lake_at_rest_is_preserved_over_bumpy_bed_with_dry_islands():
    c = inputs.lake_at_rest_case()
    assert np.count_nonzero(c.h == 0) > 10 and np.count_nonzero(c.h > 0) > 100
    s = oracle.state_from_case(c)
    s.run(100)
    scale = 1e-12 * oracle.G * c.h.max() ** 2
    assert np.abs(s.hu).max() <= scale and np.abs(s.hv).max() <= scale
    assert np.abs(s.h - c.h).max() <= 1e-13 * c.h.max()
    assert s.neg == 0


def test_mass_is_conserved_with_walls():
    c = inputs.random_flow_case()
    s = oracle.state_from_case(c)
    m0 = s.mass()
    s.run(100)
    assert abs(s.mass() - m0) <= 1e-13 * m0
    assert s.neg == 0
    assert np.all(s.h >= 0)


def test_dt_keeps_the_positivity_bound():
    """dt * (sum over faces of l * max wave speed) <= Omega for every wet cell."""
    c = inputs.random_flow_case(seed=19)
    s = oracle.state_from_case(c)
    cells = s.mesh.cells()
    dt = s.cfl_dt()
    wet = c.h > oracle.H_EPS
    u = np.where(wet, c.hu / np.where(wet, c.h, 1), 0)
    v = np.where(wet, c.hv / np.where(wet, c.h, 1), 0)
    lam = np.hypot(u, v) + np.sqrt(oracle.G * c.h)
    assert np.all(dt * lam[wet] * cells["perim"][wet] <= 0.7 * cells["area"][wet] * (1 + 1e-12))
    assert np.any(dt * lam[wet] * cells["perim"][wet] >= 0.7 * cells["area"][wet] * (1 - 1e-12))


def _stoker_l1(f):
    c = inputs.stoker_case(50 * f, 25 * f)
    s = oracle.state_from_case(c)
    s.advance(2.0)
    assert s.t == 2.0 and s.neg == 0
    cen = inputs.centroids(c.mesh)
    band = np.abs(cen[:, 1] - 25.0) <= 2.0
    he = stoker_depth(cen[band, 0], 2.0, 10.0, 1.0, 50.0)
    return np.abs(s.h[band] - he).sum() / np.abs(he).sum(), s, cen, band


def test_stoker_dam_break_closed_form():
    h_m, u_m, sp = stoker_middle(10.0, 1.0)
    assert (h_m, u_m, sp) == pytest.approx((3.96175, 7.34077, 9.81929), abs=2e-5)
    l1, s, cen, band = _stoker_l1(1)
    assert l1 <= 0.03
    x = cen[band, 0]
    c_m = math.sqrt(oracle.G * h_m)
    plateau = (x > 50 + 2.0 * (u_m - c_m) + 4.0) & (x < 50 + 2.0 * sp - 4.0)
    assert plateau.sum() > 5
    # first-order smearing rounds the plateau's corners: mean within 2 %, every cell within 4 %
    assert abs(s.h[band][plateau].mean() - h_m) <= 0.02 * h_m
    assert np.abs(s.h[band][plateau] - h_m).max() <= 0.04 * h_m
    o = np.argsort(x)
    xs, hs = x[o], s.h[band][o]
    right = xs > 60.0
    x_shock = xs[right][np.argmax(hs[right] < 0.5 * (h_m + 1.0))]
    assert abs(x_shock - (50 + 2.0 * sp)) <= 2 * 2.0  # within two cells


def test_stoker_converges_under_refinement():
    e = [_stoker_l1(f)[0] for f in (1, 2, 4)]
    orders = [math.log2(e[i] / e[i + 1]) for i in range(2)]
    assert min(orders) >= 0.6


def test_ritter_dry_bed_dam_break():
    errs = []
    for f in (1, 2, 4):
        c = inputs.ritter_case(100 * f, 4 * f)
        s = oracle.state_from_case(c)
        m0 = s.mass()
        s.advance(3.0)
        assert s.neg == 0 and abs(s.mass() - m0) <= 1e-13 * m0
        x = inputs.centroids(c.mesh)[:, 0]
        he = ritter_depth(x, 3.0, 1.0, 50.0)
        errs.append(np.abs(s.h - he).sum() / he.sum())
        # nothing runs ahead of the exact front 2 c0 t
        assert x[s.h > 1e-9].max() <= 50.0 + 2.0 * math.sqrt(oracle.G) * 3.0 + 1.0 / f
    assert errs[0] <= 0.02
    assert errs[0] > errs[1] > errs[2]


def test_friction_decay_closed_form():
    """Uniform flow on a flat bed: interior fluxes cancel, and the linearised
    implicit friction gives 1/|q^{n+1}| = 1/|q^n| + dt g n^2 / h^{7/3} exactly,
    i.e. the ODE's closed form at t = sum of dt. Walls perturb only cells
    within one cell per step of the boundary."""
    c = inputs.uniform_flow_case()
    s = oracle.state_from_case(c)
    N = 10
    dts = s.run(N)
    q0 = math.hypot(c.hu[0], c.hv[0])
    qe = friction_decay(q0, 2.0, 0.05, dts.sum())
    cen = inputs.centroids(c.mesh)
    far = (cen[:, 0] > 10 * N + 20) & (cen[:, 0] < 600 - 10 * N - 20) & \
          (cen[:, 1] > 10 * N + 20) & (cen[:, 1] < 300 - 10 * N - 20)
    assert far.sum() > 100
    q = np.hypot(s.hu[far], s.hv[far])
    assert np.abs(q - qe).max() <= 1e-13 * qe
    assert np.abs(s.h[far] - 2.0).max() <= 1e-13
    # direction of the flow is kept
    assert np.allclose(s.hu[far] / s.hv[far], c.hu[0] / c.hv[0], rtol=1e-13)


def test_advance_stops_exactly_at_end_time():
    c = inputs.random_flow_case(seed=3)
    s = oracle.state_from_case(c)
    k = s.advance(0.5)
    assert s.t == 0.5 and k >= 2
    s2 = oracle.state_from_case(c)
    dts = s2.run(k - 1)
    assert dts.sum() < 0.5


def test_all_dry_is_an_error():
    c = inputs.random_flow_case()
    s = oracle.state_from_case(c)
    s.h[:] = 0.0
    with pytest.raises(oracle.OracleError) as ei:
        s.cfl_dt()
    assert ei.value.status == oracle.E_DRY


def test_single_cell_updates_match_the_full_step():
    c = inputs.random_flow_case(seed=23)
    s = oracle.state_from_case(c)
    dt = s.cfl_dt()
    cells = np.arange(0, s.mesh.T, 7)
    one = s.cells_after_step(dt, cells)
    s.step(dt)
    assert np.array_equal(one[0], s.h[cells])
    assert np.array_equal(one[1], s.hu[cells])
    assert np.array_equal(one[2], s.hv[cells])


def test_threaded_loops_give_identical_results():
    """The oracle's OpenMP edge and cell loops (used for the all-core CPU
    baseline) change nothing: 4 threads reproduce the serial run bit for bit,
    dt sequence included."""
    case = inputs.random_flow_case(nx=40, ny=26, seed=17)
    runs = []
    for nt in (1, 4):
        oracle.set_threads(nt)
        try:
            st = oracle.state_from_case(case)
            dts = st.run(30)
            runs.append((st.h.copy(), st.hu.copy(), st.hv.copy(), np.asarray(dts).copy()))
        finally:
            oracle.set_threads(1)
    for a, b in zip(runs[0], runs[1]):
        assert np.array_equal(a, b)
