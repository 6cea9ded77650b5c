"""CUDA path vs the FP64 oracle, element by element, through the C ABI.

Bar: the FP64 path matches the oracle to 1e-11 relative after 100 steps:
per field f in (h, hu, hv), max over cells of |f_gpu - f_oracle| divided by
max |f_oracle|; a discharge field that is itself at round-off (still water)
is divided by the Froude-1 discharge h_max sqrt(g h_max) instead. The FP32
path's L1/Linf errors against the FP64 oracle are stated and gated loosely.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1807_00672_gb300 import inputs, swe

from closed_forms import stoker_depth
from gpu_util import ensure_built, field_errors, gpu_state, l1_linf, oracle_run, rel_err

pytestmark = pytest.mark.gpu

TOL64 = 1e-11

KERNELS = [("tiled", "morton", 256), ("tiled", "morton", 128), ("tiled", "none", 256),
           ("tiled", "rcm", 256), ("edge", "morton", 0), ("edge", "none", 0), ("edge", "rcm", 0)]

# tiled kernel shapes: (cells per tile, cells per thread, stages)
# (tile, cells_per_thread, stages, halo_schedule)
TILED_SHAPES = [(256, 2, 3, 0), (256, 1, 2, 0), (256, 1, 3, 0), (128, 1, 2, 0), (512, 2, 2, 0),
                (64, 1, 3, 0), (256, 2, 2, 1), (64, 1, 3, 1), (256, 1, 2, 2), (512, 2, 2, 2),
                (64, 1, 2, 2)]


def small_cases():
    # sizes span several tiles with a ragged tail (T not a multiple of 128/256)
    return [
        inputs.random_flow_case(nx=37, ny=23, seed=41),            # 1,702 cells, wet/dry
        inputs.lake_at_rest_case(nx=45, ny=19, seed=43),           # 1,710 cells, dry islands
        inputs.humps_case(nx=61, ny=33, lx=2_000.0, ly=1_000.0, seed=45),  # 4,026 cells
        inputs.uniform_flow_case(nx=29, ny=17, seed=47),           # friction
    ]


@pytest.mark.parametrize("kernel,order,tile", KERNELS)
def test_fp64_matches_oracle_100_steps(kernel, order, tile):
    for case in small_cases():
        ref, dts = oracle_run(case, 100)
        mesh, st = gpu_state(case, "f64", kernel, order, tile)
        st.run(100)
        errs, _ = field_errors(st, ref)
        assert max(errs.values()) <= TOL64, (case.name, errs)
        t, mass = st.copy_out()
        assert t == pytest.approx(dts.sum(), rel=1e-13)
        assert mass == pytest.approx(ref.mass(), rel=1e-13)
        info = st.info()
        assert info["steps"] == 100 and info["neg"] == 0 and info["err"] == 0


@pytest.mark.parametrize("tile,cpt,stages,sched", TILED_SHAPES)
def test_tiled_shapes_match_oracle(tile, cpt, stages, sched):
    """Every tiled-kernel shape and halo-gather schedule, FP64 within 1e-11
    of the oracle and FP32 within its stated error, on a mesh spanning many
    tiles with a ragged tail."""
    case = inputs.humps_case(nx=71, ny=29, lx=2_000.0, ly=1_000.0, seed=61)   # 4,118 cells
    ref, _ = oracle_run(case, 60)
    area = ref.mesh.cells()["area"]
    for prec in ("f64", "f32"):
        ensure_built()
        mesh = swe.Mesh(case.mesh.xy, case.mesh.tri, precision=prec, kernel="tiled", tile=tile,
                        cells_per_thread=cpt, stages=stages, halo_schedule=sched)
        st = swe.State(mesh, case.h, case.hu, case.hv, case.z, case.n)
        st.run(60)
        if prec == "f64":
            errs, _ = field_errors(st, ref)
            assert max(errs.values()) <= TOL64, (tile, cpt, stages, errs)
        else:
            h, _, _ = st.fields()
            assert l1_linf(h, ref.h, area)[0] <= 1e-5, (tile, cpt, stages)
        assert st.info()["err"] == 0


def test_fp64_first_dt_matches_oracle():
    case = inputs.random_flow_case(nx=30, ny=20, seed=3)
    ref = oracle.state_from_case(case)
    mesh, st = gpu_state(case, "f64")
    assert st.next_dt() == pytest.approx(ref.cfl_dt(), rel=1e-14)
    dt = st.step()
    assert dt == pytest.approx(ref.cfl_dt(), rel=1e-14)


@pytest.mark.parametrize("kernel", ["tiled", "edge"])
def test_stoker_to_end_time(kernel):
    """Config: 2,500 triangles, dam break to T_s = 2 s (FP64), walls, n = 0."""
    case = inputs.stoker_case()
    ref = oracle.state_from_case(case)
    k_ref = ref.advance(2.0)
    mesh, st = gpu_state(case, "f64", kernel)
    k = st.advance(2.0)
    assert k == k_ref
    t, _ = st.copy_out()
    assert t == 2.0
    errs, (h, hu, hv) = field_errors(st, ref)
    assert max(errs.values()) <= TOL64, errs
    # and the closed form along the centreline
    cen = inputs.centroids(case.mesh)
    band = np.abs(cen[:, 1] - 25.0) <= 2.0
    he = stoker_depth(cen[band, 0], 2.0, 10.0, 1.0, 50.0)
    assert np.abs(h[band] - he).sum() / he.sum() <= 0.03


def test_advance_in_pieces_equals_one_advance():
    case = inputs.random_flow_case(nx=20, ny=14, seed=5)
    mesh, a = gpu_state(case, "f64")
    a.advance(0.3)
    a.advance(0.7)
    _, b = gpu_state(case, "f64")
    b.advance(0.7)
    assert a.t == 0.7 and b.t == 0.7
    ref = oracle.state_from_case(case)
    ref.advance(0.3)
    ref.advance(0.7)
    errs, _ = field_errors(a, ref)
    assert max(errs.values()) <= TOL64


def test_graph_replay_equals_single_steps_bitwise():
    case = inputs.random_flow_case(nx=33, ny=21, seed=9)
    for prec in ("f64", "f32"):
        _, a = gpu_state(case, prec)
        a.run(40)   # two graphs of 16 + 8 single launches
        _, b = gpu_state(case, prec)
        for _ in range(40):
            b.step()
        for x, y in zip(a.fields(), b.fields()):
            assert np.array_equal(x, y)


def test_a_step_is_independent_of_the_tile_walk_direction():
    """Consecutive steps walk every block's tiles in opposite directions, and
    the last tiles of each walk are handed out at run time from a pool (the
    blocks that finish first take more). The order and the assignment of the
    tiles change no bit: the first step of a fresh state (walked forwards)
    equals the second step of a state restarted from the same fields by
    swe_state_set (walked backwards), with a ragged last tile, and repeated
    runs are identical. FP32 on 4,000,000 cells (about 17 tiles per block,
    the last three waves pooled in both walks), FP64 on 974,000 cells (no
    pool)."""
    for prec, (nx, ny) in (("f32", (2000, 1000)), ("f64", (1000, 487))):
        case = inputs.humps_case(nx=nx, ny=ny, lx=20_000.0, ly=10_000.0, seed=19)
        _, a = gpu_state(case, prec)
        a.step()
        _, b = gpu_state(case, prec)
        b.step()
        b.set(case.h, case.hu, case.hv)
        b.step()
        assert a.t == b.t
        for x, y in zip(a.fields(), b.fields()):
            assert np.array_equal(x, y)
        a.run(9)
        _, c = gpu_state(case, prec)
        c.run(10)
        for x, y in zip(a.fields(), c.fields()):
            assert np.array_equal(x, y)


def test_pooled_tiles_with_three_stages_give_the_same_bits():
    """A mesh large enough for the tile pool (4,000,000 cells), stepped with
    three shared-memory stages and with two: the same bits (the stages only
    change how far ahead tiles are fetched)."""
    case = inputs.humps_case(nx=2000, ny=1000, lx=20_000.0, ly=10_000.0, seed=23)
    out = []
    for stages in (2, 3):
        ensure_built()
        mesh = swe.Mesh(case.mesh.xy, case.mesh.tri, precision="f32", stages=stages)
        st = swe.State(mesh, case.h, case.hu, case.hv, case.z, case.n)
        st.run(12)
        assert st.info()["err"] == 0
        out.append(st.fields())
    for x, y in zip(*out):
        assert np.array_equal(x, y)


def test_runs_are_deterministic_bitwise():
    case = inputs.humps_case(nx=80, ny=40, lx=2_000.0, ly=1_000.0, seed=13)
    for prec in ("f64", "f32"):
        for kernel in ("tiled", "edge"):
            outs = []
            for _ in range(2):
                _, s = gpu_state(case, prec, kernel)
                s.run(50)
                outs.append(s.fields() + s.copy_out())
            for x, y in zip(outs[0], outs[1]):
                assert np.array_equal(np.asarray(x), np.asarray(y))


def test_tiled_and_edge_kernels_agree_fp64():
    case = inputs.humps_case(nx=90, ny=45, lx=3_000.0, ly=1_500.0, seed=17)
    _, a = gpu_state(case, "f64", "tiled")
    _, b = gpu_state(case, "f64", "edge")
    a.run(60)
    b.run(60)
    for x, y in zip(a.fields(), b.fields()):
        assert rel_err(x, y) <= 1e-13


def test_fp32_error_against_fp64_oracle():
    """FP32 state and fluxes with compensated face sums: stated L1/Linf error."""
    case = inputs.humps_case(nx=120, ny=60, lx=4_000.0, ly=2_000.0, seed=19)
    ref, _ = oracle_run(case, 100)
    area = ref.mesh.cells()["area"]
    for kernel in ("tiled", "edge"):
        _, st = gpu_state(case, "f32", kernel)
        st.run(100)
        h, hu, hv = st.fields()
        l1h, linfh = l1_linf(h, ref.h, area)
        assert l1h <= 1e-4, (kernel, l1h, linfh)
        for f, r in ((hu, ref.hu), (hv, ref.hv)):
            l1, _ = l1_linf(f, r, area)
            assert l1 <= 1e-3, (kernel, l1)
        info = st.info()
        assert info["neg"] == 0 and info["err"] == 0


def test_lake_at_rest_on_gpu():
    case = inputs.lake_at_rest_case(nx=50, ny=30, seed=21)
    scale = 9.81 * case.h.max() ** 2
    for prec, tol in (("f64", 1e-12), ("f32", 1e-5)):
        for kernel in ("tiled", "edge"):
            _, st = gpu_state(case, prec, kernel)
            st.run(100)
            h, hu, hv = st.fields()
            assert np.abs(hu).max() <= tol * scale and np.abs(hv).max() <= tol * scale, (prec, kernel)
            assert np.abs(h - case.h).max() <= tol * case.h.max() * 10


def test_mass_conservation_on_gpu():
    case = inputs.random_flow_case(nx=40, ny=30, seed=23)
    for prec, tol in (("f64", 1e-13), ("f32", 1e-6)):
        for kernel in ("tiled", "edge"):
            _, st = gpu_state(case, prec, kernel)
            m0 = st.mass
            st.run(100)
            assert abs(st.mass - m0) <= tol * m0, (prec, kernel)
            assert st.info()["neg"] == 0


def test_single_triangle_all_walls():
    xy = np.array([[0.0, 0.0], [2.0, 0.0], [0.5, 1.5]])
    tri = np.array([[0, 1, 2]], dtype=np.int32)
    case = inputs.Case(inputs.Mesh(xy, tri), np.array([1.0]), np.array([0.3]), np.array([-0.2]),
                       np.array([0.0]), np.array([0.02]))
    ref, _ = oracle_run(case, 10)
    for kernel in ("tiled", "edge"):
        _, st = gpu_state(case, "f64", kernel)
        st.run(10)
        errs, (h, _, _) = field_errors(st, ref)
        assert max(errs.values()) <= TOL64
        assert h[0] == pytest.approx(1.0, rel=1e-15)  # walls: no mass flux


def test_fewer_cells_than_a_tile_and_ragged_tail():
    for nx, ny in ((3, 2), (11, 6), (16, 8), (17, 8)):   # 12, 132, 256, 272 cells
        case = inputs.random_flow_case(nx=nx, ny=ny, lx=10.0 * nx, ly=10.0 * ny, seed=nx)
        ref, _ = oracle_run(case, 30)
        for kernel, order, tile in KERNELS:
            _, st = gpu_state(case, "f64", kernel, order, tile)
            st.run(30)
            errs, _ = field_errors(st, ref)
            assert max(errs.values()) <= TOL64, (nx, ny, kernel, tile, errs)


def test_all_dry_is_reported():
    ensure_built()
    case = inputs.random_flow_case(nx=8, ny=6)
    mesh = swe.Mesh(case.mesh.xy, case.mesh.tri)
    with pytest.raises(swe.SweError) as ei:
        swe.State(mesh, np.zeros(mesh.T), np.zeros(mesh.T), np.zeros(mesh.T), case.z, case.n)
    assert ei.value.status == swe.SWE_EDRY


def test_nan_input_is_reported():
    ensure_built()
    case = inputs.random_flow_case(nx=8, ny=6)
    h = case.h.copy()
    h[5] = np.nan
    mesh = swe.Mesh(case.mesh.xy, case.mesh.tri)
    with pytest.raises(swe.SweError) as ei:
        swe.State(mesh, h, case.hu, case.hv, case.z, case.n)
    assert ei.value.status == swe.SWE_ENAN


def test_state_set_restarts_from_new_fields():
    case = inputs.random_flow_case(nx=20, ny=10, seed=29)
    ref, _ = oracle_run(case, 20)
    _, st = gpu_state(case, "f64")
    st.run(7)
    st.set(case.h, case.hu, case.hv)
    assert st.t == 0.0
    st.run(20)
    errs, _ = field_errors(st, ref)
    assert max(errs.values()) <= TOL64


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_constant_manning_equals_per_cell_array(prec):
    case = inputs.uniform_flow_case(nx=20, ny=10)
    ensure_built()
    m = swe.Mesh(case.mesh.xy, case.mesh.tri, precision=prec)
    a = swe.State(m, case.h, case.hu, case.hv, case.z, case.n)
    b = swe.State(m, case.h, case.hu, case.hv, case.z, None, manning_const=0.05)
    a.run(20)
    b.run(20)
    for x, y in zip(a.fields(), b.fields()):
        assert np.array_equal(x, y)


# ------------------------------------------------------------------ full sizes

@pytest.mark.slow
def test_fp64_1m_humps_matches_oracle_after_100_steps():
    """1,000,000 triangles, bed of three Gaussian humps, wet/dry fronts."""
    case = inputs.humps_case()
    ref, dts = oracle_run(case, 100)
    mesh, st = gpu_state(case, "f64")
    st.run(100)
    errs, _ = field_errors(st, ref)
    assert max(errs.values()) <= TOL64, errs


@pytest.mark.slow
def test_fp32_10m_sinusoid_sampled_cells():
    """10,001,406 triangles in the benchmark's launch configuration: after 20
    FP32 steps, one more step checked cell by cell on a seeded sample against
    the oracle's FP64 update of the same (FP32-rounded) state with the same
    dt; and properties at full size: mass, positivity, finiteness."""
    case = inputs.sinusoid_case()
    mesh, st = gpu_state(case, "f32")
    m0 = st.mass
    st.run(20)
    h, hu, hv = st.fields()
    dt = st.next_dt()
    st.run(1)
    h1, hu1, hv1 = st.fields()
    # the FP32 step used dt rounded to float
    dt32 = float(np.float32(dt))
    o = oracle.State(oracle.Mesh(case.mesh.xy, case.mesh.tri), h, hu, hv, case.z, case.n)
    rng = np.random.default_rng(77)
    cells = rng.choice(mesh.T, size=20_000, replace=False)
    want = o.cells_after_step(dt32, cells)
    for got, w, full in ((h1, want[0], h), (hu1, want[1], hu), (hv1, want[2], hv)):
        scale = max(np.abs(full).max(), 1e-30)
        assert np.abs(got[cells] - w).max() <= 2e-6 * scale
    assert np.all(h1 >= 0) and np.all(np.isfinite(h1))
    assert abs(st.mass - m0) <= 1e-6 * m0


def test_meshes_of_different_layouts_in_any_order():
    """A tiled kernel's shared-memory limit is shared by every mesh that
    launches it: a mesh created after another one, with a smaller layout,
    must not stop the first one's steps (nor graph captures of new states
    on it)."""
    big = inputs.humps_case(nx=120, ny=60, lx=4_000.0, ly=2_000.0, seed=19)
    small = inputs.random_flow_case(nx=6, ny=4, seed=3)
    for prec in ("f64", "f32"):
        ensure_built()
        mb = swe.Mesh(big.mesh.xy, big.mesh.tri, precision=prec)
        a = swe.State(mb, big.h, big.hu, big.hv, big.z, big.n)
        a.run(20)
        ms = swe.Mesh(small.mesh.xy, small.mesh.tri, precision=prec)
        b = swe.State(ms, small.h, small.hu, small.hv, small.z, small.n)
        b.run(20)
        c = swe.State(mb, big.h, big.hu, big.hv, big.z, big.n)  # new graph on the big mesh
        c.run(20)
        a.set(big.h, big.hu, big.hv)
        a.run(20)
        for x, y in zip(a.fields(), c.fields()):
            assert np.array_equal(x, y)
        assert a.info()["err"] == 0 and c.info()["err"] == 0


@pytest.mark.parametrize("tile,cpt", [(256, 1), (512, 2), (128, 2), (32, 1), (512, 1)])
def test_pipelined_fp32_step_equals_the_two_barrier_step_bitwise(tile, cpt):
    """halo_schedule 2 (one block barrier per tile: the cell updates of a
    tile overlap the face loop of the next) computes every face and cell with
    the same arithmetic as the default kernel: the same bits, for any
    number of tiles per block and a ragged last tile."""
    ensure_built()
    for case in (inputs.humps_case(nx=71, ny=29, lx=2_000.0, ly=1_000.0, seed=61),
                 inputs.random_flow_case(nx=37, ny=23, seed=41)):
        out = []
        for sched in (0, 2):
            # 512-cell tiles with one cell per thread exist only pipelined: the
            # two-barrier reference runs them with two cells per thread
            c = 2 if (sched == 0 and tile // cpt == 512) else cpt
            mesh = swe.Mesh(case.mesh.xy, case.mesh.tri, precision="f32", kernel="tiled", tile=tile,
                            cells_per_thread=c, halo_schedule=sched)
            st = swe.State(mesh, case.h, case.hu, case.hv, case.z, case.n)
            st.run(37)
            out.append(st.fields() + (st.t,))
            assert st.info()["err"] == 0
        for x, y in zip(out[0], out[1]):
            assert np.array_equal(np.asarray(x), np.asarray(y))
