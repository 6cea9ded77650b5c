"""FP32 states with a depth residual (swe_params.compensated_depth): the
Euler update of h keeps the part of each update that FP32 rounding would
drop, so the mass stays at its FP64-integration level over long runs and
the depth follows the FP64 oracle far more closely than plain FP32.
Through the C ABI, against the FP64 oracle and the plain FP32 path."""
import numpy as np
import pytest

import oracle
from paper_1807_00672_gb300 import inputs, swe

from gpu_util import ensure_built, l1_linf, oracle_run
from test_gpu_ensemble import ensemble_state, scenario_mix, single_state, split

pytestmark = pytest.mark.gpu


def state(case, comp, **kw):
    ensure_built()
    mesh = swe.Mesh(case.mesh.xy, case.mesh.tri, precision="f32", compensated_depth=comp, **kw)
    return mesh, swe.State(mesh, case.h, case.hu, case.hv, case.z, case.n)


def test_water_drop_keeps_its_mass():
    """20,402 cells, still water 10 m deep with a 1 m hump, walls, to
    T_s = 2,400 s (3,640 steps): plain FP32 loses about 1e-6 of the mass
    (updates below half an ulp of 10 m are rounded away, unevenly), the
    residual keeps it to the FP64 integral's round-off."""
    case = inputs.water_drop_case(n=101)
    drift = {}
    for comp in (False, True):
        _, st = state(case, comp)
        m0 = st.mass
        st.advance(2400.0)
        assert st.t == 2400.0 and st.info()["err"] == 0
        drift[comp] = abs(st.mass - m0) / m0
    assert drift[True] <= 1e-11, drift
    assert drift[False] >= 1e3 * drift[True], drift


def test_depth_follows_the_fp64_oracle():
    """Wet/dry humps, 4,026 cells, 100 steps: L1(h) against the FP64 oracle
    smaller than plain FP32's, and within 1e-7."""
    case = inputs.humps_case(nx=61, ny=33, lx=2_000.0, ly=1_000.0, seed=45)
    ref, _ = oracle_run(case, 100)
    area = ref.mesh.cells()["area"]
    err = {}
    for comp in (False, True):
        _, st = state(case, comp)
        st.run(100)
        h, _, _ = st.fields()
        err[comp] = l1_linf(h, ref.h, area)[0]
        assert st.info()["err"] == 0 and st.info()["neg"] == 0
    print("L1(h) plain / compensated", err[False], err[True])
    assert err[True] <= 1e-7 and err[True] < err[False], err


def test_copy_out_returns_depth_plus_residual():
    """The FP64 copy-out holds h + residual (exact in FP64), the FP32 one its
    rounding to FP32; the mass integral is that of h + residual."""
    case = inputs.water_drop_case(n=41)
    _, st = state(case, True)
    st.run(300)
    T = case.h.size
    h64 = np.empty(T)
    t, mass = st.copy_out(h64)
    h32 = np.empty(T, np.float32)
    st.copy_out_f32(h32)
    assert np.array_equal(h64.astype(np.float32), h32)
    d = h64 - h32.astype(np.float64)
    assert np.any(d != 0.0)  # some residuals are non-zero
    assert np.all(np.abs(d) <= 0.5 * np.spacing(h32).astype(np.float64))
    ref = oracle.state_from_case(case)
    area32 = ref.mesh.cells()["area"].astype(np.float32).astype(np.float64)  # the mesh's areas
    assert mass == pytest.approx(float(np.sum(area32 * h64)), rel=1e-12)


def test_set_clears_the_residual():
    case = inputs.random_flow_case(nx=37, ny=23, seed=41)
    _, a = state(case, True)
    a.run(25)
    a.set(case.h, case.hu, case.hv)
    a.run(25)
    _, b = state(case, True)
    b.run(25)
    for x, y in zip(a.fields(), b.fields()):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("tile,cpt", [(512, 2), (256, 1), (128, 2), (64, 1)])
def test_every_tile_shape_gives_the_same_bits(tile, cpt):
    case = inputs.humps_case(nx=71, ny=29, lx=2_000.0, ly=1_000.0, seed=61)
    out = []
    for t, c in ((512, 2), (tile, cpt)):
        _, st = state(case, True, tile=t, cells_per_thread=c)
        st.run(40)
        out.append(st.fields())
    for x, y in zip(*out):
        assert np.array_equal(x, y)


def test_pooled_tiles_give_the_same_bits():
    """On 4,000,000 cells (about 17 tiles per block) the last tiles of each
    walk are handed out at run time; a step walked backwards equals the same
    step walked forwards, and repeated runs are identical."""
    case = inputs.humps_case(nx=2000, ny=1000, lx=20_000.0, ly=10_000.0, seed=19)
    _, a = state(case, True)
    a.step()
    _, b = state(case, True)
    b.step()
    b.set(case.h, case.hu, case.hv)
    b.step()
    for x, y in zip(a.fields(), b.fields()):
        assert np.array_equal(x, y)
    a.run(7)
    _, c = state(case, True)
    c.run(8)
    for x, y in zip(a.fields(), c.fields()):
        assert np.array_equal(x, y)
    assert c.info()["err"] == 0


def test_ensemble_scenarios_equal_their_own_runs():
    cs = scenario_mix()
    mesh, st = ensemble_state(cs, precision="f32", compensated_depth=True)
    st.advance(2.0)
    got = [split(mesh, f) for f in st.fields()]
    for i, c in enumerate(cs):
        _, s1 = single_state(c, precision="f32", compensated_depth=True)
        s1.advance(2.0)
        for k, f in enumerate(s1.fields()):
            assert np.array_equal(got[k][i], f), (i, k)


def test_unsupported_combinations_are_rejected():
    case = inputs.random_flow_case(nx=9, ny=7, seed=2)
    for kw in (dict(precision="f64"), dict(precision="f32", kernel="edge"),
               dict(precision="f32", stages=3), dict(precision="f32", halo_schedule=1)):
        with pytest.raises(swe.SweError) as e:
            swe.Mesh(case.mesh.xy, case.mesh.tri, compensated_depth=True, **kw)
        assert e.value.status == swe.SWE_EINVAL, kw
    _, st = state(case, True)
    with pytest.raises(swe.SweError) as e:
        swe.Tape(st, 4, 2, np.array([0], dtype=np.int32))
    assert e.value.status == swe.SWE_ESTATE
