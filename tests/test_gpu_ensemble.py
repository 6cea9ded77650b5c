"""Ensembles (swe_mesh_create_batch): several independent scenarios in one
mesh, advanced by the same launches.

A scenario's result must not depend on the company it keeps: its cells go
through the same per-cell arithmetic whether it runs alone or in a batch, so
the fields must be bitwise identical to a run of that scenario on its own
mesh, and its FP64 fields must match the oracle like any single mesh.
"""
import numpy as np
import pytest

import oracle
from paper_1807_00672_gb300 import inputs, swe

from gpu_util import ensure_built, errors_of, rel_err

pytestmark = pytest.mark.gpu

TOL64 = 1e-11


def scenario_mix():
    """Six scenarios: dam breaks of several sizes (ragged tails), wet/dry
    random flows (one smaller than a tile) and bumps over a dry bed top."""
    cases = inputs.ensemble_cases(3, t_min=300, t_max=9_000, seed=11)
    cases.append(inputs.random_flow_case(nx=21, ny=13, seed=5))
    cases.append(inputs.humps_case(nx=30, ny=20))
    cases.append(inputs.random_flow_case(nx=7, ny=5, seed=6))
    return cases


def areas(case):
    xy, tri = case.mesh.xy, case.mesh.tri
    p0, p1, p2 = xy[tri[:, 0]], xy[tri[:, 1]], xy[tri[:, 2]]
    return 0.5 * np.abs((p1[:, 0] - p0[:, 0]) * (p2[:, 1] - p0[:, 1])
                        - (p2[:, 0] - p0[:, 0]) * (p1[:, 1] - p0[:, 1]))


def ensemble_state(cases, **kw):
    ensure_built()
    mesh = swe.Mesh.ensemble([(c.mesh.xy, c.mesh.tri) for c in cases], **kw)
    cat = lambda name: np.concatenate([getattr(c, name) for c in cases])
    st = swe.State(mesh, cat("h"), cat("hu"), cat("hv"), cat("z"), cat("n"))
    return mesh, st


def single_state(case, **kw):
    mesh = swe.Mesh(case.mesh.xy, case.mesh.tri, **kw)
    return mesh, swe.State(mesh, case.h, case.hu, case.hv, case.z, case.n)


def split(mesh, a):
    return [a[o:o + n] for o, n in zip(mesh.scenario_offsets, mesh.scenario_cells)]


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_ensemble_equals_scenarios_run_alone_bitwise(precision):
    cases = scenario_mix()
    mesh, st = ensemble_state(cases, precision=precision)
    assert mesh.n_scenarios == len(cases)
    assert mesh.scenario_cells == [c.mesh.n_tris for c in cases]
    assert mesh.T == sum(c.mesh.n_tris for c in cases)
    st.run(37)  # two graph replays and five single launches
    got = [split(mesh, f) for f in st.fields()]
    for i, c in enumerate(cases):
        m1, s1 = single_state(c, precision=precision)
        s1.run(37)
        ref = s1.fields()
        for k in range(3):
            assert np.array_equal(got[k][i], ref[k]), (i, k)
        info = st.scenario(i)
        assert info["steps"] == 37
        assert info["t"] == s1.t
        assert info["dt"] == s1.next_dt()
        assert info["mass"] == pytest.approx(s1.mass, rel=1e-13)


def test_ensemble_fp64_matches_oracle_per_scenario():
    cases = scenario_mix()
    mesh, st = ensemble_state(cases, precision="f64")
    st.run(100)
    h, hu, hv = (split(mesh, f) for f in st.fields())
    for i, c in enumerate(cases):
        ref = oracle.state_from_case(c)
        ref.run(100)
        errs = errors_of((h[i], hu[i], hv[i]), (ref.h, ref.hu, ref.hv))
        assert max(errs.values()) <= TOL64, (i, errs)
        assert st.scenario(i)["t"] == pytest.approx(ref.t, rel=1e-13)


def test_ensemble_advance_stops_every_scenario_at_the_end_time():
    """Scenarios take different step counts to reach t_end, so they end in
    different state buffers; each must stop exactly at t_end and equal its
    own advance bitwise."""
    cases = scenario_mix()
    mesh, st = ensemble_state(cases, precision="f64")
    t_end = 2.0  # the oracle takes 43, 26, 28, 32, 1 and 5 steps
    st.advance(t_end)
    steps = [st.scenario(i)["steps"] for i in range(len(cases))]
    assert len(set(steps)) > 1 and len({s % 2 for s in steps}) == 2
    got = [split(mesh, f) for f in st.fields()]
    for i, c in enumerate(cases):
        info = st.scenario(i)
        assert info["t"] == t_end
        m1, s1 = single_state(c, precision="f64")
        n1 = s1.advance(t_end)
        assert info["steps"] == n1
        ref = s1.fields()
        for k in range(3):
            assert np.array_equal(got[k][i], ref[k]), (i, k)


def test_ensemble_total_mass_is_the_sum_of_scenario_masses():
    cases = scenario_mix()
    mesh, st = ensemble_state(cases, precision="f64")
    st.run(20)
    parts = [st.scenario(i)["mass"] for i in range(len(cases))]
    assert st.mass == pytest.approx(sum(parts), rel=1e-15)
    exact = sum(float((areas(c) * c.h).sum()) for c in cases)
    assert st.mass == pytest.approx(exact, rel=1e-12)


def test_ensemble_of_one_equals_a_plain_mesh():
    case = inputs.random_flow_case(nx=33, ny=17, seed=9)
    mesh, st = ensemble_state([case], precision="f32")
    m1, s1 = single_state(case, precision="f32")
    st.run(25)
    s1.run(25)
    for a, b in zip(st.fields(), s1.fields()):
        assert np.array_equal(a, b)


def test_ensemble_reports_a_dry_scenario_at_init():
    cases = scenario_mix()[:2]
    dry = cases[1]
    dry.h[:] = 0.0
    with pytest.raises(swe.SweError) as e:
        ensemble_state(cases, precision="f64")
    assert e.value.status == swe.SWE_EDRY


def test_scenario_index_is_checked():
    mesh, st = ensemble_state(scenario_mix()[:2], precision="f64")
    with pytest.raises(swe.SweError) as e:
        st.scenario(2)
    assert e.value.status == swe.SWE_EINVAL


def test_mesh_closed_before_its_state_stays_alive_until_the_state_goes():
    """Destroying a mesh that a state still uses only marks it; the state
    keeps working and frees the mesh when it is destroyed itself (garbage
    collection may finalise the two in either order)."""
    cases = scenario_mix()[:3]
    mesh, st = ensemble_state(cases, precision="f32")
    ref_mesh, ref = ensemble_state(cases, precision="f32")
    mesh.close()
    st.run(5)
    ref.run(5)
    for a, b in zip(st.fields(), ref.fields()):
        assert np.array_equal(a, b)
    st.close()


def test_autotuner_picks_a_measured_shape_and_caches_it(tmp_path, monkeypatch):
    pytest.importorskip("torch")
    from paper_1807_00672_gb300 import autotune
    ensure_built()
    monkeypatch.setenv("SWE_TUNE_CACHE", str(tmp_path / "tune.json"))
    cases = scenario_mix()[:3]
    cand = ((256, 2, 2), (256, 2, 2, 1), (128, 1, 2), (64, 2, 2))
    r = autotune.tune(cases, "f32", candidates=cand, steps=8)
    assert not r["cached"]
    picked = (r["tile"], r["cells_per_thread"], r["stages"])
    assert picked + (r["halo_schedule"],) in cand or (r["halo_schedule"] == 0 and picked in cand)
    timed = [t for t in r["trials"] if "sec_per_step" in t]
    assert len(timed) == 4
    assert r["sec_per_step"] == min(t["sec_per_step"] for t in timed)
    again = autotune.tune(cases, "f32", candidates=cand, steps=8)
    assert again["cached"] and again["tile"] == r["tile"]
    # the chosen shape runs and matches the default shape bitwise
    mesh, st = ensemble_state(cases, precision="f32", tile=r["tile"],
                              cells_per_thread=r["cells_per_thread"], stages=r["stages"],
                              halo_schedule=r["halo_schedule"])
    ref_mesh, ref = ensemble_state(cases, precision="f32")
    st.run(10)
    ref.run(10)
    for a, b in zip(st.fields(), ref.fields()):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("precision", ["f64", "f32"])
@pytest.mark.parametrize("tile,cpt", [(256, 2), (64, 1)])
def test_early_halo_schedule_is_bitwise_equal(precision, tile, cpt):
    """halo_schedule = 1 moves only when each tile's halo gather is issued,
    and 2 (FP32) overlaps a tile's cell updates with the next tile's faces;
    the arithmetic and its order are those of the default schedule, on an
    ensemble whose chunks mix scenarios."""
    cases = scenario_mix()
    runs = []
    for sched in ((0, 1, 2) if precision == "f32" else (0, 1)):
        mesh, st = ensemble_state(cases, precision=precision, tile=tile, cells_per_thread=cpt,
                                  halo_schedule=sched)
        st.run(21)
        runs.append(st.fields())
        assert st.info()["err"] == 0
    for other in runs[1:]:
        for a, b in zip(runs[0], other):
            assert np.array_equal(a, b)
