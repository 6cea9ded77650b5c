"""Failure detection on the GPU without a GPU fault.

The tiled kernels wait for their tile copies with bounded waits and latch
SWE_ETIMEOUT when a wait runs out (instead of hanging). A mesh built with
swe_params.wait_rounds = -1 makes the first wait of every step give up at
once, so the timeout path runs deterministically: the copies already in
flight are still waited for (with the normal limit) before each block
exits, the step reports SWE_ETIMEOUT, later steps are skipped, and the
device stays usable: a fresh state on the same device then steps and
matches the oracle.
"""
import numpy as np
import pytest

from paper_1807_00672_gb300 import inputs, swe

from gpu_util import ensure_built, field_errors, oracle_run

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec,sched", [("f64", 0), ("f32", 0), ("f32", 1)])
def test_wait_that_runs_out_reports_timeout_and_device_recovers(prec, sched):
    ensure_built()
    case = inputs.random_flow_case(nx=37, ny=23, seed=41)   # 1,702 cells, several tiles
    mesh = swe.Mesh(case.mesh.xy, case.mesh.tri, precision=prec, kernel="tiled", tile=128,
                    halo_schedule=sched, wait_rounds=-1)
    st = swe.State(mesh, case.h, case.hu, case.hv, case.z, case.n)  # init has no waits
    h0, _, _ = st.fields()
    with pytest.raises(swe.SweError) as ei:
        st.step()
    assert ei.value.status == swe.SWE_ETIMEOUT
    # later steps are skipped: the error stays latched, the clock stays at 0
    st.run(20, sync=False)
    with pytest.raises(swe.SweError) as ei:
        st.sync()
    assert ei.value.status == swe.SWE_ETIMEOUT
    info = st.info()
    assert info["err"] & 4 and info["steps"] <= 1
    st.close()
    mesh.close()

    # the device is still usable: a fresh mesh and state with the default limit
    ref, _ = oracle_run(case, 20)
    mesh2 = swe.Mesh(case.mesh.xy, case.mesh.tri, precision=prec, kernel="tiled", tile=128,
                     halo_schedule=sched)
    st2 = swe.State(mesh2, case.h, case.hu, case.hv, case.z, case.n)
    st2.run(20)
    if prec == "f64":
        errs, _ = field_errors(st2, ref)
        assert max(errs.values()) <= 1e-11, errs
    else:
        h, _, _ = st2.fields()
        assert np.abs(h - ref.h).max() <= 1e-4 * np.abs(ref.h).max()
    assert st2.info()["err"] == 0


def test_gradient_recording_reports_timeout():
    ensure_built()
    case = inputs.random_flow_case(nx=20, ny=12, seed=7)
    mesh = swe.Mesh(case.mesh.xy, case.mesh.tri, precision="f64", tile=128, wait_rounds=-1)
    st = swe.State(mesh, case.h, case.hu, case.hv, case.z, case.n)
    with pytest.raises(swe.SweError) as ei:
        swe.Tape(st, 5, 2, [0, 3])
    assert ei.value.status == swe.SWE_ETIMEOUT


@pytest.mark.parametrize("kernel", ["tiled", "edge"])
def test_negative_input_depths_are_clipped_and_counted(kernel):
    """A negative depth injected into the initial state is not a fault: the
    first step clips it at 0 and counts it (swe_state_info), as the oracle
    does; the state then matches the oracle's to 1e-11 and stays >= 0."""
    ensure_built()
    case = inputs.random_flow_case(nx=37, ny=23, seed=41)
    # a dry disc (no inflow within 10 steps) whose inner cells hold -1 cm
    c = inputs.centroids(case.mesh)
    r = np.hypot(c[:, 0] - 60.0, c[:, 1] - 40.0)
    for f in (case.h, case.hu, case.hv):
        f[r < 40.0] = 0.0
    case.h[r < 15.0] = -0.01
    ref, _ = oracle_run(case, 10)
    assert ref.neg == int((case.h < 0).sum()) > 0
    mesh = swe.Mesh(case.mesh.xy, case.mesh.tri, precision="f64", kernel=kernel)
    st = swe.State(mesh, case.h, case.hu, case.hv, case.z, case.n)
    st.run(10)
    info = st.info()
    assert info["neg"] == ref.neg and info["err"] == 0
    errs, (h, _, _) = field_errors(st, ref)
    assert max(errs.values()) <= 1e-11, errs
    assert np.all(h >= 0.0)
