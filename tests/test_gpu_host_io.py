"""Host-array transfers through the C ABI: swe_state_set / swe_copy_out with
FP64 arrays and their FP32 forms swe_state_set_f32 / swe_copy_out_f32, from
and into page-locked host memory (read and written by a kernel across the
host link) and ordinary host memory (through the staging buffer). Every
path gives bitwise the same state and the same copied values."""
import numpy as np
import pytest

from paper_1807_00672_gb300 import inputs, swe

from gpu_util import ensure_built
from test_gpu_ensemble import ensemble_state, scenario_mix, single_state, split

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def pinned(n, dtype):
    """A numpy view of page-locked host memory (kept alive by the view's base)."""
    t = torch.empty(n, dtype=torch.float64 if dtype == np.float64 else torch.float32).pin_memory()
    a = t.numpy()
    assert a.ctypes.data == t.data_ptr()
    return a


def pinned_copy(a, dtype):
    out = pinned(a.size, dtype)
    out[:] = a
    return out


def state(case, prec, tile=0):
    ensure_built()
    mesh = swe.Mesh(case.mesh.xy, case.mesh.tri, precision=prec, kernel="tiled", tile=tile)
    return mesh, swe.State(mesh, case.h, case.hu, case.hv, case.z, case.n)


def cases():
    # several tiles with a ragged last one; wet/dry; 37 x 23 x 2 = 1,702 cells
    return [inputs.random_flow_case(nx=37, ny=23, seed=41),
            inputs.humps_case(nx=71, ny=29, lx=2_000.0, ly=1_000.0, seed=61)]


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_set_from_pinned_and_pageable_fp64_arrays_is_the_same_state(prec):
    for case in cases():
        outs = []
        for where in ("pageable", "pinned"):
            _, st = state(case, prec)
            st.run(3)  # a state in the other buffer, then replaced
            f = [np.ascontiguousarray(a, dtype=np.float64) for a in (case.h, case.hu, case.hv)]
            if where == "pinned":
                f = [pinned_copy(a, np.float64) for a in f]
            st.set(*f)
            assert st.t == 0.0
            st.run(11)
            outs.append(st.fields() + (st.t, st.mass))
        for x, y in zip(*outs):
            assert np.array_equal(np.asarray(x), np.asarray(y))


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_copy_out_to_pinned_equals_copy_out_to_pageable(prec):
    for case in cases():
        _, st = state(case, prec)
        st.run(9)
        T = case.h.size
        ref = [np.empty(T) for _ in range(3)]
        t0, m0 = st.copy_out(*ref)
        got = [pinned(T, np.float64) for _ in range(3)]
        for a in got:
            a[:] = np.nan
        t1, m1 = st.copy_out(*got)
        assert (t0, m0) == (t1, m1)
        for x, y in zip(ref, got):
            assert np.array_equal(x, y)
        # only some of the fields
        part = pinned(T, np.float64)
        part[:] = np.nan
        st.copy_out(None, part, None)
        assert np.array_equal(part, ref[1])


def test_fp32_arrays_give_the_state_of_the_rounded_fp64_arrays():
    """An SWE_F32 state holds FP32 values: swe_state_set rounds FP64 inputs to
    the nearest FP32, so FP32 arrays holding those rounded values give the
    same state, and swe_copy_out_f32 returns exactly what swe_copy_out
    widens."""
    for case in cases():
        _, a = state(case, "f32")
        a.run(7)
        ref64 = a.fields()
        f32 = [np.asarray(x, dtype=np.float64).astype(np.float32) for x in (case.h, case.hu, case.hv)]
        for where in ("pageable", "pinned"):
            _, b = state(case, "f32")
            b.set_f32(*(pinned_copy(x, np.float32) if where == "pinned" else x for x in f32))
            b.run(7)
            assert b.t == a.t
            got64 = b.fields()
            for x, y in zip(ref64, got64):
                assert np.array_equal(x, y)
            T = case.h.size
            out = [pinned(T, np.float32) if where == "pinned" else np.empty(T, np.float32)
                   for _ in range(3)]
            b.copy_out_f32(*out)
            for x, y in zip(ref64, out):
                assert np.array_equal(x.astype(np.float32), y)
                assert np.array_equal(y.astype(np.float64), x)  # exact: FP32 values


def test_fp32_arrays_on_an_fp64_state():
    """An SWE_F64 state widens FP32 inputs exactly and rounds its values to
    the nearest FP32 on swe_copy_out_f32 (as numpy's float32 cast does)."""
    case = cases()[0]
    f32 = [np.asarray(x, dtype=np.float64).astype(np.float32) for x in (case.h, case.hu, case.hv)]
    _, a = state(case, "f64")
    a.set(*(x.astype(np.float64) for x in f32))
    a.run(5)
    _, b = state(case, "f64")
    b.set_f32(*f32)
    b.run(5)
    ref = a.fields()
    for x, y in zip(ref, b.fields()):
        assert np.array_equal(x, y)
    for where in ("pageable", "pinned"):
        T = case.h.size
        out = [pinned(T, np.float32) if where == "pinned" else np.empty(T, np.float32)
               for _ in range(3)]
        b.copy_out_f32(*out)
        for x, y in zip(ref, out):
            assert np.array_equal(x.astype(np.float32), y)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_ensemble_scenarios_in_different_buffers_copy_out_to_pinned(prec):
    """Scenarios that stopped at different step counts are copied from the
    buffer each one is in, by one kernel per run of scenarios in the same
    buffer, into page-locked arrays as into ordinary ones."""
    cs = scenario_mix()
    mesh, st = ensemble_state(cs, precision=prec)
    st.advance(2.0)
    steps = [st.scenario(i)["steps"] for i in range(len(cs))]
    assert len({s % 2 for s in steps}) == 2
    T = sum(c.h.size for c in cs)
    ref = [np.empty(T) for _ in range(3)]
    st.copy_out(*ref)
    got = [pinned(T, np.float64) for _ in range(3)]
    st.copy_out(*got)
    g32 = [pinned(T, np.float32) for _ in range(3)]
    st.copy_out_f32(*g32)
    for x, y, z in zip(ref, got, g32):
        assert np.array_equal(x, y)
        assert np.array_equal(x.astype(np.float32), z)
    parts = [split(mesh, f) for f in got]
    for i, c in enumerate(cs):
        _, s1 = single_state(c, precision=prec)
        s1.advance(2.0)
        for k, f in enumerate(s1.fields()):
            assert np.array_equal(parts[k][i], f), (i, k)


def test_bad_arguments_are_rejected():
    case = cases()[0]
    _, st = state(case, "f32")
    T = case.h.size
    with pytest.raises(swe.SweError):
        swe._check(swe.lib().swe_state_set_f32(st._h, None, None, None), "swe_state_set_f32")
    with pytest.raises(TypeError):
        st.copy_out_f32(np.empty(T))  # float64 array
