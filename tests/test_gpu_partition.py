"""Decomposed runs on one GPU (partition.LocalRun: every sub-domain a
library mesh with ghost cells, halos packed and unpacked by the library's
kernels, the global time step as a minimum on the device) against the
whole mesh's run: the owned cells equal it bit for bit, FP64 and FP32, and
the FP64 result matches the oracle."""
import numpy as np
import pytest

from paper_1807_00672_gb300 import inputs, swe

from gpu_util import ensure_built, errors_of, oracle_run

pytestmark = pytest.mark.gpu


def fields(case):
    return (case.h, case.hu, case.hv, case.z, case.n)


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("P", [2, 3])
def test_decomposed_run_equals_the_whole_mesh_bitwise(prec, P):
    pytest.importorskip("torch")
    from paper_1807_00672_gb300.partition import LocalRun
    ensure_built()
    case = inputs.humps_case(nx=71, ny=29, lx=2_000.0, ly=1_000.0, seed=61)  # 4,118 cells
    whole = swe.Mesh(case.mesh.xy, case.mesh.tri, precision=prec, tile=128)
    ref = swe.State(whole, *fields(case))
    m0 = ref.mass
    run = LocalRun(case.mesh.xy, case.mesh.tri, fields(case), P, precision=prec, tile=128)
    assert run.mass() == pytest.approx(m0, rel=1e-12)
    for _ in range(2):
        ref.run(20)
        run.run(20)
        got = run.fields()
        want = ref.fields()
        for a, b in zip(got, want):
            assert np.array_equal(a, b)
        assert run.parts[0].state.t == ref.t
    assert run.mass() == pytest.approx(ref.mass, rel=1e-12)
    for s in run.parts:
        assert s.state.info()["err"] == 0
    run.close()


def test_decomposed_fp64_run_matches_the_oracle():
    pytest.importorskip("torch")
    from paper_1807_00672_gb300.partition import LocalRun
    ensure_built()
    case = inputs.random_flow_case(nx=37, ny=23, seed=41)  # wet/dry, walls
    ref, _ = oracle_run(case, 60)
    run = LocalRun(case.mesh.xy, case.mesh.tri, fields(case), 4, precision="f64")
    run.run(60)
    errs = errors_of(run.fields(), (ref.h, ref.hu, ref.hv))
    assert max(errs.values()) <= 1e-11, errs
    run.close()


def test_halo_calls_need_a_mesh_with_ghosts():
    ensure_built()
    torch = pytest.importorskip("torch")
    case = inputs.random_flow_case(nx=8, ny=6, seed=3)
    mesh = swe.Mesh(case.mesh.xy, case.mesh.tri, precision="f64")
    st = swe.State(mesh, *fields(case))
    ids = torch.zeros(4, dtype=torch.int32, device="cuda")
    buf = torch.zeros(12, dtype=torch.float64, device="cuda")
    with pytest.raises(swe.SweError) as e:
        st.halo_pack(ids.data_ptr(), 4, buf.data_ptr())
    assert e.value.status == swe.SWE_ESTATE
    # and gradients are not taken on a sub-domain mesh
    pmesh = swe.Mesh.part(case.mesh.xy, case.mesh.tri, np.zeros(mesh.T, np.uint8))
    pst = swe.State(pmesh, *fields(case))
    with pytest.raises(swe.SweError) as e:
        swe.Tape(pst, 2, 1)
    assert e.value.status == swe.SWE_ESTATE


def test_sub_domains_whose_own_cells_are_all_dry():
    """The three-mound dam break starts with most of the basin dry: some
    sub-domains own no wet cell (their CFL step is +inf, the global minimum
    decides). The decomposed run still equals the whole mesh bitwise, and
    the whole mesh's mass is the sum of the parts' (ghosts excluded)."""
    pytest.importorskip("torch")
    from paper_1807_00672_gb300.partition import LocalRun
    ensure_built()
    case = inputs.three_mounds_case(80, 32)  # 5,120 cells, wet behind the dam only
    whole = swe.Mesh(case.mesh.xy, case.mesh.tri, precision="f64", tile=128)
    ref = swe.State(whole, *fields(case))
    run = LocalRun(case.mesh.xy, case.mesh.tri, fields(case), 6, precision="f64", tile=128)
    dry_parts = sum(1 for s in run.parts if np.all(case.h[s.cells[~s.ghost]] == 0.0))
    assert dry_parts >= 2
    ref.run(40)
    run.run(40)
    for a, b in zip(run.fields(), ref.fields()):
        assert np.array_equal(a, b)
    assert run.mass() == pytest.approx(ref.mass, rel=1e-13)
    run.close()


def test_many_small_sub_domains_on_one_gpu():
    """132 cells in 11 sub-domains of 12 cells (most cells of a part have a
    ghost neighbour): bitwise equal to the whole mesh, FP64 and FP32."""
    pytest.importorskip("torch")
    from paper_1807_00672_gb300.partition import LocalRun
    ensure_built()
    case = inputs.random_flow_case(nx=11, ny=6, lx=110.0, ly=60.0, seed=11)
    for prec in ("f64", "f32"):
        whole = swe.Mesh(case.mesh.xy, case.mesh.tri, precision=prec)
        ref = swe.State(whole, *fields(case))
        run = LocalRun(case.mesh.xy, case.mesh.tri, fields(case), 11, precision=prec)
        ref.run(30)
        run.run(30)
        for a, b in zip(run.fields(), ref.fields()):
            assert np.array_equal(a, b), prec
        run.close()
