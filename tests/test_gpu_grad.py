"""Gradients through many steps (swe_grad_record / swe_grad) against the
FP64 oracle: its forward-mode derivative (dot-product test: <g, J v> from
the dual-number run must equal <J^T g, v> from the adjoint) and central
finite differences of its plain steps, both with the recorded time steps
held fixed."""
import numpy as np
import pytest

import oracle
from paper_1807_00672_gb300 import inputs, swe

from gpu_util import ensure_built
from test_oracle_tangent import smooth_wet_case

pytestmark = pytest.mark.gpu


def record(case, n_steps, K, gauges, precision="f64", tile=0):
    ensure_built()
    mesh = swe.Mesh(case.mesh.xy, case.mesh.tri, precision=precision, tile=tile)
    st = swe.State(mesh, case.h, case.hu, case.hv, case.z, case.n)
    tape = swe.Tape(st, n_steps, K, gauges)
    return mesh, st, tape


def seeds(case, n_steps, G, seed):
    rng = np.random.default_rng(seed)
    T = case.mesh.n_tris
    return dict(g_h=rng.standard_normal(T), g_hu=rng.standard_normal(T),
                g_hv=rng.standard_normal(T), g_gauge=rng.standard_normal((n_steps, G)))


def directions(case, seed, which="all"):
    rng = np.random.default_rng(seed)
    T = case.mesh.n_tris
    v = dict(h=0.1 * rng.standard_normal(T), hu=0.2 * rng.standard_normal(T),
             hv=0.2 * rng.standard_normal(T), z=0.05 * rng.standard_normal(T),
             n=0.005 * rng.standard_normal(T))
    if which != "all":
        v = {k: (a if k == which else np.zeros(T)) for k, a in v.items()}
    return v


def oracle_jvp(case, n_steps, gauges, v):
    """Directional derivative of (final h, hu, hv, gauge depths) along v,
    with the oracle's own CFL time steps held fixed."""
    dts = oracle.state_from_case(case).run(n_steps)
    s = oracle.state_from_case(case)
    t, gh, gd = s.run_tangent(dts, v["h"], v["hu"], v["hv"], v["z"], v["n"], gauges)
    return t, gd, dts


def pair(g, v, t, gd, grads):
    lhs = float(g["g_h"] @ t[0] + g["g_hu"] @ t[1] + g["g_hv"] @ t[2] + (g["g_gauge"] * gd).sum())
    rhs = float(sum(grads[k] @ v[k] for k in ("h", "hu", "hv", "z", "n")))
    return lhs, rhs


@pytest.mark.parametrize("which", ["h", "hu", "hv", "z", "n", "all"])
def test_adjoint_matches_dual_number_oracle(which):
    c = smooth_wet_case()
    N, gauges = 12, [3, 50, 101, 50]
    mesh, st, tape = record(c, N, 5, gauges)
    g = seeds(c, N, len(gauges), 1)
    grads = tape.grad(**g)
    v = directions(c, 2, which)
    t, gd, dts = oracle_jvp(c, N, gauges, v)
    lhs, rhs = pair(g, v, t, gd, grads)
    assert abs(lhs - rhs) <= 1e-10 * max(abs(lhs), 1e-300), (lhs, rhs)


def test_recorded_dts_and_gauges_match_the_oracle():
    c = smooth_wet_case()
    N, gauges = 12, [3, 50, 101]
    mesh, st, tape = record(c, N, 5, gauges)
    o = oracle.state_from_case(c)
    dts = o.run(N)
    s2 = oracle.state_from_case(c)
    gh = s2.run_dts(dts, gauges)
    assert np.abs(tape.gauge_h - gh).max() <= 1e-12 * np.abs(gh).max()
    assert st.t == pytest.approx(float(dts.sum()), rel=1e-13)


def test_adjoint_matches_central_differences():
    """L = sum of seeded outputs; (L(x + e v) - L(x - e v)) / 2e from the plain
    FP64 oracle steps with the same dt sequence against <grad L, v>: 1e-5."""
    c = smooth_wet_case(seed=4)
    N, gauges = 10, [7, 60]
    mesh, st, tape = record(c, N, 4, gauges)
    g = seeds(c, N, len(gauges), 5)
    grads = tape.grad(**g)
    dts = oracle.state_from_case(c).run(N)
    v = directions(c, 6)

    def loss(sign, eps):
        s = oracle.State(oracle.Mesh(c.mesh.xy, c.mesh.tri), c.h + sign * eps * v["h"],
                         c.hu + sign * eps * v["hu"], c.hv + sign * eps * v["hv"],
                         c.z + sign * eps * v["z"], c.n + sign * eps * v["n"])
        gh = s.run_dts(dts, gauges)
        return float(g["g_h"] @ s.h + g["g_hu"] @ s.hu + g["g_hv"] @ s.hv + (g["g_gauge"] * gh).sum())

    eps = 1e-6
    fd = (loss(+1, eps) - loss(-1, eps)) / (2 * eps)
    ad = float(sum(grads[k] @ v[k] for k in ("h", "hu", "hv", "z", "n")))
    assert abs(fd - ad) <= 1e-5 * abs(ad)


def test_checkpoint_interval_does_not_change_the_gradient():
    c = smooth_wet_case(seed=1)
    N, gauges = 13, [5, 40]
    g = seeds(c, N, len(gauges), 3)
    ref = None
    for K in (1, 4, 13, 50):
        mesh, st, tape = record(c, N, K, gauges)
        r = tape.grad(**g)
        if ref is None:
            ref = r
        else:
            for k in ref:
                assert np.array_equal(r[k], ref[k]), (K, k)


def test_wet_dry_case_matches_dual_number_oracle():
    """Moving shorelines and dry cells: the derivative follows the branches
    the forward took (the oracle and the kernels take the same ones)."""
    c = inputs.random_flow_case(nx=21, ny=13, seed=5)
    N, gauges = 8, [10, 200]
    mesh, st, tape = record(c, N, 3, gauges)
    g = seeds(c, N, len(gauges), 7)
    grads = tape.grad(**g)
    for which in ("h", "hu", "z", "n"):
        v = directions(c, 8, which)
        v = {k: np.where(c.h > 0.05, a, 0.0) for k, a in v.items()}
        t, gd, dts = oracle_jvp(c, N, gauges, v)
        lhs, rhs = pair(g, v, t, gd, grads)
        assert abs(lhs - rhs) <= 1e-9 * max(abs(lhs), abs(rhs)), (which, lhs, rhs)


@pytest.mark.parametrize("tile", [128, 512])
def test_gradient_does_not_depend_on_the_tile_size(tile):
    c = smooth_wet_case(seed=3)
    N, gauges = 6, [9]
    g = seeds(c, N, 1, 4)
    _, _, t0 = record(c, N, 3, gauges)
    _, _, t1 = record(c, N, 3, gauges, tile=tile)
    a, b = t0.grad(**g), t1.grad(**g)
    for k in a:
        assert np.abs(a[k] - b[k]).max() <= 1e-12 * np.abs(a[k]).max(), k


def test_fp32_gradient_close_to_fp64():
    c = smooth_wet_case(seed=2)
    N, gauges = 10, [3, 30]
    g = seeds(c, N, len(gauges), 9)
    _, _, t64 = record(c, N, 5, gauges, precision="f64")
    _, _, t32 = record(c, N, 5, gauges, precision="f32")
    a, b = t64.grad(**g), t32.grad(**g)
    for k in a:
        assert np.abs(a[k] - b[k]).max() <= 1e-3 * np.abs(a[k]).max(), k


def test_torch_autograd_function_matches_the_tape():
    torch = pytest.importorskip("torch")
    from paper_1807_00672_gb300 import grad as sgrad
    c = smooth_wet_case()
    ensure_built()
    mesh = swe.Mesh(c.mesh.xy, c.mesh.tri, precision="f64")
    dev = torch.device("cuda", 0)
    x = [torch.tensor(a, device=dev, requires_grad=True) for a in (c.h, c.hu, c.hv, c.z, c.n)]
    gauges = [3, 50]
    h, hu, hv, gh = sgrad.rollout(mesh, *x, n_steps=9, checkpoint_every=4, gauges=gauges)
    obs = torch.linspace(1.5, 2.5, 9, device=dev, dtype=torch.float64)
    loss = ((gh[:, 0] - obs) ** 2).sum() + 0.1 * (hu ** 2).sum()
    loss.backward()
    # same seeds through the tape directly
    st = swe.State(mesh, c.h, c.hu, c.hv, c.z, c.n)
    tape = swe.Tape(st, 9, 4, gauges)
    gg = np.zeros((9, 2))
    gg[:, 0] = 2 * (tape.gauge_h[:, 0] - obs.cpu().numpy())
    _, hu_n, _ = st.fields()
    r = tape.grad(g_hu=0.2 * hu_n, g_gauge=gg)
    for k, t in zip(("h", "hu", "hv", "z", "n"), x):
        assert np.allclose(t.grad.cpu().numpy(), r[k], rtol=1e-12, atol=1e-14 * np.abs(r[k]).max())


def test_grad_needs_the_tiled_single_scenario_mesh():
    c = smooth_wet_case()
    ensure_built()
    mesh = swe.Mesh(c.mesh.xy, c.mesh.tri, precision="f64", kernel="edge")
    st = swe.State(mesh, c.h, c.hu, c.hv, c.z, c.n)
    with pytest.raises(swe.SweError) as e:
        swe.Tape(st, 3, 2)
    assert e.value.status == swe.SWE_ESTATE
    mesh2 = swe.Mesh.ensemble([(c.mesh.xy, c.mesh.tri)] * 2, precision="f64")
    cat = lambda a: np.concatenate([a, a])
    st2 = swe.State(mesh2, cat(c.h), cat(c.hu), cat(c.hv), cat(c.z), cat(c.n))
    with pytest.raises(swe.SweError) as e:
        swe.Tape(st2, 3, 2)
    assert e.value.status == swe.SWE_ESTATE


def test_grad_edge_cases():
    """One step, no gauges, interval longer than the run, no seeds."""
    c = smooth_wet_case(seed=6)
    mesh, st, tape = record(c, 1, 1, None)
    assert tape.gauge_h.shape == (1, 0)
    g = seeds(c, 1, 0, 2)
    r = tape.grad(g_h=g["g_h"], g_hu=g["g_hu"], g_hv=g["g_hv"])
    v = directions(c, 3)
    t, gd, _ = oracle_jvp(c, 1, [], v)
    lhs = float(g["g_h"] @ t[0] + g["g_hu"] @ t[1] + g["g_hv"] @ t[2])
    rhs = float(sum(r[k] @ v[k] for k in ("h", "hu", "hv", "z", "n")))
    assert abs(lhs - rhs) <= 1e-10 * abs(lhs)
    zero = tape.grad()
    for k, a in zero.items():
        assert np.all(a == 0.0), k
    _, _, t2 = record(c, 3, 10, [4])  # K > N: one segment
    assert t2.info()["checkpoint_every"] == 3
    r2 = t2.grad(g_gauge=np.ones((3, 1)))
    assert np.isfinite(r2["n"]).all() and np.abs(r2["h"]).max() > 0


def test_grad_rejects_bad_arguments():
    c = smooth_wet_case()
    ensure_built()
    mesh = swe.Mesh(c.mesh.xy, c.mesh.tri, precision="f64")
    st = swe.State(mesh, c.h, c.hu, c.hv, c.z, c.n)
    for n, k, gauges in ((0, 1, None), (3, 0, None), (3, 1, [mesh.T]), (3, 1, [-1])):
        with pytest.raises(swe.SweError) as e:
            swe.Tape(st, n, k, gauges)
        assert e.value.status == swe.SWE_EINVAL


# ------------------------------------------------- multi-tile, multi-chunk scale

def large_cases():
    """307,200 cells each (1,200 tiles of 256 cells, more than the adjoint
    launch has resident blocks, so every block walks several tiles and most
    faces between tiles are halo faces): a smooth fully wet case and the
    random wet/dry case."""
    return {"wet": smooth_wet_case(nx=400, ny=384, seed=11),
            "wetdry": inputs.random_flow_case(nx=400, ny=384, lx=4_000.0, ly=3_840.0, seed=13)}


@pytest.mark.parametrize("name", ["wet", "wetdry"])
def test_adjoint_matches_dual_number_oracle_on_many_tiles(name):
    """The dot-product test at 307,200 cells, 20 steps, checkpoints every 7
    steps (segments of 7, 7 and 6 steps), default 256-cell FP64 tiles: the
    tile walk of each block, the halo lists between tiles, the registers
    loaded one tile ahead and the early copies before the launch's
    dependency wait all take part. Each input direction alone and all at
    once; 1e-10 relative (wet/dry: 1e-9)."""
    c = large_cases()[name]
    N, K = 20, 7
    rng = np.random.default_rng(17)
    gauges = sorted(rng.choice(c.mesh.n_tris, size=16, replace=False).tolist())
    mesh, st, tape = record(c, N, K, gauges, tile=256)
    assert tape.info()["checkpoint_every"] == K
    g = seeds(c, N, len(gauges), 19)
    grads = tape.grad(**g)
    tol = 1e-10 if name == "wet" else 1e-9
    for which in ("h", "hu", "hv", "z", "n", "all"):
        v = directions(c, 23, which)
        if name == "wetdry":
            v = {k: np.where(c.h > 0.05, a, 0.0) for k, a in v.items()}
        t, gd, dts = oracle_jvp(c, N, gauges, v)
        lhs, rhs = pair(g, v, t, gd, grads)
        assert abs(lhs - rhs) <= tol * max(abs(lhs), abs(rhs)), (name, which, lhs, rhs)


def test_adjoint_matches_central_differences_on_many_tiles():
    """Central differences of the plain FP64 oracle steps at 307,200 cells
    along a smooth direction, against the GPU gradient: 1e-5 relative. The
    direction is smooth in space: a per-cell random one makes the perturbed
    runs cross kinks of the flux (the min/max of the wave-speed estimates,
    the upwind side of the transverse momentum) at a few of the 9 million
    face evaluations, where a difference quotient differs from the
    piecewise derivative by about 1e-5 whatever the step size."""
    c = large_cases()["wet"]
    N, K = 20, 7
    gauges = [1_000, 150_000, 300_000]
    mesh, st, tape = record(c, N, K, gauges, tile=256)
    g = seeds(c, N, len(gauges), 29)
    grads = tape.grad(**g)
    dts = oracle.state_from_case(c).run(N)
    cen = inputs.centroids(c.mesh)
    x, y = cen[:, 0] / c.mesh.lx, cen[:, 1] / c.mesh.ly
    v = dict(h=0.1 * np.sin(5 * x + 1) * np.cos(3 * y), hu=0.2 * np.cos(4 * x) * np.sin(2 * y + 0.5),
             hv=0.2 * np.sin(3 * x + 2 * y), z=0.05 * np.cos(6 * x - y),
             n=0.005 * np.sin(2 * x + 3 * y))

    def loss(sign, eps):
        s = oracle.State(oracle.Mesh(c.mesh.xy, c.mesh.tri), c.h + sign * eps * v["h"],
                         c.hu + sign * eps * v["hu"], c.hv + sign * eps * v["hv"],
                         c.z + sign * eps * v["z"], c.n + sign * eps * v["n"])
        gh = s.run_dts(dts, gauges)
        return float(g["g_h"] @ s.h + g["g_hu"] @ s.hu + g["g_hv"] @ s.hv + (g["g_gauge"] * gh).sum())

    eps = 1e-6
    fd = (loss(+1, eps) - loss(-1, eps)) / (2 * eps)
    ad = float(sum(grads[k] @ v[k] for k in ("h", "hu", "hv", "z", "n")))
    assert abs(fd - ad) <= 1e-5 * abs(ad), (fd, ad)


def test_fp32_calibration_gradient_when_misfits_exceed_fp32_resolution():
    """The calibration loss (squared gauge misfits, observations from a run
    with a perturbed Manning n) on a reduced calibration mesh: 40,000 fully
    wet cells, 64 gauges, 100 steps, checkpoints every 10. The FP32 gauge
    depths differ from the FP64 ones by about 1e-6 m after the run, so the
    gradient is only as good as the misfits are large against that: with
    observations offset by 5 cm the FP32 gradient matches the FP64 one to
    1e-4 (max norm, relative). The FP32 adjoint itself, seeded with the FP64
    run's residuals, matches to 2e-5 whatever the misfits (its own rounding;
    the FP32 forward's depth error is what limits tiny misfits)."""
    case = inputs.humps_case(nx=200, ny=100, lx=2_000.0, ly=1_000.0, fully_wet=True)
    gauges = inputs.gauge_cells(case, 64, seed=5, radius=300.0)
    n_obs = inputs.perturbed_manning(case, seed=5)
    N, K = 100, 10
    ensure_built()
    res = {}
    for prec in ("f64", "f32"):
        mesh = swe.Mesh(case.mesh.xy, case.mesh.tri, precision=prec, tile=256)
        o = swe.State(mesh, case.h, case.hu, case.hv, case.z, n_obs)
        obs = swe.Tape(o, N, K, gauges).gauge_h.copy() + 0.05
        st = swe.State(mesh, case.h, case.hu, case.hv, case.z, case.n)
        tape = swe.Tape(st, N, K, gauges)
        resid = tape.gauge_h - obs
        res[prec] = dict(mesh=mesh, st=st, tape=tape, resid=resid, grad=tape.grad(g_gauge=2 * resid))
    assert np.abs(res["f32"]["resid"] - res["f64"]["resid"]).max() <= 1e-5
    seeded = res["f32"]["tape"].grad(g_gauge=2 * res["f64"]["resid"])
    for k in ("n", "z", "h"):
        ref = res["f64"]["grad"][k]
        den = np.abs(ref).max()
        assert np.abs(res["f32"]["grad"][k] - ref).max() <= 1e-4 * den, k
        assert np.abs(seeded[k] - ref).max() <= 2e-5 * den, k
