"""The oracle's forward-mode derivative (oracle_run_tangent), pinned to things
other than itself: central finite differences of the plain FP64 steps, the
closed-form derivatives of the friction decay, the lake at rest (a direction
that keeps the water still must keep it still), and linearity.

Every run holds the time-step sequence fixed (it is recorded once and passed
in), as the gradient of the solver does.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1807_00672_gb300 import inputs


def smooth_wet_case(nx=12, ny=8, seed=0):
    """Fully wet, smooth state over a smooth bed: no wet/dry switch and no
    shock within a few steps, so the step is differentiable and finite
    differences converge."""
    m = inputs.jittered_grid(nx, ny, 10.0 * nx, 10.0 * ny, jitter=0.25, seed=seed)
    c = inputs.centroids(m)
    x, y = c[:, 0] / (10.0 * nx), c[:, 1] / (10.0 * ny)
    z = 0.4 * np.sin(2.1 * x + 0.3) * np.cos(1.7 * y)
    h = 2.0 + 0.3 * np.sin(3.0 * x + 1.1 * y) - z
    hu = h * (0.4 * np.cos(2.0 * y) + 0.1)
    hv = h * (0.3 * np.sin(2.5 * x) - 0.05)
    n = 0.02 + 0.01 * x
    return inputs.Case(m, h, hu, hv, z, n, name="smooth_wet")


def directions(case, seed):
    rng = np.random.default_rng(seed)
    T = case.mesh.n_tris
    return [rng.standard_normal(T) * s for s in (0.1, 0.2, 0.2, 0.05, 0.005)]


def run_plain(case, dts, h, hu, hv, z, n, gauges):
    s = oracle.State(oracle.Mesh(case.mesh.xy, case.mesh.tri), h, hu, hv, z, n)
    gh = s.run_dts(dts, gauges)
    return np.concatenate([s.h, s.hu, s.hv, gh.ravel()])


@pytest.mark.parametrize("which", ["h", "hu", "hv", "z", "n", "all"])
def test_tangent_matches_central_differences(which):
    c = smooth_wet_case()
    dts = oracle.state_from_case(c).run(6)
    gauges = [3, 50, 101]
    d = directions(c, 7)
    names = ["h", "hu", "hv", "z", "n"]
    v = [di if (which == "all" or which == nm) else np.zeros_like(di) for di, nm in zip(d, names)]
    s = oracle.state_from_case(c)
    t, gh, gd = s.run_tangent(dts, v[0], v[1], v[2], v[3], v[4], gauges)
    jv = np.concatenate([t[0], t[1], t[2], gd.ravel()])
    base = [c.h, c.hu, c.hv, c.z, c.n]
    eps = 1e-6
    plus = run_plain(c, dts, *[b + eps * vi for b, vi in zip(base, v)], gauges)
    minus = run_plain(c, dts, *[b - eps * vi for b, vi in zip(base, v)], gauges)
    fd = (plus - minus) / (2 * eps)
    scale = np.abs(jv).max()
    assert scale > 0
    assert np.abs(fd - jv).max() <= 1e-6 * scale


def test_friction_decay_derivatives_closed_form():
    """Uniform flow on a flat bed: 1/|q_N| = 1/|q_0| + g n^2 t / h^{7/3}
    (t = sum of dt). Differentiating the closed form: d|q_N|/dn =
    -2 g n t h^{-7/3} |q_N|^2, d|q_N|/d|q_0| = |q_N|^2 / |q_0|^2, and
    d|q_N|/dh = (7/3) g n^2 t h^{-10/3} |q_N|^2 for a uniform change of h."""
    c = inputs.uniform_flow_case()
    N = 8
    dts = oracle.state_from_case(c).run(N)
    t = float(dts.sum())
    g, h, n = 9.81, 2.0, 0.05
    q0 = math.hypot(c.hu[0], c.hv[0])
    qN = 1.0 / (1.0 / q0 + g * n * n * t / h ** (7.0 / 3.0))
    cen = inputs.centroids(c.mesh)
    far = (cen[:, 0] > 10 * N + 20) & (cen[:, 0] < 600 - 10 * N - 20) & \
          (cen[:, 1] > 10 * N + 20) & (cen[:, 1] < 300 - 10 * N - 20)
    assert far.sum() > 100
    T = c.mesh.n_tris
    zero, one = np.zeros(T), np.ones(T)
    ux, uy = c.hu[0] / q0, c.hv[0] / q0

    def dq(tan):  # derivative of |q| along the flow direction
        return tan[1][far] * ux + tan[2][far] * uy

    tn, _, _ = oracle.state_from_case(c).run_tangent(dts, zero, zero, zero, zero, one)
    assert np.abs(dq(tn) - (-2 * g * n * t * h ** (-7.0 / 3.0) * qN ** 2)).max() <= 1e-10 * qN
    tq, _, _ = oracle.state_from_case(c).run_tangent(dts, zero, one * ux, one * uy, zero, zero)
    assert np.abs(dq(tq) - qN ** 2 / q0 ** 2).max() <= 1e-10
    th, _, _ = oracle.state_from_case(c).run_tangent(dts, one, zero, zero, zero, zero)
    assert np.abs(dq(th) - (7.0 / 3.0) * g * n * n * t * h ** (-10.0 / 3.0) * qN ** 2).max() \
        <= 1e-10 * qN
    assert np.abs(th[0][far] - 1.0).max() <= 1e-12  # depth tangent is carried unchanged


def test_lake_at_rest_direction_keeps_the_water_still():
    """Raising the bed of wet cells by dz and lowering their depth by the
    same amount is another lake at rest, so the tangent of the state after
    any number of steps is exactly (-dz, 0, 0)."""
    c = inputs.lake_at_rest_case()
    dts = oracle.state_from_case(c).run(10)
    rng = np.random.default_rng(3)
    wet = c.h > 0.05
    dz = np.where(wet, rng.standard_normal(c.mesh.n_tris), 0.0)
    zero = np.zeros(c.mesh.n_tris)
    t, _, _ = oracle.state_from_case(c).run_tangent(dts, -dz, zero, zero, dz, zero)
    assert np.abs(t[0] + dz).max() <= 1e-12
    assert np.abs(t[1]).max() <= 1e-11 and np.abs(t[2]).max() <= 1e-11


def test_tangent_is_linear_in_the_direction():
    c = smooth_wet_case(seed=2)
    dts = oracle.state_from_case(c).run(4)
    a, b = directions(c, 1), directions(c, 2)
    ta, _, _ = oracle.state_from_case(c).run_tangent(dts, *a)
    tb, _, _ = oracle.state_from_case(c).run_tangent(dts, *b)
    tab, _, _ = oracle.state_from_case(c).run_tangent(dts, *[2.0 * x - 3.0 * y for x, y in zip(a, b)])
    for k in range(3):
        ref = 2.0 * ta[k] - 3.0 * tb[k]
        assert np.abs(tab[k] - ref).max() <= 1e-12 * np.abs(ref).max()


def test_tangent_run_values_equal_the_plain_run():
    c = smooth_wet_case()
    dts = oracle.state_from_case(c).run(5)
    s1 = oracle.state_from_case(c)
    s1.run_tangent(dts, *directions(c, 4))
    s2 = oracle.state_from_case(c)
    s2.run_dts(dts)
    for a, b in ((s1.h, s2.h), (s1.hu, s2.hu), (s1.hv, s2.hv)):
        assert np.array_equal(a, b)
