"""Pins of the oracle's interface flux (HLLC + hydrostatic reconstruction + walls).

Each test checks the oracle against something other than itself: the physical
flux of Eq. 1, symmetries the exact Riemann problem has, the HLL integral
relations, Riemann-invariant constructions, or closed forms of special cases.
"""
import math

import numpy as np
import pytest

import oracle

G = oracle.G
rng = np.random.default_rng(1234)


def phys_flux(h, hu, hv, nx, ny, g=G):
    """G(U) nx + H(U) ny from Eq. 1."""
    u, v = hu / h, hv / h
    un = u * nx + v * ny
    return np.array([h * un, hu * un + 0.5 * g * h * h * nx, hv * un + 0.5 * g * h * h * ny])


def rand_state(wet=True):
    h = rng.uniform(0.1, 5.0)
    return np.array([h, h * rng.uniform(-4, 4), h * rng.uniform(-4, 4), rng.uniform(-1, 1)])


def rand_normal():
    a = rng.uniform(0, 2 * math.pi)
    return math.cos(a), math.sin(a)


def test_consistency_equal_states_give_physical_flux():
    for _ in range(300):
        s = rand_state()
        nx, ny = rand_normal()
        out = oracle.interface_flux(s, s, nx, ny)
        ref = phys_flux(s[0], s[1], s[2], nx, ny)
        scale = max(1.0, np.abs(ref).max())
        assert np.abs(out[:3] - ref).max() <= 1e-13 * scale
        # equal beds: no bed pressure beyond the rounding of (h + z) - z
        assert abs(out[3]) <= 1e-14 * scale and abs(out[4]) <= 1e-14 * scale


def test_antisymmetry_swapping_sides_and_normal():
    for _ in range(300):
        a, b = rand_state(), rand_state()
        nx, ny = rand_normal()
        f = oracle.interface_flux(a, b, nx, ny)
        r = oracle.interface_flux(b, a, -nx, -ny)
        scale = max(1.0, np.abs(f).max())
        assert np.abs(f[:3] + r[:3]).max() <= 1e-12 * scale
        assert abs(f[3] - r[4]) <= 1e-12 * scale and abs(f[4] - r[3]) <= 1e-12 * scale


def test_rotation_invariance():
    for _ in range(200):
        a, b = rand_state(), rand_state()
        nx, ny = rand_normal()
        th = rng.uniform(0, 2 * math.pi)
        c, s = math.cos(th), math.sin(th)

        def rot(st):
            return np.array([st[0], c * st[1] - s * st[2], s * st[1] + c * st[2], st[3]])

        f = oracle.interface_flux(a, b, nx, ny)
        g_ = oracle.interface_flux(rot(a), rot(b), c * nx - s * ny, s * nx + c * ny)
        fr = np.array([f[0], c * f[1] - s * f[2], s * f[1] + c * f[2]])
        scale = max(1.0, np.abs(f).max())
        assert np.abs(g_[:3] - fr).max() <= 1e-12 * scale


def _subsonic_pair():
    while True:
        hL, hR = rng.uniform(0.2, 4.0, 2)
        uL, uR = rng.uniform(-2.0, 2.0, 2)
        S = oracle.hllc_speeds(hL, uL, hR, uR)
        if S[0] < 0 < S[1]:
            return hL, uL, hR, uR, S


def test_hll_integral_relations():
    """Subsonic case: the mass flux is the HLL flux of the Riemann fan average.

    h_hll = (S_R hR - S_L hL - (qR - qL)) / (S_R - S_L) is the fan average;
    conservation over each half fan gives F = F_L + S_L (h_hll - hL)
    = F_R + S_R (h_hll - hR), and the contact speed is S* = F / h_hll.
    """
    for _ in range(300):
        hL, uL, hR, uR, S = _subsonic_pair()
        SL, SR, Ss = S
        utL, utR = rng.uniform(-1, 1, 2)
        F = oracle.hllc(hL, uL, utL, hR, uR, utR)
        qL, qR = hL * uL, hR * uR
        hh = (SR * hR - SL * hL - (qR - qL)) / (SR - SL)
        assert F[0] == pytest.approx(qL + SL * (hh - hL), rel=1e-12, abs=1e-12)
        assert F[0] == pytest.approx(qR + SR * (hh - hR), rel=1e-12, abs=1e-12)
        # normal momentum: the same relation on the momentum component
        fL1 = qL * uL + 0.5 * G * hL * hL
        fR1 = qR * uR + 0.5 * G * hR * hR
        qh = (SR * qR - SL * qL - (fR1 - fL1)) / (SR - SL)
        assert F[1] == pytest.approx(fL1 + SL * (qh - qL), rel=1e-12, abs=1e-11)
        assert Ss == pytest.approx(F[0] / hh, rel=1e-10, abs=1e-12)
        # transverse momentum is carried by the mass flux from the upwind side
        assert F[2] == pytest.approx(F[0] * (utL if Ss >= 0 else utR), rel=1e-13, abs=1e-14)


def test_supersonic_states_are_upwinded():
    # both waves to the right: flux is the left physical flux, and vice versa
    F = oracle.hllc(1.0, 10.0, 0.3, 0.8, 9.0, -0.2)
    assert np.allclose(F, [10.0, 100.0 + 0.5 * G, 3.0], rtol=1e-15)
    F = oracle.hllc(1.0, -9.0, 0.3, 0.8, -10.0, -0.2)
    assert np.allclose(F, [-8.0, 80.0 + 0.5 * G * 0.64, 1.6], rtol=1e-15)


def test_two_rarefaction_speeds_are_exact():
    """Two rarefactions: u + 2c is constant across the left wave, u - 2c across
    the right one. Build the states from a middle state; the estimated wave
    speeds must then be the exact rarefaction heads, and the middle state the
    estimate is built from must be the one chosen."""
    for _ in range(200):
        hs = rng.uniform(0.2, 2.0)
        us = rng.uniform(-1.0, 1.0)
        cs = math.sqrt(G * hs)
        cL = cs + rng.uniform(0.1, 2.0)
        cR = cs + rng.uniform(0.1, 2.0)
        uL = us + 2 * cs - 2 * cL
        uR = us - 2 * cs + 2 * cR
        hL, hR = cL * cL / G, cR * cR / G
        SL, SR, _ = oracle.hllc_speeds(hL, uL, hR, uR)
        assert SL == pytest.approx(uL - cL, rel=1e-12, abs=1e-12)
        assert SR == pytest.approx(uR + cR, rel=1e-12, abs=1e-12)


def test_shock_side_uses_two_rarefaction_middle_state():
    """Converging states: the left estimate is u* - c*, where (u*, c*) solve the
    two Riemann-invariant relations uL + 2cL = u* + 2c*, uR - 2cR = u* - 2c*."""
    for _ in range(200):
        hL, hR = rng.uniform(0.5, 3.0, 2)
        cL, cR = math.sqrt(G * hL), math.sqrt(G * hR)
        uL = rng.uniform(2.0, 5.0)
        uR = -rng.uniform(2.0, 5.0)
        us, cs = np.linalg.solve([[1.0, 2.0], [1.0, -2.0]], [uL + 2 * cL, uR - 2 * cR])
        SL, SR, _ = oracle.hllc_speeds(hL, uL, hR, uR)
        assert SL == pytest.approx(min(uL - cL, us - cs), rel=1e-12, abs=1e-12)
        assert SR == pytest.approx(max(uR + cR, us + cs), rel=1e-12, abs=1e-12)


def test_dry_bed_speeds_are_ritter_front():
    for _ in range(100):
        h = rng.uniform(0.1, 3.0)
        u = rng.uniform(-2.0, 2.0)
        c = math.sqrt(G * h)
        SL, SR, Ss = oracle.hllc_speeds(h, u, 0.0, 0.0)
        assert SL == pytest.approx(u - c, rel=1e-14, abs=1e-14)
        assert SR == pytest.approx(u + 2 * c, rel=1e-14, abs=1e-14)
        assert Ss == pytest.approx(SR, rel=1e-14)
        SL, SR, Ss = oracle.hllc_speeds(0.0, 0.0, h, u)
        assert SL == pytest.approx(u - 2 * c, rel=1e-14, abs=1e-14)
        assert SR == pytest.approx(u + c, rel=1e-14, abs=1e-14)
        assert Ss == pytest.approx(SL, rel=1e-14)


def test_both_dry_is_zero_flux():
    assert np.all(oracle.hllc(0.0, 0.0, 0.0, 0.0, 0.0, 0.0) == 0.0)


def test_wall_flux_closed_form():
    """Mirror ghost: symmetric fan S_L = -S_R, so the mass flux vanishes and the
    normal momentum flux is F(U) + S_R h un with S_R = max(c - un, c + un/2)."""
    for _ in range(200):
        h = rng.uniform(0.1, 4.0)
        u, v = rng.uniform(-3, 3, 2)
        nx, ny = rand_normal()
        s = np.array([h, h * u, h * v, rng.uniform(-1, 1)])
        out = oracle.interface_flux(s, s, nx, ny, wall=True)
        un = u * nx + v * ny
        c = math.sqrt(G * h)
        if un >= 0:
            F1 = 0.5 * G * h * h + h * un * c + 1.5 * h * un * un
        else:
            F1 = 0.5 * G * h * h + h * un * c
        assert out[0] == 0.0
        assert out[1] == pytest.approx(F1 * nx, rel=1e-12, abs=1e-12)
        assert out[2] == pytest.approx(F1 * ny, rel=1e-12, abs=1e-12)
        assert abs(out[3]) <= 1e-14 * max(1.0, 0.5 * G * h * h)  # rounding of (h + z) - z only


def test_still_water_over_a_bed_step_is_balanced():
    """Hydrostatic reconstruction: at rest with a flat free surface, the flux
    out of each side (F + P_side n) is that side's own hydrostatic thrust
    g h_side^2 / 2 n, and no mass moves, wet or partly dry."""
    for _ in range(200):
        eta = rng.uniform(0.5, 3.0)
        zL, zR = rng.uniform(-1.0, 3.5, 2)
        hL, hR = max(0.0, eta - zL), max(0.0, eta - zR)
        nx, ny = rand_normal()
        out = oracle.interface_flux([hL, 0, 0, zL], [hR, 0, 0, zR], nx, ny)
        assert abs(out[0]) <= 1e-14
        tol = 1e-13 * max(1.0, eta * eta)
        left = out[1:3] + out[3] * np.array([nx, ny])
        right = out[1:3] + out[4] * np.array([nx, ny])
        assert np.abs(left - 0.5 * G * hL * hL * np.array([nx, ny])).max() <= tol
        assert np.abs(right - 0.5 * G * hR * hR * np.array([nx, ny])).max() <= tol


def test_reconstructed_depths_never_exceed_cell_depths():
    """h* <= h per side: the bed pressure terms are never negative (beyond the
    rounding of (h + z) - z*)."""
    for _ in range(300):
        a, b = rand_state(), rand_state()
        a[3], b[3] = rng.uniform(-3, 3, 2)
        nx, ny = rand_normal()
        out = oracle.interface_flux(a, b, nx, ny)
        tol = 1e-14 * 0.5 * G * max(a[0], b[0]) ** 2
        assert out[3] >= -tol and out[4] >= -tol
