"""Closed-form solutions the oracle and the CUDA path are checked against.

Independent of both implementations: textbook results, written from their
definitions.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.optimize import brentq

G = 9.81


def stoker_middle(h_l: float, h_r: float, g: float = G):
    """Middle depth, velocity and shock speed of the wet-bed dam break.

    Left rarefaction (Riemann invariant u + 2c constant) meets a right shock
    (Rankine-Hugoniot): 2(c_l - c_m) = (h_m - h_r) sqrt(g/2 (1/h_m + 1/h_r)).
    """
    c_l = math.sqrt(g * h_l)

    def f(hm):
        return 2.0 * (c_l - math.sqrt(g * hm)) - (hm - h_r) * math.sqrt(0.5 * g * (1.0 / hm + 1.0 / h_r))

    h_m = brentq(f, h_r, h_l, xtol=1e-15, rtol=1e-15)
    u_m = 2.0 * (c_l - math.sqrt(g * h_m))
    s = h_m * u_m / (h_m - h_r)
    return h_m, u_m, s


def stoker_depth(x, t: float, h_l: float, h_r: float, x0: float, g: float = G):
    h_m, u_m, s = stoker_middle(h_l, h_r, g)
    c_l = math.sqrt(g * h_l)
    c_m = math.sqrt(g * h_m)
    xi = (np.asarray(x) - x0) / t
    fan = (2.0 * c_l - xi) ** 2 / (9.0 * g)
    return np.where(xi < -c_l, h_l, np.where(xi < u_m - c_m, fan, np.where(xi < s, h_m, h_r)))


def ritter_depth(x, t: float, h0: float, x0: float, g: float = G):
    """Dam break onto a dry bed: h = (2 c0 - xi)^2 / (9 g) on -c0 <= xi <= 2 c0."""
    c0 = math.sqrt(g * h0)
    xi = (np.asarray(x) - x0) / t
    return np.where(xi < -c0, h0, np.where(xi < 2.0 * c0, (2.0 * c0 - xi) ** 2 / (9.0 * g), 0.0))


def friction_decay(q0: float, h: float, n: float, t: float, g: float = G) -> float:
    """|q(t)| of dq/dt = -g n^2 |q| q / h^{7/3} at fixed h: 1/|q| grows linearly."""
    return 1.0 / (1.0 / q0 + g * n * n * t / h ** (7.0 / 3.0))
