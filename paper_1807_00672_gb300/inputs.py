"""Seeded synthetic inputs: triangle meshes and initial fields.

This module is the only code that the CUDA path and the FP64 CPU oracle share.
It draws meshes and fields; it holds none of the method's arithmetic (no
areas, normals, fluxes, updates or time steps). Both sides receive the arrays
it returns, in the caller's cell order, and build everything else themselves.

The workloads stand in for the paper's own test grids (Table 2: 1,036 to
10,261,932 triangles) and its dam-break / water-drop cases (Sec. 2.3, Sec. 3),
whose mesh files and parameters the paper does not give.

Every array is float64 (coordinates, fields) or int32 (triangles), C-contiguous.
Triangles are listed counter-clockwise.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Mesh",
    "Case",
    "jittered_grid",
    "centroids",
    "stoker_case",
    "ritter_case",
    "humps_case",
    "sinusoid_case",
    "lake_at_rest_case",
    "uniform_flow_case",
    "random_flow_case",
    "ensemble_cases",
    "water_drop_case",
    "three_mounds_case",
    "gauge_cells",
    "perturbed_manning",
    "CONFIGS",
    "make_config",
]


@dataclass
class Mesh:
    xy: np.ndarray  # (V, 2) float64 node coordinates
    tri: np.ndarray  # (T, 3) int32 node ids, counter-clockwise
    lx: float = 0.0
    ly: float = 0.0
    nx: int = 0
    ny: int = 0

    @property
    def n_nodes(self) -> int:
        return int(self.xy.shape[0])

    @property
    def n_tris(self) -> int:
        return int(self.tri.shape[0])


@dataclass
class Case:
    """A mesh plus an initial state, all in the caller's cell order."""

    mesh: Mesh
    h: np.ndarray
    hu: np.ndarray
    hv: np.ndarray
    z: np.ndarray
    n: np.ndarray  # per-cell Manning coefficient
    name: str = ""
    meta: dict = field(default_factory=dict)


def jittered_grid(nx: int, ny: int, lx: float, ly: float, *, jitter: float = 0.0,
                  diagonal: str = "random", seed: int = 0) -> Mesh:
    """Triangulate an nx x ny grid of quads over [0,lx] x [0,ly].

    Interior nodes move by U(-jitter, +jitter) cell widths in x and y (the
    boundary stays a rectangle). Each quad is cut along one diagonal:
    ``"random"`` picks it by a seeded coin, ``"shorter"`` takes the shorter
    diagonal of the (jittered) quad, ties broken by the coin, ``"ac"`` cuts
    every quad from its lower-left to its upper-right node.
    Counts: V = (nx+1)(ny+1), T = 2 nx ny.
    """
    if nx < 1 or ny < 1:
        raise ValueError("grid needs at least one quad")
    rng = np.random.default_rng(seed)
    dx = lx / nx
    dy = ly / ny
    xs = np.arange(nx + 1, dtype=np.float64) * dx
    ys = np.arange(ny + 1, dtype=np.float64) * dy
    xs[-1] = lx
    ys[-1] = ly
    X, Y = np.meshgrid(xs, ys, indexing="xy")  # (ny+1, nx+1)
    if jitter > 0.0 and nx > 1 and ny > 1:
        jx = rng.uniform(-jitter, jitter, size=(ny - 1, nx - 1)) * dx
        jy = rng.uniform(-jitter, jitter, size=(ny - 1, nx - 1)) * dy
        X[1:-1, 1:-1] += jx
        Y[1:-1, 1:-1] += jy
    xy = np.stack([X.ravel(), Y.ravel()], axis=1)

    j, i = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    a = (j * (nx + 1) + i).ravel()
    b = a + 1
    c = a + (nx + 1) + 1
    d = a + (nx + 1)
    coin = rng.integers(0, 2, size=a.shape[0]).astype(bool)
    if diagonal == "random":
        use_ac = coin
    elif diagonal == "ac":  # every quad cut the same way: point-symmetric about the centre
        use_ac = np.ones(a.shape[0], dtype=bool)
    elif diagonal == "shorter":
        lac = np.sum((xy[a] - xy[c]) ** 2, axis=1)
        lbd = np.sum((xy[b] - xy[d]) ** 2, axis=1)
        use_ac = np.where(lac == lbd, coin, lac < lbd)
    else:
        raise ValueError(f"unknown diagonal rule {diagonal!r}")
    t1 = np.where(use_ac[:, None], np.stack([a, b, c], 1), np.stack([a, b, d], 1))
    t2 = np.where(use_ac[:, None], np.stack([a, c, d], 1), np.stack([b, c, d], 1))
    tri = np.empty((2 * a.shape[0], 3), dtype=np.int32)
    tri[0::2] = t1
    tri[1::2] = t2
    return Mesh(xy=np.ascontiguousarray(xy), tri=tri, lx=lx, ly=ly, nx=nx, ny=ny)


def centroids(mesh: Mesh) -> np.ndarray:
    """Mean of each triangle's three nodes, (T, 2). Used only to place fields."""
    return mesh.xy[mesh.tri].mean(axis=1)


def _zeros(t: int) -> np.ndarray:
    return np.zeros(t, dtype=np.float64)


def stoker_case(nx: int = 50, ny: int = 25, *, lx: float = 100.0, ly: float = 50.0,
                h_left: float = 10.0, h_right: float = 1.0, x_dam: float = 50.0,
                seed: int = 1) -> Case:
    """1D dam break on a triangulated strip: flat bed, no friction, walls.

    Default: 100 m x 50 m, 50 x 25 squares cut along seeded random diagonals
    (2,500 triangles), h = 10 m for x < 50 m and 1 m elsewhere, at rest.
    """
    m = jittered_grid(nx, ny, lx, ly, jitter=0.0, diagonal="random", seed=seed)
    c = centroids(m)
    t = m.n_tris
    h = np.where(c[:, 0] < x_dam, h_left, h_right).astype(np.float64)
    return Case(m, h, _zeros(t), _zeros(t), _zeros(t), _zeros(t), name="stoker",
                meta=dict(h_left=h_left, h_right=h_right, x_dam=x_dam, seed=seed))


def ritter_case(nx: int = 100, ny: int = 4, *, lx: float = 100.0, ly: float = 4.0,
                h_left: float = 1.0, x_dam: float = 50.0, seed: int = 11) -> Case:
    """Dam break onto a dry flat bed (h = 0 downstream), no friction, walls."""
    m = jittered_grid(nx, ny, lx, ly, jitter=0.0, diagonal="random", seed=seed)
    c = centroids(m)
    t = m.n_tris
    h = np.where(c[:, 0] < x_dam, h_left, 0.0).astype(np.float64)
    return Case(m, h, _zeros(t), _zeros(t), _zeros(t), _zeros(t), name="ritter",
                meta=dict(h_left=h_left, x_dam=x_dam, seed=seed))


def _gaussian_humps(c: np.ndarray, rng, k: int, lx: float, ly: float,
                    amp=(0.5, 2.0), sigma=(300.0, 800.0)) -> np.ndarray:
    z = np.zeros(c.shape[0])
    for _ in range(k):
        a = rng.uniform(*amp)
        s = rng.uniform(*sigma)
        x0 = rng.uniform(0.0, lx)
        y0 = rng.uniform(0.0, ly)
        r2 = (c[:, 0] - x0) ** 2 + (c[:, 1] - y0) ** 2
        z += a * np.exp(-r2 / (2.0 * s * s))
    return z


def humps_case(nx: int = 1000, ny: int = 500, *, lx: float = 10_000.0, ly: float = 5_000.0,
               eta0: float = 2.0, bump: float = 1.0, bump_size: float = 1_000.0,
               manning: float = 0.03, jitter: float = 0.3, seed: int = 2,
               fully_wet: bool = False, dry_top: float = 0.3) -> Case:
    """Jittered grid, bed = 3 Gaussian humps (0.5-2 m, sigma 300-800 m).

    Free surface eta0 with +bump inside a bump_size square at the domain
    centre; h = max(0, eta - z). The bed is shifted vertically so that its
    highest point lies dry_top above eta0, so the highest hump starts with a
    dry top and wet/dry fronts are present. ``fully_wet`` instead leaves the
    bed and raises the surface to max(z) + 1 m (+bump), which gives h >= 1 m
    everywhere. Sizes scale the hump widths with the domain.
    """
    m = jittered_grid(nx, ny, lx, ly, jitter=jitter, diagonal="shorter", seed=seed)
    rng = np.random.default_rng(seed + 1000)
    c = centroids(m)
    scale = lx / 10_000.0
    z = _gaussian_humps(c, rng, 3, lx, ly, sigma=(300.0 * scale, 800.0 * scale))
    if not fully_wet:
        z += (eta0 + dry_top) - float(z.max())
    base = (float(z.max()) + 1.0) if fully_wet else eta0
    inside = (np.abs(c[:, 0] - lx / 2) <= bump_size * scale / 2) & (
        np.abs(c[:, 1] - ly / 2) <= bump_size * scale / 2)
    eta = base + np.where(inside, bump, 0.0)
    h = np.maximum(0.0, eta - z)
    t = m.n_tris
    return Case(m, h, _zeros(t), _zeros(t), z, np.full(t, manning), name="humps",
                meta=dict(seed=seed, eta0=base, bump=bump, manning=manning))


def sinusoid_case(nx: int = 3163, ny: int = 1581, *, lx: float = 100_000.0, ly: float = 50_000.0,
                  n_waves: int = 8, amp_max: float = 3.0, wavelength=(2_000.0, 50_000.0),
                  r_dam: float = 5_000.0, h_in: float = 5.0, h_out: float = 1.0,
                  manning=(0.02, 0.05), jitter: float = 0.3, seed: int = 3) -> Case:
    """Radial dam break over a bed of random sinusoids, per-cell Manning n.

    Bed z = sum of n_waves plane waves with random direction, wavelength and
    phase; weights w_k ~ U[0,1] scaled so the summed amplitude is amp_max,
    i.e. |z| <= amp_max. Depth h = h_in within r_dam of the centre, else h_out;
    n ~ U[manning] per cell; at rest. Wavelengths scale with the domain.
    """
    m = jittered_grid(nx, ny, lx, ly, jitter=jitter, diagonal="shorter", seed=seed)
    rng = np.random.default_rng(seed + 1000)
    c = centroids(m)
    scale = lx / 100_000.0
    w = rng.uniform(0.0, 1.0, size=n_waves)
    w = amp_max * w / w.sum()
    z = np.zeros(c.shape[0])
    for k in range(n_waves):
        lam = rng.uniform(*wavelength) * scale
        th = rng.uniform(0.0, 2.0 * math.pi)
        ph = rng.uniform(0.0, 2.0 * math.pi)
        kx = 2.0 * math.pi / lam * math.cos(th)
        ky = 2.0 * math.pi / lam * math.sin(th)
        z += w[k] * np.sin(kx * c[:, 0] + ky * c[:, 1] + ph)
    r = np.hypot(c[:, 0] - lx / 2, c[:, 1] - ly / 2)
    h = np.where(r < r_dam * scale, h_in, h_out).astype(np.float64)
    n = rng.uniform(*manning, size=m.n_tris)
    t = m.n_tris
    return Case(m, h, _zeros(t), _zeros(t), z, n, name="sinusoid",
                meta=dict(seed=seed, n_waves=n_waves, amp_max=amp_max))


def lake_at_rest_case(nx: int = 40, ny: int = 20, *, lx: float = 400.0, ly: float = 200.0,
                      eta: float = 1.0, jitter: float = 0.3, seed: int = 5,
                      manning: float = 0.03) -> Case:
    """Still water over a bumpy bed with dry islands: eta = const, u = v = 0.

    The bed mixes Gaussian bumps (some poking above eta, so dry islands) with
    a random per-cell jitter so that neighbouring beds always differ.
    """
    m = jittered_grid(nx, ny, lx, ly, jitter=jitter, diagonal="shorter", seed=seed)
    rng = np.random.default_rng(seed + 1000)
    c = centroids(m)
    z = _gaussian_humps(c, rng, 4, lx, ly, amp=(0.6, 1.8), sigma=(0.05 * lx, 0.12 * lx))
    z += rng.uniform(-0.05, 0.05, size=z.shape[0])
    h = np.maximum(0.0, eta - z)
    t = m.n_tris
    return Case(m, h, _zeros(t), _zeros(t), z, np.full(t, manning), name="lake",
                meta=dict(eta=eta, seed=seed))


def uniform_flow_case(nx: int = 60, ny: int = 30, *, lx: float = 600.0, ly: float = 300.0,
                      h0: float = 2.0, u0: float = 1.5, v0: float = -0.7,
                      manning: float = 0.05, seed: int = 7) -> Case:
    """Uniform depth and velocity on a flat bed with friction (walls around)."""
    m = jittered_grid(nx, ny, lx, ly, jitter=0.0, diagonal="random", seed=seed)
    t = m.n_tris
    h = np.full(t, h0)
    return Case(m, h, h * u0, h * v0, _zeros(t), np.full(t, manning), name="uniform",
                meta=dict(h0=h0, u0=u0, v0=v0, manning=manning))


def random_flow_case(nx: int = 24, ny: int = 16, *, lx: float = 240.0, ly: float = 160.0,
                     jitter: float = 0.3, seed: int = 9, dry_fraction: float = 0.2,
                     manning=(0.0, 0.05)) -> Case:
    """Random wet/dry state with random velocities over a random bed.

    About dry_fraction of the cells start dry (h = 0); the others get
    h ~ U[0.2, 3] m and velocities ~ U[-2, 2] m/s; bed ~ U[-0.5, 0.5] m.
    Exercises every branch of the flux (dry sides, supercritical states).
    """
    m = jittered_grid(nx, ny, lx, ly, jitter=jitter, diagonal="shorter", seed=seed)
    rng = np.random.default_rng(seed + 1000)
    t = m.n_tris
    h = rng.uniform(0.2, 3.0, size=t)
    h[rng.uniform(size=t) < dry_fraction] = 0.0
    u = rng.uniform(-2.0, 2.0, size=t)
    v = rng.uniform(-2.0, 2.0, size=t)
    z = rng.uniform(-0.5, 0.5, size=t)
    n = rng.uniform(*manning, size=t)
    return Case(m, h, h * u, h * v, z, n, name="random", meta=dict(seed=seed))


def ensemble_cases(n_scen: int = 256, *, t_min: int = 5_000, t_max: int = 500_000,
                   cell: float = 10.0, seed: int = 4) -> list[Case]:
    """Independent dam-break scenarios on jittered grids of log-uniform size.

    Triangle counts are log-uniform in [t_min, t_max] (rounded to a 2:1 grid,
    10 m cells), flat bed, dam at mid-x with H ~ U[2, 10] m upstream and 1 m
    downstream, n ~ U[0.01, 0.05].
    """
    rng = np.random.default_rng(seed)
    out = []
    for s in range(n_scen):
        t_target = math.exp(rng.uniform(math.log(t_min), math.log(t_max)))
        ny = max(1, int(round(math.sqrt(t_target / 4.0))))
        nx = 2 * ny
        m = jittered_grid(nx, ny, nx * cell, ny * cell, jitter=0.3, diagonal="shorter",
                          seed=seed * 100_003 + s)
        c = centroids(m)
        hh = rng.uniform(2.0, 10.0)
        nn = rng.uniform(0.01, 0.05)
        t = m.n_tris
        h = np.where(c[:, 0] < nx * cell / 2, hh, 1.0).astype(np.float64)
        out.append(Case(m, h, _zeros(t), _zeros(t), _zeros(t), np.full(t, nn),
                        name=f"ensemble{s}", meta=dict(H=hh, n=nn)))
    return out


# Quads per side of the water-drop meshes whose 2 n^2 triangles approximate
# the paper's test grids 1-5 (Table 2: 1,036 to 10,261,932 triangles).
WATER_DROP_N = {1: 23, 2: 71, 3: 229, 4: 727, 5: 2265}


def water_drop_case(n: int = 71, *, l: float = 10_000.0, h0: float = 10.0, amp: float = 1.0,
                    sigma: float = 500.0, jitter: float = 0.15, diagonal: str = "shorter",
                    manning: float = 0.0, seed: int = 21) -> Case:
    """The paper's water drop (Sec. 3): water at rest in a square basin closed
    by walls, with a Gaussian hump of the free surface at the centre; the
    paper runs it to T_s = 2,400 s. Its parameters are not printed; these are
    project choices: a 10 km square, 10 m deep, a 1 m hump of width sigma =
    500 m, flat bed, no friction, an n x n jittered grid (T = 2 n^2; see
    WATER_DROP_N for the Table 2 sizes)."""
    m = jittered_grid(n, n, l, l, jitter=jitter, diagonal=diagonal, seed=seed)
    c = centroids(m)
    r2 = (c[:, 0] - 0.5 * l) ** 2 + (c[:, 1] - 0.5 * l) ** 2
    h = h0 + amp * np.exp(-r2 / (2.0 * sigma * sigma))
    t = m.n_tris
    return Case(m, h, _zeros(t), _zeros(t), _zeros(t), np.full(t, manning), name="water_drop",
                meta=dict(n=n, l=l, h0=h0, amp=amp, sigma=sigma, seed=seed))


# Three conical mounds (x, y, height, base radius) of the three-mound case.
THREE_MOUNDS = ((32.0, 8.0, 1.2, 9.0), (32.0, 24.0, 1.2, 9.0), (52.0, 16.0, 2.8, 11.0))


def three_mounds_case(nx: int = 160, ny: int = 64, *, lx: float = 80.0, ly: float = 32.0,
                      x_dam: float = 18.0, h_up: float = 2.0, mounds=THREE_MOUNDS,
                      manning: float = 0.02, jitter: float = 0.3, seed: int = 31) -> Case:
    """A dam break over three mounds onto a dry bed, with wetting and drying
    (the paper's three-mound case, Sec. 2.3 and Fig. 4, whose parameters it
    does not print; these are project choices): an 80 m x 32 m basin closed
    by walls, still water 2 m deep behind a dam at x = 18 m, a dry bed beyond
    it carrying two 1.2 m cones and one 2.8 m cone, Manning n = 0.02."""
    m = jittered_grid(nx, ny, lx, ly, jitter=jitter, diagonal="shorter", seed=seed)
    c = centroids(m)
    z = np.zeros(m.n_tris)
    for (mx, my, height, radius) in mounds:
        d = np.hypot(c[:, 0] - mx, c[:, 1] - my)
        z = np.maximum(z, height * np.maximum(0.0, 1.0 - d / radius))
    h = np.where(c[:, 0] < x_dam, np.maximum(0.0, h_up - z), 0.0)
    t = m.n_tris
    return Case(m, h, _zeros(t), _zeros(t), z, np.full(t, manning), name="three_mounds",
                meta=dict(x_dam=x_dam, h_up=h_up, manning=manning, seed=seed))


def gauge_cells(case: Case, count: int = 64, seed: int = 5, radius: float | None = None) -> np.ndarray:
    """Gauge cells sampled without replacement (seeded), from the cells whose
    centroid lies within ``radius`` of the domain centre if given (so that
    the gauges see the flow within the run)."""
    rng = np.random.default_rng(seed)
    pool = np.arange(case.mesh.n_tris)
    if radius is not None:
        c = centroids(case.mesh)
        lx, ly = case.mesh.lx, case.mesh.ly
        pool = pool[np.hypot(c[:, 0] - 0.5 * lx, c[:, 1] - 0.5 * ly) <= radius]
    return np.sort(rng.choice(pool, size=count, replace=False)).astype(np.int32)


def perturbed_manning(case: Case, rel: float = 0.1, seed: int = 5) -> np.ndarray:
    """Target roughness of the calibration workload: n (1 + rel xi), xi ~ N(0, 1)."""
    rng = np.random.default_rng(seed + 17)
    return case.n * (1.0 + rel * rng.standard_normal(case.mesh.n_tris))


# The five workloads the benchmark and the parity tests are built on.
CONFIGS = {
    "stoker_2500": dict(fn=stoker_case, kw={}, steps=None, t_end=2.0, prec="f64"),
    "humps_1m": dict(fn=humps_case, kw={}, steps=500, t_end=None, prec="f64+f32"),
    "sinusoid_10m": dict(fn=sinusoid_case, kw={}, steps=1000, t_end=None, prec="f32"),
    "ensemble_256": dict(fn=ensemble_cases, kw={}, steps=200, t_end=None, prec="f32"),
    "calibration_1m": dict(fn=humps_case, kw=dict(fully_wet=True), steps=500, t_end=None,
                           prec="f32"),
}


def make_config(name: str, **overrides):
    spec = CONFIGS[name]
    kw = dict(spec["kw"])
    kw.update(overrides)
    return spec["fn"](**kw)
