"""FP64 CPU oracle for the HLLC shallow-water step (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package; the CUDA library never does. The arithmetic lives
in ``swe_oracle.cpp``; this module is ctypes marshalling.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

_lib = None

G = 9.81
COURANT = 0.7
H_EPS = 1e-6


class _Params(ctypes.Structure):
    _fields_ = [("g", ctypes.c_double), ("courant", ctypes.c_double), ("h_eps", ctypes.c_double)]


def params(g: float = G, courant: float = COURANT, h_eps: float = H_EPS) -> _Params:
    return _Params(g, courant, h_eps)


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        vp, i64, dbl, i32p = ctypes.c_void_p, ctypes.c_int64, ctypes.c_double, ctypes.c_void_p
        pp = ctypes.POINTER(_Params)
        L.oracle_mesh_new.restype = vp
        L.oracle_mesh_new.argtypes = [vp, i64, vp, i64, ctypes.POINTER(ctypes.c_int)]
        L.oracle_mesh_free.argtypes = [vp]
        L.oracle_mesh_counts.argtypes = [vp, vp]
        L.oracle_mesh_cells.argtypes = [vp, vp, vp, vp, vp]
        L.oracle_mesh_edges.argtypes = [vp, vp, vp, vp, vp, vp]
        L.oracle_hllc.argtypes = [dbl] * 7 + [vp]
        L.oracle_hllc_speeds.argtypes = [dbl] * 5 + [vp]
        L.oracle_interface_flux.argtypes = [vp, vp, dbl, dbl, ctypes.c_int, pp, vp]
        L.oracle_edge_fluxes.argtypes = [vp, pp, vp, vp, vp, vp, vp]
        L.oracle_cfl_dt.argtypes = [vp, pp, vp, vp, vp, vp]
        L.oracle_cfl_dt.restype = ctypes.c_int
        L.oracle_mass.argtypes = [vp, vp]
        L.oracle_mass.restype = dbl
        L.oracle_step.argtypes = [vp, pp, dbl, vp, vp, vp, vp, vp]
        L.oracle_step.restype = i64
        L.oracle_run.argtypes = [vp, pp, i64, vp, vp, vp, vp, vp, vp, vp]
        L.oracle_run.restype = ctypes.c_int
        L.oracle_advance.argtypes = [vp, pp, dbl, i64, vp, vp, vp, vp, vp, vp, vp, vp]
        L.oracle_advance.restype = ctypes.c_int
        L.oracle_cells_after_step.argtypes = [vp, pp, dbl, vp, vp, vp, vp, vp, vp, i64, vp]
        L.oracle_run_tangent.argtypes = [vp, pp, i64, vp] + [vp] * 5 + [vp] * 5 + [vp, i64, vp, vp]
        L.oracle_run_tangent.restype = i64
        L.oracle_run_dts.argtypes = [vp, pp, i64, vp] + [vp] * 5 + [vp, i64, vp]
        L.oracle_run_dts.restype = i64
        L.oracle_set_threads.argtypes = [ctypes.c_int]
        _lib = L
    return _lib


def set_threads(n: int) -> None:
    """Host threads of the FP64 edge and cell loops (1: serial, the default).
    The results do not depend on it."""
    lib().oracle_set_threads(int(n))


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


class OracleError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: oracle status {status}")
        self.status = status


E_INVAL, E_MESH, E_DRY = -1, -2, -8


class Mesh:
    """Oracle-side mesh: edges, normals, lengths, areas built from (xy, tri)."""

    def __init__(self, xy: np.ndarray, tri: np.ndarray):
        L = lib()
        self._xy = _f64(xy).reshape(-1, 2)
        self._tri = np.ascontiguousarray(tri, dtype=np.int32).reshape(-1, 3)
        st = ctypes.c_int(0)
        self._h = L.oracle_mesh_new(_p(self._xy), self._xy.shape[0], _p(self._tri),
                                    self._tri.shape[0], ctypes.byref(st))
        if not self._h:
            raise OracleError(st.value, "mesh")
        c = np.zeros(4, dtype=np.int64)
        L.oracle_mesh_counts(self._h, _p(c))
        self.V, self.T, self.E, self.Eb = (int(x) for x in c)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.oracle_mesh_free(h)
            self._h = None

    def cells(self):
        area = np.zeros(self.T)
        perim = np.zeros(self.T)
        tri = np.zeros((self.T, 3), dtype=np.int32)
        ce = np.zeros((self.T, 3), dtype=np.int32)
        lib().oracle_mesh_cells(self._h, _p(area), _p(perim), _p(tri), _p(ce))
        return dict(area=area, perim=perim, tri=tri, cell_edge=ce)

    def edges(self):
        L_ = np.zeros(self.E, dtype=np.int32)
        R_ = np.zeros(self.E, dtype=np.int32)
        nx = np.zeros(self.E)
        ny = np.zeros(self.E)
        ln = np.zeros(self.E)
        lib().oracle_mesh_edges(self._h, _p(L_), _p(R_), _p(nx), _p(ny), _p(ln))
        return dict(L=L_, R=R_, nx=nx, ny=ny, len=ln)


class State:
    """Mutable FP64 state (h, hu, hv) plus static z, n, stepped by the oracle."""

    def __init__(self, mesh: Mesh, h, hu, hv, z, n, prm=None):
        self.mesh = mesh
        self.h = _f64(h).copy()
        self.hu = _f64(hu).copy()
        self.hv = _f64(hv).copy()
        self.z = _f64(z).copy()
        self.n = _f64(n).copy()
        self.t = 0.0
        self.neg = 0
        self.prm = prm if prm is not None else params()

    def cfl_dt(self) -> float:
        dt = ctypes.c_double(0.0)
        st = lib().oracle_cfl_dt(self.mesh._h, ctypes.byref(self.prm), _p(self.h), _p(self.hu),
                                 _p(self.hv), ctypes.byref(dt))
        if st != 0:
            raise OracleError(st, "cfl_dt")
        return dt.value

    def step(self, dt: float) -> int:
        neg = lib().oracle_step(self.mesh._h, ctypes.byref(self.prm), dt, _p(self.h),
                                _p(self.hu), _p(self.hv), _p(self.z), _p(self.n))
        self.neg += int(neg)
        self.t += dt
        return int(neg)

    def run(self, n_steps: int) -> np.ndarray:
        dts = np.zeros(n_steps)
        neg = ctypes.c_int64(0)
        st = lib().oracle_run(self.mesh._h, ctypes.byref(self.prm), n_steps, _p(self.h),
                              _p(self.hu), _p(self.hv), _p(self.z), _p(self.n), _p(dts),
                              ctypes.byref(neg))
        self.neg += neg.value
        if st != 0:
            raise OracleError(st, "run")
        self.t += float(dts.sum())
        return dts

    def advance(self, t_end: float, max_steps: int = 10_000_000) -> int:
        t = ctypes.c_double(self.t)
        k = ctypes.c_int64(0)
        neg = ctypes.c_int64(0)
        st = lib().oracle_advance(self.mesh._h, ctypes.byref(self.prm), t_end, max_steps,
                                  _p(self.h), _p(self.hu), _p(self.hv), _p(self.z), _p(self.n),
                                  ctypes.byref(t), ctypes.byref(k), ctypes.byref(neg))
        self.t = t.value
        self.neg += neg.value
        if st != 0:
            raise OracleError(st, "advance")
        return k.value

    def mass(self) -> float:
        return float(lib().oracle_mass(self.mesh._h, _p(self.h)))

    def edge_fluxes(self) -> np.ndarray:
        out = np.zeros((5, self.mesh.E))
        lib().oracle_edge_fluxes(self.mesh._h, ctypes.byref(self.prm), _p(self.h), _p(self.hu),
                                 _p(self.hv), _p(self.z), _p(out))
        return out

    def cells_after_step(self, dt: float, cells) -> np.ndarray:
        cells = np.ascontiguousarray(cells, dtype=np.int64)
        out = np.zeros((3, cells.shape[0]))
        lib().oracle_cells_after_step(self.mesh._h, ctypes.byref(self.prm), dt, _p(self.h),
                                      _p(self.hu), _p(self.hv), _p(self.z), _p(self.n),
                                      _p(cells), cells.shape[0], _p(out))
        return out


    def run_dts(self, dts, gauges=None):
        """Steps with the prescribed time steps dts (state advanced in place).
        Returns the gauge depths [len(dts), len(gauges)] after each step."""
        dts = _f64(dts)
        g = np.ascontiguousarray(gauges if gauges is not None else [], dtype=np.int32)
        gh = np.zeros((dts.shape[0], g.shape[0]))
        neg = lib().oracle_run_dts(self.mesh._h, ctypes.byref(self.prm), dts.shape[0], _p(dts),
                                   _p(self.h), _p(self.hu), _p(self.hv), _p(self.z), _p(self.n),
                                   _p(g), g.shape[0], _p(gh))
        self.neg += int(neg)
        self.t += float(dts.sum())
        return gh

    def run_tangent(self, dts, dh, dhu, dhv, dz=None, dn=None, gauges=None):
        """Forward-mode derivative of run_dts along the direction (dh, dhu,
        dhv, dz, dn). Advances the state; returns (tangent of (h, hu, hv) at
        the end, gauge depths, gauge tangents)."""
        dts = _f64(dts)
        t = [_f64(a).copy() for a in (dh, dhu, dhv)]
        dz = None if dz is None else _f64(dz)
        dn = None if dn is None else _f64(dn)
        g = np.ascontiguousarray(gauges if gauges is not None else [], dtype=np.int32)
        gh = np.zeros((dts.shape[0], g.shape[0]))
        gd = np.zeros((dts.shape[0], g.shape[0]))
        neg = lib().oracle_run_tangent(
            self.mesh._h, ctypes.byref(self.prm), dts.shape[0], _p(dts), _p(self.h), _p(self.hu),
            _p(self.hv), _p(self.z), _p(self.n), _p(t[0]), _p(t[1]), _p(t[2]),
            None if dz is None else _p(dz), None if dn is None else _p(dn), _p(g), g.shape[0],
            _p(gh), _p(gd))
        self.neg += int(neg)
        self.t += float(dts.sum())
        return t, gh, gd


def hllc(hL, unL, utL, hR, unR, utR, g=G) -> np.ndarray:
    F = np.zeros(3)
    lib().oracle_hllc(hL, unL, utL, hR, unR, utR, g, _p(F))
    return F


def hllc_speeds(hL, unL, hR, unR, g=G) -> np.ndarray:
    S = np.zeros(3)
    lib().oracle_hllc_speeds(hL, unL, hR, unR, g, _p(S))
    return S


def interface_flux(sL, sR, nx, ny, wall=False, prm=None) -> np.ndarray:
    """(F_h, F_hu, F_hv, PL, PR) for states (h, hu, hv, z) on each side."""
    a = _f64(sL)
    b = _f64(sR)
    out = np.zeros(5)
    prm = prm if prm is not None else params()
    lib().oracle_interface_flux(_p(a), _p(b), nx, ny, int(wall), ctypes.byref(prm), _p(out))
    return out


def state_from_case(case, prm=None) -> State:
    m = Mesh(case.mesh.xy, case.mesh.tri)
    return State(m, case.h, case.hu, case.hv, case.z, case.n, prm)
