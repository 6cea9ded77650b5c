"""ctypes binding of libswe.so (the C ABI declared in include/swe.h).

Argument marshalling only: every step of the method runs in the library's
CUDA kernels. The library must have been built (``build.build()``); if it is
missing, ``lib()`` raises instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libswe.so")

SWE_OK = 0
SWE_EINVAL = -1
SWE_EMESH = -2
SWE_ENOMEM = -3
SWE_ECUDA = -4
SWE_ENAN = -5
SWE_ETIMEOUT = -7
SWE_EDRY = -8
SWE_ESTATE = -9

PRECISION = {"f64": 0, "f32": 1}
ORDER = {"none": 0, "morton": 1, "rcm": 2}
KERNEL = {"auto": 0, "edge": 1, "tiled": 2}

# Every symbol include/swe.h declares.
EXPORTS = (
    "swe_params_default", "swe_mesh_create", "swe_mesh_create_batch", "swe_mesh_counts",
    "swe_mesh_scenarios", "swe_mesh_device_bytes", "swe_mesh_destroy", "swe_state_init",
    "swe_state_set", "swe_step", "swe_run", "swe_advance", "swe_sync", "swe_copy_out",
    "swe_state_info", "swe_next_dt", "swe_scenario_info", "swe_state_destroy", "swe_strerror",
    "swe_last_cuda_error", "swe_step_edges_static", "swe_grad_record", "swe_grad",
    "swe_tape_info", "swe_tape_destroy", "swe_fp64_fma_rate", "swe_state_init_device",
    "swe_state_set_device", "swe_copy_out_device", "swe_grad_device", "swe_tape_gauges_device",
    "swe_partition_create", "swe_partition_sizes", "swe_partition_local_mesh",
    "swe_partition_exchange", "swe_partition_destroy", "swe_mesh_create_part",
    "swe_state_halo_pack", "swe_state_halo_unpack", "swe_state_dt_device",
    "swe_state_set_dt_min_device", "swe_state_set_f32", "swe_copy_out_f32", "swe_cell_order",
)


class Params(ctypes.Structure):
    _fields_ = [
        ("g", ctypes.c_double),
        ("courant", ctypes.c_double),
        ("h_eps", ctypes.c_double),
        ("precision", ctypes.c_int32),
        ("order", ctypes.c_int32),
        ("kernel", ctypes.c_int32),
        ("tile", ctypes.c_int32),
        ("stages", ctypes.c_int32),
        ("cells_per_thread", ctypes.c_int32),
        ("halo_schedule", ctypes.c_int32),
        ("wait_rounds", ctypes.c_int32),
        ("compensated_depth", ctypes.c_int32),
    ]


class SweError(RuntimeError):
    def __init__(self, status: int, what: str):
        msg = lib().swe_strerror(status).decode()
        extra = lib().swe_last_cuda_error().decode() if status == SWE_ECUDA else ""
        super().__init__(f"{what}: {msg} ({status}){' - ' + extra if extra else ''}")
        self.status = status


_lib = None


def lib():
    """Loads libswe.so once. Raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                           "`python -m paper_1807_00672_gb300.build` (needs nvcc)")
    L = ctypes.CDLL(LIB_PATH)
    vp, i64, dbl, st = ctypes.c_void_p, ctypes.c_int64, ctypes.c_double, ctypes.c_int
    P = ctypes.POINTER(Params)
    pp = ctypes.POINTER(ctypes.c_void_p)
    sig = {
        "swe_params_default": (None, [P]),
        "swe_mesh_create": (st, [vp, i64, vp, i64, P, vp, pp]),
        "swe_mesh_create_batch": (st, [ctypes.c_int32, vp, vp, vp, vp, P, vp, pp]),
        "swe_mesh_counts": (st, [vp, vp]),
        "swe_mesh_scenarios": (st, [vp, vp, vp]),
        "swe_mesh_device_bytes": (st, [vp, vp]),
        "swe_mesh_destroy": (None, [vp]),
        "swe_state_init": (st, [vp, vp, vp, vp, vp, vp, dbl, pp]),
        "swe_state_set": (st, [vp, vp, vp, vp]),
        "swe_step": (st, [vp, vp]),
        "swe_run": (st, [vp, i64]),
        "swe_advance": (st, [vp, dbl, vp]),
        "swe_sync": (st, [vp]),
        "swe_copy_out": (st, [vp, vp, vp, vp, vp, vp]),
        "swe_state_set_f32": (st, [vp, vp, vp, vp]),
        "swe_cell_order": (st, [vp, i64, vp, i64, ctypes.c_int32, vp]),
        "swe_copy_out_f32": (st, [vp, vp, vp, vp, vp, vp]),
        "swe_state_info": (st, [vp, vp]),
        "swe_next_dt": (st, [vp, vp]),
        "swe_scenario_info": (st, [vp, ctypes.c_int32, vp, vp, vp, vp]),
        "swe_state_destroy": (None, [vp]),
        "swe_strerror": (ctypes.c_char_p, [st]),
        "swe_last_cuda_error": (ctypes.c_char_p, []),
        "swe_grad_record": (st, [vp, i64, i64, vp, ctypes.c_int32, vp, pp]),
        "swe_grad": (st, [vp] + [vp] * 9),
        "swe_tape_info": (st, [vp, vp]),
        "swe_tape_destroy": (None, [vp]),
        "swe_step_edges_static": (st, [i64, i64] + [vp] * 13 + [dbl] * 4 + [vp] * 3
                                  + [vp, vp, vp]),
        "swe_fp64_fma_rate": (st, [vp, vp]),
        "swe_state_init_device": (st, [vp, vp, vp, vp, vp, vp, dbl, vp, pp]),
        "swe_state_set_device": (st, [vp, vp, vp, vp, vp]),
        "swe_copy_out_device": (st, [vp, vp, vp, vp, vp, vp, vp]),
        "swe_grad_device": (st, [vp] + [vp] * 9 + [vp]),
        "swe_tape_gauges_device": (st, [vp, vp, vp]),
        "swe_partition_create": (st, [vp, i64, vp, i64, ctypes.c_int32, pp]),
        "swe_partition_sizes": (st, [vp, ctypes.c_int32, vp]),
        "swe_partition_local_mesh": (st, [vp, ctypes.c_int32, vp, vp, vp, vp, vp]),
        "swe_partition_exchange": (st, [vp, ctypes.c_int32, ctypes.c_int32, vp, vp, vp]),
        "swe_partition_destroy": (None, [vp]),
        "swe_mesh_create_part": (st, [vp, i64, vp, i64, vp, P, vp, pp]),
        "swe_state_halo_pack": (st, [vp, vp, i64, vp]),
        "swe_state_halo_unpack": (st, [vp, vp, i64, vp]),
        "swe_state_dt_device": (st, [vp, vp]),
        "swe_state_set_dt_min_device": (st, [vp, vp, ctypes.c_int32]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _vp(addr):
    """A device address or stream handle (int, or None) as a void pointer."""
    return None if addr is None else ctypes.c_void_p(int(addr))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _f32(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float32)


def _check(status: int, what: str):
    if status != SWE_OK:
        raise SweError(status, what)


def params(precision="f64", order="morton", kernel="auto", tile=0, g=9.81, courant=0.7,
           h_eps=1e-6, stages=0, cells_per_thread=0, halo_schedule=0, wait_rounds=0,
           compensated_depth=False) -> Params:
    p = Params()
    lib().swe_params_default(ctypes.byref(p))
    p.g, p.courant, p.h_eps = g, courant, h_eps
    p.precision = PRECISION[precision]
    p.order = ORDER[order]
    p.kernel = KERNEL[kernel]
    p.tile = tile
    p.stages = stages
    p.cells_per_thread = cells_per_thread
    p.halo_schedule = halo_schedule
    p.wait_rounds = wait_rounds
    p.compensated_depth = int(compensated_depth)
    return p


def cell_order(xy, tri, order="morton") -> np.ndarray:
    """swe_cell_order (host only): perm[j] = caller index of the cell at
    internal position j under `order` ("none", "morton" or "rcm")."""
    xy = np.ascontiguousarray(xy, dtype=np.float64).reshape(-1, 2)
    tri = np.ascontiguousarray(tri, dtype=np.int32).reshape(-1, 3)
    perm = np.empty(tri.shape[0], dtype=np.int32)
    _check(lib().swe_cell_order(_p(xy), xy.shape[0], _p(tri), tri.shape[0], ORDER[order], _p(perm)),
           "swe_cell_order")
    return perm


class Mesh:
    """Device-resident mesh (swe_mesh_create), or an ensemble of independent
    scenario meshes (``Mesh.ensemble``, swe_mesh_create_batch)."""

    def __init__(self, xy, tri, *, precision="f64", order="morton", kernel="auto", tile=0,
                 stages=0, cells_per_thread=0, stream=None, g=9.81, courant=0.7, h_eps=1e-6,
                 halo_schedule=0, wait_rounds=0, compensated_depth=False):
        self._build([(xy, tri)], precision, order, kernel, tile, stages, cells_per_thread,
                    stream, g, courant, h_eps, batch=False, halo_schedule=halo_schedule,
                    wait_rounds=wait_rounds, compensated_depth=compensated_depth)

    @classmethod
    def ensemble(cls, meshes, *, precision="f64", order="morton", kernel="auto", tile=0,
                 stages=0, cells_per_thread=0, stream=None, g=9.81, courant=0.7, h_eps=1e-6,
                 halo_schedule=0, compensated_depth=False):
        """One mesh holding the scenarios ``meshes`` = [(xy, tri), ...]; cell
        arrays are the scenarios' cells concatenated in this order."""
        self = cls.__new__(cls)
        self._build(list(meshes), precision, order, kernel, tile, stages, cells_per_thread,
                    stream, g, courant, h_eps, batch=True, halo_schedule=halo_schedule,
                    compensated_depth=compensated_depth)
        return self

    def _build(self, meshes, precision, order, kernel, tile, stages, cpt, stream, g, courant,
               h_eps, batch, halo_schedule=0, wait_rounds=0, compensated_depth=False):
        xys = [_f64(xy).reshape(-1, 2) for xy, _ in meshes]
        tris = [np.ascontiguousarray(t, dtype=np.int32).reshape(-1, 3) for _, t in meshes]
        self.prm = params(precision, order, kernel, tile, g, courant, h_eps, stages, cpt,
                          halo_schedule, wait_rounds, compensated_depth)
        self.precision = precision
        h = ctypes.c_void_p()
        if batch:
            n = len(meshes)
            xp = (ctypes.c_void_p * n)(*[a.ctypes.data for a in xys])
            tp = (ctypes.c_void_p * n)(*[a.ctypes.data for a in tris])
            nn = np.array([a.shape[0] for a in xys], dtype=np.int64)
            nt = np.array([a.shape[0] for a in tris], dtype=np.int64)
            s = lib().swe_mesh_create_batch(n, xp, _p(nn), tp, _p(nt), ctypes.byref(self.prm),
                                            stream, ctypes.byref(h))
            _check(s, "swe_mesh_create_batch")
        else:
            xy, tri = xys[0], tris[0]
            s = lib().swe_mesh_create(_p(xy), xy.shape[0], _p(tri), tri.shape[0],
                                      ctypes.byref(self.prm), stream, ctypes.byref(h))
            _check(s, "swe_mesh_create")
        self._h = h
        c = np.zeros(4, dtype=np.int64)
        lib().swe_mesh_counts(self._h, _p(c))
        self.V, self.T, self.E, self.Eb = (int(x) for x in c)
        ns = ctypes.c_int32()
        _check(lib().swe_mesh_scenarios(self._h, ctypes.byref(ns), None), "swe_mesh_scenarios")
        counts = np.zeros(ns.value, dtype=np.int64)
        _check(lib().swe_mesh_scenarios(self._h, ctypes.byref(ns), _p(counts)),
               "swe_mesh_scenarios")
        self.scenario_cells = [int(x) for x in counts]
        self.scenario_offsets = [0] + list(np.cumsum(counts)[:-1].astype(int))

    @classmethod
    def part(cls, xy, tri, ghost, *, precision="f64", order="morton", tile=0, stages=0,
             cells_per_thread=0, stream=None, g=9.81, courant=0.7, h_eps=1e-6):
        """A sub-domain's local mesh with ghost cells (swe_mesh_create_part);
        ghost: one flag per triangle, nonzero for a ghost."""
        self = cls.__new__(cls)
        xy = _f64(xy).reshape(-1, 2)
        tri = np.ascontiguousarray(tri, dtype=np.int32).reshape(-1, 3)
        gh = np.ascontiguousarray(ghost, dtype=np.uint8).reshape(-1)
        if gh.shape[0] != tri.shape[0]:
            raise ValueError("one ghost flag per triangle")
        self.prm = params(precision, order, "tiled", tile, g, courant, h_eps, stages,
                          cells_per_thread)
        self.precision = precision
        h = ctypes.c_void_p()
        _check(lib().swe_mesh_create_part(_p(xy), xy.shape[0], _p(tri), tri.shape[0], _p(gh),
                                          ctypes.byref(self.prm), stream, ctypes.byref(h)),
               "swe_mesh_create_part")
        self._h = h
        c = np.zeros(4, dtype=np.int64)
        lib().swe_mesh_counts(self._h, _p(c))
        self.V, self.T, self.E, self.Eb = (int(x) for x in c)
        self.scenario_cells = [self.T]
        self.scenario_offsets = [0]
        return self

    @property
    def n_scenarios(self) -> int:
        return len(self.scenario_cells)

    def device_bytes(self) -> int:
        b = ctypes.c_int64()
        _check(lib().swe_mesh_device_bytes(self._h, ctypes.byref(b)), "swe_mesh_device_bytes")
        return b.value

    def close(self):
        if getattr(self, "_h", None):
            lib().swe_mesh_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class State:
    """Device-resident state on a Mesh (swe_state_init and friends)."""

    def __init__(self, mesh: Mesh, h, hu, hv, z, n=None, manning_const: float = 0.0):
        self.mesh = mesh
        h, hu, hv, z = (_f64(a) for a in (h, hu, hv, z))
        for a in (h, hu, hv, z):
            if a.shape != (mesh.T,):
                raise ValueError("cell arrays must have one value per triangle")
        nn = None if n is None else _f64(n)
        hdl = ctypes.c_void_p()
        s = lib().swe_state_init(mesh._h, _p(h), _p(hu), _p(hv), _p(z),
                                 None if nn is None else _p(nn), float(manning_const),
                                 ctypes.byref(hdl))
        _check(s, "swe_state_init")
        self._h = hdl

    @classmethod
    def from_device(cls, mesh: Mesh, h, hu, hv, z, n=None, manning_const: float = 0.0,
                    stream=None):
        """swe_state_init_device: h, hu, hv, z, n are device addresses (ints)
        of mesh.T contiguous float64 values each in caller order (n may be
        None); stream: the CUDA stream handle (int) they were written on."""
        self = cls.__new__(cls)
        self.mesh = mesh
        hdl = ctypes.c_void_p()
        s = lib().swe_state_init_device(mesh._h, _vp(h), _vp(hu), _vp(hv), _vp(z), _vp(n),
                                        float(manning_const), _vp(stream), ctypes.byref(hdl))
        _check(s, "swe_state_init_device")
        self._h = hdl
        return self

    def set(self, h, hu, hv):
        h, hu, hv = (_f64(a) for a in (h, hu, hv))
        _check(lib().swe_state_set(self._h, _p(h), _p(hu), _p(hv)), "swe_state_set")

    def set_f32(self, h, hu, hv):
        """swe_state_set_f32 from float32 arrays (page-locked ones, e.g.
        views of pinned torch tensors, are read directly by the device)."""
        h, hu, hv = (_f32(a) for a in (h, hu, hv))
        _check(lib().swe_state_set_f32(self._h, _p(h), _p(hu), _p(hv)), "swe_state_set_f32")

    def set_device(self, h, hu, hv, stream=None):
        """swe_state_set_device: device addresses (ints) of float64 arrays."""
        _check(lib().swe_state_set_device(self._h, _vp(h), _vp(hu), _vp(hv), _vp(stream)),
               "swe_state_set_device")

    def halo_pack(self, cells, n, buf):
        """swe_state_halo_pack: device addresses (ints) of n int32 local cell
        ids and of a 3 n float64 buffer."""
        _check(lib().swe_state_halo_pack(self._h, _vp(cells), int(n), _vp(buf)),
               "swe_state_halo_pack")

    def halo_unpack(self, cells, n, buf):
        """swe_state_halo_unpack (device addresses as for halo_pack)."""
        _check(lib().swe_state_halo_unpack(self._h, _vp(cells), int(n), _vp(buf)),
               "swe_state_halo_unpack")

    def dt_device(self, dst):
        """swe_state_dt_device: the current CFL dt into a device double."""
        _check(lib().swe_state_dt_device(self._h, _vp(dst)), "swe_state_dt_device")

    def set_dt_min_device(self, dts, n):
        """swe_state_set_dt_min_device: next dt = min of n device doubles."""
        _check(lib().swe_state_set_dt_min_device(self._h, _vp(dts), int(n)),
               "swe_state_set_dt_min_device")

    def copy_out_device(self, h=None, hu=None, hv=None, stream=None):
        """swe_copy_out_device into device addresses (ints, any may be None);
        returns (t, mass)."""
        t = ctypes.c_double()
        m = ctypes.c_double()
        _check(lib().swe_copy_out_device(self._h, _vp(h), _vp(hu), _vp(hv), ctypes.byref(t),
                                         ctypes.byref(m), _vp(stream)), "swe_copy_out_device")
        return t.value, m.value

    def step(self) -> float:
        dt = ctypes.c_double()
        _check(lib().swe_step(self._h, ctypes.byref(dt)), "swe_step")
        return dt.value

    def run(self, n_steps: int, sync: bool = True):
        _check(lib().swe_run(self._h, int(n_steps)), "swe_run")
        if sync:
            self.sync()

    def advance(self, t_end: float) -> int:
        k = ctypes.c_int64()
        _check(lib().swe_advance(self._h, float(t_end), ctypes.byref(k)), "swe_advance")
        return k.value

    def sync(self):
        _check(lib().swe_sync(self._h), "swe_sync")

    def copy_out(self, h=None, hu=None, hv=None):
        """Fills the given float64 arrays (any may be None); returns (t, mass)."""
        t = ctypes.c_double()
        m = ctypes.c_double()
        args = [None if a is None else _p(a) for a in (h, hu, hv)]
        _check(lib().swe_copy_out(self._h, *args, ctypes.byref(t), ctypes.byref(m)), "swe_copy_out")
        return t.value, m.value

    def copy_out_f32(self, h=None, hu=None, hv=None):
        """swe_copy_out_f32 into the given float32 arrays (any may be None);
        returns (t, mass)."""
        for a in (h, hu, hv):
            if a is not None and (a.dtype != np.float32 or not a.flags["C_CONTIGUOUS"]):
                raise TypeError("copy_out_f32 needs contiguous float32 arrays")
        t = ctypes.c_double()
        m = ctypes.c_double()
        args = [None if a is None else _p(a) for a in (h, hu, hv)]
        _check(lib().swe_copy_out_f32(self._h, *args, ctypes.byref(t), ctypes.byref(m)),
               "swe_copy_out_f32")
        return t.value, m.value

    def fields(self):
        T = self.mesh.T
        h, hu, hv = np.empty(T), np.empty(T), np.empty(T)
        self.copy_out(h, hu, hv)
        return h, hu, hv

    @property
    def t(self) -> float:
        return self.copy_out()[0]

    @property
    def mass(self) -> float:
        return self.copy_out()[1]

    def info(self):
        a = np.zeros(3, dtype=np.int64)
        _check(lib().swe_state_info(self._h, _p(a)), "swe_state_info")
        return dict(steps=int(a[0]), neg=int(a[1]), err=int(a[2]))

    def next_dt(self) -> float:
        dt = ctypes.c_double()
        _check(lib().swe_next_dt(self._h, ctypes.byref(dt)), "swe_next_dt")
        return dt.value

    def scenario(self, i: int):
        """(t, mass, steps, next dt) of scenario i of an ensemble."""
        t, m, dt = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        k = ctypes.c_int64()
        _check(lib().swe_scenario_info(self._h, int(i), ctypes.byref(t), ctypes.byref(m),
                                       ctypes.byref(k), ctypes.byref(dt)), "swe_scenario_info")
        return dict(t=t.value, mass=m.value, steps=k.value, dt=dt.value)

    def close(self):
        if getattr(self, "_h", None):
            lib().swe_state_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Tape:
    """Steps recorded for gradients (swe_grad_record): advances ``state`` by
    ``n_steps`` CFL steps, keeping every dt, the depths at ``gauges`` (caller
    cell indices) after every step, and checkpoints every
    ``checkpoint_every`` steps. ``gauge_h`` is [n_steps, len(gauges)]."""

    def __init__(self, state: State, n_steps: int, checkpoint_every: int = 50, gauges=None,
                 host_gauges: bool = True):
        g = np.ascontiguousarray(gauges if gauges is not None else [], dtype=np.int32).reshape(-1)
        self.gauges = g
        self.n_steps = int(n_steps)
        # host_gauges=False: the gauge depths stay on the device (gauges_device)
        self.gauge_h = np.zeros((self.n_steps, g.shape[0])) if host_gauges else None
        self.mesh = state.mesh
        h = ctypes.c_void_p()
        s = lib().swe_grad_record(state._h, self.n_steps, int(checkpoint_every),
                                  _p(g) if g.size else None, g.shape[0],
                                  _p(self.gauge_h) if (g.size and host_gauges) else None,
                                  ctypes.byref(h))
        _check(s, "swe_grad_record")
        self._h = h

    def grad(self, g_h=None, g_hu=None, g_hv=None, g_gauge=None):
        """Gradient of a loss given by dL/d(final h, hu, hv) and dL/d gauge_h.
        Returns dict(h, hu, hv, z, n) of dL/d(initial h, hu, hv), dL/dz, dL/dn."""
        T = self.mesh.T
        seeds = [None if a is None else _f64(a).reshape(T) for a in (g_h, g_hu, g_hv)]
        gg = None
        if g_gauge is not None and self.gauges.size:
            gg = _f64(g_gauge).reshape(self.n_steps, self.gauges.shape[0])
        out = {k: np.empty(T) for k in ("h", "hu", "hv", "z", "n")}
        s = lib().swe_grad(self._h, *[None if a is None else _p(a) for a in seeds],
                           None if gg is None else _p(gg),
                           *[_p(out[k]) for k in ("h", "hu", "hv", "z", "n")])
        _check(s, "swe_grad")
        return out

    def grad_device(self, seeds, outs, stream=None):
        """swe_grad_device: seeds = (g_h, g_hu, g_hv, g_gauge), outs = (h, hu,
        hv, z, n), device addresses (ints) or None each."""
        s = lib().swe_grad_device(self._h, *[_vp(a) for a in seeds], *[_vp(a) for a in outs],
                                  _vp(stream))
        _check(s, "swe_grad_device")

    def gauges_device(self, dst, stream=None):
        """swe_tape_gauges_device: the recorded gauge depths into a device
        address (int) of n_steps * len(gauges) float64 values."""
        _check(lib().swe_tape_gauges_device(self._h, _vp(dst), _vp(stream)),
               "swe_tape_gauges_device")

    def info(self):
        a = np.zeros(5)
        _check(lib().swe_tape_info(self._h, _p(a)), "swe_tape_info")
        return dict(steps=int(a[0]), checkpoint_every=int(a[1]), record_ms=float(a[2]),
                    grad_ms=float(a[3]), bytes=int(a[4]))

    def close(self):
        if getattr(self, "_h", None):
            lib().swe_tape_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def fp64_fma_rate(stream=None) -> float:
    """Measured FP64 fused multiply-add throughput of the current device in
    TFLOP/s (swe_fp64_fma_rate)."""
    r = ctypes.c_double()
    _check(lib().swe_fp64_fma_rate(stream, ctypes.byref(r)), "swe_fp64_fma_rate")
    return r.value


class Partition:
    """swe_partition: the mesh (xy, tri) cut into n_parts sub-domains, each a
    local mesh of its own cells plus one ring of ghost cells, and the halo
    exchange lists between them."""

    def __init__(self, xy, tri, n_parts: int):
        self.xy = _f64(xy).reshape(-1, 2)
        t = np.ascontiguousarray(tri, dtype=np.int32).reshape(-1, 3)
        h = ctypes.c_void_p()
        _check(lib().swe_partition_create(_p(self.xy), self.xy.shape[0], _p(t), t.shape[0],
                                          int(n_parts), ctypes.byref(h)), "swe_partition_create")
        self._h = h
        self.n_parts = int(n_parts)
        self.n_tris = t.shape[0]

    def local(self, part: int) -> dict:
        """cells (global ids, ascending), ghost flags, local xy and tri."""
        sz = np.zeros(3, dtype=np.int64)
        _check(lib().swe_partition_sizes(self._h, int(part), _p(sz)), "swe_partition_sizes")
        n, _, nv = (int(x) for x in sz)
        cells = np.zeros(n, dtype=np.int32)
        ghost = np.zeros(n, dtype=np.uint8)
        xy = np.zeros((nv, 2))
        tri = np.zeros((n, 3), dtype=np.int32)
        _check(lib().swe_partition_local_mesh(self._h, int(part), _p(self.xy), _p(cells),
                                              _p(ghost), _p(xy), _p(tri)),
               "swe_partition_local_mesh")
        return dict(cells=cells, ghost=ghost, xy=xy, tri=tri)

    def exchange(self, src: int, dst: int):
        """(src-side local ids, dst-side local ids) of the cells owned by
        part src that part dst holds as ghosts."""
        n = ctypes.c_int64()
        _check(lib().swe_partition_exchange(self._h, int(src), int(dst), ctypes.byref(n), None,
                                            None), "swe_partition_exchange")
        a = np.zeros(n.value, dtype=np.int32)
        b = np.zeros(n.value, dtype=np.int32)
        if n.value:
            _check(lib().swe_partition_exchange(self._h, int(src), int(dst), ctypes.byref(n),
                                                _p(a), _p(b)), "swe_partition_exchange")
        return a, b

    def close(self):
        if getattr(self, "_h", None):
            lib().swe_partition_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
