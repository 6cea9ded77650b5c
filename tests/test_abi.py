"""The C ABI without a GPU: the library loads, exports every declared entry
point, and rejects bad arguments and invalid meshes before touching a device."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_1807_00672_gb300 import build, inputs, swe

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    build.build()
    return swe.lib()


def declared_functions():
    text = open(os.path.join(ROOT, "include", "swe.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b(swe_[a-z_0-9]+)\s*\(", text)
    return sorted(set(names))


def test_header_and_binding_agree():
    assert sorted(swe.EXPORTS) == declared_functions()


def test_library_exports_every_declared_symbol(L):
    for name in declared_functions():
        assert hasattr(L, name), name


def test_strerror_and_defaults(L):
    assert L.swe_strerror(0) == b"ok"
    assert b"mesh" in L.swe_strerror(swe.SWE_EMESH)
    assert L.swe_strerror(12345) == b"unknown status"
    p = swe.Params()
    L.swe_params_default(ctypes.byref(p))
    assert (p.g, p.courant, p.h_eps) == (9.81, 0.7, 1e-6)
    assert (p.precision, p.order, p.kernel, p.tile, p.stages, p.cells_per_thread,
            p.halo_schedule, p.wait_rounds) == (0, 1, 0, 0, 0, 0, 0, 0)


def _create(xy, tri, prm=None):
    h = ctypes.c_void_p()
    xy = np.ascontiguousarray(xy, dtype=np.float64)
    tri = np.ascontiguousarray(tri, dtype=np.int32)
    st = swe.lib().swe_mesh_create(xy.ctypes.data_as(ctypes.c_void_p), xy.shape[0],
                                   tri.ctypes.data_as(ctypes.c_void_p), tri.shape[0],
                                   None if prm is None else ctypes.byref(prm), None,
                                   ctypes.byref(h))
    return st, h


def test_null_and_empty_arguments(L):
    h = ctypes.c_void_p()
    assert L.swe_mesh_create(None, 3, None, 1, None, None, ctypes.byref(h)) == swe.SWE_EINVAL
    m = inputs.jittered_grid(2, 2, 1.0, 1.0)
    st, _ = _create(m.xy, m.tri[:0])
    assert st == swe.SWE_EMESH
    assert L.swe_mesh_create(None, 0, None, 0, None, None, None) == swe.SWE_EINVAL
    assert L.swe_state_init(None, None, None, None, None, None, 0.0, ctypes.byref(h)) == swe.SWE_EINVAL
    assert L.swe_step(None, None) == swe.SWE_EINVAL
    assert L.swe_run(None, 1) == swe.SWE_EINVAL
    assert L.swe_copy_out(None, None, None, None, None, None) == swe.SWE_EINVAL


@pytest.mark.parametrize("bad", ["index", "negative", "degenerate", "nonmanifold", "collinear"])
def test_invalid_meshes_rejected_on_the_host(L, bad):
    m = inputs.jittered_grid(3, 3, 3.0, 3.0)
    xy, tri = m.xy.copy(), m.tri.copy()
    if bad == "index":
        tri[4, 1] = m.n_nodes
    elif bad == "negative":
        tri[1, 0] = -1
    elif bad == "degenerate":
        tri[2, 2] = tri[2, 0]
    elif bad == "nonmanifold":
        tri = np.concatenate([tri, tri[:1, [0, 2, 1]]])
    else:
        xy[tri[0, 1]] = 0.5 * (xy[tri[0, 0]] + xy[tri[0, 2]])
    st, _ = _create(xy, tri)
    assert st == swe.SWE_EMESH


@pytest.mark.parametrize("field,val", [("precision", 7), ("order", 5), ("kernel", 9), ("tile", 100),
                                       ("stages", 5), ("cells_per_thread", 3),
                                       ("halo_schedule", 3), ("wait_rounds", -2),
                                       ("compensated_depth", 2), ("compensated_depth", 1)])
def test_bad_params_rejected(L, field, val):
    m = inputs.jittered_grid(3, 3, 3.0, 3.0)
    p = swe.params()
    setattr(p, field, val)
    st, _ = _create(m.xy, m.tri, p)
    assert st == swe.SWE_EINVAL


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    monkeypatch.setattr(swe, "_lib", None)
    monkeypatch.setattr(swe, "LIB_PATH", str(tmp_path / "libswe.so"))
    with pytest.raises(RuntimeError, match="missing"):
        swe.lib()


def _create_batch(meshes, prm=None, n=None):
    k = len(meshes)
    xys = [np.ascontiguousarray(xy, dtype=np.float64) for xy, _ in meshes]
    tris = [np.ascontiguousarray(t, dtype=np.int32) for _, t in meshes]
    xp = (ctypes.c_void_p * max(k, 1))(*[a.ctypes.data for a in xys])
    tp = (ctypes.c_void_p * max(k, 1))(*[a.ctypes.data for a in tris])
    nn = np.array([a.shape[0] for a in xys] or [0], dtype=np.int64)
    nt = np.array([a.shape[0] for a in tris] or [0], dtype=np.int64)
    h = ctypes.c_void_p()
    st = swe.lib().swe_mesh_create_batch(k if n is None else n, xp,
                                         nn.ctypes.data_as(ctypes.c_void_p), tp,
                                         nt.ctypes.data_as(ctypes.c_void_p),
                                         None if prm is None else ctypes.byref(prm), None,
                                         ctypes.byref(h))
    return st, h


def test_batch_rejects_bad_counts_and_an_invalid_scenario(L):
    a = inputs.jittered_grid(3, 3, 3.0, 3.0)
    b = inputs.jittered_grid(4, 2, 4.0, 2.0, seed=3)
    st, _ = _create_batch([(a.xy, a.tri)], n=0)
    assert st == swe.SWE_EINVAL
    st, _ = _create_batch([(a.xy, a.tri)], n=-3)
    assert st == swe.SWE_EINVAL
    bad = b.tri.copy()
    bad[0, 0] = b.n_nodes  # the second scenario has a node index out of range
    st, _ = _create_batch([(a.xy, a.tri), (b.xy, bad)])
    assert st == swe.SWE_EMESH
    st, _ = _create_batch([(a.xy, a.tri), (b.xy, b.tri[:0])])
    assert st == swe.SWE_EMESH
    h = ctypes.c_void_p()
    assert L.swe_mesh_create_batch(2, None, None, None, None, None, None, ctypes.byref(h)) == swe.SWE_EINVAL


def test_batch_needs_the_tiled_kernel(L):
    a = inputs.jittered_grid(3, 3, 3.0, 3.0)
    st, _ = _create_batch([(a.xy, a.tri), (a.xy, a.tri)], swe.params(kernel="edge"))
    assert st == swe.SWE_EINVAL


def test_scenario_queries_reject_null_handles(L):
    n = ctypes.c_int32()
    assert L.swe_mesh_scenarios(None, ctypes.byref(n), None) == swe.SWE_EINVAL
    assert L.swe_scenario_info(None, 0, None, None, None, None) == swe.SWE_EINVAL
