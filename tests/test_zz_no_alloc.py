"""The allocation-free entry point swe_step_edges_static, through the C ABI.

It serves callers that cannot call cudaMalloc (no allocation once running,
device memory owned by the host's own pool): every input and output is a
device buffer the caller already has, and the scratch lives in a static
device array. Two calls in a row must reproduce two steps of the existing
entry points (swe_step on a handle with the two-launch kernels, caller cell
order) within the FP64 parity tolerance of the other GPU tests.

This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

from paper_1807_00672_gb300 import inputs, swe

from gpu_util import ensure_built, errors_of

pytestmark = pytest.mark.gpu

TOL64 = 1e-11
G = 9.81


def edge_layout(xy, tri, n_manning):
    """Edge and cell arrays in the layout swe_step_edges_static documents,
    built here with numpy: edges between the lower and the higher cell index,
    unit normal out of the lower cell along its counter-clockwise traversal,
    wall edges with right = -1, faces k = 0, 1, 2 joining nodes k and k+1."""
    T = tri.shape[0]
    p0, p1, p2 = xy[tri[:, 0]], xy[tri[:, 1]], xy[tri[:, 2]]
    area = 0.5 * ((p1[:, 0] - p0[:, 0]) * (p2[:, 1] - p0[:, 1])
                  - (p2[:, 0] - p0[:, 0]) * (p1[:, 1] - p0[:, 1]))
    assert np.all(area > 0)
    a = tri.reshape(-1)                       # half-edge h = 3 i + k: node k -> k+1
    b = tri[:, [1, 2, 0]].reshape(-1)
    key = np.minimum(a, b).astype(np.int64) << 32 | np.maximum(a, b)
    order = np.lexsort((np.arange(3 * T), key))
    ks = key[order]
    first = np.ones(ks.shape[0], dtype=bool)
    first[1:] = ks[1:] != ks[:-1]
    edge_of_sorted = np.cumsum(first) - 1
    E = int(edge_of_sorted[-1]) + 1
    edge_of_half = np.empty(3 * T, dtype=np.int64)
    edge_of_half[order] = edge_of_sorted
    left_half = order[first]                  # lowest half-edge id = lowest cell
    cnt = np.bincount(edge_of_sorted, minlength=E)
    assert cnt.max() <= 2
    right = np.full(E, -1, dtype=np.int32)
    second = order[~first]
    right[edge_of_sorted[~first]] = second // 3
    left = (left_half // 3).astype(np.int32)
    dx = xy[b[left_half], 0] - xy[a[left_half], 0]
    dy = xy[b[left_half], 1] - xy[a[left_half], 1]
    ln = np.sqrt(dx * dx + dy * dy)
    nx, ny = dy / ln, -dx / ln
    cell = np.repeat(np.arange(T), 3)
    is_right = left[edge_of_half] != cell
    face = (edge_of_half | np.where(is_right, 1 << 31, 0)).astype(np.uint32).view(np.int32)
    face = face.reshape(T, 3).T.copy()         # [k * T + i]
    fl = ln[edge_of_half].reshape(T, 3)
    perim = ((0.0 + fl[:, 0]) + fl[:, 1]) + fl[:, 2]
    return dict(T=T, E=E, left=left, right=right, nx=nx, ny=ny, len=ln, face=face.reshape(-1),
                area=area, irp=perim / area, gn2=G * (n_manning * n_manning))


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def test_static_entry_point_matches_swe_step_twice():
    torch = pytest.importorskip("torch")
    ensure_built()
    L = swe.lib()
    case = inputs.random_flow_case(nx=37, ny=23, seed=41)   # 1,702 cells, wet/dry, walls
    lay = edge_layout(case.mesh.xy, case.mesh.tri, case.n)

    mesh = swe.Mesh(case.mesh.xy, case.mesh.tri, precision="f64", kernel="edge", order="none")
    ref = swe.State(mesh, case.h, case.hu, case.hv, case.z, case.n)
    assert (mesh.T, mesh.E) == (lay["T"], lay["E"])

    dev = torch.device("cuda", 0)
    d = {k: torch.from_numpy(np.ascontiguousarray(lay[k])).to(dev)
         for k in ("left", "right", "nx", "ny", "len", "face", "area", "irp", "gn2")}
    z = torch.from_numpy(case.z).to(dev)
    U = [torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in (case.h, case.hu, case.hv)]
    stream = torch.cuda.current_stream(dev)

    dt = ref.next_dt()
    for call in range(2):
        out = [torch.empty_like(U[0]) for _ in range(3)]
        next_dt = ctypes.c_double()
        mass = ctypes.c_double()
        s = L.swe_step_edges_static(
            lay["T"], lay["E"], _ptr(d["left"]), _ptr(d["right"]), _ptr(d["nx"]), _ptr(d["ny"]),
            _ptr(d["len"]), _ptr(d["face"]), _ptr(d["area"]), _ptr(d["irp"]), _ptr(d["gn2"]),
            _ptr(z), _ptr(U[0]), _ptr(U[1]), _ptr(U[2]), G, 0.7, 1e-6, dt,
            _ptr(out[0]), _ptr(out[1]), _ptr(out[2]), ctypes.byref(next_dt), ctypes.byref(mass),
            ctypes.c_void_p(stream.cuda_stream))
        assert s == swe.SWE_OK, L.swe_strerror(s)
        used = ref.step()
        assert used == pytest.approx(dt, rel=1e-15)
        h, hu, hv = ref.fields()
        got = [o.cpu().numpy() for o in out]
        errs = errors_of(got, (h, hu, hv))
        assert max(errs.values()) <= TOL64, (call, errs)
        assert next_dt.value == pytest.approx(ref.next_dt(), rel=1e-13)
        assert mass.value == pytest.approx(ref.mass, rel=1e-13)
        U, dt = out, next_dt.value


def test_static_entry_point_rejects_oversized_meshes():
    ensure_built()
    L = swe.lib()
    one = ctypes.c_void_p(1)   # never dereferenced: the size check comes first
    args = [one] * 13
    too_many = 417_792 + 1
    s = L.swe_step_edges_static(too_many // 2, too_many, *args, G, 0.7, 1e-6, 0.1,
                                one, one, one, None, None, None)
    assert s == swe.SWE_EINVAL
    s = L.swe_step_edges_static(0, 10, *args, G, 0.7, 1e-6, 0.1, one, one, one, None, None, None)
    assert s == swe.SWE_EINVAL
    for dt in (float("inf"), float("nan"), -1.0):
        s = L.swe_step_edges_static(5, 10, *args, G, 0.7, 1e-6, dt, one, one, one, None, None, None)
        assert s == swe.SWE_EINVAL
