"""Helpers shared by the GPU tests: run the CUDA path and the oracle on one case."""
from __future__ import annotations

import numpy as np

import oracle
from paper_1807_00672_gb300 import build, swe

_built = False


def ensure_built():
    global _built
    if not _built:
        build.build()
        _built = True


def gpu_state(case, precision="f64", kernel="auto", order="morton", tile=0):
    ensure_built()
    mesh = swe.Mesh(case.mesh.xy, case.mesh.tri, precision=precision, kernel=kernel, order=order,
                    tile=tile)
    st = swe.State(mesh, case.h, case.hu, case.hv, case.z, case.n)
    return mesh, st


def rel_err(a: np.ndarray, ref: np.ndarray) -> float:
    """max |a - ref| / max |ref| (absolute if ref is identically 0)."""
    scale = float(np.abs(ref).max())
    d = float(np.abs(a - ref).max()) if a.size else 0.0
    return d / scale if scale > 0 else d


def froude_scale(h_ref, g=9.81) -> float:
    """h_max sqrt(g h_max): the discharge of a Froude-1 flow at the largest
    depth. Used as the error scale of a discharge field only where that
    field is round-off (still water), which would make max |q_ref| a
    meaningless denominator."""
    hmax = float(np.abs(h_ref).max()) if h_ref.size else 0.0
    return hmax * np.sqrt(g * hmax)


def field_rel_err(a, ref, h_ref, g=9.81, roundoff=1e-6) -> tuple[float, str]:
    """max |a - ref| / max |ref| per field (Eq. 4's state components); for a
    field whose largest value is at round-off level (below roundoff times
    the Froude-1 discharge, i.e. still water) the denominator is the
    Froude-1 discharge instead. Returns (error, which denominator)."""
    d = float(np.abs(a - ref).max()) if a.size else 0.0
    fmax = float(np.abs(ref).max()) if ref.size else 0.0
    fs = froude_scale(h_ref, g)
    if fmax > roundoff * fs:
        return d / fmax, "max|ref|"
    return (d / fs if fs > 0 else d), "froude"


def field_errors(st, ref):
    """Per field max |gpu - oracle| over cells divided by the field's own
    max |ref| (hu and hv on still water: by the Froude-1 discharge)."""
    h, hu, hv = st.fields()
    return errors_of((h, hu, hv), (ref.h, ref.hu, ref.hv)), (h, hu, hv)


def errors_of(got, want):
    """field_errors on arrays: got, want = (h, hu, hv) each."""
    errs = {}
    for name, a, r in zip(("h", "hu", "hv"), got, want):
        if name == "h":
            errs[name] = rel_err(a, r)
        else:
            errs[name], _ = field_rel_err(a, r, want[0])
    return errs


def l1_linf(a, ref, area):
    """Area-weighted L1 and Linf errors relative to the reference field."""
    den = float((area * np.abs(ref)).sum())
    l1 = float((area * np.abs(a - ref)).sum()) / den if den > 0 else float(np.abs(a - ref).max())
    return l1, rel_err(a, ref)


def oracle_run(case, n_steps):
    o = oracle.state_from_case(case)
    dts = o.run(n_steps)
    return o, dts
