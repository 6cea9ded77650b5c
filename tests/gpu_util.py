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


def momentum_scale(h_ref, hu_ref, hv_ref, g=9.81) -> float:
    """Scale of the discharge error: the larger of the reference's largest
    |(hu, hv)| and the Froude-1 discharge h_max sqrt(g h_max). A still lake
    has |(hu, hv)| at round-off, which would make max |q_ref| meaningless as a
    denominator; the momentum fluxes it comes from are of size g h^2 / 2."""
    hmax = float(np.abs(h_ref).max())
    qmax = float(np.hypot(hu_ref, hv_ref).max()) if hu_ref.size else 0.0
    return max(qmax, hmax * np.sqrt(g * hmax))


def field_errors(st, ref):
    """Per field max |gpu - oracle| over cells, divided by max |h_ref| for h
    and by momentum_scale for hu, hv."""
    h, hu, hv = st.fields()
    qs = momentum_scale(ref.h, ref.hu, ref.hv)
    errs = dict(h=rel_err(h, ref.h),
                hu=float(np.abs(hu - ref.hu).max()) / qs,
                hv=float(np.abs(hv - ref.hv).max()) / qs)
    return errs, (h, hu, hv)


def l1_linf(a, ref, area):
    """Area-weighted L1 and Linf errors relative to the reference field."""
    den = float((area * np.abs(ref)).sum())
    l1 = float((area * np.abs(a - ref)).sum()) / den if den > 0 else float(np.abs(a - ref).max())
    return l1, rel_err(a, ref)


def oracle_run(case, n_steps):
    o = oracle.state_from_case(case)
    dts = o.run(n_steps)
    return o, dts
