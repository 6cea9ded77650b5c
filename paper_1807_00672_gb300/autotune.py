"""Autotuner for the tiled step kernel's shape: cells per tile, cells per
thread, shared-memory pipeline stages and halo-gather schedule
(``swe_params.tile``, ``cells_per_thread``, ``stages``, ``halo_schedule``).

The best shape depends on the mesh (how many faces and halo cells a tile
has, how many tiles each block walks) and on the precision, so it is chosen
by measurement: each candidate builds the mesh (or ensemble) with that shape,
takes a few untimed steps, then times ``steps`` steps with CUDA events on the
mesh's stream. Results are cached in a JSON file keyed by GPU name,
precision, scenario count and the log2 bucket of the cell count, so a later
run on a similar problem reuses the answer without measuring again.

Cache file: ``$SWE_TUNE_CACHE`` if set, else ``~/.cache/swe_gb300/tune.json``.
"""
from __future__ import annotations

import json
import math
import os
import time

from . import swe

# (tile, cells_per_thread, stages[, halo_schedule]); threads per block =
# tile / cells_per_thread; a missing halo_schedule is 0 (2: the pipelined
# kernel, FP32 only; in FP64 those shapes run as schedule 0 or are skipped).
CANDIDATES = (
    (256, 2, 2), (256, 2, 2, 1), (256, 2, 3), (256, 1, 2), (256, 1, 3),
    (512, 2, 2), (512, 2, 2, 1), (128, 1, 2), (128, 2, 3),
    (256, 1, 2, 2), (512, 2, 2, 2), (512, 1, 2, 2),
)


def cache_path() -> str:
    p = os.environ.get("SWE_TUNE_CACHE")
    if p:
        return p
    return os.path.join(os.path.expanduser("~"), ".cache", "swe_gb300", "tune.json")


def problem_key(device_name: str, precision: str, n_cells: int, n_scenarios: int) -> str:
    bucket = int(math.floor(math.log2(max(1, n_cells))))
    return f"{device_name}|{precision}|s{n_scenarios}|c2^{bucket}"


def _load(path):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(path, data):
    d = os.path.dirname(path)
    if d:
        os.makedirs(d, exist_ok=True)
    tmp = path + f".{os.getpid()}.tmp"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def _build(cases, precision, shape, stream):
    tile, cpt, stages = shape[:3]
    kw = dict(precision=precision, kernel="tiled", tile=tile, cells_per_thread=cpt,
              stages=stages, halo_schedule=shape[3] if len(shape) > 3 else 0, stream=stream)
    if len(cases) == 1:
        c = cases[0]
        mesh = swe.Mesh(c.mesh.xy, c.mesh.tri, **kw)
        st = swe.State(mesh, c.h, c.hu, c.hv, c.z, c.n)
    else:
        import numpy as np
        mesh = swe.Mesh.ensemble([(c.mesh.xy, c.mesh.tri) for c in cases], **kw)
        cat = lambda name: np.concatenate([getattr(c, name) for c in cases])
        st = swe.State(mesh, cat("h"), cat("hu"), cat("hv"), cat("z"), cat("n"))
    return mesh, st


def measure(cases, precision: str, shape, steps: int = 32, warmup: int = 16) -> float:
    """Seconds per step of one shape on these cases (a list of inputs.Case;
    more than one = an ensemble)."""
    import ctypes

    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.Stream(device=dev)
    mesh, st = _build(cases, precision, shape, ctypes.c_void_p(stream.cuda_stream))
    try:
        st.run(warmup)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        st.run(steps, sync=False)
        b.record(stream)
        torch.cuda.synchronize(dev)
        st.sync()
        return a.elapsed_time(b) * 1e-3 / steps
    finally:
        st.close()
        mesh.close()


def tune(cases, precision: str = "f32", *, candidates=CANDIDATES, steps: int = 32,
         use_cache: bool = True, key_cells: int | None = None, key_scenarios: int | None = None,
         log=None) -> dict:
    """Best (tile, cells_per_thread, stages, halo_schedule) for these cases.

    ``cases`` may be a representative sample of a larger problem; key_cells
    and key_scenarios then name the full problem's size for the cache key.
    Returns {"tile", "cells_per_thread", "stages", "halo_schedule",
    "sec_per_step", "cached", "trials": [...]}.
    """
    import torch
    n_cells = key_cells if key_cells is not None else sum(c.mesh.n_tris for c in cases)
    n_scen = key_scenarios if key_scenarios is not None else len(cases)
    name = torch.cuda.get_device_name(torch.cuda.current_device())
    key = problem_key(name, precision, n_cells, n_scen)
    path = cache_path()
    if use_cache:
        hit = _load(path).get(key)
        if hit:
            return dict({"halo_schedule": 0}, **hit, cached=True, key=key)
    trials = []
    for shape in candidates:
        t0 = time.perf_counter()
        try:
            sec = measure(cases, precision, shape, steps=steps)
        except swe.SweError as e:  # a shape that does not fit (shared memory) is skipped
            trials.append(dict(shape=list(shape), error=str(e)))
            continue
        trials.append(dict(shape=list(shape), sec_per_step=sec,
                           wall_s=time.perf_counter() - t0))
        if log:
            log(f"autotune {shape}: {sec * 1e6:.1f} us/step")
    ok = [t for t in trials if "sec_per_step" in t]
    if not ok:
        raise RuntimeError("autotune: no candidate shape could run")
    best = min(ok, key=lambda t: t["sec_per_step"])
    tile, cpt, stages = best["shape"][:3]
    sched = best["shape"][3] if len(best["shape"]) > 3 else 0
    res = dict(tile=tile, cells_per_thread=cpt, stages=stages, halo_schedule=sched,
               sec_per_step=best["sec_per_step"],
               sample_cells=sum(c.mesh.n_tris for c in cases), trials=trials)
    if use_cache:
        data = _load(path)
        data[key] = res
        _store(path, data)
    return dict(res, cached=False, key=key)
