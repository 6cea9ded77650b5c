"""The FP32 tiled layout's bank-aware record order (host side, mesh_build.cpp):
within every tile it is a permutation of the stored records that keeps each
record's geometry and keeps the record classes contiguous and in order, so
every face is still computed exactly once per tile and the step's results
cannot change. Compiles tests/record_order_check.cpp against the library's
mesh builder and runs it on several meshes and tile sizes."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from paper_1807_00672_gb300 import inputs

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("g++ not available")
    out = tmp_path_factory.mktemp("rec") / "record_order_check"
    subprocess.run([cxx, "-O2", "-std=c++17", "-pthread", "-o", str(out),
                    os.path.join(HERE, "record_order_check.cpp"),
                    os.path.join(ROOT, "paper_1807_00672_gb300", "csrc", "mesh_build.cpp"),
                    "-I", os.path.join(ROOT, "include")], check=True)
    return str(out)


def write_mesh(path, mesh):
    xy = np.ascontiguousarray(mesh.xy, dtype=np.float64)
    tri = np.ascontiguousarray(mesh.tri, dtype=np.int32)
    with open(path, "wb") as f:
        f.write(np.int64(xy.shape[0]).tobytes())
        f.write(np.int64(tri.shape[0]).tobytes())
        f.write(xy.tobytes())
        f.write(tri.tobytes())


@pytest.mark.parametrize("tile", [64, 128, 256, 512])
def test_record_order_is_a_permutation_within_classes(checker, tmp_path, tile):
    meshes = [inputs.random_flow_case(nx=37, ny=23, seed=41).mesh,
              inputs.humps_case(nx=300, ny=150, lx=6_000.0, ly=3_000.0, seed=7).mesh,
              inputs.stoker_case().mesh,
              # above the size at which the order is computed on several host threads
              inputs.humps_case(nx=400, ny=300, lx=8_000.0, ly=6_000.0, seed=8).mesh]
    for i, mesh in enumerate(meshes):
        path = tmp_path / f"m{i}.bin"
        write_mesh(path, mesh)
        r = subprocess.run([checker, str(path), str(tile)], capture_output=True, text=True)
        assert r.returncode == 0, r.stdout + r.stderr
        assert r.stdout.startswith("ok "), r.stdout
