"""Host logic of bench.py that needs no GPU: the kernel-source key under which
the committed ncu counters (profiles/traffic.txt, profiles/fp64_ops.txt) are
reported, and the lookups that use it."""
import types

import bench


def _digest_of(tmp_path, monkeypatch, text):
    src = tmp_path / "paper_1807_00672_gb300" / "csrc"
    src.mkdir(parents=True, exist_ok=True)
    (src / "swe_kernels.cuh").write_text(text)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    return bench.kernel_source_digest()


def test_digest_ignores_comments_and_blank_lines(tmp_path, monkeypatch):
    code = "int f(int x) {\n  return x + 1;\n}\n"
    commented = "// header\nint f(int x) {  // add one\n\n  return x + 1;   \n}\n// end\n"
    assert _digest_of(tmp_path, monkeypatch, code) == _digest_of(tmp_path, monkeypatch, commented)


def test_digest_changes_with_the_code(tmp_path, monkeypatch):
    a = _digest_of(tmp_path, monkeypatch, "int f(int x) { return x + 1; }\n")
    b = _digest_of(tmp_path, monkeypatch, "int f(int x) { return x + 2; }\n")
    assert a != b and len(a) == 16


def test_counter_lookups_follow_the_key_and_the_shape(tmp_path, monkeypatch):
    """A counter line is used only for the workload and kernel source it was
    captured on, and only for the captured shape."""
    digest = _digest_of(tmp_path, monkeypatch, "int f(int x) { return x + 1; }\n")
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "traffic.txt").write_text(f"# comment\nsinusoid_10m {digest} 686274816 ncu ...\n"
                                      "sinusoid_10m 0000000000000000 1 ncu ...\n")
    (prof / "fp64_ops.txt").write_text(f"sinusoid_10m {digest} 377.55 254.90 ncu ...\n")
    args = types.SimpleNamespace(precision="f32", kernel="auto", tile=0, cpt=0, stages=0,
                                 workload="sinusoid_10m")
    assert bench.profiled_traffic(args) == 686274816.0
    args.tile = 256  # not the captured FP32 shape
    assert bench.profiled_traffic(args) is None
    args.precision, args.tile = "f64", 0
    assert bench.profiled_fp64_flops(args) == 377.55
    assert bench.profiled_fp64_flops(args, field=3) == 254.90
    args.workload = "calibration_1m"
    assert bench.profiled_fp64_flops(args) is None
    # a code change lapses every line
    _digest_of(tmp_path, monkeypatch, "int f(int x) { return x + 2; }\n")
    args.precision, args.workload = "f32", "sinusoid_10m"
    assert bench.profiled_traffic(args) is None
