"""Host logic of bench.py that needs no GPU: the JSON line of the reference
arm (the FP64 oracle timed on the host cores), the source hashing that keeps a
recorded ncu traffic figure tied to the kernel it was measured on, and the
table lookup that scales it to a launch."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench as B  # noqa: E402


def test_reference_arm_prints_one_contract_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
                          "bumps_64", "--steps", "1", "--warmup", "1"], capture_output=True, text=True,
                         timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == "unknowns/s"
    assert d["metric"] == B.METRIC and d["higher_is_better"] is True and d["steps"] == 1
    assert d["e2e"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["config"]["workload"] == "bumps_64"


def test_function_text_is_one_global_function():
    src = open(os.path.join(ROOT, "paper_1002_3094_gb300", "csrc", "ax_stencil.cu")).read()
    text = B._function_text(src, "residual_df_kernel")
    assert text.splitlines()[0].startswith("__global__") and "residual_df_kernel(" in text.splitlines()[0]
    assert text.rstrip().endswith("}") and "stencil_kernel(" not in text
    assert len(B.source_hash("stencil")) == 16 and B.source_hash("stencil") != B.source_hash("outer_residual")


def test_source_hash_ignores_comments_but_not_code():
    src = {"ax_stencil.cu": open(os.path.join(ROOT, "paper_1002_3094_gb300", "csrc", "ax_stencil.cu")).read(),
           "ax_common.cuh": open(os.path.join(ROOT, "paper_1002_3094_gb300", "csrc", "ax_common.cuh")).read()}
    base = B.source_hash("stencil", src.__getitem__)
    assert base == B.source_hash("stencil")
    decl = "__global__"
    commented = dict(src)
    i = src["ax_stencil.cu"].index(decl, src["ax_stencil.cu"].index("stencil_kernel(") - 400)
    body = src["ax_stencil.cu"]
    j = body.index("{", body.index("stencil_kernel(", i)) + 1
    commented["ax_stencil.cu"] = body[:j] + "\n  // a new comment\n  /* and a block\n  comment */\n" + body[j:]
    assert B.source_hash("stencil", commented.__getitem__) == base
    changed = dict(src)
    changed["ax_stencil.cu"] = body[:j] + "\n  int unused_probe = 0;\n" + body[j:]
    assert B.source_hash("stencil", changed.__getitem__) != base


def test_traffic_row_applies_only_to_the_source_it_was_measured_on(tmp_path, monkeypatch):
    table = tmp_path / "traffic.json"
    table.write_text(json.dumps({"entries": [
        {"class": "stencil", "dram_bytes_per_unknown": 6.5, "source_sha": B.source_hash("stencil")},
        {"class": "pcg_update", "dram_bytes_per_unknown": 12.0, "source_sha": "0000000000000000"}]}))
    monkeypatch.setattr(B, "TRAFFIC_TABLE", str(table))
    assert B.measured_traffic("stencil", 1000.0) == pytest.approx(6500.0)
    assert B.measured_traffic("pcg_update", 1000.0) is None  # recorded on other code
    assert B.measured_traffic("mode_solve", 1000.0) is None  # never recorded
    table.write_text("not json")
    assert B.measured_traffic("stencil", 1000.0) is None


def test_kernel_class_follows_the_kernels_the_solve_ran():
    assert B.kernel_class("dst_inverse", True, 14) == "dst_inverse_tc"
    assert B.kernel_class("dst_inverse", False, 9) == "dst_inverse"
    assert B.kernel_class("mode_solve", True, 9) == "mode_solve_scaled"
    assert B.kernel_class("mode_solve", True, 14) == "mode_solve_modemajor"
    assert B.kernel_class("mode_solve", True, 1) == "mode_solve"
    assert B.kernel_class("mode_solve", True, 0) == "mode_solve_tall"
    assert B.kernel_class("mode_solve", True, 5) == "mode_solve_pipe"
    assert B.kernel_class("stencil", True, 14) == "stencil"
    for c in ("mode_solve_scaled", "mode_solve_reuse", "mode_solve_pipe", "mode_solve_modemajor"):
        assert len(B.source_hash(c)) == 16 and B.source_hash(c) != B.source_hash("stencil")


def test_both_arms_describe_the_same_workload():
    """The reference arm's line carries the GPU arm's config (arm_config) for
    the single-operator workloads, sizes and right-hand-side count included."""
    import argparse
    for name, shape in (("layered_1024_m64", (1024, 1024, 64)), ("large_4096_m16", (4096, 4096, 16)),
                        ("bumps_64", (64, 64, 1))):
        args = argparse.Namespace(workload=name, bc_z=0, method="pcg_mixed", option=[], rhs=0, gpus=1)
        nr, nz, med = B.workload(name, rhs=0)
        cfg = B.arm_config(args, nr, nz, med.n_rhs, 1)
        assert (cfg["nr"], cfg["nz"], cfg["rhs"]) == shape
        assert cfg["workload"] == name and cfg["tol"] == B.TOL and cfg["parallelism"] == "replicas x1"
        assert ("larger than L2" in cfg["l2"]) == (name != "bumps_64")
