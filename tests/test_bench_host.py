"""Host logic of bench.py that needs no GPU: the DRAM traffic lines it reads
from profiles/ are used only while the sha256 of the named kernel sources
matches, and lines marked as growing with the point count are scaled."""
import hashlib
import os

import bench


def _write(root, rel, text):
    p = os.path.join(root, rel)
    os.makedirs(os.path.dirname(p), exist_ok=True)
    with open(p, "w") as fh:
        fh.write(text)
    return p


def _line(cls, bytes_, points, scales, sha, sources):
    return (f"traffic class={cls} bytes_per_step={bytes_:.4e} points={points} scales={scales} "
            f"sha256={sha} sources={','.join(sources)}\n")


def test_profile_traffic_keeps_matching_lines_and_drops_stale_ones(tmp_path, monkeypatch):
    root = str(tmp_path)
    _write(root, "src/a.cu", "kernel a\n")
    _write(root, "src/b.cu", "kernel b\n")
    good = hashlib.sha256(b"kernel a\nkernel b\n").hexdigest()
    stale = hashlib.sha256(b"kernel a (old)\n").hexdigest()
    _write(root, "profiles/p.md",
           "# capture\n\n" +
           _line("layer_gemm", 5.0e10, 2560, 0, good, ["src/a.cu", "src/b.cu"]) +
           _line("gram", 1.0e10, 1280, 1, good, ["src/a.cu", "src/b.cu"]) +
           _line("eig", 5.0e9, 2560, 0, stale, ["src/a.cu"]) +
           _line("precond", 1.0e8, 2560, 0, good, ["src/missing.cu"]))
    monkeypatch.setattr(bench, "ROOT", root)
    t = bench.profile_traffic(2560)
    assert set(t) == {"layer_gemm", "gram"}
    assert t["layer_gemm"]["bytes"] == 5.0e10
    assert t["layer_gemm"]["source"] == os.path.join("profiles", "p.md")
    assert t["gram"]["bytes"] == 2.0e10                  # scaled from 1280 to 2560 points
    assert "scaled from 1280 to 2560" in t["gram"]["source"]
    # a changed source drops the line
    _write(root, "src/b.cu", "kernel b, edited\n")
    assert bench.profile_traffic(2560) == {}


def test_reference_arm_line(monkeypatch):
    # the oracle arm's JSON line (run at N = 1 on the host cores), on a
    # two-point sample so that it takes seconds
    import json

    monkeypatch.setattr(bench, "REF_SAMPLE", (2, 1))

    class Args:
        steps, warmup = 1, 0

    out = bench.run_reference(Args, 0, 1)
    json.dumps(out)
    assert out["impl"] == "reference" and out["metric"] == bench.METRIC
    assert out["unit"] == "steps/s" and out["higher_is_better"] is True and out["value"] > 0
    assert out["config"]["workload"] == bench.WORKLOAD_NAME and out["dtype"] == "f64"
    assert out["e2e"] == {"value": out["value"], "unit": "steps/s", "h2d_bytes_per_step": 0,
                          "d2h_bytes_per_step": 0}
    cb = out["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == out["value"] and cb["cores"] >= 1
    assert cb["extrapolated"] is True and cb["scale"] == bench.WORKLOAD.n_int // 2 and "sample" in cb
