"""bench.py's reference arm (the oracle timed on the host cores) keeps the
JSON-line contract: one line with the metric, value, unit, step counts,
direction, scaling, dtype, data, config, a cpu_baseline describing the run and
an e2e object with zero copies; under a multi-rank launch only rank 0
prints."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run(env_extra):
    env = dict(os.environ)
    env.update(env_extra)
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload", "mixed_small",
           "--steps", "2", "--warmup", "1"]
    p = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert p.returncode == 0, p.stderr[-2000:]
    return [ln for ln in p.stdout.splitlines() if ln.startswith("{")]


def test_reference_line():
    lines = run({})
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for k in ("metric", "unit", "data", "dtype", "scaling"):
        assert isinstance(d[k], str) and d[k]
    assert d["value"] > 0 and d["ms_per_step"] > 0
    assert d["steps"] == 2 and d["warmup"] == 1 and d["n_gpus"] == 1
    assert d["higher_is_better"] is True and d["vs_baseline"] is None
    assert "workload" in d["config"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_reference_other_ranks_are_silent():
    lines = run({"RANK": "1", "LOCAL_RANK": "1", "WORLD_SIZE": "2"})
    assert lines == []


def test_roofline_models():
    """The algorithmic-byte and flop models bench.py divides by: the CG
    products of the large mixed program move 8 nnz + 4(m+1) + 4n + 4m bytes
    (q = A p) and 8 nnz + 4(n+1) + 4m + 24n + 20m bytes (A^T q with its CG
    update and its side task y_acc += alpha q, az += alpha q: q, y_acc, az
    read, y_acc, az written), 179.9 MB and 235.9 MB; the FP32 ALU peak is
    152 SMs x 128 lanes x 2 flops a clock."""
    sys.path.insert(0, ROOT)
    import bench

    class P:
        m, n = 2_000_000, 1_000_000

        class A:
            nnz = 19_986_983          # synth.mixed(0): 2e7 drawn entries, duplicates merged

    b = bench.spmv_bytes(P, 5, 7)
    k3 = 8 * P.A.nnz + 4 * (P.m + 1) + 4 * P.n + 4 * P.m
    k4 = 8 * P.A.nnz + 4 * (P.n + 1) + 4 * P.m + 24 * P.n + 20 * P.m
    assert b["per_launch"]["A_cg"] == k3 and b["per_launch"]["At_cg"] == k4
    assert b[0] == 7 * k3                      # only the CG products q = A p are timed as kind 0
    k2 = 8 * P.A.nnz + 4 * (P.n + 1) + 4 * P.m + (8 + 8 + 4 + 4) * P.n + 8 * P.n
    assert b[1] == 5 * k2 + 7 * k4
    assert (k3, k4) == (179_895_868, 235_895_868)
    assert abs(bench.fp32_alu_peak_tflops(2070.0) - 152 * 128 * 2 * 2.07e9 / 1e12) < 1e-9
