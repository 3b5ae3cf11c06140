"""bench.py's reference arm (the CPU oracle timed on the host) runs without a
GPU and prints one JSON line with the keys the benchmark contract needs (the
multi-rank helpers are covered by test_multirank_cpu.py)."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e", "impl"):
        assert key in d, key
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
    assert d["dtype"] == "f64" and "workload" in d["config"]


def test_roofline_instruction_tables_are_consistent():
    """The op-class split (general FMAs + DADD-rate operations, counted on the
    op-class build) accounts for the production kernels' FP64 instruction
    counts to within 1% (the op-class build forms a few FMAs of its own), and
    the mix ceiling it implies is never below the all-DFMA time."""
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench", os.path.join(ROOT, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    for order in (4, 8):
        for name in ("z4c_derivs", "z4c_stage"):
            total = bench.FP64_INSTR_PER_CELL[order][name]
            gen, slow = bench.FP64_OP_CLASSES[order][name]
            assert gen > 0 and slow > 0
            assert abs(gen + slow - total) <= 0.01 * total, (order, name, gen + slow, total)
            dfma, dadd = 626.7, 527.9  # G/s, as measured in the bench run
            assert gen / dfma + slow / dadd >= total / dfma
