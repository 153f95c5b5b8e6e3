"""The benchmark's reference arm (the CPU oracle) prints one JSON line with the
keys the benchmark contract names; run here on a small mesh (no GPU)."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_the_contract_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0", "--nel", "12"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["value"] > 0 and d["dtype"] == "f64"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0


def test_kernel_table_and_rounding():
    """The per-kernel rows of the bench line: [total ms, launches, algorithmic
    TFLOP/s, fraction of the peak], the flops being the oracle's per-DOF count
    of the kernel's step times the DOFs of one launch; kernels without a step
    count (time step, indicator) carry times only; idle ones are left out."""
    sys.path.insert(0, ROOT)
    import bench
    prof = {"dg_volume": (10.0, 5), "face_flux": (3.0, 5), "dt": (1.0, 2), "remap": (0.0, 0)}
    per_step = {bench.KERNEL_STEP["dg_volume"]: 1000.0, bench.KERNEL_STEP["face_flux"]: 0.0}
    t = bench.kernel_table(prof, per_step, 1.0e6, 1.25)
    # 1000 flop per DOF x 1e6 DOFs in 2 ms per launch: 0.5 TFLOP/s, 0.4 of 1.25
    assert t["dg_volume"] == [10.0, 5, 0.5, 0.4]
    assert t["face_flux"] == [3.0, 5, None, None]
    assert t["dt"] == [1.0, 2, None, None]
    assert "remap" not in t
    assert bench.r4(123456.0) == 123500.0 and bench.r4(0.000123456) == 0.0001235 and bench.r4(None) is None


def test_target_summary_reads_the_legs_and_tolerates_missing_ones():
    """The closing `targets` object of the bench line takes each ratio from its
    leg (kernel-table rows by position) and gives None where a leg was
    skipped."""
    sys.path.insert(0, ROOT)
    import bench
    line = {"roofline": {"frac": 0.8, "whole_rhs_frac": 0.79},
            "hp_shock": {"whole_rhs_frac": 0.52, "kernels": {"fv": [12.0, 30, 0.6, 0.48]}},
            "adjoint": {"mixing_layer": {"adj_over_fwd_stored": 2.2, "adj_over_fwd_recomputed": 2.9}},
            "batched_domains": None}
    t = bench.target_summary(line)
    assert t == {"dominant_frac": 0.8, "whole_rhs_frac": 0.79, "hp_shock_whole_rhs_frac": 0.52,
                 "hp_shock_fv_frac": 0.48, "adj_over_fwd_stored": 2.2, "adj_over_fwd_recomputed": 2.9,
                 "batched_over_per_degree": None}
    assert all(v is None for v in bench.target_summary({}).values())
