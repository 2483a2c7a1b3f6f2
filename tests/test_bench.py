"""Host logic of bench.py (no GPU): both arms name the same metric per
workload, the roofline classification of the dominant kernel, and measured
DRAM traffic applied only at the settings (workload, ND leaf, amalgamation)
and the kernel source it was captured with."""
import types

import pytest

import bench


def _args(**kw):
    a = dict(workload="2d", theta_steps=150, batch_count=256, nd_leaf=None, relax_k=None, relax_pct=None)
    a.update(kw)
    return types.SimpleNamespace(**a)


def test_metric_names_per_workload():
    names = {w: bench.metric_name(_args(workload=w)) for w in ("2d", "batch", "theta")}
    assert len(set(names.values())) == 3
    assert "150 steps" in names["theta"] and "batch" in names["batch"]
    assert bench.batch_name(_args()) == "batch_256_instances_1d2d_exp_nugget1e-2_1rhs"


def test_amalgamation_defaults_and_overrides(wdlib):
    d = wdlib.DEFAULTS
    assert bench.amalgamation(_args()) == (d["nd_leaf"], d["relax_k"], d["relax_pct"])
    assert bench.amalgamation(_args(nd_leaf=64, relax_k=16, relax_pct=10)) == (64, 16, 10)


def test_roofline_classification(monkeypatch):
    monkeypatch.setattr(bench, "load_peaks", lambda: {"hbm_gbs": 6000.0, "bf16_tflops_sustained": 1800.0})
    monkeypatch.setattr(bench, "device_units", lambda: (152, 2070.0, "test"))
    key = ("2d", (128, 64, 10))
    tc = bench.roofline({"name": "tc_schur_syrk_fp32", "ms": 1000.0, "flops": 84e12, "bytes": 0}, 64, key)
    assert tc["bound"] == "tensor"
    assert tc["peak"] == pytest.approx(1800.0 * 1.1 / 2.25)
    assert tc["achieved"] == pytest.approx(84.0)
    alu = bench.roofline({"name": "panel_fp32", "ms": 1000.0, "flops": 8e12, "bytes": 0}, 64, key)
    assert alu["bound"] == "alu" and alu["peak"] == pytest.approx(152 * 256 * 2070e6 / 1e12)
    df = bench.roofline({"name": "spmv_residual_df", "ms": 1000.0, "flops": 2e12, "bytes": 0}, 64, key)
    assert df["achieved"] == pytest.approx(bench.DF_OPS_PER_TERM * 1.0)
    hbm = bench.roofline({"name": "fwd_gather_fp32", "ms": 1000.0, "flops": 0, "bytes": 3e12}, 64, key)
    assert hbm["bound"] == "hbm" and hbm["frac"] == pytest.approx(0.5)


def test_measured_traffic_only_where_it_was_taken(monkeypatch, tmp_path):
    src = tmp_path / "k.cu"
    src.write_text("kernel")
    import hashlib
    sha = hashlib.sha1(b"kernel").hexdigest()
    entry = {"bytes": 1.5e6, "source": str(src), "sha1": sha}
    monkeypatch.setitem(bench.MEASURED_TRAFFIC, ("2d", "tc_schur_update_fp32", 128, 64, 10), entry)
    assert bench.measured_traffic(("2d", (128, 64, 10)), "tc_schur_update_fp32") == 1.5e6
    assert bench.measured_traffic(("2d", (64, 64, 10)), "tc_schur_update_fp32") is None
    assert bench.measured_traffic(("batch", (128, 64, 10)), "tc_schur_update_fp32") is None
    # a changed source file voids the figure
    src.write_text("kernel v2")
    assert bench.measured_traffic(("2d", (128, 64, 10)), "tc_schur_update_fp32") is None
    # every committed entry names a source file of the repository
    for k, t in bench.MEASURED_TRAFFIC.items():
        if k[1] != "tc_schur_update_fp32":
            assert t["source"].startswith("paper_2007_01541_gb300/csrc/")


def test_reference_arm_and_cpu_baseline_share_the_config(capsys):
    """The reference arm prints the same metric, unit and config as this
    build's line for the workload, with the oracle's bounded sample stated."""
    import json
    bench.run_reference(_args(workload="1d", nrhs=None, cpu_flops=1e7, steps=2, warmup=1, gpus=1))
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["metric"] == bench.metric_name(_args(workload="1d"))
    w = bench.make_workload("1d", None, "cpu")
    r = bench.oracle_sample(w, 1e7, repeats=1)
    assert line["config"] == bench.step_config(_args(workload="1d"), w, r["nnz_L"], r["flops_factor"], 1)
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] == 1
    assert r["factor_flops"] <= 1e7 and r["solve_flops"] > 0 and r["nproc"] >= 1


def test_batch_cpu_baseline_runs_the_oracle_in_parallel_processes():
    spec = {"dim": 1, "J": 10, "ell": 0.2, "nugget": 1e-2}
    params = [dict(spec), dict(spec, ell=0.3), dict(spec, J=9)]
    costs = [2.0, 3.0, 1.0]
    r = bench.batch_cpu_baseline(params, costs, 2)
    assert r is not None and r["cores"] == 2 and r["kind"] == "oracle"
    assert r["value"] > 0 and r["per_process"] > 0
    assert "(1, 10)" in r["sample"] and "(1, 9)" not in r["sample"]   # the two most expensive


def test_cpu_baseline_default_is_the_whole_factorization_and_solve():
    """With no flop budget the cpu_baseline times the oracle's whole
    factorization and both whole substitutions, once."""
    w = bench.make_workload("1d", None, "cpu")
    r = bench.oracle_sample(w, bench.parse([]).cpu_flops)
    assert r["sample_columns"] == w["basis"].N and r["repeats"] == 1
    assert r["factor_flops"] == r["flops_factor"] and "whole" in r["sample"]
    assert abs(r["solve_flops"] - 4.0 * r["nnz_L"] * w["nrhs"]) <= 1e-9 * r["solve_flops"]
