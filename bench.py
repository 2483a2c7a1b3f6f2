#!/usr/bin/env python
"""Benchmark: factor + solve of the wavelet-compressed 2D kernel matrix.

Workload (default): unit square with 256 x 256 cells, isotropic Haar
wavelets (N = 65,536), Matern-3/2 kernel (ell = 0.1) by the cell-centroid
rule, a = 2 compression, nugget 1e-3, 64 right-hand sides ~ N(0, 1), seed 0.
Inputs are synthetic (seeded generator; no dataset).

One step = wd_factor + wd_solve (64 RHS, refined in FP64 to a backward error
<= 1e-12 in mixed precision) + wd_logdet, with the matrix values and the
right-hand sides already resident in HBM.  The front pool (about 4 GB) is
far larger than L2, so no L2 flush is needed between steps.

value = (sum_j c_j^2 + 4 nnz(L) nrhs) / step time, in TFLOP/s, for the mixed
path.  The FP64 path is measured the same way and reported beside it.

Other workloads (--workload): batch (256 independent 1D / 2D instances, one
right-hand side each, sharded over ranks by longest-processing-time; strong
scaling), theta (the theta-scheme: M = I + theta dt K factored once, then
--theta-steps steps of product and refined solve, one right-hand side),
2d_small and 1d (smaller cases for profiling).

--impl reference times the CPU oracle (plain left-looking FP64 Cholesky and
the substitutions) on one host core, each step a bounded share of the same
factorization and solve: the factor of the first columns of P A P^T and both
substitutions over them.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
# derived ALU peaks: unit counts per SM x the device's SM count x its maximum
# SM clock (both read from the device at run time, see device_units)
FP32_LANES_PER_SM = 128
FP64_FLOPS_PER_SM_CLK = 4     # 2 FP64 FMA per SM per clock (GB300: 1.25 TFLOP/s nominal)
THETA, THETA_DT = 0.5, 1e-2      # theta workload: Crank-Nicolson, time step
DF_OPS_PER_TERM = 12.75       # FP32 instructions per double-float multiply-add (12, plus a 6-op TwoSum every 8 terms)
DF32_OPS_PER_TERM = 11.75     # the same with x exactly FP32 (one FMA less)

# tf32 / bf16 dense tensor rates (nominal 1.1 and 2.25 PFLOP/s): a tf32
# contraction's peak is the measured bf16 peak times this ratio
TF32_PER_BF16 = 1.1 / 2.25
# flop budget of each step of the reference arm (the oracle's factor of the
# first columns plus both substitutions over them), so that the whole
# --steps K --warmup W run stays within minutes
REF_STEP_FLOPS = 3e9

# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of a
# kernel from one ncu capture, keyed by (workload, kernel, nd_leaf, relax_k,
# relax_pct), with the SHA-1 of the source file the kernel was built from:
# reported as null once that file has changed.
MEASURED_TRAFFIC = {
    # 2D 256^2, tc_schur_kernel in its pivot-block update mode: 112 launches of
    # one timed step, dram__bytes_read.sum + dram__bytes_write.sum averaged over
    # the launches (a one-pass capture, gpu__time_duration.sum beside it)
    ("2d", "tc_schur_update_fp32", 128, 64, 10): {
        "bytes": 1.432e7, "source": "paper_2007_01541_gb300/csrc/tc_schur.cu",
        "sha1": "8ef397c4b80e9b17fb26b02b8d48367e5067f5c1"},
    # 2D 256^2, tc_chain_kernel: the 8 launches (one per level the tuner gives
    # it) of one timed step, averaged (one-pass capture)
    ("2d", "tc_chain_fp32", 128, 64, 10): {
        "bytes": 8.011e7, "source": "paper_2007_01541_gb300/csrc/tc_chain.cu",
        "sha1": "8a715ab56dd0b6a60e38e2f7e397db9be256ade1"},
}


def amalgamation(args):
    """(nd_leaf, relax_k, relax_pct) in effect: the options given, else the library's defaults."""
    from paper_2007_01541_gb300 import DEFAULTS
    return (args.nd_leaf if args.nd_leaf is not None else DEFAULTS["nd_leaf"],
            args.relax_k if args.relax_k is not None else DEFAULTS["relax_k"],
            args.relax_pct if args.relax_pct is not None else DEFAULTS["relax_pct"])


def measured_traffic(key, kernel):
    import hashlib
    workload, relax = key
    t = MEASURED_TRAFFIC.get((workload, kernel) + tuple(relax))
    if not t:
        return None
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), t["source"])   # absolute paths stay
    try:
        with open(path, "rb") as f:
            if hashlib.sha1(f.read()).hexdigest() != t["sha1"]:
                return None
    except OSError:
        return None
    return t["bytes"]


def parse(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--workload", choices=["2d", "2d_small", "1d", "batch", "theta"], default="2d",
                   help="2d: 256x256 cells (N=65,536, the benchmark); 2d_small: 128x128 "
                        "(N=16,384, for profiler captures); 1d: 1024 cells; batch: the 256 "
                        "independent 1D/2D instances (N 1024..16384), sharded over the ranks")
    p.add_argument("--batch-count", type=int, default=256)
    p.add_argument("--nd-leaf", type=int, default=None,
                   help="nested dissection: leaf size (library default if unset)")
    p.add_argument("--relax-k", type=int, default=None,
                   help="supernode amalgamation: merge while the width is <= this (library default if unset)")
    p.add_argument("--relax-pct", type=int, default=None,
                   help="supernode amalgamation: or while explicit zeros stay <= this percent")
    p.add_argument("--diag64-min-k", type=int, default=None,
                   help="mixed precision: factor the diagonal blocks of supernodes at least this wide "
                        "in FP64 (library default if unset)")
    p.add_argument("--no-tune", action="store_true",
                   help="keep the default schedule (one launch per level) instead of the tuner's per-level choice")
    p.add_argument("--step-launches", action="store_true",
                   help="factor the pivot columns with a (panel, update) launch pair per 64-column block "
                        "instead of one launch per level")
    p.add_argument("--theta-steps", type=int, default=150,
                   help="theta workload: time steps per factorization")
    p.add_argument("--nrhs", type=int, default=None)
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-fp64", action="store_true")
    p.add_argument("--no-replay", action="store_true",
                   help="skip the profiled replay (per-kernel events)")
    p.add_argument("--cpu-flops", type=float, default=0.0,
                   help="flop budget of the oracle's cpu_baseline sample (0: the whole factorization and "
                        "both substitutions, once)")
    return p.parse_args(argv)


# ---------------------------------------------------------------------------
def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class Dist:
    def __init__(self, backend):
        self.ws, self.rank, self.local = dist_env()
        self.pg = None
        if self.ws > 1:
            import torch.distributed as dist
            dist.init_process_group(backend)
            self.pg = dist

    def barrier(self):
        if self.pg:
            self.pg.barrier()

    def max(self, x: float) -> float:
        if not self.pg:
            return x
        import torch
        t = torch.tensor([x], dtype=torch.float64,
                         device="cuda" if torch.cuda.is_available() else "cpu")
        self.pg.all_reduce(t, op=self.pg.ReduceOp.MAX)
        return float(t.item())

    def sum(self, x: float) -> float:
        if not self.pg:
            return x
        import torch
        t = torch.tensor([x], dtype=torch.float64,
                         device="cuda" if torch.cuda.is_available() else "cpu")
        self.pg.all_reduce(t)
        return float(t.item())

    def close(self):
        if self.pg:
            self.pg.destroy_process_group()


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str | None):
        self.gpu_id = gpu_id
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                   "-lms", "200"]
            if self.gpu_id:
                cmd += ["-i", self.gpu_id]
            self.proc = subprocess.Popen(cmd, stdout=open(self.path, "w"),
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def gpu_id_for_smi():
    try:
        import torch
        u = getattr(torch.cuda.get_device_properties(torch.cuda.current_device()), "uuid", None)
        if u is not None:
            s = str(u)
            return s if s.startswith("GPU-") else "GPU-" + s
    except Exception:
        pass
    v = os.environ.get("CUDA_VISIBLE_DEVICES")
    return v.split(",")[0] if v else None


_UNITS = {}


def device_units():
    """(SM count, maximum SM clock in MHz, where the clock came from) of the
    current device: the SM count from the CUDA device properties, the clock
    from nvidia-smi (clocks.max.sm), else from MEASURED_PEAKS.json."""
    if _UNITS:
        return _UNITS["sms"], _UNITS["mhz"], _UNITS["src"]
    import torch
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    mhz, src = None, None
    try:
        cmd = ["nvidia-smi", "--query-gpu=clocks.max.sm", "--format=csv,noheader,nounits"]
        g = gpu_id_for_smi()
        if g:
            cmd += ["-i", g]
        out = subprocess.run(cmd, capture_output=True, text=True, timeout=20).stdout.split()
        mhz, src = float(out[0]), "nvidia-smi clocks.max.sm"
    except Exception:
        pass
    if mhz is None:
        mhz = load_peaks().get("sm_max_mhz")
        src = "MEASURED_PEAKS.json sm_max_mhz" if mhz else None
    if mhz is None:
        raise RuntimeError("cannot read the maximum SM clock (nvidia-smi and MEASURED_PEAKS.json failed)")
    _UNITS.update(sms=sms, mhz=float(mhz), src=src)
    return sms, float(mhz), src


def cpu_model() -> str:
    """The host CPU's model name (/proc/cpuinfo, else lscpu, else the machine type)."""
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    try:
        for line in subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.machine()


def load_peaks():
    try:
        return json.load(open(PEAKS_FILE))
    except Exception:
        return {}


# ---------------------------------------------------------------------------
def metric_name(args) -> str:
    """The metric of a workload's line, the same for both arms."""
    if args.workload == "batch":
        return "factor+solve TFLOP/s of the batch (mixed+IR path) at backward error <= 1e-12"
    if args.workload == "theta":
        return (f"theta-scheme TFLOP/s (M factored once + {args.theta_steps} steps of product and refined "
                f"solve, mixed+IR) at backward error <= 1e-12")
    return "factor+solve TFLOP/s (mixed+IR path; FP64 path beside it) at backward error <= 1e-12"


def batch_name(args) -> str:
    return f"batch_{args.batch_count}_instances_1d2d_exp_nugget1e-2_1rhs"


def solver_opts(args, **kw):
    """Solver options: the library's defaults unless --nd-leaf / --relax-k / --relax-pct are given."""
    if args.nd_leaf is not None:
        kw["nd_leaf"] = args.nd_leaf
    if args.relax_k is not None:
        kw["relax_k"] = args.relax_k
    if args.relax_pct is not None:
        kw["relax_pct"] = args.relax_pct
    if getattr(args, "diag64_min_k", None) is not None:
        kw["diag64_min_k"] = args.diag64_min_k
    if getattr(args, "step_launches", False):
        kw["step_launches"] = True
    return kw


# ---------------------------------------------------------------------------
def roofline(top, nr, key):
    """Roofline entry of the dominant kernel `top` (its accumulated launches,
    event time and algorithmic flops / bytes from the profiled replay)."""
    peaks = load_peaks()
    name = top["name"]
    sec = top["ms"] / 1e3
    if name.startswith(("tc_schur", "tc_chain")):
        # tcgen05 kind::tf32, three MMAs per product (3xTF32): useful flops
        # against the tf32 rate derived from the measured (sustained) bf16 peak
        bf16 = peaks.get("bf16_tflops_sustained", 1700.0)
        peak = bf16 * TF32_PER_BF16
        ach = top["flops"] / sec / 1e12
        return {"bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                "traffic": measured_traffic(key, name), "kernel": name,
                "peak_source": ("measured bf16 sustained %.1f x nominal tf32/bf16 1.1/2.25" % bf16)
                if "bf16_tflops_sustained" in peaks else "fallback 1700 x nominal tf32/bf16 1.1/2.25",
                "work": ("2 k flops per updated lower entry (the 3xTF32 split's extra MMAs count against it)"
                         if name.startswith("tc_schur") else
                         "sum over 64-column pivot blocks of the pivot-column update (2 nb per updated lower "
                         "entry), the panel (nb^2 per row below) and the diagonal block (2 nb^3 / 3); the "
                         "3xTF32 split's extra MMAs count against it")}
    if name in ("spmv_residual_df", "spmv_residual_df32"):
        # double-float multiply-add: 12 FP32 instructions per (entry, right-hand
        # side) term (4 for the product, 6 for TwoSum, 2 to collect the error
        # terms) plus a 6-instruction renormalisation every 8 terms; the bound
        # is the FP32 lane-operation rate
        terms = top["flops"] / 2.0
        sms, mhz, src = device_units()
        peak = sms * FP32_LANES_PER_SM * mhz * 1e6 / 1e12
        ops = DF_OPS_PER_TERM if name == "spmv_residual_df" else DF32_OPS_PER_TERM
        ach = ops * terms / sec / 1e12
        return {"bound": "alu", "achieved": ach, "peak": peak, "unit": "Tops/s (FP32 lane operations)",
                "frac": ach / peak, "traffic": measured_traffic(key, name), "kernel": name,
                "peak_source": f"derived: {sms} SMs x 128 FP32 lanes x {mhz:.0f} MHz ({src})",
                "work": f"{ops} FP32 operations per stored entry of A and right-hand side"}
    # the FP64 residual product with 8 or more right-hand sides does ~10 flops
    # per byte of A, above GB300's FP64 ridge point: bounded by the FP64 pipe
    alu = name.startswith(("schur_", "panel", "diag_factor", "fwd_xapply", "fwd_bupdate", "bwd_reduce",
                           "bwd_xapply", "sbinv_stage")) or (name.startswith("spmv_residual") and nr >= 8)
    if alu:
        fp64 = name.endswith("_fp64")
        per_clk = FP64_FLOPS_PER_SM_CLK if fp64 else 2 * FP32_LANES_PER_SM
        sms, mhz, src = device_units()
        peak = sms * per_clk * mhz * 1e6 / 1e12
        ach = top["flops"] / sec / 1e12
        return {"bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                "traffic": measured_traffic(key, name), "kernel": name,
                "peak_source": (f"derived: {sms} SMs x 128 FP32 lanes x 2 x {mhz:.0f} MHz ({src})" if not fp64
                                else f"derived: {sms} SMs x 4 FP64 flop/clk x {mhz:.0f} MHz ({src})")}
    peak = peaks.get("hbm_gbs", 6800.0)
    ach = top["bytes"] / sec / 1e9
    return {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
            "traffic": measured_traffic(key, name), "kernel": name,
            "peak_source": "measured" if "hbm_gbs" in peaks else "fallback"}


# ---------------------------------------------------------------------------
def make_workload(kind: str, nrhs: int | None, device: str):
    from wdgen import Kernel, batch_instances, compressed_pattern, compressed_values, haar_basis, rhs

    if kind == "batch":
        # the oracle's sample of the batch: its smallest instance
        p = min(batch_instances(256, 0), key=lambda q: q["N"])
        dim, J, ker, nug, nr = p["dim"], p["J"], Kernel("exponential", p["ell"]), p["nugget"], 1
        name = f"batch_instance_{dim}d_J{J}_exp_l{p['ell']:.3f}"
    elif kind == "2d":
        dim, J, ker, nug, nr = 2, 8, Kernel("matern32", 0.1), 1e-3, 64
        name = "2d_haar_256x256_matern32_l0.1_nugget1e-3"
    elif kind == "theta":
        # the matrix of the theta-scheme, M = I + theta dt K, for K the 2D 256^2 one
        dim, J, ker, nug, nr = 2, 8, Kernel("matern32", 0.1), 1e-3, 1
        name = f"theta_M=I+{THETA * THETA_DT:g}K_2d_haar_256x256_matern32_l0.1_nugget1e-3"
    elif kind == "2d_small":
        dim, J, ker, nug, nr = 2, 7, Kernel("matern32", 0.1), 1e-3, 64
        name = "2d_haar_128x128_matern32_l0.1_nugget1e-3"
    else:
        dim, J, ker, nug, nr = 1, 10, Kernel("exponential", 0.2), 1e-2, 1
        name = "1d_haar_1024_exp_l0.2_nugget1e-2"
    nr = nrhs or nr
    b = haar_basis(dim, J)
    cp, ri = compressed_pattern(b)
    vals = compressed_values(b, cp, ri, ker, nug, device=device)
    if kind == "theta":
        vals = THETA * THETA_DT * vals
        vals[cp[:-1]] += 1.0          # the diagonal is the first entry of every column
    B = rhs(b.N, nr, seed=0)
    return dict(name=f"{name}_{nr}rhs", basis=b, colptr=cp, rowidx=ri, values=vals, B=B, nrhs=nr)


def oracle_sample(w, budget_flops: float, repeats: int = 3, analyze: bool = True):
    """The CPU oracle on one host core: the full analysis (nested dissection
    and symbolic, timed for the record), then either (budget_flops <= 0) the
    whole left-looking FP64 factorization of P A P^T and both substitutions
    for all right-hand sides, once, or a bounded share of them: the factor of
    the first columns up to `budget_flops` of sum c_j^2 (the bottom of the
    elimination tree) and both substitutions over those columns (4 nnz(L
    prefix) nrhs flops), each part timed `repeats` times, the median kept."""
    import numpy as np

    import oracle

    ta = []
    for _ in range(repeats if analyze else 1):
        t = time.perf_counter()
        o = oracle.Oracle(w["colptr"], w["rowidx"], w["basis"])
        ta.append(time.perf_counter() - t)
    c2 = np.cumsum(o.colcount.astype(np.float64) ** 2)
    whole = budget_flops <= 0
    if whole:
        ncols, repeats = o.n, 1
    else:
        ncols = max(1, min(int(np.searchsorted(c2, budget_flops, side="right")), o.n))
    ff = float(c2[ncols - 1])
    nr = int(w["nrhs"])
    fs = 4.0 * float(o.Lp[ncols]) * nr
    B = np.asarray(w["B"], dtype=np.float64).reshape(o.n, -1)[:, :nr]
    Y0 = np.asfortranarray(B[o.perm])
    tf, ts = [], []
    for _ in range(repeats):
        t = time.perf_counter()
        rc = o.factor_prefix(w["values"], ncols)
        tf.append(time.perf_counter() - t)
        if rc != 0:
            raise RuntimeError(f"oracle factor failed: {rc}")
        Y = Y0.copy(order="F")
        t = time.perf_counter()
        o.solve_prefix(Y, ncols)
        ts.append(time.perf_counter() - t)
    mf, ms_, ma = statistics.median(tf), statistics.median(ts), statistics.median(ta)
    return {"value": (ff + fs) / (mf + ms_) / 1e12, "unit": "TFLOP/s", "cores": 1, "kind": "oracle",
            "sample": ((f"one host core, once: the whole left-looking FP64 factorization of P A P^T ({ff:.3e} "
                        f"flop of sum c_j^2) in {mf:.2f} s, then both substitutions with {nr} right-hand sides "
                        f"({fs:.3e} flop) in {ms_:.2f} s") if whole else
                       (f"one host core, median of {repeats}: left-looking FP64 factor of the first {ncols} of "
                        f"{o.n} columns of P A P^T ({ff:.3e} flop of sum c_j^2, bottom of the elimination tree) "
                        f"in {mf:.2f} s, then both substitutions over those columns with {nr} right-hand sides "
                        f"({fs:.3e} flop) in {ms_:.2f} s")),
            "analyze_s": ma if analyze else None, "factor_s": mf, "factor_flops": ff, "solve_s": ms_,
            "solve_flops": fs, "sample_columns": ncols, "repeats": repeats,
            "nproc": os.cpu_count(), "cpu_model": cpu_model(),
            "nnz_L": int(o.nnzL), "flops_factor": float(c2[-1])}


def step_config(args, w, nnz_L: int, flops_factor: float, ws: int) -> dict:
    """The `config` of a single-matrix workload's line, the same for both arms."""
    N = w["basis"].N
    c = {"workload": w["name"], "N": N, "nnz_A": 2 * int(w["rowidx"].size) - N, "nnz_L": int(nnz_L),
         "flops_factor": float(flops_factor), "nrhs": int(w["nrhs"])}
    if args.workload == "theta":
        c.update(theta=THETA, dt=THETA_DT, time_steps=args.theta_steps)
    c["parallelism"] = "replicas" if ws > 1 else "single"
    mb = 4e-6 * nnz_L
    c["l2"] = (("inputs larger than L2 (L alone holds %.1e entries, %.0f MB in FP32)" % (nnz_L, mb))
               if mb > 129 else ("no L2 flush: a small case whose factor (%.0f MB) fits in L2" % mb))
    return c


def run_reference(args):
    """The reference arm: the CPU oracle (this build's FP64 reference), each
    step a bounded sample of the workload's factor + solve on one host core."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    try:
        import torch
        dev = "cuda" if torch.cuda.is_available() else "cpu"
    except Exception:
        dev = "cpu"
    if args.workload == "batch":
        w = make_workload("batch", args.nrhs, dev)
    else:
        w = make_workload(args.workload, args.nrhs, dev)
    budget = args.cpu_flops / 4 if args.cpu_flops > 0 else REF_STEP_FLOPS
    samples = []
    for i in range(args.warmup + args.steps):
        r = oracle_sample(w, budget, repeats=1, analyze=(i == 0))
        if i >= args.warmup:
            samples.append(r)
    tot = sum(r["factor_s"] + r["solve_s"] for r in samples)
    fl = sum(r["factor_flops"] + r["solve_flops"] for r in samples)
    value = fl / tot / 1e12
    last = samples[-1]
    sample = last["sample"].replace("median of 1: ", "per step: ")
    if args.workload == "batch":
        sample = f"{w['name']} (the smallest instance of the batch): " + sample
        config = {"workload": batch_name(args), "instances": args.batch_count,
                  "N_total": int(sum(p["N"] for p in __import__("wdgen").batch_instances(args.batch_count, 0))),
                  "parallelism": "single", "l2": "inputs larger than L2"}
    else:
        config = step_config(args, w, last["nnz_L"], last["flops_factor"], 1)
    cpu = {"value": value, "unit": "TFLOP/s", "cores": 1, "kind": "oracle", "sample": sample,
           "nproc": last["nproc"], "cpu_model": last["cpu_model"]}
    line = {"impl": "reference", "metric": metric_name(args),
            "value": value, "unit": "TFLOP/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": tot / len(samples) * 1e3, "higher_is_better": True,
            "scaling": "strong" if args.workload == "batch" else "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config, "cpu_baseline": cpu,
            "e2e": {"value": value, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
def run_ours(args):
    import numpy as np
    import torch

    import paper_2007_01541_gb300 as wd
    from paper_2007_01541_gb300 import build as wdbuild

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = Dist("nccl")
    wdbuild.build()
    w = make_workload(args.workload, args.nrhs, "cuda")
    N, nr = w["basis"].N, w["nrhs"]
    s = wd.Solver(**solver_opts(args, profile=False)).analyze(w["colptr"], w["rowidx"], w["basis"])
    sp = None if args.no_replay else wd.Solver(**solver_opts(args, profile=True)).analyze(
        w["colptr"], w["rowidx"], w["basis"])
    info = s.info()
    flops_factor = info["flops_factor"]
    flops_solve = 4.0 * info["nnz_L"] * nr
    flops_step = flops_factor + flops_solve
    vals = torch.from_numpy(w["values"]).cuda()
    B0 = torch.from_numpy(np.ascontiguousarray(w["B"].T)).cuda()   # (nrhs, N) = column-major B
    Bw = torch.empty_like(B0)
    stream = torch.cuda.current_stream()
    # per-level schedule of the mixed factorization, chosen by measurement
    # (or taken from the tuner's cache) before anything is timed
    tuned = None
    if not args.no_tune:
        from paper_2007_01541_gb300 import tune
        t_tune = time.perf_counter()
        tuned = tune.tune_schedule(s, vals)
        tuned["tuning_s"] = time.perf_counter() - t_tune
        if sp is not None:
            sp.set_level_schedule(tuned["schedule"])

    phase = {"factor": 0.0, "solve": 0.0, "logdet": 0.0}

    def step(sv, prec, record=False):
        t0 = time.perf_counter()
        sv.factor(vals, prec)
        t1 = time.perf_counter()
        Bw.copy_(B0)
        sv.solve(Bw.T)
        t2 = time.perf_counter()
        sv.logdet()
        t3 = time.perf_counter()
        if record:
            phase["factor"] += t1 - t0
            phase["solve"] += t2 - t1
            phase["logdet"] += t3 - t2

    def timed(sv, prec, K, W):
        for _ in range(W):
            step(sv, prec)
        sv.kernel_stats(reset=True)
        sv.launch_count(reset=True)
        dist.barrier()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        for key in phase:
            phase[key] = 0.0
        e0.record(stream)
        for _ in range(K):
            step(sv, prec, record=True)
        e1.record(stream)
        torch.cuda.synchronize()
        dist.barrier()
        ms = e0.elapsed_time(e1) / K
        ph = {k: round(v / K * 1e3, 3) for k, v in phase.items()}
        return (dist.max(ms), sv.kernel_stats(reset=True), sv.launch_count(reset=True),
                dict(sv.last_solve, phases_ms=ph))

    # headline: graphs replayed with no per-kernel events
    clocks = ClockSampler(gpu_id_for_smi())
    clocks.start()
    ms_mixed, _, launches, solve_info = timed(s, "mixed", args.steps, args.warmup)
    clk = clocks.stop()
    # the same steps again with CUDA events around every kernel launch
    ms_mixed_prof, kstats = None, []
    if not args.no_replay:
        ms_mixed_prof, kstats, _, _ = timed(sp, "mixed", args.steps, 1)
    res_fp64 = None
    if not args.no_fp64:
        ms64, _, _, si64 = timed(s, "fp64", max(2, args.steps // 2), 2)
        kst64 = [] if args.no_replay else timed(sp, "fp64", 1, 1)[1]
        res_fp64 = {"ms_per_step": ms64,
                    "tflops": dist.sum(flops_step) / (ms64 / 1e3) / 1e12,
                    "backward_error": si64["backward_error"], "phases_ms": si64["phases_ms"],
                    "top_kernels": _top(kst64, 4)}
        # the FP64 factorization with its Schur updates on the tensor cores
        # (bf16 slices): same arithmetic bar, no refinement
        s_tc = wd.Solver(**solver_opts(args, profile=False), fp64_tc_schur=True).analyze(
            w["colptr"], w["rowidx"], w["basis"])
        ms64t, _, _, si64t = timed(s_tc, "fp64", max(2, args.steps // 2), 2)
        kst64t = []
        if not args.no_replay:
            sp_tc = wd.Solver(**solver_opts(args, profile=True), fp64_tc_schur=True).analyze(
                w["colptr"], w["rowidx"], w["basis"])
            kst64t = timed(sp_tc, "fp64", 1, 1)[1]
            sp_tc.close()
        s_tc.close()
        res_fp64["tensor_core_updates"] = {
            "ms_per_step": ms64t, "tflops": dist.sum(flops_step) / (ms64t / 1e3) / 1e12,
            "backward_error": si64t["backward_error"], "phases_ms": si64t["phases_ms"],
            "speedup_vs_fp64": ms64 / ms64t, "top_kernels": _top(kst64t, 4)}
    value = dist.sum(flops_step) / (ms_mixed / 1e3) / 1e12

    # roofline of the dominant kernel of the mixed step
    top = max(kstats, key=lambda k: k["ms"]) if kstats else None
    roof = None
    if top:
        roof = roofline(top, nr, (args.workload, amalgamation(args)))
        roof["launches_per_step"] = top["launches"] / args.steps
        roof["ms_per_launch"] = top["ms"] / max(1, top["launches"])
        roof["timing"] = ("CUDA events around every launch of this kernel during a profiled "
                          "replay of the timed steps (%.2f ms/step with events)" % ms_mixed_prof)

    # end to end through the C ABI with pinned host buffers
    e2e = None
    if not args.no_e2e:
        vh = torch.from_numpy(w["values"]).pin_memory()
        Bh0 = torch.from_numpy(np.ascontiguousarray(w["B"].T)).pin_memory()
        Bh = torch.empty_like(Bh0).pin_memory()

        def step_host():
            s.factor(vh, "mixed")
            Bh.copy_(Bh0)
            s.solve(Bh.T)
            s.logdet()

        for _ in range(2):
            step_host()
        dist.barrier()
        torch.cuda.synchronize()
        t = time.perf_counter()
        for _ in range(args.steps):
            step_host()
        torch.cuda.synchronize()
        dt = dist.max((time.perf_counter() - t) / args.steps)
        e2e = {"value": dist.sum(flops_step) / dt / 1e12, "unit": "TFLOP/s",
               "h2d_bytes_per_step": 8 * int(w["rowidx"].size) + 8 * N * nr,
               "d2h_bytes_per_step": 8 * N * nr + 8 + 8 * 3 * nr * (1 + solve_info["iterations"]),
               "ms_per_step": dt * 1e3}

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = oracle_sample(w, args.cpu_flops)

    if rank == 0:
        line = {
            "metric": metric_name(args),
            "value": value, "unit": "TFLOP/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_mixed, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": step_config(args, w, info["nnz_L"], flops_factor, ws),
            "schedule": (None if tuned is None else
                         {"per_level_launch_pairs": tuned["schedule"], "tuner_ms_tuned": tuned["ms"],
                          "tuner_ms_all_tasks": tuned["ms_default"], "from_cache": tuned["cached"],
                          "tuning_s": tuned["tuning_s"]}),
            "front_pool_gb": info["front_bytes"] / 1e9,
            "backward_error": solve_info["backward_error"], "ir_iterations": solve_info["iterations"],
            "phases_ms": solve_info["phases_ms"],
            "fp64": res_fp64,
            "speedup_mixed_vs_fp64": (res_fp64["ms_per_step"] / ms_mixed) if res_fp64 else None,
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
            "clocks": clk, "top_kernels": _top(kstats, 12),
            "analyze_s": info["analyze_seconds"],
        }
        print(json.dumps(line), flush=True)
    dist.close()


def _oracle_instance_worker(spec, barrier):
    """One batch instance in one host process: build it, wait for the other
    processes, then time the oracle's factorization."""
    import time as _time

    import torch

    import oracle
    from wdgen import Kernel, compressed_pattern, compressed_values, haar_basis

    torch.set_num_threads(1)
    b = haar_basis(spec["dim"], spec["J"])
    cp, ri = compressed_pattern(b)
    v = compressed_values(b, cp, ri, Kernel("exponential", spec["ell"]), spec["nugget"])
    o = oracle.Oracle(cp, ri, b)
    flops = float((o.colcount.astype("float64") ** 2).sum())
    barrier.wait(timeout=600)
    t = _time.perf_counter()
    rc = o.factor(v)
    return flops, _time.perf_counter() - t, rc


def batch_cpu_baseline(params, costs, workers: int):
    """The oracle on `workers` host processes at once, one instance each: the
    most expensive instances (those that carry the batch's work), all factored
    concurrently after a barrier; throughput = their flops / the slowest
    process's factorization time.  Processes are spawned (never forked)."""
    import multiprocessing as mp

    order = sorted(range(len(params)), key=lambda i: (-costs[i], i))[:max(1, workers)]
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        barrier = mgr.Barrier(len(order))
        with ctx.Pool(processes=len(order)) as pool:
            res = pool.starmap(_oracle_instance_worker, [(params[i], barrier) for i in order])
    if any(r[2] != 0 for r in res):
        return None
    fl = sum(r[0] for r in res)
    tmax = max(r[1] for r in res)
    return {"value": fl / tmax / 1e12, "unit": "TFLOP/s", "cores": len(order), "kind": "oracle",
            "per_process": sum(r[0] / r[1] for r in res) / len(res) / 1e12,
            "sample": (f"{len(order)} instances (the most expensive: {sorted(set((params[i]['dim'], params[i]['J']) for i in order))} "
                       f"as (dim, J)), one per host process, left-looking FP64 factor run concurrently: "
                       f"{fl:.3e} flop in {tmax:.2f} s (slowest process); solve not sampled")}


def run_theta(args):
    """Repeated solves of the theta-scheme (Section 5, Eq. (theta), G = I):
    M = I + theta dt K (K the 2D 256^2 compressed matrix) is factored once,
    then --theta-steps steps each form (1/theta) U - ((1-theta)/theta) M U +
    dt F and solve with M, refined to backward error <= 1e-12
    (wd_theta_step).  One bench step = the factorization plus all time steps;
    value = (sum_j c_j^2 + steps (4 nnz(L) + 2 nnz(A)) nrhs) / its time."""
    import numpy as np
    import torch

    import paper_2007_01541_gb300 as wd
    from paper_2007_01541_gb300 import build as wdbuild
    from wdgen import rhs

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = Dist("nccl")
    wdbuild.build()
    w = make_workload("theta", args.nrhs, "cuda")
    N, nr, T = w["basis"].N, w["nrhs"], args.theta_steps
    s = wd.Solver(**solver_opts(args)).analyze(w["colptr"], w["rowidx"], w["basis"])
    sp = None if args.no_replay else wd.Solver(**solver_opts(args, profile=True)).analyze(
        w["colptr"], w["rowidx"], w["basis"])
    info = s.info()
    nnz_a = 2 * int(w["rowidx"].size) - N
    flops_step = info["flops_factor"] + T * (4.0 * info["nnz_L"] + 2.0 * nnz_a) * nr
    vals = torch.from_numpy(w["values"]).cuda()
    U0 = torch.from_numpy(np.ascontiguousarray(w["B"].T)).cuda()       # (nrhs, N): U0.T column-major
    F = torch.from_numpy(np.ascontiguousarray(rhs(N, nr, seed=1).T)).cuda()
    Uw = torch.empty_like(U0)
    stream = torch.cuda.current_stream()

    def job(sv):
        sv.factor(vals, "mixed")
        Uw.copy_(U0)
        for _ in range(T):
            sv.theta_step(Uw.T, F.T, theta=THETA, dt=THETA_DT)

    def timed(sv, K, W):
        for _ in range(W):
            job(sv)
        sv.kernel_stats(reset=True)
        sv.launch_count(reset=True)
        dist.barrier()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(K):
            job(sv)
        e1.record(stream)
        torch.cuda.synchronize()
        dist.barrier()
        return dist.max(e0.elapsed_time(e1) / K), sv.kernel_stats(reset=True), sv.launch_count(reset=True)

    clocks = ClockSampler(gpu_id_for_smi())
    clocks.start()
    ms, _, launches = timed(s, args.steps, args.warmup)
    clk = clocks.stop()
    be, its = s.last_solve["backward_error"], s.last_solve["iterations"]
    # the factorization alone, to report the time of one step
    f0 = torch.cuda.Event(enable_timing=True)
    f1 = torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    for _ in range(args.steps):
        s.factor(vals, "mixed")
    f1.record(stream)
    torch.cuda.synchronize()
    ms_factor = dist.max(f0.elapsed_time(f1) / args.steps)
    kstats = [] if args.no_replay else timed(sp, args.steps, 1)[1]
    value = dist.sum(flops_step) / (ms / 1e3) / 1e12
    roof = None
    top = max(kstats, key=lambda k: k["ms"]) if kstats else None
    if top:
        roof = roofline(top, nr, ("theta", amalgamation(args)))
        roof["launches_per_step"] = top["launches"] / args.steps
        roof["ms_per_launch"] = top["ms"] / max(1, top["launches"])
    e2e = None
    if not args.no_e2e:
        vh = torch.from_numpy(w["values"]).pin_memory()
        Uh0 = torch.from_numpy(np.ascontiguousarray(w["B"].T)).pin_memory()
        Fh = F.cpu().pin_memory()
        Uh = torch.empty_like(Uh0).pin_memory()

        def job_host():
            s.factor(vh, "mixed")
            Uh.copy_(Uh0)
            for _ in range(T):
                s.theta_step(Uh.T, Fh.T, theta=THETA, dt=THETA_DT)

        job_host()
        dist.barrier()
        torch.cuda.synchronize()
        t = time.perf_counter()
        for _ in range(max(1, args.steps // 2)):
            job_host()
        torch.cuda.synchronize()
        dt = dist.max((time.perf_counter() - t) / max(1, args.steps // 2))
        e2e = {"value": dist.sum(flops_step) / dt / 1e12, "unit": "TFLOP/s",
               "h2d_bytes_per_step": 8 * int(w["rowidx"].size) + T * 2 * 8 * N * nr,
               "d2h_bytes_per_step": T * 8 * N * nr, "ms_per_step": dt * 1e3}
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = oracle_sample(w, args.cpu_flops)
    if rank == 0:
        line = {"metric": metric_name(args),
                "value": value, "unit": "TFLOP/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": ms, "ms_factor": ms_factor, "ms_per_theta_step": (ms - ms_factor) / T, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
                "config": step_config(args, w, info["nnz_L"], info["flops_factor"], ws),
                "front_pool_gb": info["front_bytes"] / 1e9,
                "backward_error": be, "ir_iterations_last_step": its,
                "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
                "clocks": clk, "top_kernels": _top(kstats, 12)}
        print(json.dumps(line), flush=True)
    dist.close()


def run_batch(args):
    """Independent instances, one right-hand side each, mixed precision with
    refinement.  Ranks take their longest-processing-time shares of the
    instances (no data-path collective); value = all instances' factor + solve
    flops over the slowest rank's time (the total work is fixed: strong scaling)."""
    import numpy as np
    import torch

    import paper_2007_01541_gb300 as wd
    from paper_2007_01541_gb300 import build as wdbuild
    from paper_2007_01541_gb300.shard import instance_costs, lpt_partition
    from wdgen import batch_instances, batch_workload, compressed_pattern, haar_basis

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = Dist("nccl")
    wdbuild.build()
    params = batch_instances(args.batch_count, 0)
    cache = {}
    pats, bases = [], []
    for p in params:
        key = (p["dim"], p["J"])
        if key not in cache:
            b = haar_basis(*key)
            cache[key] = (b, compressed_pattern(b))
        bases.append(cache[key][0])
        pats.append(cache[key][1])
    costs = instance_costs(pats, bases)
    idx = lpt_partition(costs, ws)[rank]
    w = batch_workload(params=[params[i] for i in idx], nrhs=1, seed=rank, device="cuda")
    s = wd.Solver(**solver_opts(args)).analyze_batch(w.patterns, w.bases)
    sp = None if args.no_replay else wd.Solver(**solver_opts(args, profile=True)).analyze_batch(w.patterns,
                                                                                              w.bases)
    info = s.info()
    flops_step = info["flops_factor"] + 4.0 * info["nnz_L"]
    vals = torch.tensor(np.concatenate(w.values), device="cuda")
    B0 = torch.tensor(np.ascontiguousarray(w.B.T), device="cuda")
    Bw = torch.empty_like(B0)
    stream = torch.cuda.current_stream()

    def step(sv):
        sv.factor(vals, "mixed")
        Bw.copy_(B0)
        sv.solve(Bw.T)
        sv.logdet_batch()

    def timed(sv, K, W):
        for _ in range(W):
            step(sv)
        sv.kernel_stats(reset=True)
        sv.launch_count(reset=True)
        dist.barrier()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(K):
            step(sv)
        e1.record(stream)
        torch.cuda.synchronize()
        dist.barrier()
        return dist.max(e0.elapsed_time(e1) / K), sv.kernel_stats(reset=True), sv.launch_count(reset=True)

    clocks = ClockSampler(gpu_id_for_smi())
    clocks.start()
    ms, _, launches = timed(s, args.steps, args.warmup)
    clk = clocks.stop()
    be = s.last_solve["backward_error"]
    kstats = [] if args.no_replay else timed(sp, args.steps, 1)[1]
    total = dist.sum(flops_step)
    value = total / (ms / 1e3) / 1e12
    roof = None
    top = max(kstats, key=lambda k: k["ms"]) if kstats else None
    if top:
        roof = roofline(top, 1, ("batch", amalgamation(args)))
        roof["launches_per_step"] = top["launches"] / args.steps
    e2e = None
    if not args.no_e2e:
        vh = torch.tensor(np.concatenate(w.values)).pin_memory()
        Bh0 = torch.tensor(np.ascontiguousarray(w.B.T)).pin_memory()
        Bh = torch.empty_like(Bh0).pin_memory()

        def step_host():
            s.factor(vh, "mixed")
            Bh.copy_(Bh0)
            s.solve(Bh.T)
            s.logdet_batch()

        for _ in range(2):
            step_host()
        dist.barrier()
        t = time.perf_counter()
        for _ in range(args.steps):
            step_host()
        torch.cuda.synchronize()
        dt = dist.max((time.perf_counter() - t) / args.steps)
        n_loc = int(w.B.shape[0])
        e2e = {"value": total / dt / 1e12, "unit": "TFLOP/s",
               "h2d_bytes_per_step": 8 * int(vals.numel()) + 8 * n_loc,
               "d2h_bytes_per_step": 8 * n_loc + 8 * len(idx), "ms_per_step": dt * 1e3}
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = batch_cpu_baseline(params, costs, os.cpu_count() or 1)
    if rank == 0:
        line = {"metric": metric_name(args),
                "value": value, "unit": "TFLOP/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": ms, "higher_is_better": True, "scaling": "strong", "vs_baseline": None,
                "dtype": "f32+f64", "data": "synthetic",
                "config": {"workload": batch_name(args),
                           "instances": args.batch_count, "N_total": int(sum(p["N"] for p in params)),
                           "parallelism": f"lpt-shards x{ws}" if ws > 1 else "single",
                           "l2": "inputs larger than L2"},
                "backward_error": be, "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": launches, "clocks": clk, "top_kernels": _top(kstats, 8)}
        print(json.dumps(line), flush=True)
    dist.close()


def _top(kstats, n):
    out = []
    for k in sorted(kstats, key=lambda k: -k["ms"])[:n]:
        out.append({"name": k["name"], "ms": round(k["ms"], 3), "launches": k["launches"],
                    "tflops": k["flops"] / max(k["ms"], 1e-9) / 1e9,
                    "gbs": k["bytes"] / max(k["ms"], 1e-9) / 1e6})
    return out


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch":
        run_batch(args)
    elif args.workload == "theta":
        run_theta(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
