"""Benchmark: space-time DOF * cycles / s of the multigrid waveform-relaxation solve.

Workload (default): 1D time-fractional heat equation, N = 4095 interior points, M = 4096 graded
time steps, alpha = 0.5, gamma = (2 - alpha)/alpha, H-matrix with leaf 64 and recompression
tolerance 1e-10, manufactured u = t^alpha sin(pi x), zero initial guess, V(1,1) cycles until the
max-norm residual drops by 1e-8.  One step = one complete solve (all hot-path kernels: smoother
half-sweeps, residual + restriction, prolongation, coarsest solve, residual norms).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--alpha A]

value       = DOF * cycles summed over the K timed solves / device time (CUDA events, max over
              ranks), DOF = N * M.  Inputs (u, f: 134 MB each) exceed the 129 MB L2.
e2e         = the same metric through fhmg_solve_host with pinned host buffers (the H2D copy of u
              and f and the D2H copy of u inside the timed region).
roofline    = the finest-grid smoother kernel (the dominant launch), FP64-ALU bound: algorithmic
              FP64 flops per launch / its CUDA-event time, against 152 SMs x 2 DFMA/clk x 2 flop
              x 2.07 GHz = 1.258 TFLOP/s.
cpu_baseline / --impl reference = the CPU oracle's direct solve (implicit time stepping with the
              dense L1 history sum) on the host cores, expressed as DOF * (the GPU's cycle count)
              / s so that the ratio is a time-to-solution ratio.
N > 1 (torchrun): replicas only -- every rank solves its own instance, no collective on the data
path; value is the sum over ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12     # 1.258, DFMA units x clock
MEASURED_DFMA_TFLOPS = 1.202                        # dependent-free DFMA loop on this machine's GB300
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12   # 80.5, FFMA units x clock (a loop measured 75.1)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--alpha", type=float, default=0.5)
    ap.add_argument("--N", type=int, default=4095)
    ap.add_argument("--M", type=int, default=4096)
    ap.add_argument("--rtol", type=float, default=1e-8)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    return ap.parse_args()


def workload(a):
    gamma = (2 - a.alpha) / a.alpha
    return {"workload": f"1D H-matrix FP64, N={a.N}, M={a.M}, alpha={a.alpha}, gamma={gamma:.4g}, "
                        f"leaf 64, tol 1e-10, V(1,1) to relres {a.rtol:g}",
            "dim": 1, "N": a.N, "M": a.M, "alpha": a.alpha, "gamma": gamma, "leaf": 64, "tol": 1e-10,
            "cycle": "V(1,1)", "rtol": a.rtol, "source": "manufactured t^alpha sin(pi x)",
            "l2": "inputs larger than L2 (u, f 134 MB each)"}


class Clocks:
    """nvidia-smi sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.file, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        self.proc.wait()
        self.file.seek(0)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.file.read().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.file.name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup(a):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if ws > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        dist.init_process_group("nccl")
        return dist, rank, ws
    return None, 0, 1


def oracle_direct_sample(a, cores_env=None):
    """Times the oracle's direct solve of the full workload (dense R history, O1)."""
    import numpy as np
    from oracle import direct, l1
    from paper_1706_07632_gb300 import inputs
    gamma = (2 - a.alpha) / a.alpha
    t0 = time.perf_counter()
    t = l1.graded_mesh(1.0, a.M, gamma)
    R = l1.l1_matrix(t, a.alpha)
    t_build = time.perf_counter() - t0
    amp, s = inputs.manufactured(t[1:], a.N, 1, a.alpha)
    F = np.outer(amp, s)
    t0 = time.perf_counter()
    direct.solve_o1(R, F, 1.0 / (a.N + 1))
    t_solve = time.perf_counter() - t0
    return t_solve, t_build


def run_reference(a):
    """--impl reference: the CPU oracle on the host cores (rank 0 only)."""
    dist, rank, ws = dist_setup(a)
    if rank != 0:
        return
    # the cycle unit of the metric: FP64 V(1,1) cycles to 1e-8 measured on GB300 for the default
    # workload (other workloads: set FHMG_REF_CYCLES)
    cyc = int(os.environ.get("FHMG_REF_CYCLES", "8"))
    dof = a.N * a.M
    for _ in range(max(0, min(a.warmup, 1))):
        oracle_direct_sample(a)
    times = []
    for _ in range(a.steps):
        ts, tb = oracle_direct_sample(a)
        times.append(ts)
    tot = sum(times)
    value = dof * cyc * a.steps / tot
    cores = os.cpu_count()
    line = {"impl": "reference", "metric": "space-time DOF*cycles/s (time-to-1e-8 solve)", "value": value,
            "unit": "DOF*cycles/s", "n_gpus": a.gpus, "steps": a.steps, "warmup": a.warmup,
            "ms_per_step": 1e3 * tot / a.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic", "config": workload(a),
            "cpu_baseline": {"value": value, "unit": "DOF*cycles/s", "cores": cores, "kind": "oracle",
                             "sample": f"full direct solve N={a.N} M={a.M} (implicit time stepping, dense L1 history, "
                                       f"numpy/OpenBLAS); DOF*cycles with {cyc} cycles = the GPU FP64 count"},
            "e2e": {"value": value, "unit": "DOF*cycles/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def timed_solves(P, f, a, stream, rank, dist):
    """W untimed + K timed solves from u = 0 on one problem; CUDA events on the launching stream."""
    import torch
    u = torch.zeros_like(f)
    for _ in range(a.warmup):
        u.zero_()
        P.solve(u, f, None, 1, 1, a.rtol, 80)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    P.profile(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    cycles, rr_last = 0, None
    e0.record(stream)
    for _ in range(a.steps):
        u.zero_()
        k, rr_last = P.solve(u, f, None, 1, 1, a.rtol, 80)
        cycles += k
    e1.record(stream)
    torch.cuda.synchronize()
    cnt = P.counters()
    P.profile(False)
    if dist:
        dist.barrier()
    return e0.elapsed_time(e1), cycles, rr_last, cnt, u


def main():
    a = parse()
    if a.impl == "reference":
        return run_reference(a)
    import torch

    import __graft_entry__
    __graft_entry__.build()
    import paper_1706_07632_gb300 as fh
    from paper_1706_07632_gb300 import inputs

    dist, rank, ws = dist_setup(a)
    dev = torch.device("cuda", torch.cuda.current_device())
    gamma = (2 - a.alpha) / a.alpha
    t_h0 = time.perf_counter()
    H = fh.HMatrix(a.alpha, gamma, 1.0, a.M, 64, 0, 1e-10)
    t_hbuild = time.perf_counter() - t_h0
    stream = torch.cuda.current_stream()
    tmesh, _ = H.mesh()
    amp, s = inputs.manufactured(tmesh[1:], a.N, 1, a.alpha)
    f = torch.as_tensor(amp, device=dev)[:, None] * torch.as_tensor(s, device=dev)[None, :]
    dof = a.N * a.M

    clocks = Clocks(torch.cuda.current_device()) if rank == 0 else None
    res = {}
    for name, prec in (("fp64", fh.FP64), ("mixed", fh.MIXED_FP32)):
        P = fh.Problem(H, 1, a.N, 1.0, prec, stream)
        ms, cycles, rr, cnt, u = timed_solves(P, f, a, stream, rank, dist)
        if dist:
            mx = torch.tensor([ms], device=dev)
            dist.all_reduce(mx, op=dist.ReduceOp.MAX)
            ms = float(mx[0])
        res[name] = {"P": P, "ms": ms, "cycles": cycles, "relres": rr, "cnt": cnt}
    clk = clocks.stop() if clocks else None

    # common cycle unit: the FP64 V(1,1) cycle count of this workload
    k_ref = res["fp64"]["cycles"] / a.steps
    for name in res:
        r = res[name]
        r["time_to_rtol_s"] = r["ms"] / a.steps / 1e3
        r["value"] = dof * k_ref * ws / r["time_to_rtol_s"]
    head = res["mixed"]
    value = head["value"]

    def roofline(r, kind):
        c = r["cnt"]
        flops_launch = H.flops_per_column() * (a.N / 2.0)
        sm_ms = c["smooth_ms"] / max(c["smooth_launches"], 1)
        achieved = flops_launch / (sm_ms / 1e3) / 1e12
        if kind == "fp64":
            peak, note = FP64_PEAK_TFLOPS, "152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz (a DFMA loop measured 1.202)"
            kern = "hwalk_kernel<double,double,64,*,SMOOTH> (finest-grid half-sweep)"
        else:
            peak, note = FP32_PEAK_TFLOPS, "152 SMs x 128 FFMA/clk x 2 flop x 2.07 GHz (an FFMA loop measured 75.1)"
            kern = "hwalk_kernel<double,float,64,*,SMOOTH> (finest-grid half-sweep, FP32 products)"
        return {"kernel": kern, "bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "peak_note": note, "traffic": None, "avg_launch_ms": sm_ms,
                "launches_timed": c["smooth_launches"], "algorithmic_flops_per_launch": flops_launch,
                "share_of_step": c["smooth_ms"] / r["ms"] if r["ms"] > 0 else None}

    # end to end through the C-ABI with host buffers (headline path)
    e2e = None
    if not a.no_e2e:
        P = head["P"]
        fh_host = f.cpu().pin_memory()
        uh = torch.zeros(f.shape, dtype=torch.float64).pin_memory()
        P.solve_host(uh, fh_host, None, 1, 1, a.rtol, 80)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(a.steps):
            uh.zero_()
            P.solve_host(uh, fh_host, None, 1, 1, a.rtol, 80)
        te = time.perf_counter() - t0
        e2e = {"value": dof * k_ref * ws * a.steps / te, "unit": "DOF*cycles/s", "h2d_bytes_per_step": 2 * dof * 8,
               "d2h_bytes_per_step": dof * 8, "ms_per_step": 1e3 * te / a.steps}

    cpu = None
    if rank == 0 and not a.no_cpu_baseline:
        ts, tb = oracle_direct_sample(a)
        cpu = {"value": dof * k_ref / ts, "unit": "DOF*cycles/s", "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"full direct solve of this workload (N={a.N}, M={a.M}), implicit time stepping with the "
                         f"dense L1 history sum, numpy/OpenBLAS on all host threads: {ts:.2f} s (+{tb:.2f} s to "
                         f"build R, not timed); cycles = the FP64 V(1,1) count to 1e-8 ({k_ref:.0f})"}

    if rank == 0:
        def summary(r):
            return {"value": r["value"], "time_to_rtol_s": r["time_to_rtol_s"], "cycles_per_solve": r["cycles"] / a.steps,
                    "relres": r["relres"], "gpu_launches_per_solve": r["cnt"]["launches"] / a.steps}
        line = {"metric": "space-time DOF*cycles/s (time-to-1e-8 solve)", "value": value, "unit": "DOF*cycles/s",
                "n_gpus": ws, "steps": a.steps, "warmup": a.warmup, "ms_per_step": head["ms"] / a.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64+f32",
                "data": "synthetic", "config": workload(a),
                "headline": "mixed: FP64 defect correction, FP32 H-matrix products in the V-cycles",
                "cycle_unit": f"FP64 V(1,1) cycles to relres {a.rtol:g} on this workload = {k_ref:.0f}",
                "fp64": summary(res["fp64"]), "mixed": summary(res["mixed"]),
                "speedup_mixed_vs_fp64": res["fp64"]["time_to_rtol_s"] / res["mixed"]["time_to_rtol_s"],
                "hbuild_s": t_hbuild, "roofline": roofline(res["mixed"], "mixed"),
                "roofline_fp64": roofline(res["fp64"], "fp64"), "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": head["cnt"]["launches"], "clocks": clk}
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
