"""Benchmark: time-to-1e-8 solves of multigrid waveform relaxation for the time-fractional heat
equation, mixed precision + learned warm start against plain FP64, on one GB300.

Headline workload (the learned-warm-start configuration): 2D unit square, N = 1023^2 interior
points, M = 512 graded time steps (gamma = 2), alpha = 0.55, H-matrix leaf 64 with recompression
tolerance 1e-10, source = a Gaussian random field (length scale 0.1) drawn as a 2D sine series,
constant in time; V(1,1) cycles until the max-norm defect is <= 1e-8 max|F| (the same absolute
target for every initial guess); the coarse-grid correction on the 31^2 level is solved exactly.
One step = one complete warm-started solve: the network's prediction of the initial iterate
(projection, BF16 inference, synthesis) and the mixed-precision solve from it (defect correction:
FP64-accurate double-float outer defects around V-cycles with FP32 storage whose H-matrix products
run in BF16 on the tcgen05 tensor cores with FP32 accumulation in tensor memory).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--quick]

value     = DOF * K_ref * ranks / (device time per step), DOF = N^2 M, K_ref = the FP64 path's V(1,1)
            cycle count on the headline source: every arm is expressed in FP64-cycle equivalents,
            so values compare time to solution.  Arms beside it: plain FP64 from zero, mixed (BF16
            products) from zero, each the median of >= 5 timed solves, and the mixed form with FP32
            products (3xTF32 mma.sync) from zero (median of 3); err_vs_oracle of every arm at 4096
            sampled grid points against the per-mode oracle.
sources   = 16 unseen GRF sources with alpha ~ U[.3, .8]: cycles and time from zero and from the
            warm start, and the error against the per-mode oracle, per source.
e2e       = the same metric through fhmg_ws_solve_host (pinned host buffers: f in, u out, inside
            the timed region).
roofline  = the dominant kernel of the headline step (the finest-grid smoother half-sweeps or the
            outer defect, whichever takes the larger share), timed live with CUDA events on the
            launching stream inside the timed steps; the other one: roofline_secondary.  Peaks:
            the measured copy bandwidth and the sustained BF16 rate (MEASURED_PEAKS.json).
cpu_baseline / --impl reference = the oracle's direct solver (implicit time stepping with the dense
            L1 history sum and a DST-I spatial solve per step, numpy/scipy) on the host cores, on the
            first time levels of the headline workload (a bounded sample).
Secondary workloads (keys workload_1d, workload_2d, workload_batched): 1D N=4095, M=4096,
alpha=0.5; 2D N=511^2, M=1024, alpha=0.4; 64 batched 1D instances.
N > 1 (torchrun): replicas only -- each rank solves its own instance; no data-path collective.
Inputs (u, f: 4.3 GB each) exceed the 129 MB L2.
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

FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12     # 1.258: DFMA units x clock (a DFMA loop measured 1.202)
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12   # 80.5: FFMA units x clock (an FFMA loop measured 75.1)
# double-float multiply-add = 11 FP32 instructions (TwoProd by FMA, two cross-term FMAs, TwoSum,
# low-word update): 2 algorithmic flops per 11 FP32 lane-instructions
DF_PEAK_TFLOPS = 152 * 128 * 2.07e9 * 2 / 11 / 1e12  # 7.32
HEAD = dict(dim=2, N=1023, M=512, alpha=0.55, gamma=2.0, seed=999, K=24, nc=31)
METRIC = "space-time DOF*cycles/s (time-to-1e-8 solve): mixed+warm-start vs plain FP64"
# DRAM bytes per column of one launch at M time levels, from the ncu captures named beside each
# (same kernels and tiles on the 2D 255^2 x 512 case, scaled by columns); traffic is reported as
# null for another M, and the entries are dropped whenever the kernel they describe changes
TRAFFIC_PER_COLUMN = {
    "smooth": (512, 349.2e6 / 32513),                     # profiles/humma_smooth_2d_255x512.md
    "defect": (512, (770.95e6 + 770.24e6) / 65025),       # profiles/split_defect_2d_255x512.md (both kernels)
}


def traffic(kind, M, ncols):
    e = TRAFFIC_PER_COLUMN.get(kind)
    return e[1] * ncols if e and e[0] == M else None


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--rtol", type=float, default=1e-8)
    ap.add_argument("--sources", type=int, default=16, help="unseen GRF sources of the warm-start sweep")
    ap.add_argument("--quick", action="store_true", help="headline only (no sweep, secondary workloads, CPU baseline)")
    ap.add_argument("--grid", type=int, default=1023,
                    help="interior points per dimension of the headline grid (2^k - 1; 1023 is the workload; smaller "
                         "grids serve profiling captures that must stay small)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the heuristic column tiles (deterministic kernel choice, e.g. for profiling)")
    return ap.parse_args()


def peaks():
    """HBM copy bandwidth and the BF16 dense rate sustained over seconds (the kernels are timed inside
    a long step): the measured figures, else the fallback ones."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), float(d.get("bf16_tflops_sustained", d["bf16_tflops"])), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, 1700.0, "fallback"


class Clocks:
    """nvidia-smi sampling during the timed work."""

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
                "reasons": sorted(reasons), "samples": len(sm),
                "span": "every workload of the run (headline, sweep, secondary workloads)"}


def dist_setup():
    """Rank, world size and the process group of a torchrun launch (replicas only: the group is
    used for the barrier and the max-over-ranks timing, never on the data path).  NCCL between
    GPUs; gloo when no GPU is visible (host-only runs of the multi-process tests).  Idempotent."""
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if ws > 1:
        import torch
        import torch.distributed as dist
        if not dist.is_initialized():
            if torch.cuda.is_available():
                torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
                dist.init_process_group("nccl")
            else:
                dist.init_process_group("gloo")
        return dist, rank, ws
    return None, 0, 1


def max_over_ranks(x, dist):
    """The largest value of x over all ranks (the timing rule: the slowest rank sets the time)."""
    if not dist:
        return x
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t[0])


def job_value(units_per_rank, ranks, seconds):
    """Whole-job throughput: the units every rank processed over the slowest rank's time."""
    return units_per_rank * ranks / seconds


def head_config(rtol, tuned=True):
    h = HEAD
    return {"workload": (f"2D N={h['N']}^2, M={h['M']}, alpha={h['alpha']}, gamma={h['gamma']}, GRF source "
                         f"(length scale 0.1, seed {h['seed']}), H-matrix leaf 64 tol 1e-10, V(1,1) to "
                         f"max|r| <= {rtol:g} max|F|; mixed precision + learned warm start vs plain FP64"),
            "dim": 2, "N": h["N"], "M": h["M"], "alpha": h["alpha"], "gamma": h["gamma"], "leaf": 64, "tol": 1e-10,
            "cycle": "V(1,1)", "rtol": rtol, "rtol_reference": "max|F|",
            "coarse_solve": f"exact solve of the {h['nc']}^2 level (DST-I in space, one H-matrix walk per mode)",
            "tiles": "autotuned (fhmg_problem_autotune)" if tuned else "heuristic",
            "warm_start": f"spectral MLP 6->320->320->320->1 (SiLU), BF16 inference, K={h['K']} modes per dimension",
            "l2": f"inputs larger than L2 (u, f {h['N'] ** 2 * h['M'] * 8 / 1e9:.2f} GB each)"}


# ------------------------------------------------------------------ oracle (timing + error checks)

def oracle_R(alpha, gamma, M, cache={}):
    from oracle import l1
    key = (alpha, gamma, M)
    if key not in cache:
        t = l1.graded_mesh(1.0, M, gamma)
        cache[key] = (t, l1.l1_matrix(t, alpha))
    return cache[key]


def grf_oracle_at(alpha, gamma, M, N, seed, iy, ix):
    """Per-mode oracle of a GRF source at sampled grid points (every time level)."""
    import numpy as np
    from oracle import direct
    from paper_1706_07632_gb300 import inputs
    t, R = oracle_R(alpha, gamma, M)
    _, _, c = inputs.grf_2d(seed, t[1:], N)
    kmax = c.shape[0]
    lam = direct.laplacian_eigs_1d(N, 1.0 / (N + 1))[:kmax]
    x = inputs.grid(N)
    W = np.zeros((M, len(iy)))
    for p in range(kmax):
        sy = np.sin((p + 1) * math.pi * x[iy])
        for q in range(kmax):
            if c[p, q] != 0.0:
                w = direct.solve_o2_mode(R, lam[p] + lam[q], np.full(M, c[p, q]))
                W += np.outer(w, sy * np.sin((q + 1) * math.pi * x[ix]))
    return W


def sampled_err(u, ref, iy, ix):
    import numpy as np
    import torch
    got = u[:, torch.as_tensor(iy, device=u.device), torch.as_tensor(ix, device=u.device)].cpu().numpy()
    return float(np.abs(got - ref).max() / np.abs(ref).max())


def oracle_direct_c5_sample(m_stop):
    """The oracle's direct solver (O1) on the first m_stop time levels of the headline workload;
    returns (seconds, DOF processed)."""
    import numpy as np
    from oracle import direct
    from paper_1706_07632_gb300 import inputs
    h = HEAD
    t, R = oracle_R(h["alpha"], h["gamma"], h["M"])
    a, s, _ = inputs.grf_2d(h["seed"], t[1:], h["N"])
    F = np.empty((m_stop, h["N"], h["N"]))
    F[:] = s[None]
    t0 = time.perf_counter()
    direct.solve_o1(R[:m_stop, :m_stop], F, 1.0 / (h["N"] + 1))
    return time.perf_counter() - t0, h["N"] ** 2 * m_stop


def run_reference(a):
    """--impl reference: the CPU oracle on the host cores (rank 0 only; other ranks exit)."""
    dist, rank, ws = dist_setup()
    if rank != 0:
        return
    k_ref = int(os.environ.get("FHMG_REF_CYCLES", "7"))  # FP64 V(1,1) cycles of the headline (GB300 run)
    m_stop = 48
    oracle_R(HEAD["alpha"], HEAD["gamma"], HEAD["M"])   # R is set-up, not timed
    for _ in range(max(0, min(a.warmup, 1))):
        oracle_direct_c5_sample(m_stop)
    samples = [oracle_direct_c5_sample(m_stop) for _ in range(a.steps)]
    tot = sum(s for s, _ in samples)
    dof = samples[0][1]
    value = dof * k_ref * a.steps / tot
    sample = (f"direct solve (implicit time stepping, dense L1 history sum, DST-I spatial solve per step; numpy/scipy "
              f"on the host threads) of the first {m_stop} of {HEAD['M']} time levels of the headline workload per step; "
              f"DOF*cycles with the FP64 cycle count {k_ref}")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "DOF*cycles/s", "n_gpus": a.gpus,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1e3 * tot / a.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": head_config(a.rtol),
            "cpu_baseline": {"value": value, "unit": "DOF*cycles/s", "cores": os.cpu_count(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "DOF*cycles/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# ------------------------------------------------------------------ GPU measurements

def events():
    import torch
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def train_net(fh, stream):
    """The warm-start network, trained on library solves (N=255^2, M=512, 11 alphas, sources with
    seeds 200..210 -- none of them used below)."""
    import torch
    from paper_1706_07632_gb300 import warmstart
    alphas = [0.3 + 0.05 * k for k in range(11)]
    t0 = time.perf_counter()
    X, Y = warmstart.generate(2, 255, HEAD["M"], HEAD["gamma"], alphas, seeds=list(range(200, 211)), K=HEAD["K"])
    t_data = time.perf_counter() - t0
    net = fh.WSNet(320, 3, seed=0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    losses = warmstart.train(net, X, Y, steps=4500, batch=4096, lr=2e-3)
    torch.cuda.synchronize()
    return net, {"samples": int(X.shape[0]), "data_s": t_data, "train_s": time.perf_counter() - t0,
                 "loss": losses[-1], "params": net.num_params(),
                 "train_grid": "N=255^2, M=512, 11 alphas 0.30..0.80, seeds 200-210, 4500 Adam steps"}


def problem(fh, H, prec, stream, tune):
    P = fh.Problem(H, 2, HEAD["N"], 1.0, prec, stream)
    P.set_coarse_direct(HEAD["nc"])
    P.set_rtol_reference(1)
    if tune:
        P.autotune()
    return P


def timed(fn, stream, n):
    """n calls of fn, each bracketed by CUDA events on the launching stream; returns the times (s)
    and the last result."""
    import torch
    ts, out = [], None
    for _ in range(n):
        e0, e1 = events()
        torch.cuda.synchronize()
        e0.record(stream)
        out = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1) / 1e3)
    return ts, out


def measure_headline(fh, a, stream, dist):
    import numpy as np
    import torch
    from paper_1706_07632_gb300 import warmstart
    h = HEAD
    net, training = train_net(fh, stream)
    t0 = time.perf_counter()
    H = fh.HMatrix(h["alpha"], h["gamma"], 1.0, h["M"], 64, 0, 1e-10)
    t_hbuild = time.perf_counter() - t0
    t, _ = H.mesh()
    f = warmstart.source_field(2, h["seed"], t[1:], h["N"])
    Pm = problem(fh, H, fh.MIXED_BF16, stream, not a.no_autotune)
    u = torch.zeros_like(f)
    rtol = a.rtol

    def warm_step():
        net.predict(Pm, f, h["alpha"], K=h["K"], bf16=True, u0=u)
        return Pm.solve(u, f, None, 1, 1, rtol, 60)

    for _ in range(a.warmup):
        warm_step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    Pm.profile(True)
    l0 = fh.wsnet_launches()
    e0, e1 = events()
    torch.cuda.cudart().cudaProfilerStart()  # a profiler started with capture off records the timed steps only
    e0.record(stream)
    k_warm = 0
    for _ in range(a.steps):
        k_warm, rr_warm = warm_step()
    e1.record(stream)
    torch.cuda.synchronize()
    torch.cuda.cudart().cudaProfilerStop()
    ms = max_over_ranks(e0.elapsed_time(e1), dist)
    cnt = Pm.counters()
    cnt.update(Pm.defect_timing())
    split_flops = Pm.split_flops()
    nn_launches = fh.wsnet_launches() - l0
    Pm.profile(False)
    if dist:
        dist.barrier()
    rng = np.random.default_rng(77)
    iy, ix = rng.integers(0, h["N"], 4096), rng.integers(0, h["N"], 4096)
    ref = grf_oracle_at(h["alpha"], h["gamma"], h["M"], h["N"], h["seed"], iy, ix)
    arms = {"mixed_warm": {"time_to_rtol_s": ms / a.steps / 1e3, "cycles": k_warm, "relres_vs_maxF": rr_warm,
                           "err_vs_oracle": sampled_err(u, ref, iy, ix), "steps_timed": a.steps}}
    arms["mixed_warm"]["predict_s"] = statistics.median(
        timed(lambda: net.predict(Pm, f, h["alpha"], K=h["K"], bf16=True, u0=u), stream, 3)[0])
    # mixed from zero: median of 5 solves
    def zero_solve(P):
        u.zero_()
        return P.solve(u, f, None, 1, 1, rtol, 60)
    zero_solve(Pm)
    ts, (k, rr) = timed(lambda: zero_solve(Pm), stream, 5)
    arms["mixed_zero"] = {"time_to_rtol_s": statistics.median(ts), "times_s": ts, "cycles": k, "relres_vs_maxF": rr,
                          "err_vs_oracle": sampled_err(u, ref, iy, ix)}
    # the mixed form with FP32 products (3xTF32 mma.sync walks), from zero
    Pf = problem(fh, H, fh.MIXED_FP32, stream, not a.no_autotune)
    zero_solve(Pf)
    ts, (k, rr) = timed(lambda: zero_solve(Pf), stream, 3)
    arms["mixed_fp32_zero"] = {"time_to_rtol_s": statistics.median(ts), "times_s": ts, "cycles": k,
                               "relres_vs_maxF": rr, "err_vs_oracle": sampled_err(u, ref, iy, ix)}
    del Pf
    torch.cuda.empty_cache()
    # e2e: the warm-started solve from pinned host buffers through fhmg_ws_solve_host
    f_host = f.cpu().pin_memory()
    u_host = torch.empty(f.shape, dtype=torch.float64).pin_memory()
    net.solve_host(Pm, u_host, f_host, h["alpha"], h["K"], True, 1, 1, rtol, 60)
    n_e2e = min(a.steps, 5)
    t0 = time.perf_counter()
    for _ in range(n_e2e):
        net.solve_host(Pm, u_host, f_host, h["alpha"], h["K"], True, 1, 1, rtol, 60)
    te = max_over_ranks(time.perf_counter() - t0, dist)
    del f_host, u_host
    del Pm
    torch.cuda.empty_cache()
    # plain FP64 from zero: median of 5 solves (heuristic tiles: autotuning the FP64 walks on this
    # grid takes minutes)
    Pd = problem(fh, H, fh.FP64, stream, False)
    zero_solve(Pd)
    ts, (k, rr) = timed(lambda: zero_solve(Pd), stream, 5)
    arms["fp64_zero"] = {"time_to_rtol_s": statistics.median(ts), "times_s": ts, "cycles": k, "relres_vs_maxF": rr,
                         "err_vs_oracle": sampled_err(u, ref, iy, ix)}
    del Pd
    torch.cuda.empty_cache()
    return {"H": H, "arms": arms, "cnt": cnt, "ms": ms, "nn_launches": nn_launches, "training": training,
            "split_flops": split_flops,
            "hbuild_s": t_hbuild, "e2e_s": te / n_e2e, "dof": h["N"] ** 2 * h["M"], "nbytes": f.numel() * 8}


def measure_sources(fh, net_holder, a, stream):
    """Unseen GRF sources, alpha ~ U[.3, .8]: cycles and time from zero and from the warm start."""
    import numpy as np
    import torch
    from paper_1706_07632_gb300 import warmstart
    h = HEAD
    net = net_holder
    rng = np.random.default_rng(4242)
    rows = []
    for i in range(a.sources):
        alpha = float(rng.uniform(0.3, 0.8))
        seed = 1000 + i
        H = fh.HMatrix(alpha, h["gamma"], 1.0, h["M"], 64, 0, 1e-10)
        t, _ = H.mesh()
        f = warmstart.source_field(2, seed, t[1:], h["N"])
        P = problem(fh, H, fh.MIXED_BF16, stream, False)
        u = torch.zeros_like(f)

        def zero():
            u.zero_()
            return P.solve(u, f, None, 1, 1, a.rtol, 60)

        def warm():
            net.predict(P, f, alpha, K=h["K"], bf16=True, u0=u)
            return P.solve(u, f, None, 1, 1, a.rtol, 60)

        (tz,), (kz, _) = timed(zero, stream, 1)
        (tw,), (kw, rw) = timed(warm, stream, 1)
        r = {"alpha": alpha, "seed": seed, "cycles_zero": kz, "cycles_warm": kw, "time_zero_s": tz, "time_warm_s": tw}
        if i < 4:  # error of the warm-started solution against the per-mode oracle (sampled points)
            prs = np.random.default_rng(seed)
            iy, ix = prs.integers(0, h["N"], 1024), prs.integers(0, h["N"], 1024)
            r["err_vs_oracle"] = sampled_err(u, grf_oracle_at(alpha, h["gamma"], h["M"], h["N"], seed, iy, ix), iy, ix)
        rows.append(r)
        del P, H, f, u
        torch.cuda.empty_cache()
    saved = [r["cycles_zero"] - r["cycles_warm"] for r in rows]
    tsave = [1.0 - r["time_warm_s"] / r["time_zero_s"] for r in rows]
    errs = [r["err_vs_oracle"] for r in rows if "err_vs_oracle" in r]
    return {"workload": f"{len(rows)} unseen GRF sources (seeds 1000+), alpha ~ U[.3,.8], same grid and target as the "
                        f"headline; mixed precision from zero vs from the learned warm start (heuristic tiles)",
            "cycles_saved_mean": float(np.mean(saved)), "cycles_saved_min": int(np.min(saved)),
            "cycles_saved_max": int(np.max(saved)), "time_saved_mean": float(np.mean(tsave)),
            "time_saved_min": float(np.min(tsave)), "err_vs_oracle_max": max(errs) if errs else None, "per_source": rows}


def mode_oracle_1d(alpha, gamma, M, N, a):
    """Per-mode oracle of the manufactured single-mode source (sin(pi x) times a(t))."""
    from oracle import direct
    t, R = oracle_R(alpha, gamma, M)
    return direct.solve_o2_mode(R, direct.laplacian_eigs_1d(N, 1.0 / (N + 1))[0], a)


def measure_manufactured(fh, stream, dim, N, M, alpha, gamma, nc, steps, tune):
    """FP64 and mixed solves of the manufactured u = t^alpha prod sin(pi x_i) to relres 1e-8,
    with the error against the per-mode oracle."""
    import numpy as np
    import torch
    from paper_1706_07632_gb300 import inputs
    H = fh.HMatrix(alpha, gamma, 1.0, M, 64, 0, 1e-10)
    t, _ = H.mesh()
    amp, s = inputs.manufactured(t[1:], N, dim, alpha)
    dev = torch.device("cuda", torch.cuda.current_device())
    f = torch.as_tensor(amp, device=dev).reshape((-1,) + (1,) * dim) * torch.as_tensor(s, device=dev)[None]
    from oracle import direct
    _, R = oracle_R(alpha, gamma, M)
    lam = direct.laplacian_eigs_1d(N, 1.0 / (N + 1))[0] * dim
    w = direct.solve_o2_mode(R, lam, amp)
    ref = torch.as_tensor(w, device=dev).reshape((-1,) + (1,) * dim) * torch.as_tensor(s, device=dev)[None]
    out = {}
    for name, prec in (("fp64", fh.FP64), ("mixed", fh.MIXED_FP32), ("mixed_bf16", fh.MIXED_BF16)):
        P = fh.Problem(H, dim, N, 1.0, prec, stream)
        P.set_coarse_direct(nc)
        if tune:
            P.autotune()
        u = torch.zeros_like(f)

        def run():
            u.zero_()
            return P.solve(u, f, None, 1, 1, 1e-8, 80)
        run()
        P.profile(True)
        ts, (k, rr) = timed(run, stream, steps)
        cnt = P.counters()
        cnt.update(P.defect_timing())
        P.profile(False)
        out[name] = {"time_to_rtol_s": statistics.median(ts), "cycles": k, "relres": rr,
                     "err_vs_oracle": float((u - ref).abs().max() / ref.abs().max()),
                     "gpu_launches_per_solve": cnt["launches"] / steps}
        del P
    out["speedup_mixed_vs_fp64"] = out["fp64"]["time_to_rtol_s"] / out["mixed"]["time_to_rtol_s"]
    k_ref = out["fp64"]["cycles"]
    dof = N ** dim * M
    for name in ("fp64", "mixed", "mixed_bf16"):
        out[name]["dof_cycles_per_s"] = dof * k_ref / out[name]["time_to_rtol_s"]
    out["speedup_mixed_bf16_vs_fp64"] = out["fp64"]["time_to_rtol_s"] / out["mixed_bf16"]["time_to_rtol_s"]
    return out


def measure_batched(fh, stream, rtol, n_inst=64, seed=7):
    """64 independent 1D instances (alpha ~ U[.2,.9], gamma ~ U[1,3], M in {256,...,2048},
    N in {255, 1023, 4095}, 8-mode sine-series sources), leaf autotuned per (M, N) class, solved by
    one batched mixed solve (one launch per stage, graph-replayed cycles); error of every instance
    against the per-mode oracle."""
    import numpy as np
    import torch
    from oracle import direct
    from paper_1706_07632_gb300 import inputs
    rng = np.random.default_rng(seed)
    Hs, Ps, us, fs, dof, meta = [], [], [], [], 0, []
    leaf_cache = {}
    dev = torch.device("cuda", torch.cuda.current_device())
    for i in range(n_inst):
        alpha = float(rng.uniform(0.2, 0.9))
        gamma = float(rng.uniform(1.0, 3.0))
        M = int(rng.choice([256, 512, 1024, 2048]))
        N = int(rng.choice([255, 1023, 4095]))
        key = (M, N)
        if key not in leaf_cache:
            leaf_cache[key] = fh.autotune_leaf(alpha, gamma, 1.0, M, 1e-10, 1, N, 1.0, fh.MIXED_FP32, stream)[0]
        H = fh.HMatrix(alpha, gamma, 1.0, M, leaf_cache[key], 0, 1e-10)
        P = fh.Problem(H, 1, N, 1.0, fh.MIXED_FP32, stream)
        t, _ = H.mesh()
        a, s, c = inputs.sine_series_1d(seed * 1000 + i, t[1:], N)
        f = torch.as_tensor(a, device=dev)[:, None] * torch.as_tensor(s, device=dev)[None, :]
        Hs.append(H), Ps.append(P), fs.append(f), us.append(torch.zeros_like(f))
        meta.append((alpha, gamma, M, N, c))
        dof += N * M
    for u in us:
        u.zero_()
    fh.solve_batched(Ps, us, fs, 1, 1, rtol, 60)  # warm-up (graph capture)
    for u in us:
        u.zero_()
    (tb,), (k, rr) = timed(lambda: fh.solve_batched(Ps, us, fs, 1, 1, rtol, 60), stream, 1)
    errs = []
    for i in range(0, n_inst, 8):  # every 8th instance against the per-mode oracle
        alpha, gamma, M, N, c = meta[i]
        _, R = oracle_R(alpha, gamma, M)
        lam = direct.laplacian_eigs_1d(N, 1.0 / (N + 1))
        x = inputs.grid(N)
        ref = sum(np.outer(direct.solve_o2_mode(R, lam[q - 1], np.full(M, c[q - 1] / q ** 2)),
                           np.sin(q * math.pi * x)) for q in range(1, 9))
        errs.append(float(np.abs(us[i].cpu().numpy() - ref).max() / np.abs(ref).max()))
    for u in us:
        u.zero_()

    def seq():
        ks = []
        for P, u, f in zip(Ps, us, fs):
            ks.append(P.solve(u, f, None, 1, 1, rtol, 60)[0])
        return ks
    (ts,), ks = timed(seq, stream, 1)
    return {"workload": f"{n_inst} 1D instances, alpha~U[.2,.9], gamma~U[1,3], M in {{256..2048}}, "
                        f"N in {{255,1023,4095}}, 8-mode sine sources, relres {rtol:g}",
            "dof_total": dof, "leaves": sorted(set(leaf_cache.values())),
            "leaf_by_size": {f"M={m},N={n}": l for (m, n), l in sorted(leaf_cache.items())},
            "batched_s": tb, "sequential_s": ts, "speedup_batched_vs_sequential": ts / tb,
            "batched_dof_cycles_per_s": dof * float(np.mean(k)) / tb,
            "cycles_mean": float(np.mean(k)), "cycles_max": int(np.max(k)), "relres_max": float(np.max(rr)),
            "err_vs_oracle_max": max(errs), "err_checked_instances": len(errs)}


def roofline_smoother(H, cnt, ms_total, ncols, M, hbm_peak, bf16_peak, peak_kind):
    """Finest-grid smoother half-sweeps of the mixed path (FP32 storage, BF16 products on the
    tcgen05 tensor cores), timed live.  Algorithmic HBM bytes per column: the column's right-hand
    side, the neighbours' values (each value of the other colour once) and the column written, 4
    bytes each per time level (12 M bytes); algorithmic tensor work: the H-matrix flops of one
    walk.  The bound is whichever takes longer at its peak."""
    n = max(cnt["smooth_launches"], 1)
    t = cnt["smooth_ms"] / n / 1e3
    bytes_launch = 12.0 * M * ncols
    flops_launch = H.flops_per_column() * ncols
    t_hbm = bytes_launch / (hbm_peak * 1e9)
    t_tc = flops_launch / (bf16_peak * 1e12)
    common = {"kernel": "humma_kernel<SMOOTH> (finest-grid half-sweep, FP32 storage, BF16 tcgen05.mma, TMEM accumulators)",
              "avg_launch_ms": t * 1e3, "launches_timed": cnt["smooth_launches"],
              "share_of_step": cnt["smooth_ms"] / ms_total if ms_total > 0 else None,
              "algorithmic_bytes_per_launch": bytes_launch, "algorithmic_flops_per_launch": flops_launch,
              "traffic": traffic("smooth", M, ncols)}
    if t_hbm >= t_tc:
        ach = bytes_launch / t / 1e9
        return dict(common, bound="hbm", achieved=ach, peak=hbm_peak, unit="GB/s", frac=ach / hbm_peak,
                    peak_note=f"copy bandwidth, {peak_kind}")
    ach = flops_launch / t / 1e12
    return dict(common, bound="tensor", achieved=ach, peak=bf16_peak, unit="TFLOP/s", frac=ach / bf16_peak,
                peak_note=f"BF16 dense, {peak_kind}")


def roofline_defect(H, cnt, ms_total, ncols, M, split_flops, bf16_peak, peak_kind):
    """The outer FP64-accurate defect, timed live (the split_prep_kernel pass and the defect kernel).
    With digit splitting (split_flops: BF16 tensor flops per grid point of the digit-tile products)
    it is bounded by the tensor pipe; the double-float walk by the FP32 pipe."""
    n = max(cnt["defect_launches"], 1)
    t = cnt["defect_ms"] / n / 1e3
    flops_launch = H.flops_per_column() * ncols
    common = {"avg_launch_ms": t * 1e3, "launches_timed": cnt["defect_launches"],
              "share_of_step": cnt["defect_ms"] / ms_total if ms_total > 0 else None,
              "fp64_equivalent_tflops": flops_launch / t / 1e12, "algorithmic_fp64_flops_per_launch": flops_launch,
              "traffic": traffic("defect", M, ncols)}
    if split_flops:
        mma = split_flops * ncols
        ach = mma / t / 1e12
        return dict(common, kernel="split_prep_kernel + split_defect_kernel (finest-grid FP64-accurate defect by "
                    "BF16 digit splitting on tcgen05, exact FP32 group sums in TMEM)", bound="tensor", achieved=ach, peak=bf16_peak,
                    unit="TFLOP/s", frac=ach / bf16_peak, peak_note=f"BF16 dense sustained, {peak_kind}",
                    algorithmic_flops_per_launch=mma)
    ach = flops_launch / t / 1e12
    return dict(common, kernel="hdf_kernel<64,8,MATVEC> (finest-grid FP64-accurate defect, double-float)",
                bound="alu", achieved=ach, peak=DF_PEAK_TFLOPS, unit="TFLOP/s", frac=ach / DF_PEAK_TFLOPS,
                peak_note="152 SMs x 128 FP32 lanes/clk x 2.07 GHz x 2 flop per 11-instruction double-float multiply-add",
                algorithmic_flops_per_launch=flops_launch)


def main():
    a = parse()
    if a.grid != HEAD["N"]:
        if a.grid < 63 or (a.grid + 1) & a.grid:
            raise SystemExit("--grid must be 2^k - 1 >= 63")
        HEAD["N"] = a.grid
    if a.impl == "reference":
        return run_reference(a)
    import torch

    import __graft_entry__
    __graft_entry__.build()
    import paper_1706_07632_gb300 as fh

    dist, rank, ws = dist_setup()
    stream = torch.cuda.current_stream()
    hbm_peak, bf16_peak, peak_kind = peaks()
    clocks = Clocks(torch.cuda.current_device()) if rank == 0 else None

    hd = measure_headline(fh, a, stream, dist)
    arms = hd["arms"]
    k_ref = arms["fp64_zero"]["cycles"]
    dof = hd["dof"]
    for r in arms.values():
        r["value"] = job_value(dof * k_ref, ws, r["time_to_rtol_s"])
    value = arms["mixed_warm"]["value"]
    e2e = {"value": job_value(dof * k_ref, ws, hd["e2e_s"]), "unit": "DOF*cycles/s",
           "h2d_bytes_per_step": hd["nbytes"], "d2h_bytes_per_step": hd["nbytes"], "ms_per_step": 1e3 * hd["e2e_s"],
           "call": "fhmg_ws_solve_host (pinned host f in, warm start + solve, u out)"}

    sweep = w1d = w2d = bat = cpu = None
    if not a.quick:
        # the sweep reuses a freshly trained network (same recipe and seed as the headline's)
        net, _ = train_net(fh, stream)
        sweep = measure_sources(fh, net, a, stream)
        del net
        torch.cuda.empty_cache()
        w1d = measure_manufactured(fh, stream, 1, 4095, 4096, 0.5, 3.0, 255, 3, not a.no_autotune)
        w1d["workload"] = "1D H-matrix, N=4095, M=4096, alpha=0.5, gamma=3, leaf 64, tol 1e-10, V(1,1) to relres 1e-8"
        torch.cuda.empty_cache()
        w2d = measure_manufactured(fh, stream, 2, 511, 1024, 0.4, 2.5, 31, 2, not a.no_autotune)
        w2d["workload"] = "2D H-matrix, N=511^2, M=1024, alpha=0.4, gamma=2.5, leaf 64, tol 1e-10, V(1,1) to relres 1e-8"
        torch.cuda.empty_cache()
        bat = measure_batched(fh, stream, a.rtol)
        torch.cuda.empty_cache()
    clk = clocks.stop() if clocks else None

    if rank == 0 and not a.quick:
        m_stop = 192
        ts, ndof = oracle_direct_c5_sample(m_stop)
        cpu = {"value": ndof * k_ref / ts, "unit": "DOF*cycles/s", "cores": os.cpu_count(), "kind": "oracle",
               "sample": (f"direct solve (implicit time stepping, dense L1 history sum, DST-I spatial solve per step; "
                          f"numpy/scipy on the host threads) of the first {m_stop} of {HEAD['M']} time levels of the "
                          f"headline workload: {ts:.2f} s for {ndof} DOF; DOF*cycles with the FP64 cycle count {k_ref}")}

    ncol_colour = (HEAD["N"] ** 2 + 1) // 2
    if rank == 0 and HEAD["N"] != 1023:
        print(f"note: headline grid {HEAD['N']}^2 (profiling size), not the workload's 1023^2", file=sys.stderr)
    rl_s = roofline_smoother(hd["H"], hd["cnt"], hd["ms"], ncol_colour, HEAD["M"], hbm_peak, bf16_peak, peak_kind)
    rl_d = roofline_defect(hd["H"], hd["cnt"], hd["ms"], HEAD["N"] ** 2, HEAD["M"], hd["split_flops"], bf16_peak,
                           peak_kind)
    rl_head, rl_second = (rl_s, rl_d) if (rl_s["share_of_step"] or 0) >= (rl_d["share_of_step"] or 0) else (rl_d, rl_s)
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "DOF*cycles/s", "n_gpus": ws, "steps": a.steps,
                "warmup": a.warmup, "ms_per_step": hd["ms"] / a.steps, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64+f32+bf16", "data": "synthetic",
                "config": head_config(a.rtol, not a.no_autotune),
                "headline": ("mixed precision + learned warm start: network prediction of u0, then defect correction "
                             "with FP64-accurate outer defects (BF16 digit splitting on the tcgen05 tensor cores) around "
                             "V-cycles with FP32 storage and "
                             "BF16 H-matrix products on the tcgen05 tensor cores (FP32 accumulation in tensor memory)"),
                "cycle_unit": f"FP64 V(1,1) cycles to the target on the headline source = {k_ref}",
                "arms": arms,
                "speedup_mixed_warm_vs_fp64": arms["fp64_zero"]["time_to_rtol_s"] / arms["mixed_warm"]["time_to_rtol_s"],
                "speedup_mixed_warm_vs_mixed_zero": arms["mixed_zero"]["time_to_rtol_s"] / arms["mixed_warm"]["time_to_rtol_s"],
                "cycles_saved_by_warm_start": arms["mixed_zero"]["cycles"] - arms["mixed_warm"]["cycles"],
                "training": hd["training"], "hbuild_s": hd["hbuild_s"],
                "roofline": rl_head, "roofline_secondary": rl_second,
                "sources": sweep, "workload_1d": w1d, "workload_2d": w2d, "workload_batched": bat,
                "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": hd["cnt"]["launches"] + hd["nn_launches"], "clocks": clk}
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
