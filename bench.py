"""Benchmark: time to relative residual 1e-10 of the RaNN domain-decomposition
solver, and the bandwidth of its block matrix-vector products.

Headline workload (the largest configured problem that one GPU holds): the
space-time heat equation u_t = 0.1 Lap u on [0,1]^2 x [0,1], u(0) =
sin(pi x) sin(pi y) (exact solution known); 8 x 8 x 4 space-time subdomains
(overlap ratio 1.4), 400 tanh neurons per subdomain with weights U[-1, 1]
(seeded), 16 x 16 x 8 collocation points per subdomain cell (128 x 128 x 32
global); PCA keeping 1 - 1e-12 of the variance; additive-Schwarz
preconditioned CG on the normal equations to rtol 1e-10.  One step = the
whole hot path: assembly, right-hand side, PCA and reduction, preconditioner
set-up, Krylov solve.  Synthetic, seeded inputs.

The line also carries the 2D multiscale workload (8 x 8 subdomains, m = 300,
SAS-preconditioned GMRES(50)) in both precision modes: plain float64
(mode 0) and the double-float preconditioner and inner iterations with
float64 refinement (mode 1); and the differentiable batch of 64
piecewise-coefficient diffusion instances (forward RAS-GMRES, adjoint
solve, gradients with respect to the coefficient cells and the source).

Prints one JSON line.  --impl reference times the CPU oracle (float64 numpy)
on a bounded sample of the workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import rann_inputs as ri  # noqa: E402

METRIC = "time to rel. residual 1e-10 (AS-CG, RAS-GMRES) & block-matvec HBM GB/s"
WORKLOAD_DESC = ("heat3d (space-time heat u_t = 0.1 Lap u) 8x8x4 subdomains, m=400, 16x16x8 pts/subdomain "
                 "(128x128x32), overlap ratio 1.4, PCA 1-1e-12, AS-CG on the normal equations, rtol 1e-10")
DTYPE = ("mixed: f64 residuals, PCA eigenvalues and reduced blocks; df32 (float32 hi+lo) local factors, "
         "Schwarz apply and inner Krylov operator; bf16 digit-slice (Ozaki) tensor-core products, f64-accurate")
FP64_PEAK_TFLOPS = 152 * 4 * 2.07e9 / 1e12   # 152 SMs x 2 float64 FMA/clk x 2 flop x 2.07 GHz
DF32_PEAK_TFLOPS = 152 * 128 * 2.07e9 / 12 * 2 / 1e12   # double-float multiply-add: 12 float32 instructions
CSRC = os.path.join(ROOT, "paper_2412_19207_gb300", "csrc")
# DRAM bytes per launch of a kernel family (dram__bytes_read.sum +
# dram__bytes_write.sum from one ncu capture on this workload, as the
# profiles/ summary states), valid only for the kernel source it was taken
# on: (bytes, file, kernel, sha256 prefix of the kernel's source text).  A
# changed kernel reports null.
TRAFFIC = {"schwarz_apply_df32": (17946.9e6, "apply.cu", "schwarz_apply_rows_df_kernel", "7c262b33f7dc")}
# families whose profiled bracket spans a multi-stream pipeline of many kernels
# (the Cholesky with lookahead and the row-block inverse): no single launch
# duration, so they are reported as pipelines, not as the roofline kernel
PIPELINED = {"cholesky", "cholesky_tc"}


SMALL = False          # --small: the headline problem on 3 x 3 x 2 subdomains (12 x 12 x 6 points each), for profiling


def headline_workload():
    p = ri.heat3d(sub=(3, 3, 2), pts=(12, 12, 6), neurons=400) if SMALL else ri.config("heat3d")
    p.solver, p.precond = "cg_as", "as"
    return p


def multiscale_workload():
    p = ri.config("multiscale2d")
    p.precond = "sas"
    return p


def kernel_source_sha(fname, kernel):
    """sha256 prefix of one kernel's source text: from the line that declares
    `kernel` to the first line holding only a closing brace."""
    lines = open(os.path.join(CSRC, fname)).read().split("\n")
    start = next(i for i, l in enumerate(lines) if kernel + "(" in l and "__global__" in l)
    end = next(i for i in range(start, len(lines)) if lines[i] == "}")
    return hashlib.sha256("\n".join(lines[start:end + 1]).encode()).hexdigest()[:12]


def traffic_of(family):
    t = TRAFFIC.get(family)
    if not t:
        return None
    bytes_per_launch, fname, kernel, sha = t
    return bytes_per_launch if kernel_source_sha(fname, kernel) == sha else None


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "_fallback": True}


def local_gpu_index():
    """The nvidia-smi index of this rank's GPU: entry LOCAL_RANK of
    CUDA_VISIBLE_DEVICES, or LOCAL_RANK itself when the variable is unset."""
    lr = int(os.environ.get("LOCAL_RANK", "0"))
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis:
        ids = [v.strip() for v in vis.split(",") if v.strip()]
        if ids:
            return ids[min(lr, len(ids) - 1)]
    return str(lr)


class Clocks:
    """Samples nvidia-smi during the timed region."""

    def __init__(self):
        self.samples = []
        self.proc = None

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", local_gpu_index(),
                                          f"--query-gpu={q}", "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) == 7:
                self.samples.append(parts)

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in self.samples for i in range(4) if s[3 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples)}


def run_step(s, p, F, events=None):
    """One pass of the hot path; with events (5 CUDA events) the phase
    boundaries are recorded on the handle's stream."""
    rec = (lambda i: events[i].record(s.stream)) if events else (lambda i: None)
    rec(0)
    s.assemble()
    s.rhs(F)
    rec(1)
    ranks = s.pca(p.pca_mode, p.pca_thr)
    rec(2)
    s.setup_precond(p.precond)
    rec(3)
    if p.solver == "cg_as":
        W, st = s.solve_cg_as(F, p.rtol, p.maxit)
    else:
        W, st = s.solve_gmres_ras(F, p.rtol, p.restart, p.maxit)
    rec(4)
    return W, st, ranks


def max_over_ranks(value: float, world: int, device: str = "cuda") -> float:
    """The largest value over the ranks of the process group (the job's time
    per step is its slowest replica's); the value itself when world == 1."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def roofline(prof, pk):
    """The roofline object of the dominant single kernel of a profiled step."""
    dom_name, dom = max(((k, v) for k, v in prof.items() if k not in PIPELINED and v["ms"] > 0),
                        key=lambda kv: kv[1]["ms"])
    bound = dom["bound"]
    if bound == "hbm":
        ach = dom["bytes"] / (dom["ms"] * 1e-3) / 1e9
        peak, unit = pk["hbm_gbs"], "GB/s"
        note = "measured HBM copy (MEASURED_PEAKS.json)"
    elif bound == "tensor":
        ach = dom["flops"] / (dom["ms"] * 1e-3) / 1e12
        peak, unit = pk.get("bf16_tflops_sustained", pk.get("bf16_tflops")), "TFLOP/s"
        note = "measured cuBLAS bf16, sustained (MEASURED_PEAKS.json); flops of the digit-slice products"
    elif bound == "alu_df32":
        ach = dom["flops"] / (dom["ms"] * 1e-3) / 1e12
        peak, unit = pk["df32_tflops"], "TFLOP/s"
        note = ("double-float multiply-add rate measured by rann_dd_device_rates (float64-equivalent flops)"
                if pk.get("rates_measured") else "double-float multiply-add: unit counts x max clock / 12 instructions")
        bound = "alu"
    else:
        ach = dom["flops"] / (dom["ms"] * 1e-3) / 1e12
        peak, unit = pk["fp64_tflops"], "TFLOP/s"
        note = ("float64 FMA rate measured by rann_dd_device_rates" if pk.get("rates_measured")
                else "float64 FMA: 152 SMs x 2 FMA/clk x 2.07 GHz (unit counts x max clock)")
    tr = traffic_of(dom_name)
    return {"kernel": dom_name, "bound": bound, "achieved": round(ach, 3), "peak": peak, "unit": unit,
            "frac": round(ach / peak, 4), "traffic": (tr if tr is None else round(tr)),
            "launches": dom["launches"], "ms_per_launch": round(dom["ms"] / max(dom["launches"], 1), 4),
            "alg_bytes_per_launch": round(dom["bytes"] / max(dom["launches"], 1)),
            "peak_source": note}


def pipeline_entry(f, pk):
    """A multi-stream pipeline family: its time per step and its rate against
    the peak of its class (double-float pipe, or the bf16 tensor cores for the
    digit-slice products; the tensor pipeline also runs its 32-column panel
    steps on the float32 pipe, inside the same bracket)."""
    ach = f["flops"] / (f["ms"] * 1e-3) / 1e12
    if f["bound"] == "tensor":
        peak = pk.get("bf16_tflops_sustained", pk.get("bf16_tflops"))
        return {"ms_per_step": round(f["ms"], 3), "launches_per_step": f["launches"], "achieved_tflops": round(ach, 3),
                "peak_tflops": peak, "frac_of_bf16_sustained": round(ach / peak, 4),
                "flops": "digit-slice products (36 per float64-accurate product)"}
    return {"ms_per_step": round(f["ms"], 3), "launches_per_step": f["launches"], "achieved_tflops": round(ach, 3),
            "frac_of_df32_rate": round(ach / pk["df32_tflops"], 4)}


def bandwidths(prof, pk):
    def gbps(names):
        fam = [prof[n] for n in names if prof.get(n, {}).get("ms")]
        if not fam:
            return None
        by, t = sum(f["bytes"] for f in fam), sum(f["ms"] for f in fam)
        return {"GBps": round(by / (t * 1e-3) / 1e9, 1), "frac_of_hbm": round(by / (t * 1e-3) / 1e9 / pk["hbm_gbs"], 4),
                "launches_per_step": sum(f["launches"] for f in fam), "ms_per_step": round(t, 3)}
    return {"normal_rows_df32": gbps(["gramop_df32"]), "H_f64": gbps(["matvec_H"]), "HT_f64": gbps(["matvec_HT"]),
            "schwarz_apply_df32": gbps(["schwarz_apply_df32", "trmv_lower_df32", "trmv_upper_df32"]),
            "schwarz_apply_f64": gbps(["trmv_lower", "trmv_upper"])}


def time_steps(torch, s, p, F, n):
    """Mean CUDA-event time of n steps (after the caller's warm-up)."""
    stream = torch.cuda.current_stream()
    out = []
    for _ in range(n):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        W, st, ranks = run_step(s, p, F)
        e1.record(stream)
        e1.synchronize()
        out.append(e0.elapsed_time(e1))
    return out, W, st, ranks


def multiscale_arms(g, torch, steps=3):
    """The 2D multiscale workload (SAS-GMRES(50)) in precision mode 0 (plain
    float64) and mode 1 (double-float preconditioner and inner iterations,
    float64 refinement), each after one warm-up step."""
    p = multiscale_workload()
    R, b = ri.weights(p)
    out = {"workload": "multiscale2d 8x8 subdomains, m=300, 40x40 pts/subdomain (320x320), overlap 0.05, "
                       "PCA 1-1e-12, SAS-GMRES(50), rtol 1e-10"}
    for mode in (0, 1):
        s = g.RannDD(p, R, b)
        s.set_precision(mode)
        F = s._empty(s.sizes()["n_points"])
        run_step(s, p, F)
        times, W, st, ranks = time_steps(torch, s, p, F, steps)
        out[f"mode{mode}"] = {"precision": "f64" if mode == 0 else "df32 preconditioner+inner, f64 refinement",
                              "ms_per_step": round(float(np.mean(times)), 3), "iters": st["iters"],
                              "rel_res_true": st["rel_res_true"], "rel_res_prec": st["rel_res_prec"],
                              "dof": int(np.sum(ranks))}
        s.close()
    out["mode1_speedup_over_mode0"] = round(out["mode0"]["ms_per_step"] / out["mode1"]["ms_per_step"], 3)
    return out


def bench_ours(args, rank, world):
    import torch
    import paper_2412_19207_gb300 as g
    from paper_2412_19207_gb300 import build
    if rank == 0 or not os.path.exists(build.LIB):
        build.build()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    g.load_library()
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
    p = headline_workload()
    R, b = ri.weights(p)
    s = g.RannDD(p, R, b)
    F = s._empty(s.sizes()["n_points"])

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    for _ in range(args.warmup):
        W, st, ranks = run_step(s, p, F)
    barrier()
    with Clocks() as clk:
        times, W, st, ranks = time_steps(torch, s, p, F, args.steps)
        barrier()
    ms = max_over_ranks(float(np.mean(times)), world)
    # one further step with the phase boundaries on CUDA events, and one with
    # every launch bracketed by CUDA events on the handle's stream (kernel
    # breakdown and roofline); neither is part of the timed steps
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
    run_step(s, p, F, ev)
    torch.cuda.synchronize()
    phases = {k: round(ev[i].elapsed_time(ev[i + 1]), 3)
              for i, k in enumerate(["assemble_rhs", "pca", "setup_precond", "solve"])}
    s.profile(True)
    run_step(s, p, F)
    torch.cuda.synchronize()
    prof = s.profile_read()
    s.profile(False)
    s.close()
    # end to end through the public API with host buffers: weights in, W out
    Rh = torch.tensor(R).pin_memory()
    bh = torch.tensor(b).pin_memory()
    e2e = []
    for _ in range(2):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s2 = g.RannDD(p, Rh.numpy(), bh.numpy())
        F2 = s2._empty(s2.sizes()["n_points"])
        W2, st2, _ = run_step(s2, p, F2)
        Wh = torch.empty(W2.shape, dtype=torch.float64).pin_memory()
        Wh.copy_(W2)
        torch.cuda.synchronize()
        e2e.append(time.perf_counter() - t0)
        s2.close()
        del s2, F2, W2
    pk = peaks()
    try:                                  # measured double-float and float64 rates of this GPU
        pk["df32_tflops"], pk["fp64_tflops"] = g.device_rates()
        pk["rates_measured"] = True
    except Exception:
        pk["df32_tflops"], pk["fp64_tflops"], pk["rates_measured"] = DF32_PEAK_TFLOPS, FP64_PEAK_TFLOPS, False
    launches = sum(v["launches"] for v in prof.values())
    kernels = {k: {"ms_per_step": round(v["ms"], 3), "launches_per_step": v["launches"]}
               for k, v in sorted(prof.items(), key=lambda kv: -kv[1]["ms"]) if v["launches"]}
    out = {
        "metric": METRIC, "value": round(ms / 1e3, 6), "unit": "s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms, 3), "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": DTYPE,
        "data": "synthetic (seeded SplitMix64 weights, manufactured PDE data)",
        "config": {"workload": WORKLOAD_DESC, "solver": "AS-CG", "precision_mode": 1,
                   "dof": int(np.sum(ranks)), "J": p.J, "m": p.neurons, "iters": st["iters"],
                   "rel_res_true": st["rel_res_true"], "rel_res_rec": st["rel_res_rec"],
                   "n_shifted": st["n_shifted"], "parallelism": f"replicas x{world}",
                   "l2": "working set > L2 (reduced blocks 8*sum N_j p_j bytes, local factors), no flush"},
        "phases_ms": phases,
        "roofline": roofline(prof, pk),
        "matvec": bandwidths(prof, pk),
        "pipelines": {k: pipeline_entry(prof[k], pk) for k in sorted(PIPELINED) if prof.get(k, {}).get("ms")},
        "device_rates": {"df32_tflops": round(pk["df32_tflops"], 2), "fp64_tflops": round(pk["fp64_tflops"], 3),
                         "measured": pk["rates_measured"]},
        "kernels": kernels,
        "gpu_launches": int(launches) * args.steps,
        "gpu_launches_per_step": int(launches),
        "e2e": {"value": round(float(np.median(e2e)), 6), "unit": "s",
                "h2d_bytes_per_step": int(R.nbytes + b.nbytes), "d2h_bytes_per_step": int(W.numel() * 8),
                "what": "fresh handle from pinned host weights R, b; full hot path; W copied to pinned host memory"},
        "clocks": clk.summary(),
    }
    if not args.no_multiscale:
        out["multiscale2d"] = multiscale_arms(g, torch)
    if not args.no_batch:
        out["piecewise_batch"] = piecewise_batch(g, torch)
    if args.multi_rhs > 0:
        out["multi_rhs"] = [multi_rhs_timing(g, args.multi_rhs, "cg"), multi_rhs_timing(g, args.multi_rhs, "gmres")]
    return out


def piecewise_batch(g, torch, kind="ras", nworkers=8):
    """The differentiable batch of the piecewise-coefficient diffusion
    workload: 64 instances (subdomain grids 4x4 .. 16x16 by instance, 200
    neurons, 24x24 points per cell, a smoothed 4x4 piecewise coefficient with
    cell values U[0.5, 2] and an 8-mode Fourier source, all seeded), each run
    forward (assembly, PCA, Schwarz set-up, preconditioned GMRES(50) to
    1e-10) and backward for l = ||u_hat - u_obs||^2 on its collocation grid
    (u_obs = 0.01 sin(pi x) sin(pi y)): dl/dW through the grid evaluation's
    adjoint, the adjoint solve, dl/da_c (16 cells) and dl/dF.  Timed two
    ways, wall time with the device synchronised on both sides: all 64
    through one rann_dd_batch_run (native worker threads, one CUDA stream
    each, Schwarz apply tuned per size class), and one instance after the
    other through the single-instance calls."""
    out = {"instances": 64, "solver": f"{kind.upper()}-GMRES(50)", "rtol": 1e-10, "workers": nworkers}
    ps = [ri.piecewise2d(i) for i in range(64)]

    def uobs(X):
        return (0.01 * torch.sin(np.pi * X[:, 0]) * torch.sin(np.pi * X[:, 1])).contiguous()

    # batched
    hs = [g.RannDD(p) for p in ps]
    uo = [uobs(h.points()) for h in hs]
    b = g.Batch(nworkers)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    res = b.run(hs, ps[0].pca_mode, ps[0].pca_thr, prec=kind, solver=g.SOLVER_GMRES, rtol=1e-10, restart=50,
                maxit=3000, autotune=True, u_obs=uo)
    torch.cuda.synchronize()
    tb = time.perf_counter() - t0
    b.close()
    for h in hs:
        h.close()
    cfgs = [r["apply_config"] for r in res]
    out["batched"] = {"s_per_batch": round(tb, 3), "ms_per_instance": round(tb * 1e3 / 64, 2),
                      "forward_and_adjoint_converged": sum(r["status"] == "RANN_OK" for r in res),
                      "iters_min_max": [int(min(r["forward"]["iters"] for r in res)),
                                        int(max(r["forward"]["iters"] for r in res))],
                      "apply_configs": {str(c): cfgs.count(c) for c in sorted(set(cfgs))}}
    # one instance after the other
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    conv = adj = 0
    for p in ps:
        s = g.RannDD(p)
        s.assemble()
        F = s.rhs()
        s.pca(p.pca_mode, p.pca_thr)
        s.setup_precond(kind)
        W, st = s.solve_gmres_ras(F, 1e-10, 50, 3000, allow_not_converged=True)
        X = s.points()
        u = s.eval(W, X)
        gW = s.eval_grid_t(2.0 * (u - uobs(X)))
        lam, sb = s.solve_backward(gW, 1e-10, 3000, allow_not_converged=True)
        s.grad_coef(F, W, lam)
        s.matvec(lam)
        conv += st["status"] == "RANN_OK"
        adj += sb["status"] == "RANN_OK"
        s.close()
    torch.cuda.synchronize()
    ts = time.perf_counter() - t0
    out["sequential"] = {"s_per_batch": round(ts, 3), "ms_per_instance": round(ts * 1e3 / 64, 2),
                         "forward_converged": conv, "adjoint_converged": adj}
    out["batched_speedup"] = round(ts / tb, 3)
    return out


def multi_rhs_timing(g, k, solver="cg"):
    """k right-hand sides of the multiscale workload (F scaled by 1..k, so every
    column runs the same iterations): k one-column solves one after another
    against one lockstep solve of all k (every operator and preconditioner
    launch serves all columns).  solver "cg": AS-preconditioned CG; "gmres":
    SAS-preconditioned GMRES(50).  Both after a warm-up solve; wall time with
    the device synchronised on both sides (the solves include their host
    round trips)."""
    import torch
    p = multiscale_workload()
    R, b = ri.weights(p)
    s = g.RannDD(p, R, b)
    s.assemble()
    F = s.rhs()
    s.pca(p.pca_mode, p.pca_thr)
    s.setup_precond("as" if solver == "cg" else p.precond)
    Fs = torch.stack([F * float(c + 1) for c in range(k)])
    if solver == "cg":
        one = lambda f: s.solve_cg_as(f, p.rtol, 4000)
        multi = lambda fs: s.solve_cg_as_multi(fs, p.rtol, 4000)
        ok = lambda st: st["rel_res_true"] <= p.rtol
    else:
        one = lambda f: s.solve_gmres_ras(f, p.rtol, p.restart, 4000)
        multi = lambda fs: s.solve_gmres_ras_multi(fs, p.rtol, p.restart, 4000)
        ok = lambda st: st["rel_res_prec"] <= p.rtol
    one(F)
    multi(Fs[:1].contiguous())
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    iters = []
    for c in range(k):
        _, st = one(Fs[c].contiguous())
        iters.append(st["iters"])
    torch.cuda.synchronize()
    t_one = time.perf_counter() - t0
    t0 = time.perf_counter()
    _, sts = multi(Fs)
    torch.cuda.synchronize()
    t_multi = time.perf_counter() - t0
    s.close()
    return {"nrhs": k, "solver": "AS-CG" if solver == "cg" else f"{p.precond.upper()}-GMRES({p.restart})",
            "iters": iters[0], "ms_one_at_a_time": round(t_one * 1e3, 3),
            "ms_lockstep": round(t_multi * 1e3, 3), "ms_per_rhs_lockstep": round(t_multi * 1e3 / k, 3),
            "speedup": round(t_one / t_multi, 3), "all_converged": all(ok(x) for x in sts)}


# --------------------------------------------------------------- CPU oracle --

def oracle_sample_problem():
    """A scaled-down instance of the headline workload that the oracle solves
    completely in seconds: the same space-time heat problem, overlap ratio,
    weight range and rank rule on 3 x 3 x 2 subdomains (one interior
    subdomain, so the Schwarz sets overlap as in the full grid) with
    6 x 6 x 4 points per cell and 40 neurons."""
    p = ri.heat3d(sub=(3, 3, 2), pts=(6, 6, 4), neurons=40)
    p.solver, p.precond = "cg_as", "as"
    return p


def oracle_pass(p):
    """The oracle's whole hot path on problem p (assembly and PCA, AS set-up
    by Householder QR of every A_i, AS-CG to rtol); seconds per phase."""
    from oracle import solver as sv
    t0 = time.perf_counter()
    S = sv.build_system(p)
    t1 = time.perf_counter()
    M = sv.schwarz(S, "as")
    t2 = time.perf_counter()
    sol = sv.solve(S, "cg", M, p.rtol, p.restart, p.maxit)
    t3 = time.perf_counter()
    return {"build": t1 - t0, "setup": t2 - t1, "solve": t3 - t2, "total": t3 - t0, "iters": sol.iters,
            "dof": S.dof, "rel_res": sol.rel_res_normal}


def oracle_extrapolation(iters):
    """The oracle's time for one step of the full headline workload, scaled
    from measured units of that workload: the assembly and PCA of one full
    subdomain (x J), one Householder QR of a 1200 x 1200 local matrix scaled
    by (n_i / 1200)^3 over the J extended sets (n_i from the full workload's
    sizes at the measured ranks), and one normal product over that subdomain
    and one local solve per set per iteration (x the GPU's iteration count).
    Returns (seconds, description)."""
    from oracle import assembly as asm
    from oracle import linalg as la
    from oracle import solver as sv
    p = headline_workload()
    R, b = ri.weights(p)
    j = 4 + 8 * 4 + 64 * 2
    t0 = time.perf_counter()
    rows, Psi, Hj = asm.block(p, R, b, j)
    pc = sv.pca(Psi, p.pca_mode, p.pca_thr)
    B = Hj @ pc.V
    t_block = time.perf_counter() - t0
    x = np.random.default_rng(1).standard_normal(B.shape[1])
    t0 = time.perf_counter()
    B.T @ (B @ x)
    t_mv = time.perf_counter() - t0
    n0 = 1200
    A = np.random.default_rng(2).standard_normal((n0, n0))
    A = A @ A.T + n0 * np.eye(n0)
    t0 = time.perf_counter()
    qr = la.householder_qr(A)
    t_qr = time.perf_counter() - t0
    y = np.ones(n0)
    t0 = time.perf_counter()
    la.back_substitute(qr[2], la.apply_qt(qr[0], qr[1], y))
    t_ls = time.perf_counter() - t0
    # extended-set sizes of the full workload at this block's rank
    l = p.sub
    n3 = n2 = 0.0
    for k2 in range(l[2]):
        for k1 in range(l[1]):
            for k0 in range(l[0]):
                cnt = 1
                for k, L in ((k0, l[0]), (k1, l[1]), (k2, l[2])):
                    cnt *= (1 + (k > 0) + (k < L - 1))
                n = cnt * pc.rank
                n3 += n ** 3
                n2 += n ** 2
    total = p.J * t_block + t_qr * n3 / n0 ** 3 + iters * (p.J * t_mv + t_ls * n2 / n0 ** 2)
    desc = (f"oracle units of the full workload: assembly+PCA of subdomain {j} ({Hj.shape[0]}x{p.neurons}, rank "
            f"{pc.rank}) {t_block:.2f} s x J={p.J}; Householder QR {n0}x{n0} {t_qr:.2f} s scaled by sum n_i^3; "
            f"per iteration: normal product {t_mv * 1e3:.2f} ms x J and QR solve {t_ls * 1e3:.1f} ms scaled by "
            f"sum n_i^2, x {iters} iterations (extrapolated)")
    return total, desc


def reference_arm(args):
    """The oracle as it stands, on the host cores: each step is one complete
    pass of the hot path on the scaled-down instance (a measured time); the
    full workload's time, extrapolated from measured units, is reported
    beside it."""
    p = oracle_sample_problem()
    for _ in range(args.warmup):                 # untimed, like the GPU arm's warm-up steps
        oracle_pass(p)
    vals = []
    for _ in range(args.steps):
        r = oracle_pass(p)
        vals.append(r["total"])
    v = float(np.mean(vals))
    ext, ext_desc = oracle_extrapolation(args.iters_hint)
    cores = os.cpu_count()
    sample = (f"complete oracle pass (assembly+PCA, AS set-up by Householder QR, AS-CG to 1e-10) on heat3d "
              f"3x3x2 subdomains, 6x6x4 pts/cell, m=40 (DoF {r['dof']}, {r['iters']} CG iterations): "
              f"build {r['build']:.2f} s, setup {r['setup']:.2f} s, solve {r['solve']:.2f} s; numpy default threads")
    return {"impl": "reference", "metric": METRIC, "value": round(v, 4), "unit": "s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(v * 1e3, 1), "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD_DESC, "sample": "scaled-down instance (see cpu_baseline.sample)"},
            "cpu_baseline": {"value": round(v, 4), "unit": "s", "cores": cores, "kind": "oracle", "sample": sample},
            "extrapolated_full_workload": {"value": round(ext, 2), "unit": "s", "how": ext_desc},
            "e2e": {"value": round(v, 4), "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--iters-hint", type=int, default=377)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-multiscale", action="store_true", help="skip the multiscale precision-mode arms")
    ap.add_argument("--no-batch", action="store_true", help="skip the piecewise-coefficient differentiable batch")
    ap.add_argument("--small", action="store_true",
                    help="headline problem on 3x3x2 subdomains with 12x12x6 points (a few GB, for ncu captures)")
    ap.add_argument("--multi-rhs", type=int, default=0,
                    help="also time AS-CG and the workload's GMRES on this many right-hand sides in lockstep "
                         "against one at a time (multiscale workload)")
    args = ap.parse_args()
    if args.small:
        global SMALL, WORKLOAD_DESC
        SMALL = True
        WORKLOAD_DESC = ("heat3d (space-time heat u_t = 0.1 Lap u) 3x3x2 subdomains, m=400, 12x12x6 pts/subdomain "
                         "(profiling case), overlap ratio 1.4, PCA 1-1e-12, AS-CG on the normal equations, rtol 1e-10")
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        if rank != 0:
            return
        print(json.dumps(reference_arm(args)))
        return
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    out = bench_ours(args, rank, world)
    if rank == 0:
        if not args.no_cpu_baseline:
            v, sample = oracle_extrapolation(out["config"]["iters"])
            out["cpu_baseline"] = {"value": round(v, 3), "unit": "s", "cores": os.cpu_count(), "kind": "oracle",
                                   "sample": sample}
        print(json.dumps(out))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
