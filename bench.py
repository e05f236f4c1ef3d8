"""Benchmark: time to relative residual 1e-10 of the RaNN domain-decomposition
solver on the 2D multiscale diffusion workload.

Workload: -div(a grad u) = 1 on [0,1]^2, a = 2 + sin(2 pi x/eps) sin(2 pi y/eps),
eps = 1/16; 8 x 8 subdomains, overlap 0.05; 300 tanh neurons per subdomain,
weights U[-2, 2] (seeded); 40 x 40 collocation points per subdomain cell
(320 x 320 global); PCA keeping 1 - 1e-12 of the variance; restricted additive
Schwarz GMRES(50) on the normal equations (scaled partition of unity D_i),
rtol 1e-10.  One step = the whole hot path: assembly, right-hand side, PCA and
reduction, preconditioner set-up, Krylov solve.  Synthetic, seeded inputs.

Prints one JSON line.  --impl reference times the CPU oracle (float64 numpy)
on a bounded sample of the same workload, scaled to a whole step.
"""
from __future__ import annotations

import argparse
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

METRIC = "time to rel. residual 1e-10 (RAS-GMRES, full hot path)"
WORKLOAD_DESC = ("multiscale2d 8x8 subdomains, m=300, 40x40 pts/subdomain (320x320), overlap 0.05, "
                 "PCA 1-1e-12, RAS(scaled D_i)-GMRES(50), rtol 1e-10")
FP64_PEAK_TFLOPS = 152 * 4 * 2.07e9 / 1e12   # 152 SMs x 2 float64 FMA/clk x 2 flop x 2.07 GHz
DF32_PEAK_TFLOPS = 152 * 128 * 2.07e9 / 12 * 2 / 1e12   # double-float multiply-add: 12 float32 instructions
# DRAM bytes of one launch of the kernel family (dram__bytes_read.sum +
# dram__bytes_write.sum of one ncu --set full capture of the same kernel code
# on this workload); a family missing here reports null
TRAFFIC = {"eig_tridiag": 28.54e6}
# families whose profiled bracket spans a multi-stream pipeline of many kernels
# (the Cholesky with lookahead and the row-block inverse): no single launch
# duration, so they are reported as pipelines, not as the roofline kernel
PIPELINED = {"cholesky"}


def workload():
    p = ri.multiscale2d()
    p.precond = "sas"
    return p


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "_fallback": True}


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
            self.proc = subprocess.Popen(["nvidia-smi", "-i", os.environ.get("CUDA_VISIBLE_DEVICES", "0").split(",")[0],
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


def run_step(g, s, p, F):
    s.assemble()
    s.rhs(F)
    ranks = s.pca(p.pca_mode, p.pca_thr)
    s.setup_precond(p.precond)
    W, st = s.solve_gmres_ras(F, p.rtol, p.restart, p.maxit)
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
    p = workload()
    R, b = ri.weights(p)
    s = g.RannDD(p, R, b)
    F = s._empty(s.sizes()["n_points"])
    stream = torch.cuda.current_stream()

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    for _ in range(args.warmup):
        W, st, ranks = run_step(g, s, p, F)
    barrier()
    times = []
    with Clocks() as clk:
        for _ in range(args.steps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            W, st, ranks = run_step(g, s, p, F)
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
        barrier()
    # one further step with every launch bracketed by CUDA events on the handle's
    # stream: the kernel breakdown and the roofline (not part of the timed steps)
    s.profile(True)
    run_step(g, s, p, F)
    torch.cuda.synchronize()
    prof = s.profile_read()
    s.profile(False)
    prof_steps = 1
    ms = max_over_ranks(float(np.mean(times)), world)
    # end to end through the public API with host buffers: weights in, W out
    Rh = torch.tensor(R).pin_memory()
    bh = torch.tensor(b).pin_memory()
    e2e = []
    for rep in range(max(2, min(args.steps, 3)) + 1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s2 = g.RannDD(p, Rh.numpy(), bh.numpy())
        F2 = s2._empty(s2.sizes()["n_points"])
        W2, st2, _ = run_step(g, s2, p, F2)
        Wh = torch.empty(W2.shape, dtype=torch.float64).pin_memory()
        Wh.copy_(W2)
        torch.cuda.synchronize()
        s2.close()
        if rep > 0:
            e2e.append(time.perf_counter() - t0)
    pk = peaks()
    launches = sum(v["launches"] for v in prof.values()) // prof_steps
    dom_name, dom = max(((k, v) for k, v in prof.items() if k not in PIPELINED), key=lambda kv: kv[1]["ms"])
    bound = dom["bound"]
    if bound == "hbm":
        ach = dom["bytes"] / (dom["ms"] * 1e-3) / 1e9
        peak, unit = pk["hbm_gbs"], "GB/s"
        peak_note = "measured HBM copy (MEASURED_PEAKS.json)"
    elif bound == "tensor":
        ach = dom["flops"] / (dom["ms"] * 1e-3) / 1e12
        peak, unit = pk.get("bf16_tflops_sustained", pk.get("bf16_tflops")), "TFLOP/s"
        peak_note = "measured cuBLAS bf16, sustained (MEASURED_PEAKS.json); flops of the digit-slice products"
    elif bound == "alu_df32":
        ach = dom["flops"] / (dom["ms"] * 1e-3) / 1e12
        peak, unit = DF32_PEAK_TFLOPS, "TFLOP/s"
        peak_note = ("double-float multiply-add: 152 SMs x 128 float32 lanes x 2.07 GHz / 12 float32 "
                     "instructions x 2 flops (unit counts x max clock), float64-equivalent flops")
        bound = "alu"
    else:
        ach = dom["flops"] / (dom["ms"] * 1e-3) / 1e12
        peak, unit = FP64_PEAK_TFLOPS, "TFLOP/s"
        peak_note = "float64 FMA: 152 SMs x 2 FMA/clk x 2.07 GHz (unit counts x max clock)"
    # the block products: the inner iterations' normal-matrix block rows (double-float) and the float64
    # two-pass B^T (B x) of the residuals that decide convergence
    def gbps(names):
        fam = [prof[n] for n in names if prof.get(n, {}).get("ms")]
        if not fam:
            return None
        by, t = sum(f["bytes"] for f in fam), sum(f["ms"] for f in fam)
        return {"GBps": round(by / (t * 1e-3) / 1e9, 1), "frac_of_hbm": round(by / (t * 1e-3) / 1e9 / pk["hbm_gbs"], 4),
                "launches_per_step": sum(f["launches"] for f in fam) // prof_steps}
    kernels = {k: {"ms_per_step": round(v["ms"] / prof_steps, 3), "launches_per_step": v["launches"] // prof_steps}
               for k, v in sorted(prof.items(), key=lambda kv: -kv[1]["ms"]) if v["launches"]}
    clocks = clk.summary()
    out = {
        "metric": METRIC, "value": round(ms / 1e3, 6), "unit": "s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms, 3), "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded SplitMix64 weights, manufactured PDE data)",
        "config": {"workload": WORKLOAD_DESC,
                   "dof": int(np.sum(ranks)), "iters": st["iters"], "rel_res_true": st["rel_res_true"],
                   "rel_res_prec": st["rel_res_prec"], "parallelism": f"replicas x{world}",
                   "l2": "working set > L2 (reduced blocks 8*sum N_j p_j bytes, factors), no flush"},
        "roofline": {"kernel": dom_name, "bound": bound, "achieved": round(ach, 3), "peak": peak,
                     "unit": unit, "frac": round(ach / peak, 4), "traffic": TRAFFIC.get(dom_name),
                     "peak_source": peak_note},
        "matvec": {"normal_rows_df32": gbps(["gramop_df32"]),
                   "H_f64": gbps(["matvec_H"]), "HT_f64": gbps(["matvec_HT"]),
                   "H_df32": gbps(["matvec_H_df32"]), "HT_df32": gbps(["matvec_HT_df32"]),
                   "schwarz_apply_df32": gbps(["schwarz_apply_df32", "trmv_lower_df32", "trmv_upper_df32"])},
        "pipelines": {k: {"ms_per_step": round(prof[k]["ms"] / prof_steps, 3),
                          "launches_per_step": prof[k]["launches"] // prof_steps,
                          "achieved_tflops": round(prof[k]["flops"] / (prof[k]["ms"] * 1e-3) / 1e12, 3),
                          "frac_of_df32_peak": round(prof[k]["flops"] / (prof[k]["ms"] * 1e-3) / 1e12
                                                     / DF32_PEAK_TFLOPS, 4)}
                      for k in sorted(PIPELINED) if prof.get(k, {}).get("ms")},
        "kernels": kernels,
        "gpu_launches": int(launches) * args.steps,
        "gpu_launches_per_step": int(launches),
        "e2e": {"value": round(float(np.median(e2e)), 6), "unit": "s",
                "h2d_bytes_per_step": int(R.nbytes + b.nbytes), "d2h_bytes_per_step": int(W.numel() * 8)},
        "clocks": clocks,
    }
    if args.multi_rhs > 0:
        out["multi_rhs"] = [multi_rhs_timing(g, p, R, b, args.multi_rhs, "cg"),
                            multi_rhs_timing(g, p, R, b, args.multi_rhs, "gmres")]
    return out


def multi_rhs_timing(g, p, R, b, k, solver="cg"):
    """k right-hand sides of the workload (F scaled by 1..k, so every column
    runs the same iterations): k one-column solves one after another against
    one lockstep solve of all k (every operator and preconditioner launch
    serves all columns).  solver "cg": AS-preconditioned CG; "gmres": the
    workload's SAS-preconditioned GMRES(50).  Both after a warm-up solve; wall
    time with the device synchronised on both sides (the solves include their
    host round trips)."""
    import torch
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


def cpu_sample(args):
    """The oracle, as it stands, on a bounded sample of the workload scaled to
    a whole step: the 3 x 3 neighbourhood of an interior subdomain is built
    with the oracle's own assembly and PCA (time per subdomain x J), the
    centre's extended-set matrix A_i is formed and factored by the oracle's
    Householder QR (x J sets), and one preconditioned normal-matrix product
    over the sample is timed (x J/9 for the products, x J local solves, x the
    GPU's Krylov iteration count)."""
    from oracle import linalg as la
    from oracle import solver as sv
    p = workload()
    R, b = ri.weights(p)
    J, l = p.J, p.sub[0]
    c = (l // 2) * l + l // 2
    hood = [c + dy * l + dx for dy in (-1, 0, 1) for dx in (-1, 0, 1)]
    t0 = time.perf_counter()
    S = sv.build_system(p, R, b, blocks_subset=hood)
    t_build = (time.perf_counter() - t0) / len(hood)
    t0 = time.perf_counter()
    A = sv.local_matrix(S, list(range(len(hood))))
    qr = la.householder_qr(A)
    t_setup = time.perf_counter() - t0
    x = np.random.default_rng(1).standard_normal(S.dof)
    t0 = time.perf_counter()
    y = S.normal(x)
    t_mv = time.perf_counter() - t0
    t0 = time.perf_counter()
    la.back_substitute(qr[2], la.apply_qt(qr[0], qr[1], y))
    t_ls = time.perf_counter() - t0
    iters = args.iters_hint
    total = J * (t_build + t_setup) + iters * (t_mv * J / len(hood) + t_ls * J)
    return total, (f"oracle on the 3x3 neighbourhood of subdomain {c}: assembly+PCA "
                   f"{t_build:.2f} s/subdomain, A_i ({A.shape[0]}x{A.shape[0]}) + Householder QR {t_setup:.2f} s, "
                   f"normal product {t_mv * 1e3:.1f} ms/9 blocks, local solve {t_ls * 1e3:.1f} ms; "
                   f"scaled by J={J} and {iters} Krylov iterations (extrapolated)")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--iters-hint", type=int, default=71)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--multi-rhs", type=int, default=0,
                    help="also time AS-CG and the workload's GMRES on this many right-hand sides in lockstep "
                         "against one at a time")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        if rank != 0:
            return
        vals = []
        for _ in range(args.steps):
            v, sample = cpu_sample(args)
            vals.append(v)
        v = float(np.mean(vals))
        cores = os.cpu_count()
        print(json.dumps({"impl": "reference", "metric": METRIC, "value": round(v, 4), "unit": "s",
                          "n_gpus": args.gpus, "steps": args.steps, "warmup": 0, "ms_per_step": round(v * 1e3, 1),
                          "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                          "data": "synthetic", "config": {"workload": WORKLOAD_DESC},
                          "cpu_baseline": {"value": round(v, 4), "unit": "s", "cores": cores, "kind": "oracle",
                                           "sample": sample},
                          "e2e": {"value": round(v, 4), "unit": "s", "h2d_bytes_per_step": 0,
                                  "d2h_bytes_per_step": 0}}))
        return
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    out = bench_ours(args, rank, world)
    if rank == 0:
        if not args.no_cpu_baseline:
            args.iters_hint = out["config"]["iters"]
            v, sample = cpu_sample(args)
            out["cpu_baseline"] = {"value": round(v, 3), "unit": "s", "cores": os.cpu_count(), "kind": "oracle",
                                   "sample": sample}
        print(json.dumps(out))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
