"""Benchmark of the recursive-skeletonization hot path on GB300.

One step = one pass of the whole hot path over one batch of synthetic input:
rs_build (tree, proxy compression + ID, block elimination, root) of the
131072-point starfish 2D Laplace system (eps 1e-10, leaf 64, 64 proxies)
followed by rs_solve_refined of a 256-column right-hand-side batch to
relative residual <= 1e-10 (FP32 solves, FP64 residual of the compressed
operator).  `value` = right-hand sides solved per second over whole steps.

Also reported (same run): build time, the resident-factorization refined
throughput, the plain FP64 one-RHS-at-a-time solve throughput, the roofline
of the dominant kernel (CUDA events on the library's stream), clocks during
the timed region, an end-to-end number through the C ABI with host buffers,
and the CPU oracle timed on this host.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Multi-GPU: launched under torchrun; each rank builds and solves its own
replica (no collective on the data path); value = all ranks' RHS / max time.
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import rs_inputs as ri  # noqa: E402

WORKLOAD = "laplace2d_starfish_131072"
METRIC = "RHS solves/s at rel. residual<=1e-10 (served vs plain FP64); build s; p50/p99 ms"
NRHS = 256
TOL = 1e-10
SERVE_COLS = 1024   # column cap of one served batch (continuous batching)


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return dict(hbm=float(d["hbm_gbs"]), bf16=float(d["bf16_tflops"]), src="measured")
    return dict(hbm=6800.0, bf16=1900.0, src="fallback")


# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of one launch per
# kernel category, from the ncu captures summarised in profiles/ (the leaf-level
# launch of the bench workload); None where no capture of the current kernel exists.
# FP64 pipe utilisation of the same launch (sm__inst_executed_pipe_fp64, % of
# peak sustained active): the ID's algorithmic flops exclude the fill and the
# pivoting arithmetic, so its roofline fraction reads far below the pipe.
NCU_FP64_PIPE = {"id": 0.875}
NCU_TRAFFIC = {"id": (48086272 + 795648,
                      "k_id leaf-level launch (profiles/k_id_leaf_laplace2d_starfish_131072.md): "
                      "dram__bytes_read.sum + dram__bytes_write.sum")}

# FP64 FMA throughput of GB300: 152 SMs x 2 FP64 FMA/clk x 2 flop x 2.07 GHz
# = 1.26 TFLOP/s nominal; a dependent-chain-free probe measured 1.195 TFLOP/s.
FP64_PEAK_GFLOPS = 152 * 2 * 2 * 2.07
FP32_PEAK_GFLOPS = 152 * 128 * 2 * 2.07


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, index):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={index}", f"--query-gpu={q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        self.p.wait()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.strip()]
        sm = [float(r[1]) for r in rows if len(r) > 8 and r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if len(r) > 8 and r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in rows:
            if len(r) > 8:
                for nm, v in zip(names, r[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows)}


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(ms: float, dist, device: str) -> float:
    """The slowest rank's time (each rank solves its own replica problem; the
    job is done when the last one is)."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(ws: int, nrhs: int, steps: int, ms: float) -> float:
    """Whole-job RHS/s: every rank solves nrhs columns per step (weak scaling)."""
    return ws * nrhs * steps / (ms / 1e3)


def workload_inputs():
    w = ri.WORKLOADS[WORKLOAD]
    pts, h = ri.starfish(w["n"])
    return w, pts, h


def oracle_step_sample(n_sample: int) -> float:
    """Seconds of one oracle step on a sample: build at n_sample + solve NRHS."""
    code = f"""
import sys, time, numpy as np
sys.path.insert(0, {ROOT!r})
import rs_inputs as ri
from oracle import rskel
pts, h = ri.starfish({n_sample})
B = ri.rhs({n_sample}, {NRHS}, seed=1)
t = time.perf_counter()
F = rskel.build(pts, rskel.Params(kind='laplace2d', w=h, eps=1e-10, leaf=64, nproxy=64))
X = F.solve(B)
print(time.perf_counter() - t)
"""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, check=True)
    return float(out.stdout.strip().splitlines()[-1])


def cpu_baseline(steps: int = 1):
    """The oracle on this host: single thread, sample = 1/8 of the workload."""
    w = ri.WORKLOADS[WORKLOAD]
    n_sample = w["n"] // 8
    ts = [oracle_step_sample(n_sample) for _ in range(steps)]
    t = min(ts)
    # The 2D build and solve are O(N) (Sec. 4, d = 1), so a step at full N
    # costs N / n_sample times the sample's.
    full = t * w["n"] / n_sample
    return {"value": NRHS / full, "unit": "RHS/s", "cores": 1, "kind": "oracle",
            "sample": f"oracle build + {NRHS}-column solve on the same starfish family at N={n_sample} "
                      f"({t:.2f} s), scaled by N/{n_sample} (O(N) cost in 2D, Sec. 4); single thread",
            "sample_s": t}


def run_reference(args, ws, rank):
    if rank != 0:
        return
    t_all = []
    for _ in range(args.warmup):
        oracle_step_sample(ri.WORKLOADS[WORKLOAD]["n"] // 8)
    for _ in range(args.steps):
        t_all.append(oracle_step_sample(ri.WORKLOADS[WORKLOAD]["n"] // 8))
    n = ri.WORKLOADS[WORKLOAD]["n"]
    scale = n / (n // 8)
    per_step = statistics.median(t_all) * scale
    value = NRHS / per_step
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "RHS/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_step * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "nrhs": NRHS, "tol": TOL},
            "cpu_baseline": {"value": value, "unit": "RHS/s", "cores": 1, "kind": "oracle",
                             "sample": f"each step: oracle build + {NRHS}-column solve at N={n // 8} of the "
                                       f"same starfish family, scaled by {scale:g} (O(N) in 2D)"},
            "e2e": {"value": value, "unit": "RHS/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def serving_session(rs, torch, P, h, w, window_s=1.0, rate=2000.0, seed=7):
    """Poisson arrivals (mean `rate` req/s, 1..64 columns each) for `window_s`
    seconds against the resident factorization, plus one memory-admitted
    build of a random starfish (serving mix form); returns RHS/s and
    latency percentiles of the completed requests."""
    n = w["n"]
    H = rs.rs_build(P, "laplace2d", h, w["eps"], w["leaf"], w["nproxy"])
    S = rs.Server(max_cols=SERVE_COLS)
    hid = S.add(H)
    # warm the server's buffers (and the launch autotuner) with full batches
    for cols in (SERVE_COLS, SERVE_COLS // 2):
        Bw = torch.from_numpy(ri.rhs(n, cols, seed=900)).t().contiguous().pin_memory().t()
        Xw = torch.empty((cols, n), dtype=torch.float64).pin_memory().t()
        S.wait(S.submit(hid, Bw, Xw))
    nb, arms, amp, rot = ri.serving_curve(seed, 0)
    pts2, h2 = ri.starfish(16384, arms=arms, amp=amp, rotation=rot)
    bt = S.submit_build(pts2, "laplace2d", h2, w["eps"], w["leaf"], w["nproxy"])
    S.reset_stats()
    u = ri.uniform01(seed, 200000, stream=7)
    gaps = -np.log(u) / rate
    cols = 1 + (ri.uniform01(seed, 200000, stream=8) * 64).astype(int).clip(0, 63)
    B = torch.from_numpy(ri.rhs(n, 64, seed=901)).t().contiguous().pin_memory().t()
    ring = [torch.empty((64, n), dtype=torch.float64).pin_memory().t() for _ in range(8)]
    tickets, i = [], 0
    t0 = time.perf_counter()
    t_next = t0
    while True:
        now = time.perf_counter()
        if now - t0 >= window_s:
            break
        if now < t_next:
            time.sleep(min(t_next - now, 0.0005))
            continue
        c = int(cols[i])
        tickets.append(S.submit(hid, B[:, :c], ring[i % len(ring)][:, :c]))
        t_next += gaps[i]
        i += 1
    offered = sum(int(cols[j]) for j in range(i)) / window_s
    worst, bad = 0.0, 0
    for t in tickets:
        r = S.wait(t)
        bad += r["status"] != 0
        worst = max(worst, r["relres"])
    st = S.stats()
    rb = S.wait(bt)
    S.destroy()
    H.free()
    return {"rhs_per_s": st["rhs"] / st["elapsed_s"], "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"],
            "requests": st["requests"], "failed": bad, "mean_batch_cols": st["mean_batch_cols"],
            "offered_rhs_per_s": offered, "arrival_rate_per_s": rate, "window_s": window_s,
            "relres_max": worst, "admitted_build_status": rb["status"],
            "note": "offered load above capacity: latency includes queueing"}


def run_ours(args, ws, rank, local):
    import torch
    import paper_1110_3105_gb300 as rs

    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    w, pts, h = workload_inputs()
    n = w["n"]
    Bh = ri.rhs(n, NRHS, seed=100 + rank)
    # device-resident inputs (point-major points, column-major B)
    P = torch.from_numpy(np.ascontiguousarray(pts.T)).cuda().t()
    B = torch.from_numpy(Bh).cuda().t().contiguous().t()
    X = torch.zeros_like(B)
    stream = torch.cuda.current_stream()

    def step():
        H = rs.rs_build(P, "laplace2d", h, w["eps"], w["leaf"], w["nproxy"], stream=stream)
        its, rel = rs.rs_solve_refined(H, B, X, tol=TOL, max_it=8, stream=stream)
        H.free()
        return its, rel

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        step()
    barrier()
    clk = Clocks(local)
    launches0 = rs.rs_launch_count()
    rs.rs_profile_enable(True)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    rels, itss = [], []
    for _ in range(args.steps):
        its, rel = step()
        rels.append(float(np.max(rel)))
        itss.append(its)
    e1.record(stream)
    barrier()
    clocks = clk.stop()
    launches = rs.rs_launch_count() - launches0
    prof = rs.rs_profile_read()
    rs.rs_profile_enable(False)
    ms = max_over_ranks(e0.elapsed_time(e1), dist, "cuda")
    ms_step = ms / args.steps
    value = replica_throughput(ws, NRHS, args.steps, ms)

    # breakdown on the resident factorization (outside the timed region)
    H = rs.rs_build(P, "laplace2d", h, w["eps"], w["leaf"], w["nproxy"], stream=stream)
    st = H.stats()
    torch.cuda.synchronize()
    tb, tbd = [], []
    for _ in range(3):
        Ht = rs.rs_build(P, "laplace2d", h, w["eps"], w["leaf"], w["nproxy"], stream=stream)
        tb.append(Ht.stats()["build_ms"])
        Ht.free()
        Ht = rs.rs_build(P, "laplace2d", h, w["eps"], w["leaf"], w["nproxy"], stream=stream, id_arith="dfloat")
        tbd.append(Ht.stats()["build_ms"])
        Ht.free()
    rs.rs_solve_refined(H, B, X, tol=TOL, max_it=8, stream=stream)
    torch.cuda.synchronize()
    t = time.perf_counter()
    reps = 3
    for _ in range(reps):
        its, rel = rs.rs_solve_refined(H, B, X, tol=TOL, max_it=8, stream=stream)
    torch.cuda.synchronize()
    refined_ms = (time.perf_counter() - t) / reps * 1e3
    b1 = B[:, :1].clone()
    x1 = torch.zeros_like(b1)
    for _ in range(5):
        rs.rs_solve(H, b1, x1, stream=stream)
    torch.cuda.synchronize()
    t = time.perf_counter()
    nplain = 50
    for _ in range(nplain):
        rs.rs_solve(H, b1, x1, stream=stream)
    torch.cuda.synchronize()
    plain_us = (time.perf_counter() - t) / nplain * 1e6
    # residual of the plain FP64 solve against the compressed operator
    y1 = torch.zeros_like(b1)
    rs.rs_matvec(H, x1, y1, stream=stream)
    torch.cuda.synchronize()
    plain_rel = float(torch.linalg.norm(y1 - b1) / torch.linalg.norm(b1))

    # end to end through the C ABI with host buffers (pinned), copies inside
    Bp = torch.empty((NRHS, n), dtype=torch.float64, pin_memory=True)
    Bp.copy_(torch.from_numpy(np.ascontiguousarray(Bh.T)))
    Bp = Bp.t()                                   # n x NRHS, column-major, pinned
    Xp = torch.empty((NRHS, n), dtype=torch.float64, pin_memory=True).t()
    pts_host = np.asfortranarray(pts)
    H.free()
    Hh = rs.rs_build(pts_host, "laplace2d", h, w["eps"], w["leaf"], w["nproxy"])
    rs.rs_solve_refined(Hh, Bp, Xp, tol=TOL, max_it=8)
    Hh.free()
    torch.cuda.synchronize()
    t = time.perf_counter()
    e2e_steps = max(1, min(args.steps, 3))
    for _ in range(e2e_steps):
        Hh = rs.rs_build(pts_host, "laplace2d", h, w["eps"], w["leaf"], w["nproxy"])
        rs.rs_solve_refined(Hh, Bp, Xp, tol=TOL, max_it=8)
        Hh.free()
    torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t) / e2e_steps

    serving = others = None
    if not args.no_serve:
        try:
            serving = serving_session(rs, torch, P, h, w)
        except Exception as e:   # keep the main measurement
            serving = {"error": f"{type(e).__name__}: {e}"}
    if rank == 0 and not args.no_serve:
        try:
            others = other_configs(rs, torch, stream)
        except Exception as e:
            others = {"error": f"{type(e).__name__}: {e}"}

    # roofline of the dominant kernel category in the timed region
    pk = peaks()
    dom_name, dom = max(prof.items(), key=lambda kv: kv[1]["ms"])
    if dom["bytes"] > 0 and dom["flops"] / max(dom["bytes"], 1.0) < 0.5:
        bound, achieved, peak, unit = "hbm", dom["bytes"] / dom["ms"] / 1e6, pk["hbm"], "GB/s"
        peak_src = f"{pk['src']} copy bandwidth"
    else:
        bound, achieved, peak, unit = "alu", dom["flops"] / dom["ms"] / 1e6, FP64_PEAK_GFLOPS, "GFLOP/s"
        peak_src = "FP64 FMA peak 152 SM x 2 FMA/clk x 2.07 GHz (derived)"
    traffic = NCU_TRAFFIC.get(dom_name)
    roof = {"bound": bound, "kernel": dom_name, "achieved": achieved, "peak": peak, "unit": unit,
            "frac": achieved / peak, "traffic": traffic[0] if traffic else None,
            "traffic_source": traffic[1] if traffic else None, "peak_source": peak_src,
            "launches": dom["launches"], "avg_launch_ms": dom["ms"] / dom["launches"],
            "ncu_fp64_pipe_active": NCU_FP64_PIPE.get(dom_name)}
    kernels = {k: {"ms_per_step": v["ms"] / args.steps, "launches_per_step": v["launches"] / args.steps,
                   "GB_s": v["bytes"] / v["ms"] / 1e6 if v["ms"] else 0.0,
                   "GFLOP_s": v["flops"] / v["ms"] / 1e6 if v["ms"] else 0.0} for k, v in prof.items()}

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return
    cpu = cpu_baseline() if ws == 1 and not args.no_cpu else None
    h2d = pts.size * 8 + n * NRHS * 8
    d2h = n * NRHS * 8
    line = {
        "metric": METRIC, "value": value, "unit": "RHS/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": n, "eps": w["eps"], "leaf": w["leaf"], "nproxy": w["nproxy"],
                   "nrhs_per_step": NRHS, "tol": TOL,
                   "step": "rs_build + rs_solve_refined(256 columns)",
                   "l2": "inputs larger than L2: B is 268 MB and every step rebuilds 0.33 GB of factors"},
        "clocks": clocks,
        "e2e": {"value": NRHS / e2e_s, "unit": "RHS/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": launches,
        "roofline": roof,
        "cpu_baseline": cpu,
        "build_ms": statistics.median(tb),
        "build_ms_dfloat_id": statistics.median(tbd),
        "resident_refined_ms_per_batch": refined_ms,
        "resident_refined_rhs_per_s": NRHS / (refined_ms / 1e3),
        "plain_fp64_rhs_per_s": 1e6 / plain_us,
        "batched_vs_plain": (NRHS / (refined_ms / 1e3)) / (1e6 / plain_us),
        "serving": serving,
        "served_vs_plain": (serving["rhs_per_s"] / (1e6 / plain_us)) if serving and "rhs_per_s" in serving else None,
        "refine_iterations": itss,
        "relres_max": max(rels),
        "plain_fp64_relres": plain_rel,
        "factor_bytes": st["factor_bytes"],
        "top_skeletons": st["top_skeletons"],
        "kernels": kernels,
        "other_configs": others,
    }
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def other_configs(rs, torch, stream):
    """Build time and a refined multi-RHS solve on the other workloads (one
    build each, after the main measurement; device-resident inputs)."""
    out = {}
    for name, nrhs, tol in (("helmholtz2d_starfish_65536", 64, 1e-9), ("laplace3d_sphere_32768", 256, 1e-10),
                            ("helmholtz3d_sphere_8192", 64, 1e-10)):
        wl = ri.WORKLOADS[name]
        pts, wt = ri.geometry(wl["geom"], wl["n"])
        n, kw = wl["n"], wl.get("kwave", 0.0)
        cplx = wl["kernel"].startswith("helmholtz")
        P = torch.from_numpy(np.ascontiguousarray(pts.T)).cuda().t()
        H = rs.rs_build(P, wl["kernel"], wt, wl["eps"], wl["leaf"], wl["nproxy"], k_wave=kw, stream=stream)
        st = H.stats()
        B = torch.from_numpy(ri.rhs(n, nrhs, seed=300, complex_=cplx)).cuda().t().contiguous().t()
        X = torch.zeros_like(B)
        rs.rs_solve_refined(H, B, X, tol=tol, max_it=8, stream=stream)
        torch.cuda.synchronize()
        t = time.perf_counter()
        its, rel = rs.rs_solve_refined(H, B, X, tol=tol, max_it=8, stream=stream)
        torch.cuda.synchronize()
        ms = (time.perf_counter() - t) * 1e3
        out[name] = {"build_ms": st["build_ms"], "depth": st["depth"], "top_skeletons": st["top_skeletons"],
                     "factor_bytes": st["factor_bytes"], "nrhs": nrhs, "tol": tol,
                     "refined_ms": ms, "refined_rhs_per_s": nrhs / (ms / 1e3), "refine_iterations": its,
                     "relres_max": float(np.max(rel))}
        H.free()
    return out


def profile_step():
    """One warm-up step (it also runs the launch autotuner), then one build +
    refined 256-column solve inside a profiler range (cudaProfilerStart/Stop:
    profile it with ncu --profile-from-start off)."""
    import torch
    import paper_1110_3105_gb300 as rs
    w, pts, h = workload_inputs()
    P = torch.from_numpy(np.ascontiguousarray(pts.T)).cuda().t()
    B = torch.from_numpy(ri.rhs(w["n"], NRHS, seed=100)).cuda().t().contiguous().t()
    X = torch.zeros_like(B)
    for profiled in (False, True):
        torch.cuda.synchronize()
        if profiled:
            torch.cuda.profiler.start()
        H = rs.rs_build(P, "laplace2d", h, w["eps"], w["leaf"], w["nproxy"])
        its, rel = rs.rs_solve_refined(H, B, X, tol=TOL, max_it=8)
        torch.cuda.synchronize()
        if profiled:
            torch.cuda.profiler.stop()
        H.free()
    print(json.dumps({"profile_step": WORKLOAD, "refine_iterations": its, "relres_max": float(np.max(rel))}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=15)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving session")
    ap.add_argument("--profile-step", action="store_true",
                    help="one warm-up step, then one step (build + refined solve) inside a profiler range: "
                         "the command profiled by ncu --profile-from-start off")
    args = ap.parse_args()
    ws, rank, local = dist_setup()
    if args.profile_step:
        profile_step()
        return
    if args.impl == "reference":
        run_reference(args, ws, rank)
    else:
        run_ours(args, ws, rank, local)


if __name__ == "__main__":
    main()
