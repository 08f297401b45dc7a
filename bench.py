"""Benchmark of the recursive-skeletonization hot path on GB300.

One step = one pass of the whole hot path over one batch of synthetic input:
rs_build (tree, proxy compression + ID, block elimination, root) of the
131072-point starfish 2D Laplace system (eps 1e-10, leaf 64, 64 proxies)
followed by rs_solve_refined of a 256-column right-hand-side batch to
relative residual <= 1e-10 (FP32 solves, FP64-accurate residual of the
compressed operator).  `value` = right-hand sides solved per second over
whole steps.

Also reported (same run): build time; the solve phase by itself (one-RHS
FP64 and FP32 solves and the 256-column FP32 solve, each against the HBM
peak and its FMA peak, measured in this run); refined throughput at 1, 16
and 256 columns; the plain FP64 one-RHS-at-a-time solve; the 4096-point
circle (plain FP64, one RHS); a serving session on the mix of resident
factorizations with admitted builds, at the offered rate and below
capacity; the roofline of the dominant kernel (CUDA events on the
library's stream); clocks during the timed region; an end-to-end number
through the C ABI with host buffers; and the CPU oracle timed on this host
(all cores and one core, full size).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Multi-GPU: launched under torchrun; every rank holds its own replica of the
factorization and solves its slice of one global batch of columns (no
collective on the data path); value = all ranks' RHS / max time.
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
DTYPE = "f64 build; f32 solves + double-float residual (refined to 1e-10)"


def peaks():
    """HBM and bf16 denominators: MEASURED_PEAKS.json (written on this pool's
    GPUs before the run), else the fallback figures."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return dict(hbm=float(d["hbm_gbs"]), bf16=float(d["bf16_tflops"]), src="measured")
    return dict(hbm=6800.0, bf16=1900.0, src="fallback")


def ncu_traffic(kernel: str):
    """DRAM bytes per launch of `kernel` from an ncu summary in profiles/, if
    the summary was captured on the current source of that kernel.  A
    summary states it on a line
      bench-traffic: kernel=<name> source=<file> sha256=<hex> dram_bytes=<int> launch=<what>
    where sha256 is the hash of the source file at capture time; once the
    file has changed, the counters no longer describe the kernel and the
    traffic is reported as null."""
    import glob
    import hashlib
    stale = None
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md"))):
        for line in open(path):
            if not line.startswith("bench-traffic:"):
                continue
            kv = dict(t.split("=", 1) for t in line.split()[1:] if "=" in t)
            if kv.get("kernel") != kernel:
                continue
            src = os.path.join(ROOT, kv.get("source", ""))
            cur = hashlib.sha256(open(src, "rb").read()).hexdigest() if os.path.isfile(src) else None
            where = f"of {kernel} ({kv.get('launch', '')} launch)"
            if cur == kv.get("sha256"):
                return int(kv["dram_bytes"]), f"ncu capture {where}, source unchanged since"
            stale = f"ncu capture {where} predates the current source of the kernel"
    return None, stale or "no ncu capture of this kernel"


def cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part")):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.machine()


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


def oracle_steps(n: int, steps: int, workers: int) -> list:
    """Seconds of each of `steps` oracle steps at N = n (build + NRHS-column
    solve of the starfish workload), with the boxes of each level spread
    over `workers` processes (1: one process).  Runs in a fresh interpreter
    that never touches CUDA, so the oracle's worker processes can be forked;
    BLAS is single-threaded so that the workers do not oversubscribe."""
    code = f"""
import sys, time
sys.path.insert(0, {ROOT!r})
import rs_inputs as ri
from oracle import rskel
pts, h = ri.starfish({n})
B = ri.rhs({n}, {NRHS}, seed=1)
bm = rskel.process_box_map({workers}) if {workers} > 1 else None
for _ in range({steps}):
    t = time.perf_counter()
    F = rskel.build(pts, rskel.Params(kind='laplace2d', w=h, eps=1e-10, leaf=64, nproxy=64), bm)
    X = F.solve(B)
    print('STEP', time.perf_counter() - t, flush=True)
"""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, check=True)
    return [float(l.split()[1]) for l in out.stdout.splitlines() if l.startswith("STEP")]


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_baseline():
    """The oracle on this host at the workload's full size: one step on all
    cores (the boxes of a level over worker processes) and one step on one
    core."""
    n = ri.WORKLOADS[WORKLOAD]["n"]
    cores = host_cores()
    t_all = oracle_steps(n, 1, cores)[0]
    t_one = oracle_steps(n, 1, 1)[0]
    return {"value": NRHS / t_all, "unit": "RHS/s", "cores": cores, "kind": "oracle",
            "sample": f"one full step at N={n}: oracle build (boxes of each level over {cores} processes) + "
                      f"{NRHS}-column FP64 solve, {t_all:.2f} s",
            "cpu_model": cpu_model(), "step_s": t_all,
            "single_core": {"value": NRHS / t_one, "step_s": t_one, "cores": 1}}


def run_reference(args, ws, rank):
    """The oracle as the reference arm: each step is one full-size step on all
    host cores (rank 0 only)."""
    if rank != 0:
        return
    n = ri.WORKLOADS[WORKLOAD]["n"]
    cores = host_cores()
    t_all = oracle_steps(n, args.warmup + args.steps, cores)[args.warmup:]
    per_step = sum(t_all) / len(t_all)
    value = NRHS / per_step
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "RHS/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_step * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "nrhs": NRHS, "tol": TOL},
            "cpu_baseline": {"value": value, "unit": "RHS/s", "cores": cores, "kind": "oracle",
                             "sample": f"each step: the full oracle step at N={n} (build with the boxes of each "
                                       f"level over {cores} processes + {NRHS}-column FP64 solve)",
                             "cpu_model": cpu_model()},
            "e2e": {"value": value, "unit": "RHS/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


SERVE_MIX = (("laplace2d_starfish_131072", 1e-10), ("helmholtz2d_starfish_65536", 1e-9),
             ("laplace3d_sphere_32768", 1e-10))


def _pinned(torch, n, cols, cplx, data=None):
    dt = torch.complex128 if cplx else torch.float64
    t = torch.empty((cols, n), dtype=dt).pin_memory()
    if data is not None:
        t.copy_(torch.from_numpy(np.ascontiguousarray(data.T)))
    return t.t()   # n x cols, column-major, pinned


def plain_fp64_rate(rs, torch, H, n, cplx, reps=20):
    """The plain FP64 one-RHS-at-a-time solve rate (RHS/s, host-timed) on H."""
    dt = torch.complex128 if cplx else torch.float64
    b = torch.from_numpy(ri.rhs(n, 1, seed=5, complex_=cplx)).to(dtype=dt).cuda()
    x = torch.zeros_like(b)
    for _ in range(3):
        rs.rs_solve(H, b, x)
    torch.cuda.synchronize()
    t = time.perf_counter()
    for _ in range(reps):
        rs.rs_solve(H, b, x)
    torch.cuda.synchronize()
    return reps / (time.perf_counter() - t)


def serving_session(rs, torch, resident, window_s, rate, seed, build_every_s=5.0, backlog_cols=64 * SERVE_COLS,
                    only_first=False):
    """The serving mix: the `resident` factorizations [(Handle, n, complex,
    tol)] registered with one server; Poisson arrivals at `rate` requests/s
    with U{1..64} columns each, each for a factorization drawn uniformly from
    those resident so far; every `build_every_s` a new 2D Laplace build of a
    random starfish (N in {8192 .. 65536}) is submitted, admitted by free
    HBM, and joins the mix once built.  Arrivals that find more than
    `backlog_cols` columns queued are shed (counted, not submitted).
    Returns throughput, latency percentiles and the admission record, and the
    plain FP64 one-RHS-at-a-time rate of the same column mix: each
    factorization's plain rate weighted by the columns it served (a
    factorization built by the server is timed on it after the session).
    only_first: every request goes to the first resident factorization and
    no builds are submitted."""
    S = rs.Server(max_cols=SERVE_COLS)
    targets = []
    plain = []   # per target: plain FP64 RHS/s (None: measure after the session)

    def add_target(hid, n, cplx, tol, pr=None):
        B = _pinned(torch, n, 64, cplx, ri.rhs(n, 64, seed=901 + len(targets), complex_=cplx))
        ring = [_pinned(torch, n, 64, cplx) for _ in range(4)]
        targets.append((hid, n, cplx, tol, B, ring))
        plain.append(pr)

    for H, n, cplx, tol, pr in resident:
        add_target(S.add(H), n, cplx, tol, pr)
        if only_first:
            break
    for hid, n, cplx, tol, B, ring in targets:   # warm the workers' buffers and the tile autotuner
        Bw = _pinned(torch, n, SERVE_COLS, cplx, ri.rhs(n, SERVE_COLS, seed=900, complex_=cplx))
        Xw = _pinned(torch, n, SERVE_COLS, cplx)
        S.wait(S.submit(hid, Bw, Xw, tol=tol))
    S.reset_stats()
    nreq = int(rate * window_s * 1.5) + 100
    gaps = -np.log(ri.uniform01(seed, nreq, stream=7)) / rate
    cols = 1 + (ri.uniform01(seed, nreq, stream=8) * 64).astype(int).clip(0, 63)
    pick = ri.uniform01(seed, nreq, stream=9)
    tickets, builds, built = [], [], []
    served_cols = [0] * 64
    submitted_cols = shed = shed_cols = offered_cols = 0
    done_cols = 0
    i, nb = 0, 0
    t0 = time.perf_counter()
    t_next, t_build, t_poll = t0, t0, t0
    while True:
        now = time.perf_counter()
        if now - t0 >= window_s:
            break
        if now >= t_build and not only_first:
            n2, arms, amp, rot = ri.serving_curve(seed, nb)
            pts2, h2 = ri.starfish(n2, arms=arms, amp=amp, rotation=rot)
            builds.append((S.submit_build(pts2, "laplace2d", h2, 1e-10, 64, 64), n2))
            nb += 1
            t_build += build_every_s
        if now >= t_poll:
            done_cols = S.stats()["rhs"]
            for bt in list(builds):
                try:
                    r = S.wait(bt[0], timeout_s=1e-4)
                except rs.RSError as e:
                    if e.code == -5:
                        continue
                    raise
                builds.remove(bt)
                built.append(r["status"])
                if r["status"] == 0:
                    add_target(r["result"], bt[1], False, 1e-10)
            t_poll = now + 0.1
        if now < t_next:
            time.sleep(min(t_next - now, 0.0005))
            continue
        c = int(cols[i])
        offered_cols += c
        if submitted_cols - done_cols > backlog_cols:
            shed += 1
            shed_cols += c
        else:
            ti = min(len(targets) - 1, int(pick[i] * len(targets)))
            hid, n, cplx, tol, B, ring = targets[ti]
            tickets.append(S.submit(hid, B[:, :c], ring[i % len(ring)][:, :c], tol=tol))
            submitted_cols += c
            served_cols[ti] += c
        t_next += gaps[i]
        i += 1
    worst, bad = 0.0, 0
    for t in tickets:
        r = S.wait(t)
        bad += r["status"] != 0
        worst = max(worst, r["relres"])
    st = S.stats()
    for bt in builds:
        built.append(S.wait(bt[0])["status"])
    for ti, (hid, n, cplx, tol, B, ring) in enumerate(targets):   # the server is idle now
        if plain[ti] is None and served_cols[ti] > 0:
            plain[ti] = plain_fp64_rate(rs, torch, S.handle(hid, n, cplx), n, cplx)
    S.destroy()
    tot = sum(served_cols[:len(targets)])
    plain_mix = tot / sum(served_cols[ti] / plain[ti] for ti in range(len(targets)) if served_cols[ti] > 0)
    return {"rhs_per_s": st["rhs"] / st["elapsed_s"], "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"],
            "requests": st["requests"], "failed": bad, "mean_batch_cols": st["mean_batch_cols"],
            "offered_rhs_per_s": offered_cols / window_s, "arrival_rate_per_s": rate, "window_s": window_s,
            "shed_requests": shed, "shed_rhs": shed_cols, "backlog_cap_cols": backlog_cols,
            "relres_max": worst, "builds_submitted": nb, "builds_admitted": sum(1 for b in built if b == 0),
            "builds_refused_oom": sum(1 for b in built if b == -2), "factorizations_served": len(targets),
            "resident_gb": st["resident_bytes"] / 1e9, "plain_fp64_mix_rhs_per_s": plain_mix,
            "served_vs_plain_same_mix": st["rhs"] / st["elapsed_s"] / plain_mix}


def serving(rs, torch, H2, n2, plain2, window_s, stream):
    """Configs 2-4 resident (built here besides the benchmark's handle);
    a session at the configuration's rate (2000 requests/s, ~65k RHS/s
    offered), then one at 50% of the capacity that session measured; and a
    session with the 131072-point factorization alone at the same rate."""
    resident = [(H2, n2, False, 1e-10, plain2)]
    own = []
    for name, tol in SERVE_MIX[1:]:
        wl = ri.WORKLOADS[name]
        pts, wt = ri.geometry(wl["geom"], wl["n"])
        cplx = wl["kernel"].startswith("helmholtz")
        H = rs.rs_build(pts, wl["kernel"], wt, wl["eps"], wl["leaf"], wl["nproxy"], k_wave=wl.get("kwave", 0.0))
        own.append(H)
        resident.append((H, wl["n"], cplx, tol, plain_fp64_rate(rs, torch, H, wl["n"], cplx)))
    try:
        sat = serving_session(rs, torch, resident, window_s, 2000.0, seed=7)
        # half the saturated rate: served in smaller batches (less efficient per
        # column than the ~1000-column batches of saturation), so 70% of the
        # saturated rate was measured to sit at the small-batch capacity
        rate2 = 0.5 * sat["rhs_per_s"] / 32.5
        below = serving_session(rs, torch, resident, max(10.0, window_s / 3), rate2, seed=8)
        alone = serving_session(rs, torch, resident, max(10.0, window_s / 3), 2000.0, seed=9, only_first=True)
    finally:
        for H in own:
            H.free()
    return {"mix": [name for name, _ in SERVE_MIX] + ["new 2D Laplace builds, random starfish, N in 8192..65536"],
            "at_config_rate": sat, "below_capacity": below, "laplace2d_starfish_131072_alone": alone}


def solve_phase(rs, torch, H, B, n, stream, pk, fp64_peak, fp32_peak):
    """The solve by itself on the resident factorization: device time per
    launch from the library's CUDA-event profiler, algorithmic bytes = the
    factors one solve reads (FP64 or FP32 copies) + B read and X written
    (double), flops = 2 x stored scalars per column."""
    st = H.stats()
    scal = st["factor_scalars"]
    out = {}
    cases = (("r1_fp64", 1, rs.RS_PREC_FP64, 8, "solve_fp64"), ("r1_fp32", 1, rs.RS_PREC_FP32, 4, "solve_fp32"),
             ("r16_fp64", 16, rs.RS_PREC_FP64, 8, "solve_fp64"), ("r256_fp32", NRHS, rs.RS_PREC_FP32, 4, "solve_fp32"))
    for name, R, prec, sb, cat in cases:
        b = B[:, :R].clone()
        x = torch.zeros_like(b)
        for _ in range(3):
            rs.rs_solve(H, b, x, precision=prec, stream=stream)
        torch.cuda.synchronize()
        reps = 50 if R == 1 else 10
        rs.rs_profile_enable(True)
        for _ in range(reps):
            rs.rs_solve(H, b, x, precision=prec, stream=stream)
        torch.cuda.synchronize()
        prof = rs.rs_profile_read()
        rs.rs_profile_enable(False)
        ms = prof[cat]["ms"] / prof[cat]["launches"]
        by = scal * sb + 2.0 * n * R * 8
        fl = 2.0 * scal * R
        peak = fp64_peak if prec == rs.RS_PREC_FP64 else fp32_peak
        out[name] = {"nrhs": R, "us_per_solve": ms * 1e3, "rhs_per_s": R / (ms * 1e-3),
                     "bytes": by, "GB_s": by / ms / 1e6, "hbm_frac": by / ms / 1e6 / pk["hbm"],
                     "GFLOP_s": fl / ms / 1e6, "fma_frac": fl / ms / 1e6 / peak,
                     "fma_peak": "FP64" if prec == rs.RS_PREC_FP64 else "FP32"}
    return out


def run_ours(args, ws, rank, local):
    import torch
    import paper_1110_3105_gb300 as rs
    from paper_1110_3105_gb300.replicas import column_range

    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    w, pts, h = workload_inputs()
    n = w["n"]
    # this rank's slice of one global batch of ws x NRHS columns
    c0, c1 = column_range(ws * NRHS, ws, rank)
    Bh = ri.rhs_columns(n, c0, c1, seed=100)
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

    # ---- outside the timed region: the parts of the path by themselves
    fp64_peak = rs.rs_probe_fma_peak(rs.RS_PREC_FP64)
    fp32_peak = rs.rs_probe_fma_peak(rs.RS_PREC_FP32)
    pk = peaks()
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
    phase = solve_phase(rs, torch, H, B, n, stream, pk, fp64_peak, fp32_peak)
    refined = {}
    for R in (1, 16, NRHS):
        b = B[:, :R].clone()
        x = torch.zeros_like(b)
        rs.rs_solve_refined(H, b, x, tol=TOL, max_it=8, stream=stream)
        torch.cuda.synchronize()
        reps = 20 if R < NRHS else 3
        t = time.perf_counter()
        for _ in range(reps):
            its, rel = rs.rs_solve_refined(H, b, x, tol=TOL, max_it=8, stream=stream)
        torch.cuda.synchronize()
        rms = (time.perf_counter() - t) / reps * 1e3
        refined[str(R)] = {"ms_per_batch": rms, "rhs_per_s": R / (rms / 1e3), "corrections": its,
                           "relres_max": float(np.max(rel))}
    b1 = B[:, :1].clone()
    x1 = torch.zeros_like(b1)
    for _ in range(5):
        rs.rs_solve(H, b1, x1, stream=stream)
    torch.cuda.synchronize()
    t = time.perf_counter()
    nplain = 100
    for _ in range(nplain):
        rs.rs_solve(H, b1, x1, stream=stream)
    torch.cuda.synchronize()
    plain_us = (time.perf_counter() - t) / nplain * 1e6
    # residual of the plain FP64 solve against the compressed operator
    y1 = torch.zeros_like(b1)
    rs.rs_matvec(H, x1, y1, stream=stream)
    torch.cuda.synchronize()
    plain_rel = float(torch.linalg.norm(y1 - b1) / torch.linalg.norm(b1))
    circle = config1(rs, torch, stream)

    # end to end through the C ABI with host buffers (pinned), copies inside
    Bp = torch.empty((NRHS, n), dtype=torch.float64, pin_memory=True)
    Bp.copy_(torch.from_numpy(np.ascontiguousarray(Bh.T)))
    Bp = Bp.t()                                   # n x NRHS, column-major, pinned
    Xp = torch.empty((NRHS, n), dtype=torch.float64, pin_memory=True).t()
    pts_host = np.asfortranarray(pts)
    Hh = rs.rs_build(pts_host, "laplace2d", h, w["eps"], w["leaf"], w["nproxy"])
    rs.rs_solve_refined(Hh, Bp, Xp, tol=TOL, max_it=8)
    Hh.free()
    torch.cuda.synchronize()
    t = time.perf_counter()
    e2e_steps = max(1, min(args.steps, 5))
    for _ in range(e2e_steps):
        Hh = rs.rs_build(pts_host, "laplace2d", h, w["eps"], w["leaf"], w["nproxy"])
        rs.rs_solve_refined(Hh, Bp, Xp, tol=TOL, max_it=8)
        Hh.free()
    torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t) / e2e_steps

    serve = others = fwd = dlr = None
    if not args.no_serve and rank == 0:
        try:
            serve = serving(rs, torch, H, n, 1e6 / plain_us, args.serve_window, stream)
        except Exception as e:   # keep the main measurement
            serve = {"error": f"{type(e).__name__}: {e}"}
        try:
            others = other_configs(rs, torch, stream)
        except Exception as e:
            others = {"error": f"{type(e).__name__}: {e}"}
        try:
            fwd = forward_apply(rs, torch, stream)
        except Exception as e:
            fwd = {"error": f"{type(e).__name__}: {e}"}
        try:
            dlr = double_layer(rs, torch, stream)
        except Exception as e:
            dlr = {"error": f"{type(e).__name__}: {e}"}
    H.free()

    # roofline of the dominant kernel category in the timed region
    dom_name, dom = max(prof.items(), key=lambda kv: kv[1]["ms"])
    if dom["bytes"] > 0 and dom["flops"] / max(dom["bytes"], 1.0) < 0.5:
        bound, achieved, peak, unit = "hbm", dom["bytes"] / dom["ms"] / 1e6, pk["hbm"], "GB/s"
        peak_src = f"{pk['src']} copy bandwidth (MEASURED_PEAKS.json)"
    else:
        bound, achieved, peak, unit = "alu", dom["flops"] / dom["ms"] / 1e6, fp64_peak, "GFLOP/s"
        peak_src = "FP64 FMA throughput measured in this run (rs_probe_fma_peak)"
    kernel_of = {"id": "k_id", "factor": "k_factor_smem", "solve_fp32": "k_solve_cta", "residual": "k_solve_cta"}
    traffic, traffic_src = ncu_traffic(kernel_of.get(dom_name, dom_name))
    roof = {"bound": bound, "kernel": dom_name, "achieved": achieved, "peak": peak, "unit": unit,
            "frac": achieved / peak, "traffic": traffic, "traffic_source": traffic_src, "peak_source": peak_src,
            "launches": dom["launches"], "avg_launch_ms": dom["ms"] / dom["launches"],
            "work": "algorithmic flops of the pivoted QR and T (4mnk - 2k^2(m+n) + 4k^3/3 + k^2(n-k) per box)"
                    if dom_name == "id" else "algorithmic bytes/flops counted from the block sizes"}
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
    plain = 1e6 / plain_us
    sat = serve.get("at_config_rate") if isinstance(serve, dict) else None
    line = {
        "metric": METRIC, "value": value, "unit": "RHS/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": DTYPE,
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": n, "eps": w["eps"], "leaf": w["leaf"], "nproxy": w["nproxy"],
                   "nrhs_per_step": NRHS, "tol": TOL, "columns": [c0, c1],
                   "step": "rs_build + rs_solve_refined(256 columns)",
                   "l2": "inputs larger than L2: B is 268 MB and every step rebuilds 0.33 GB of factors"},
        "clocks": clocks,
        "e2e": {"value": NRHS / e2e_s, "unit": "RHS/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": launches,
        "roofline": roof,
        "cpu_baseline": cpu,
        "peaks_measured": {"fp64_fma_gflops": fp64_peak, "fp32_fma_gflops": fp32_peak, "hbm_gbs": pk["hbm"],
                           "hbm_source": pk["src"]},
        "build_ms": statistics.median(tb),
        "build_ms_dfloat_id": statistics.median(tbd),
        "solve_phase": phase,
        "refined": refined,
        "resident_refined_rhs_per_s": refined[str(NRHS)]["rhs_per_s"],
        "plain_fp64_rhs_per_s": plain,
        "plain_fp64_relres": plain_rel,
        "batched_vs_plain": refined[str(NRHS)]["rhs_per_s"] / plain,
        "serving": serve,
        # served rate over the plain FP64 one-at-a-time rate of the same
        # request mix (each factorization's own plain rate, weighted by the
        # columns it served); beside it the 131072-point factorization alone
        "served_vs_plain": sat.get("served_vs_plain_same_mix") if sat else None,
        "served_vs_plain_starfish_alone": (serve["laplace2d_starfish_131072_alone"]["served_vs_plain_same_mix"]
                                           if sat else None),
        "refine_iterations": itss,
        "relres_max": max(rels),
        "factor_bytes": st["factor_bytes"],
        "top_skeletons": st["top_skeletons"],
        "circle_4096": circle,
        "kernels": kernels,
        "other_configs": others,
        "forward_apply": fwd,
        "double_layer": dlr,
    }
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def config1(rs, torch, stream):
    """4096 points on the unit circle, eps 1e-9, plain FP64, one RHS: build
    time and one-RHS solve time (device-resident)."""
    wl = ri.WORKLOADS["laplace2d_circle_4096"]
    pts, h = ri.circle(wl["n"])
    P = torch.from_numpy(np.ascontiguousarray(pts.T)).cuda().t()
    tb = []
    for _ in range(3):
        H = rs.rs_build(P, "laplace2d", h, wl["eps"], wl["leaf"], wl["nproxy"], stream=stream)
        tb.append(H.stats()["build_ms"])
        H.free()
    H = rs.rs_build(P, "laplace2d", h, wl["eps"], wl["leaf"], wl["nproxy"], stream=stream)
    b = torch.from_numpy(ri.rhs(wl["n"], 1, seed=0)).cuda()
    x = torch.zeros_like(b)
    for _ in range(5):
        rs.rs_solve(H, b, x, stream=stream)
    torch.cuda.synchronize()
    t = time.perf_counter()
    for _ in range(100):
        rs.rs_solve(H, b, x, stream=stream)
    torch.cuda.synchronize()
    us = (time.perf_counter() - t) / 100 * 1e6
    H.free()
    return {"build_ms": statistics.median(tb), "solve_us": us, "rhs_per_s": 1e6 / us}


# The paper's forward-apply tables (Sec. 6.1, Tables apply-lap-2ds and
# apply-lap-3ds: one CPU core at 2.66 GHz, eps 1e-9): matrix-vector time in
# seconds by N, for context beside rs_matvec's.
PAPER_TMV = {"circle": {4096: 1.0e-3, 32768: 1.4e-2, 131072: 5.7e-2}, "sphere": {4096: 1.1e-2, 8192: 2.9e-2}}


def forward_apply(rs, torch, stream):
    """rs_matvec (the compressed forward operator of eq. multilevel-compression
    applied in FP64, Sec. 3.3: the 'generalized FMM' use) on the shapes of the
    paper's forward-apply tables: the unit circle (2D Laplace) and the unit
    sphere (3D Laplace) at eps 1e-9.  Build time, one-RHS matvec time (CUDA
    events around 20 applications on the stream) and the relative error of 64
    sampled rows against the dense product."""
    out = []
    for geom, kind, n, leaf, nproxy in (("circle", "laplace2d", 4096, 64, 64), ("circle", "laplace2d", 32768, 64, 64),
                                        ("circle", "laplace2d", 131072, 64, 64),
                                        ("sphere", "laplace3d", 4096, 128, 216),
                                        ("sphere", "laplace3d", 8192, 128, 216)):
        pts, w = ri.geometry(geom, n)
        H = rs.rs_build(pts, kind, w, 1e-9, leaf, nproxy, stream=stream)
        st = H.stats()
        x = torch.from_numpy(ri.rhs(n, 1, seed=4)).cuda()
        y = torch.zeros_like(x)
        for _ in range(3):
            rs.rs_matvec(H, x, y, stream=stream)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        reps = 20
        for _ in range(reps):
            rs.rs_matvec(H, x, y, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        mv_ms = e0.elapsed_time(e1) / reps
        # Sec. 6.1's E on 64 sampled rows: (A x)_i = x_i + w sum_{j != i} G_ij x_j
        # with G from the library's own Green's-function evaluation (rs_green)
        rows = np.random.default_rng(n).choice(n, 64, replace=False)
        xh, yh = x.cpu().numpy()[:, 0], y.cpu().numpy()[:, 0]
        d = pts[:, rows][:, :, None] - pts[:, None, :]
        s2 = np.einsum("dij,dij->ij", d, d)
        s2[np.arange(64), rows] = 1.0
        G = rs.rs_green(kind, s2.ravel()).reshape(64, n)
        G[np.arange(64), rows] = 0.0
        ya = xh[rows] + w * (G @ xh)
        err = float(np.linalg.norm(yh[rows] - ya) / np.linalg.norm(ya))
        out.append({"geometry": geom, "kernel": kind, "n": n, "eps": 1e-9, "build_ms": st["build_ms"],
                    "top_skeletons": st["top_skeletons"], "factor_bytes": st["factor_bytes"],
                    "matvec_ms": mv_ms, "rel_err_sampled_rows": err,
                    "paper_tmv_ms_one_cpu_core": PAPER_TMV[geom].get(n, None) and PAPER_TMV[geom][n] * 1e3})
        H.free()
    return out


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


# The paper's 2D Laplace solver table (Sec. 6.2, Table solve-lap-2d: the
# double-layer interior Dirichlet problem on the ellipse, eps 1e-9, one CPU
# core at 2.66 GHz) at N = 131072: compression + factorization seconds,
# solve seconds, the interior error E and the storage in MB.
PAPER_DL_131072 = {"t_build_s": 4.6 + 3.7, "t_solve_s": 7.5e-2, "E": 8.5e-11, "M_MB": 220.0}


def double_layer(rs, torch, stream):
    """The non-symmetric double layer (two-sided IDs, Sec. 3.1) on the paper's
    ellipse at N = 131072: build time, the FP64 one-RHS solve, a refined
    256-column solve, and E, the error of the double-layer potential of the
    solved density at interior points against the exterior point source's
    field (the measurement of Sec. 6.2; evaluated here with numpy on 4
    points, outside the timed work)."""
    name = "laplace2d_dl_ellipse_131072"
    wl = ri.WORKLOADS[name]
    n = wl["n"]
    p, h, nrm, kap = ri.ellipse(n)
    w = -2.0 * h
    H = rs.rs_build(p, wl["kernel"], w, wl["eps"], wl["leaf"], wl["nproxy"], normals=nrm, curvature=kap,
                    stream=stream)
    st = H.stats()
    src = np.array([3.0, 2.0])
    xin = np.array([[0.5, -1.2, 1.6, 0.0], [0.2, -0.3, 0.1, 0.6]])
    f = -np.log(np.hypot(*(p - src[:, None]))) / (2 * np.pi)
    b = torch.from_numpy(-2.0 * f)[None, :].cuda().t()          # N x 1, leading dimension N
    x = torch.zeros((1, n), dtype=torch.float64, device="cuda").t()
    rs.rs_solve(H, b, x, stream=stream)   # warm-up
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(10):
        rs.rs_solve(H, b, x, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    solve_us = e0.elapsed_time(e1) / 10 * 1e3
    sig = x[:, 0].cpu().numpy()
    d = xin[:, :, None] - p[:, None, :]
    kern = np.einsum("dij,dj->ij", d, nrm) / (2 * np.pi * np.einsum("dij,dij->ij", d, d))
    u = h * (kern @ sig)
    ex = -np.log(np.hypot(*(xin - src[:, None]))) / (2 * np.pi)
    E = float(np.max(np.abs(u - ex) / np.abs(ex)))
    B = torch.from_numpy(ri.rhs(n, 256, seed=302)).cuda().t().contiguous().t()
    X = torch.zeros_like(B)
    rs.rs_solve_refined(H, B, X, tol=1e-10, max_it=8, stream=stream)
    torch.cuda.synchronize()
    t = time.perf_counter()
    its, rel = rs.rs_solve_refined(H, B, X, tol=1e-10, max_it=8, stream=stream)
    torch.cuda.synchronize()
    ms = (time.perf_counter() - t) * 1e3
    H.free()
    return {name: {"build_ms": st["build_ms"], "depth": st["depth"], "top_skeletons": st["top_skeletons"],
                   "factor_bytes": st["factor_bytes"], "fp64_solve_us": solve_us, "E_interior": E,
                   "refined_256_ms": ms, "refined_rhs_per_s": 256 / (ms / 1e3), "refine_iterations": its,
                   "relres_max": float(np.max(rel)), "paper_one_cpu_core": PAPER_DL_131072}}


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
    ap.add_argument("--no-serve", action="store_true", help="skip the serving sessions and the other workloads")
    ap.add_argument("--serve-window", type=float, default=60.0, help="seconds of the serving session at the "
                    "configuration's arrival rate (the session below capacity lasts a third of it)")
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
