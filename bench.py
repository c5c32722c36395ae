#!/usr/bin/env python
"""Benchmark of the GB300 FEM Fourier solver.

Workload (default): 2D rectangle [0,1]x[0,2], n = 9, K = 1024 x 1024
(9215^2 = 84,916,225 unknowns), -(1.0 u_xx + 2.5 u_yy) + 1.0 u = f, one seeded
N(0,1) right-hand side.  One step = one complete solve (all passes of the
algorithm plus the float64 refinement of the mixed path).  The headline
``value`` is the mixed-precision solver's DOF/s; the float64 path is timed in
the same run and reported beside it, with both results' relative error against
the FP64 CPU oracle at full size when the CPU baseline runs.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Multi-GPU (N > 1, launched with torch.distributed.run): independent replicas,
one right-hand side per rank, no collective on the data path.
"""

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "FEM DOF/s per solve, mixed vs FP64 on GPU at rel err \u22641e-10; % HBM roofline"
WORKLOADS = {
    "2d": dict(name="2d_n9_K1024x1024_X1x2_a1x2.5_c1", n=9, K=(1024, 1024), X=(1.0, 2.0), a=(1.0, 2.5), c=1.0),
    "3d": dict(name="3d_n9_K64^3", n=9, K=(64, 64, 64), X=(1.0, 1.0, 1.0), a=(1.0, 1.0, 1.0), c=0.0),
    "small": dict(name="2d_n2_K16x16", n=2, K=(16, 16), X=(1.0, 1.0), a=(1.0, 1.0), c=0.0),
    # profiling case of the 2D kernels: fields of 170 MB (above L2), about 1 GB on the device
    "2d_mid": dict(name="2d_n9_K512x512_X1x2_a1x2.5_c1", n=9, K=(512, 512), X=(1.0, 2.0), a=(1.0, 2.5), c=1.0),
}
FP64_PEAK_TFLOPS = 1.25     # nominal GB300 FP64 (profiling recipe table)
FP32_LANE_TOPS = 152 * 128 * 2.07e9 / 1e12   # float32 lane operations per second at the maximum SM clock


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[j] for r in rows for j in range(4) if r[5 + j].lower().startswith("active")})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def max_over_ranks(torch, dist, values, device):
    """Every rank's timings -> the per-quantity maximum over ranks (the job's
    time is its slowest replica's)."""
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.tolist()]


def job_value(units_per_rank, world_size, ms):
    """Whole-job throughput: the units every replica processed / the slowest
    replica's time."""
    return world_size * units_per_rank / (ms * 1e-3)


def time_pipeline(torch, plan, bh, uh, steps, warmup, barrier=None):
    """ms per step of host-to-host solves through the C ABI's host-buffer
    path (fem_fft_solve_host): every step uploads bh, solves and downloads into
    uh, the copies pipelined with neighbouring solves inside the library; the
    timed region runs from an event before the first call to the wait for the
    last download (fem_fft_host_wait)."""
    for _ in range(warmup):
        plan.solve_host(bh, uh)
    plan.host_wait()
    torch.cuda.synchronize()
    if barrier:
        barrier()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record()
    for _ in range(steps):
        plan.solve_host(bh, uh)
    plan.host_wait()
    ev1.record()
    torch.cuda.synchronize()
    if barrier:
        barrier()
    return ev0.elapsed_time(ev1) / steps


def time_steps(torch, fn, steps, warmup, barrier=None):
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    if barrier:
        barrier()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record()
    for _ in range(steps):
        fn()
    ev1.record()
    torch.cuda.synchronize()
    if barrier:
        barrier()
    return ev0.elapsed_time(ev1) / steps


# DRAM bytes (read + write) per DOF of one double-float residual apply, the
# average of the two launches of a 2D n=9 residual chain, from one ncu
# capture of the K=512x512 case (529.2 MB per launch at 21.2 M DOF), scaled
# by the unknowns
APPLY_DF_TRAFFIC_PER_DOF_2D_N9 = 529.2e6 / 21224449


def residual_bytes_per_dof(wl):
    """Algorithmic HBM bytes of one refinement residual r = b - L u per DOF:
    read u and b in float64, write r in float32 (20 B, as if fused)."""
    return 8.0 + 8.0 + 4.0


def roofline(prof, steps, peaks, wl=None, residuals_per_step=2):
    """Dominant kernel kind of the step and its achieved fraction of the HBM
    roofline: algorithmic bytes (the field reads and writes the method needs,
    per launch) / the kind's mean CUDA-event launch time / the measured copy
    bandwidth.  For the double-float residual the algorithmic bytes are the
    fused residual's 20 B/DOF, spread over the launches of one residual; its
    float32 lane-operation rate is reported beside it."""
    kind = max(prof, key=lambda k: prof[k]["ms"])
    p = prof[kind]
    if p["launches"] == 0 or p["ms"] <= 0:
        return None, kind
    per_launch_ms = p["ms"] / p["launches"]
    share = p["ms"] / sum(v["ms"] for v in prof.values())
    hbm = peaks.get("hbm_gbs")
    src = "MEASURED_PEAKS.json hbm_gbs (measured)"
    if hbm is None:
        hbm, src = 6800.0, "fallback 6.8 TB/s"
    out = {"bound": "hbm", "peak": hbm, "unit": "GB/s", "peak_source": src, "avg_launch_ms": per_launch_ms,
           "share_of_step": share}
    if kind in ("apply", "apply_df") and wl is not None:
        dof = 1
        for k in wl["K"]:
            dof *= wl["n"] * k - 1
        launches_per_residual = p["launches"] / max(1, steps * residuals_per_step)
        alg = residual_bytes_per_dof(wl) * dof / launches_per_residual
        achieved = alg / (per_launch_ms * 1e-3) / 1e9
        traffic = None
        if kind == "apply_df" and wl["n"] == 9 and len(wl["K"]) == 2:
            traffic = APPLY_DF_TRAFFIC_PER_DOF_2D_N9 * dof
        out.update({"achieved": achieved, "frac": achieved / hbm, "traffic": traffic,
                    "algorithmic_bytes_per_launch": alg,
                    "traffic_over_algorithmic": (traffic / alg) if traffic else None,
                    "kernel": "apply_kernel_df (double-float refinement residual, "
                              f"{launches_per_residual:g} launches per residual)"})
        if kind == "apply_df":
            lane = p["flops64"] / p["launches"] / (per_launch_ms * 1e-3) / 1e12
            out["secondary"] = {"fp32_lane_Tops": lane, "fp32_lane_peak_Tops": FP32_LANE_TOPS,
                                "frac": lane / FP32_LANE_TOPS,
                                "note": "float32 operations the double-float algorithm executes / "
                                        "(152 SMs x 128 lanes x 2.07 GHz)"}
        return out, kind
    alg = p["bytes"] / p["launches"]
    achieved = alg / (per_launch_ms * 1e-3) / 1e9
    out.update({"achieved": achieved, "frac": achieved / hbm, "traffic": None, "algorithmic_bytes_per_launch": alg,
                "kernel": f"pencil pass ({kind})"})
    return out, kind


def oracle_full_solve(wl, b):
    """FP64 oracle solve of the workload on the host cores: (u, seconds of the
    solve proper, seconds of the eigenbasis)."""
    from oracle import solve as osolve
    prob = osolve.Problem(wl["n"], wl["K"], wl["X"], wl["a"], wl["c"])
    t0 = time.perf_counter()
    for i in range(prob.N):
        prob.basis1d(i)
    prob.denominators()
    t_basis = time.perf_counter() - t0
    t0 = time.perf_counter()
    u = osolve.solve(prob, b)
    t_solve = time.perf_counter() - t0
    return u, t_solve, t_basis


def run_batched(torch, args, barrier):
    """The batched workload (256 seeded problems, N in {2,3}, n in 2..8, K_i in
    {16,...,512}, 1-8 right-hand sides): one graph launch of the batched
    mixed solver against the same problems solved one after another with
    stand-alone FP64 plans, with every plan on algorithm (a), then on
    algorithm (b).  Right-hand sides N(0,1) drawn on the device."""
    from paper_1701_03967_gb300 import Batch, Plan, synth
    specs = synth.batched_problems()
    plans = [Plan(s["n"], s["K"], s["X"], s["a"], s["c"], "mixed", max_nrhs=s["nrhs"]) for s in specs]
    t0 = time.time()
    batch = Batch(plans, [s["nrhs"] for s in specs])
    t_create = time.time() - t0
    g = torch.Generator(device="cuda").manual_seed(synth.SEED)
    b = torch.randn(batch.total_len, dtype=torch.float64, device="cuda", generator=g)
    u = torch.empty_like(b)
    ms_b = time_steps(torch, lambda: batch.solve(b, out=u), max(2, args.steps // 2), args.warmup, barrier)
    batch.check()
    # the same batch in stream mode: every problem by its own plan on one of k streams
    us = torch.empty_like(b)
    streams = {}
    for k in (4, 8, 16):
        batch.set_mode("streams", k)
        streams[k] = time_steps(torch, lambda: batch.solve(b, out=us), max(2, args.steps // 2), args.warmup,
                                barrier)
    batch.set_mode("graph")
    p64 = [Plan(s["n"], s["K"], s["X"], s["a"], s["c"], "fp64", max_nrhs=s["nrhs"]) for s in specs]
    u64 = torch.empty_like(b)
    views = list(zip(p64, batch.views(b), batch.views(u64)))

    def seq64():
        for pl, x, y in views:
            pl.solve(x, out=y)
    ms_64 = time_steps(torch, seq64, max(2, args.steps // 2), args.warmup, barrier)
    rel = float(torch.linalg.vector_norm(u - u64) / torch.linalg.vector_norm(u64))
    units = float(batch.total_len)
    # the same mixed plans launched one problem after another (what the batch replaces)
    umx = torch.empty_like(b)
    mviews = list(zip(plans, batch.views(b), batch.views(umx)))

    def seq_mixed():
        for pl, x, y in mviews:
            pl.solve(x, out=y)
    ms_mx = time_steps(torch, seq_mixed, max(2, args.steps // 2), args.warmup, barrier)
    out = {"workload": "256 problems, N in {2,3}, n 2..8, K_i in {16,32,48,96,128,384,512}, 1-8 rhs",
           "dof_x_rhs": batch.total_len, "steps": batch.n_steps, "items": batch.n_items,
           "value": units / (ms_b * 1e-3), "unit": "DOF/s", "ms_per_solve": ms_b,
           "fp64_sequential": {"value": units / (ms_64 * 1e-3), "ms_per_solve": ms_64},
           "mixed_sequential": {"value": units / (ms_mx * 1e-3), "ms_per_solve": ms_mx},
           "rel_vs_fp64": rel, "create_s": t_create, "launches_per_solve": len({s["n"] for s in specs}),
           "stream_mode": {"ms_per_solve": {str(k): v for k, v in streams.items()},
                           "value": units / (min(streams.values()) * 1e-3),
                           "rel_vs_fp64": float(torch.linalg.vector_norm(us - u64) / torch.linalg.vector_norm(u64))}}
    batch.close()
    # the same problems with every plan on algorithm (b), batched and sequential FP64
    for pl in plans + p64:
        pl.set_algorithm("b")
    batch = Batch(plans, [s["nrhs"] for s in specs])
    ms_bb = time_steps(torch, lambda: batch.solve(b, out=u), max(2, args.steps // 2), args.warmup, barrier)
    batch.check()
    rel_b = float(torch.linalg.vector_norm(u - u64) / torch.linalg.vector_norm(u64))
    kbest = min(streams, key=streams.get)
    batch.set_mode("streams", kbest)
    ms_bs = time_steps(torch, lambda: batch.solve(b, out=us), max(2, args.steps // 2), args.warmup, barrier)
    batch.set_mode("graph")
    ms_64b = time_steps(torch, seq64, max(2, args.steps // 2), args.warmup, barrier)
    out["algo_b"] = {"value": units / (ms_bb * 1e-3), "ms_per_solve": ms_bb, "steps": batch.n_steps,
                     "items": batch.n_items, "rel_vs_fp64_a": rel_b,
                     "stream_mode": {"streams": kbest, "ms_per_solve": ms_bs, "value": units / (ms_bs * 1e-3)},
                     "fp64_sequential": {"value": units / (ms_64b * 1e-3), "ms_per_solve": ms_64b}}
    batch.close()
    for pl in p64 + plans:
        pl.close()
    return out


def cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count()


def run_other_workloads(torch, args, barrier):
    """The other configurations, timed like the headline (device-resident
    N(0,1) right-hand sides, CUDA events): the n = 1..9 sweep of the 2D
    workload at K = 1024 x 1024, the 3D workloads n=9 K=64^3 and n=4 K=128^3
    (mixed and FP64), algorithm (b) on the 2D n=9 and 3D n=9 workloads,
    one differentiation step (forward solve + adjoint solve + coefficient
    gradients) of 3D n=5 K=64^3 in mixed precision, the headline problem with
    non-zero Dirichlet data, and the 1D transform sweep (n = 5, K = 2^5 ...)."""
    from paper_1701_03967_gb300 import Plan, fem_solve
    g = torch.Generator(device="cuda").manual_seed(1701)
    steps = max(2, args.steps // 2)

    def pair(n, K, X, a, c, algo="a"):
        out = {}
        ref = None
        for prec in ("mixed", "fp64"):
            pl = Plan(n, K, X, a, c, precision=prec)
            pl.tune()
            pl.set_algorithm(algo)
            b = torch.randn(pl.M, dtype=torch.float64, device="cuda", generator=g) if ref is None else ref[0]
            u = torch.empty_like(b)
            ms = time_steps(torch, lambda: pl.solve(b, out=u), steps, args.warmup, barrier)
            out[prec] = {"ms": ms, "dof_per_s": pl.dof / (ms * 1e-3)}
            if ref is None:
                ref = (b, u.clone())
            else:
                out["mixed_vs_fp64_rel"] = float(torch.linalg.vector_norm(ref[1] - u) / torch.linalg.vector_norm(u))
            pl.close()
        out["dof"] = (n * K[0] - 1) * (n * K[1] - 1) * ((n * K[2] - 1) if len(K) == 3 else 1)
        return out

    res = {"sweep_2d_K1024": {}}
    for n in range(1, 10):
        res["sweep_2d_K1024"][f"n{n}"] = pair(n, (1024, 1024), (1.0, 2.0), (1.0, 2.5), 1.0)
        torch.cuda.empty_cache()
    res["3d_n9_K64"] = pair(9, (64, 64, 64), (1.0, 1.0, 1.0), (1.0, 1.0, 1.0), 0.0)
    torch.cuda.empty_cache()
    res["3d_n4_K128"] = pair(4, (128, 128, 128), (1.0, 1.0, 1.0), (1.0, 1.0, 1.0), 0.0)
    torch.cuda.empty_cache()
    # algorithm (b): transforms along x_2..x_N, band solves along x_1
    res["algo_b_2d_n9_K1024"] = pair(9, (1024, 1024), (1.0, 2.0), (1.0, 2.5), 1.0, algo="b")
    torch.cuda.empty_cache()
    res["algo_b_3d_n9_K64"] = pair(9, (64, 64, 64), (1.0, 1.0, 1.0), (1.0, 1.0, 1.0), 0.0, algo="b")
    torch.cuda.empty_cache()
    pl = Plan(5, (64, 64, 64), (1.0, 1.0, 1.0), (1.0, 1.0, 1.0), 0.0, precision="mixed")
    f = torch.randn(pl.M, dtype=torch.float64, device="cuda", generator=g).requires_grad_(True)
    ut = torch.randn(pl.M, dtype=torch.float64, device="cuda", generator=g)
    av = torch.ones(3, dtype=torch.float64, requires_grad=True)
    cv = torch.zeros((), dtype=torch.float64, requires_grad=True)

    def grad_step():
        loss = torch.sum((fem_solve(pl, f, av, cv) - ut) ** 2)
        loss.backward()
    ms = time_steps(torch, grad_step, steps, args.warmup, barrier)
    res["grad_3d_n5_K64"] = {"ms": ms, "dof": pl.dof, "note": "loss.backward() of ||u - u_t||^2, u = L(a, c)^-1 f"}
    pl.close()
    torch.cuda.empty_cache()
    # non-zero Dirichlet data on the headline problem: the correction of f^h
    # by the boundary values, alone and followed by the mixed solve
    pl = Plan(9, (1024, 1024), (1.0, 2.0), (1.0, 2.5), 1.0, precision="mixed")
    gx = torch.randn(tuple(m + 2 for m in pl.M), dtype=torch.float64, device="cuda", generator=g)
    fb = torch.randn(pl.M, dtype=torch.float64, device="cuda", generator=g)
    work = fb.clone()
    ud = torch.empty_like(fb)
    ms_corr = time_steps(torch, lambda: pl.dirichlet_rhs(gx, work), steps, args.warmup, barrier)
    ms_dsolve = time_steps(torch, lambda: pl.solve_dirichlet(fb, gx, out=ud), steps, args.warmup, barrier)
    res["dirichlet_2d_n9_K1024"] = {"correction_ms": ms_corr, "corrected_mixed_solve_ms": ms_dsolve,
                                    "dof": pl.dof}
    pl.close()
    del gx, fb, work, ud
    torch.cuda.empty_cache()
    res["transform_1d_n5"] = transform_sweep(torch, args, barrier, g)
    res["transform_2d_n5_K4096"] = long_strided_transforms(torch, args, barrier, g)
    return res


def transform_sweep(torch, args, barrier, g, n=5):
    """The 1D transform timing of Section 5 (direct FC_n and inverse F_n
    transforms, n = 5, K = 2^5 .. 2^20 and 3 2^4 .. 3 2^17): float64
    transforms of a batch of pencils of 2^24 unknowns in all, reported per
    transform.  Pencils that fit one CTA's shared memory take the on-chip
    passes, longer ones the global four-step path.  A K the planner refuses
    is listed as refused."""
    from paper_1701_03967_gb300 import FemFftError, Plan
    steps = max(2, args.steps // 2)
    out = {}
    Ks = [2 ** p for p in range(5, 21)] + [3 * 2 ** p for p in range(4, 18)]
    for K in sorted(Ks):
        M = n * K - 1
        nrhs = max(1, (1 << 24) // M)
        pl = None
        try:
            pl = Plan(n, (K,), None, None, 0.0, precision="fp64", max_nrhs=nrhs)
            y = torch.randn(nrhs, M, dtype=torch.float64, device="cuda", generator=g)
            c = torch.empty_like(y)
            w = torch.empty_like(y)
            pl.forward(y, out=c)
            pl.inverse(c, out=w)
        except FemFftError as e:   # the pass planner refuses a pencil larger than a CTA's shared memory
            out[str(K)] = {"refused": str(e)[:120]}
            if pl is not None:
                pl.close()
            continue
        ms_f = time_steps(torch, lambda: pl.forward(y, out=c), steps, args.warmup, barrier)
        ms_i = time_steps(torch, lambda: pl.inverse(c, out=w), steps, args.warmup, barrier)
        # the direct transform expands calC^-1 y (Theorem 2), so the round trip
        # of the mass product returns the field itself
        pl.forward(pl.apply_mass(y), out=c)
        pl.inverse(c, out=w)
        rel = float(torch.linalg.vector_norm(w - y) / torch.linalg.vector_norm(y))
        out[str(K)] = {"M": M, "pencils": nrhs, "forward_us": ms_f * 1e3 / nrhs, "inverse_us": ms_i * 1e3 / nrhs,
                       "forward_dof_per_s": nrhs * M / (ms_f * 1e-3), "inverse_dof_per_s": nrhs * M / (ms_i * 1e-3),
                       "mass_roundtrip_rel_err": rel}
        pl.close()
        del y, c, w
    return out


def long_strided_transforms(torch, args, barrier, g, n=5, K=4096):
    """Float64 transforms of a 2D field with pencils longer than one CTA holds
    on both axes (n = 5, K = 4096 x 4096, 419 M unknowns): the strided axis 0
    and the contiguous axis 1 both take the global four-step path; per
    transform, with the mass round trip inverse(forward(calC y)) = y."""
    from paper_1701_03967_gb300 import Plan
    steps = max(2, args.steps // 4)
    pl = Plan(n, (K, K), None, None, 0.0, precision="fp64")
    y = torch.randn(tuple(pl.M), dtype=torch.float64, device="cuda", generator=g)
    c = torch.empty_like(y)
    w = torch.empty_like(y)
    ms_f = time_steps(torch, lambda: pl.forward(y, out=c), steps, args.warmup, barrier)
    ms_i = time_steps(torch, lambda: pl.inverse(c, out=w), steps, args.warmup, barrier)
    pl.forward(pl.apply_mass(y), out=c)
    pl.inverse(c, out=w)
    rel = float(torch.linalg.vector_norm(w - y) / torch.linalg.vector_norm(y))
    dof = pl.dof
    pl.close()
    del y, c, w
    return {"dof": dof, "forward_ms": ms_f, "inverse_ms": ms_i, "forward_dof_per_s": dof / (ms_f * 1e-3),
            "inverse_dof_per_s": dof / (ms_i * 1e-3), "mass_roundtrip_rel_err": rel}


def workload_config(wl, args, ws):
    """The `config` object of both arms' JSON lines."""
    dof = 1
    for k in wl["K"]:
        dof *= wl["n"] * k - 1
    mb = dof * 8 / 1e6
    return {"workload": wl["name"], "n": wl["n"], "K": list(wl["K"]), "X": list(wl["X"]),
            "a": list(wl["a"]), "c": wl["c"], "dof": dof, "nrhs": 1, "precision": "mixed",
            "refine_steps": args.refine, "parallelism": f"replicas x{ws}",
            "l2": f"inputs larger than L2 (b and u {mb:.0f} MB each, float32 workspace {mb / 2:.0f} MB)"
                  if mb > 129 else f"inputs of {mb:.1f} MB, within L2"}


def run_reference(args, wl):
    """Reference arm: the FP64 CPU oracle timed on the host cores.  Each step
    is one of the four dense axis products of the oracle's solve (a quarter of
    a solve, cycling), credited with DOF/4."""
    ws, rank, _ = _dist()
    if rank != 0:
        return
    from oracle import solve as osolve
    from paper_1701_03967_gb300 import synth
    prob = osolve.Problem(wl["n"], wl["K"], wl["X"], wl["a"], wl["c"])
    b = synth.normal_field(prob.M, synth.CFG_LARGE_2D if wl["n"] == 9 and len(wl["K"]) == 2 else synth.CFG_TEST)
    for i in range(prob.N):
        prob.basis1d(i)
    D = prob.denominators()
    stages = []
    for i in reversed(range(prob.N)):
        stages.append(("fwd", i))
    for i in range(prob.N):
        stages.append(("inv", i))
    nst = len(stages)
    state = {"x": b[None], "j": 0}

    def step():
        kind, i = stages[state["j"] % nst]
        _, S, cn = prob.basis1d(i)
        mat = S.T / cn[:, None] if kind == "fwd" else S
        x = osolve._axis_apply(state["x"], mat, i + 1)
        if kind == "fwd" and i == 0:
            x = x / D
        state["x"] = x if state["j"] % nst != nst - 1 else b[None]
        state["j"] += 1

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = (time.perf_counter() - t0) / args.steps
    dof = prob.dof
    value = dof / nst / dt
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "DOF/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(wl, args, ws),
            "cpu_baseline": {"value": value, "unit": "DOF/s", "cores": cores(), "kind": "oracle",
                             "sample": f"one of the {nst} dense axis products of the oracle solve per step "
                                       f"(credited DOF/{nst}); eigenbasis precomputed untimed"},
            "e2e": {"value": value, "unit": "DOF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


PROFILE_CASES = {
    # name: (precision, n, K, X, a, c, algorithm); small cases for kernel captures (fields above L2,
    # at most about 1 GB on the device)
    "fast2d": ("mixed", 9, (1024, 1024), (1.0, 2.0), (1.0, 2.5), 1.0, "a"),
    "mid2d": ("mixed", 9, (512, 512), (1.0, 2.0), (1.0, 2.5), 1.0, "a"),
    "f64_2d": ("fp64", 9, (512, 512), (1.0, 2.0), (1.0, 2.5), 1.0, "a"),
    "band2d": ("mixed", 9, (512, 512), (1.0, 2.0), (1.0, 2.5), 1.0, "b"),
    "fast3d": ("mixed", 5, (64, 64, 64), (1.0, 1.0, 1.0), (1.0, 1.0, 1.0), 0.0, "a"),
    "long1d": ("mixed", 5, (1 << 20,), (1.0,), (1.0,), 0.0, "a"),
}


def run_profile_case(case):
    """Two solves of a small case and nothing else (no timing): the program an ncu capture of
    one kernel runs.  "batch": 24 problems of the batched workload in one batch."""
    import torch
    from paper_1701_03967_gb300 import Batch, Plan, synth
    dev = "cuda"
    if case == "batch":
        specs = synth.batched_problems()[:24]
        plans = [Plan(s["n"], s["K"], s["X"], s["a"], s["c"], "mixed", max_nrhs=s["nrhs"]) for s in specs]
        bt = Batch(plans, [s["nrhs"] for s in specs], tune=False)
        x = torch.from_numpy(synth.normal_field((bt.total_len,), synth.CFG_TEST, 0, 0)).to(dev)
        u = torch.empty_like(x)
        for _ in range(2):
            bt.solve(x, out=u)
        bt.check()
        torch.cuda.synchronize()
        print("ok batch", bt.total_len)
        return
    prec, n, K, X, a, c, algo = PROFILE_CASES[case]
    pl = Plan(n, K, X, a, c, precision=prec)
    if algo == "b":
        pl.set_algorithm("b")
    b = torch.from_numpy(synth.normal_field(pl.M, synth.CFG_TEST, 0, 0)).to(dev)
    u = torch.empty_like(b)
    for _ in range(2):
        pl.solve(b, out=u)
    torch.cuda.synchronize()
    print("ok", case, float(u.norm()))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="2d", choices=sorted(WORKLOADS))
    ap.add_argument("--refine", type=int, default=2, help="refinement steps of the mixed path")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true", help="skip the 256-problem batched measurement")
    ap.add_argument("--no-others", action="store_true", help="skip the n-sweep, 3D and gradient measurements")
    ap.add_argument("--profile-case", choices=sorted(PROFILE_CASES) + ["batch"],
                    help="run two solves of a small case for a kernel capture and exit (no timing, no JSON)")
    args = ap.parse_args()
    if args.profile_case:
        run_profile_case(args.profile_case)
        return
    wl = WORKLOADS[args.workload]
    args.warmup = max(args.warmup, 3)
    if args.impl == "reference":
        run_reference(args, wl)
        return

    import torch
    ws, rank, local = _dist()
    dist = None
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.cuda.current_device()
    barrier = (lambda: dist.barrier()) if dist else None

    from paper_1701_03967_gb300 import Plan, synth
    cfg_id = synth.CFG_LARGE_2D if args.workload == "2d" else synth.CFG_TEST
    mixed = Plan(wl["n"], wl["K"], wl["X"], wl["a"], wl["c"], precision="mixed")
    mixed.set_refinement(0.0, args.refine)
    fp64 = Plan(wl["n"], wl["K"], wl["X"], wl["a"], wl["c"], precision="fp64")
    # launch shapes of both plans tuned on the device (plan setup, untimed)
    mixed.tune()
    fp64.tune()
    b_host = synth.normal_field(mixed.M, cfg_id, 0, rank)
    b = torch.from_numpy(b_host).to(f"cuda:{dev}")
    u = torch.empty_like(b)
    u64 = torch.empty_like(b)
    dof = mixed.dof

    # ---- mixed path (headline), with per-kernel event timing
    clocks = ClockSampler(dev)
    for _ in range(args.warmup):
        mixed.solve(b, out=u)
    torch.cuda.synchronize()
    mixed.profile(True)
    clocks.start()
    ms_mixed = time_steps(torch, lambda: mixed.solve(b, out=u), args.steps, 0, barrier)
    prof = mixed.profile_read()
    mixed.profile(False)
    # ---- float64 path in the same run
    ms_fp64 = time_steps(torch, lambda: fp64.solve(b, out=u64), args.steps, args.warmup, barrier)
    # ---- end to end through the public API from pinned host memory
    bh = torch.from_numpy(b_host).pin_memory()
    uh = torch.empty_like(bh).pin_memory()

    def e2e_step():
        b.copy_(bh, non_blocking=True)
        mixed.solve(b, out=u)
        uh.copy_(u, non_blocking=True)
    ms_e2e_serial = time_steps(torch, e2e_step, args.steps, args.warmup, barrier)
    # the same solves through the library's host-buffer entry point: step k+1's
    # upload and step k-1's download run on its copy streams under step k's solve
    ms_e2e = time_pipeline(torch, mixed, bh, uh, args.steps, args.warmup, barrier)
    clk = clocks.stop()

    batched = None if args.no_batched else run_batched(torch, args, barrier)
    others = None if args.no_others else run_other_workloads(torch, args, barrier)

    if dist:
        ms_mixed, ms_fp64, ms_e2e, ms_e2e_serial = max_over_ranks(
            torch, dist, [ms_mixed, ms_fp64, ms_e2e, ms_e2e_serial], f"cuda:{dev}")

    u_mixed = u.cpu().numpy()
    u_fp64 = u64.cpu().numpy()
    acc = {"mixed_vs_fp64_rel": float(np.linalg.norm(u_mixed - u_fp64) / np.linalg.norm(u_fp64))}
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        u_or, t_solve, t_basis = oracle_full_solve(wl, b_host)
        nrm = np.linalg.norm(u_or)
        acc["mixed_rel_err_vs_oracle"] = float(np.linalg.norm(u_mixed - u_or) / nrm)
        acc["fp64_rel_err_vs_oracle"] = float(np.linalg.norm(u_fp64 - u_or) / nrm)
        cpu = {"value": dof / t_solve, "unit": "DOF/s", "cores": cores(), "kind": "oracle",
               "sample": f"one full oracle solve of the workload (dense Theorem-1 eigenbasis products, "
                         f"{t_solve:.1f} s; eigenbasis {t_basis:.1f} s untimed)"}

    peaks = _peaks()
    roof, dom = roofline(prof, args.steps, peaks, wl, residuals_per_step=args.refine)
    launches = sum(v["launches"] for v in prof.values()) // max(args.steps, 1)
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    kernels = {k: {"launches_per_step": v["launches"] / args.steps, "ms_per_step": v["ms"] / args.steps,
                   "GB_per_s": (v["bytes"] / (v["ms"] * 1e-3) / 1e9) if v["ms"] else None,
                   "hbm_frac": (v["bytes"] / (v["ms"] * 1e-3) / 1e9 / hbm_peak) if v["ms"] else None,
                   ("fp32_Tops" if k == "apply_df" else "fp64_TFLOPs"):
                       (v["flops64"] / (v["ms"] * 1e-3) / 1e12) if v["ms"] and v["flops64"] else None}
               for k, v in prof.items()}
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    line = {
        "metric": METRIC, "value": job_value(dof, ws, ms_mixed), "unit": "DOF/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_mixed, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": workload_config(wl, args, ws),
        "fp64": {"value": job_value(dof, ws, ms_fp64), "unit": "DOF/s", "ms_per_step": ms_fp64, "dtype": "f64"},
        "accuracy": acc,
        "e2e": {"value": job_value(dof, ws, ms_e2e), "unit": "DOF/s", "h2d_bytes_per_step": dof * 8,
                "d2h_bytes_per_step": dof * 8, "ms_per_step": ms_e2e,
                "method": "fem_fft_solve_host (C ABI, host buffers): pinned host b -> device, solve, device -> "
                          "pinned host u every step; the library pipelines uploads and downloads on its own "
                          "streams under neighbouring solves",
                "serial": {"value": job_value(dof, ws, ms_e2e_serial), "ms_per_step": ms_e2e_serial}},
        "roofline": roof,
        "kernels": kernels,
        "gpu_launches": launches,
        "clocks": clk,
        "cpu_baseline": cpu,
        "batched": batched,
        "other_workloads": others,
    }
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
