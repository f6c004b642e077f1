"""Throughput benchmark of the J-CoMM / B-CoMM hot path on one GB300.

Workload (one "step" = one J-CoMM outer iteration, L = 1, over the whole tensor):
dense 3-way CP, 512 x 512 x 512 FP32 (537 MB, larger than the 129 MB L2, so no flush is
needed between steps), rank R = 32, beta = 1, data = CP model with Gamma(2,1) factors
times i.i.d. Gamma(10, 0.1) noise, init U(0.1, 1).  Secondary figures on the same tensor:
B-CoMM sweeps/s, and the time for each method to reach F*(1 + 1e-4), F* being the lowest
objective of a long FP32 B-CoMM run from the same init.

Usage:  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp32|tf32|3xtf32]
        python bench.py --impl reference ...   (the FP64 CPU oracle on a bounded sample)
Prints one JSON line on rank 0.
"""
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

METRIC = "J-CoMM time-to-1e-4 rel objective vs FP32 block-MU; sweeps/s; served p99"
DIMS = (512, 512, 512)
RANK = 32
BETA = 1.0
# arithmetic of each precision option: FP32 CUDA-core passes, or TF32 (split TF32 for 3xtf32)
# reconstruction with BF16 contraction operands and FP32 accumulation
DTYPES = {"fp32": "f32", "tf32": "tf32+bf16", "3xtf32": "3xtf32+bf16"}
WORKLOAD = ("dense CP 512x512x512 FP32, R=32, beta=1 (KL), J-CoMM outer iteration (L=1); "
            "Gamma(2,1) factors x Gamma(10,0.1) noise, U(0.1,1) init")


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=200)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="ntf", choices=["ntf", "reference"])
    p.add_argument("--precision", default="tf32", choices=["fp32", "tf32", "3xtf32"])
    p.add_argument("--no-ttt", action="store_true", help="skip the time-to-target runs")
    p.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    p.add_argument("--no-other", action="store_true",
                   help="skip the Tucker 400^3, sparse 3.3M-nonzero, 4-way CP / Tucker and 5-way Tucker "
                        "measurements")
    p.add_argument("--serve-jobs", type=int, default=1000,
                   help="jobs of the serving-mix measurement in the default run (0: skip)")
    p.add_argument("--serve", action="store_true", help="print only the serving-mix line")
    p.add_argument("--slots", type=int, default=16)
    p.add_argument("--c2-betas", default="0,0.5,1,1.5",
                   help="betas of the C2 table (block-MU vs J-CoMM L = 1, 3; time to target at each)")
    p.add_argument("--profile-n", type=int, default=0,
                   help="profiling driver: three J-CoMM steps and three block-MU sweeps on an n^3, "
                        "R = 32, beta = 1 tensor at --precision, then exit (no measurement)")
    p.add_argument("--profile-case", default="", choices=["", "tucker", "coo", "cp4", "tucker4", "tucker5", "jcache"],
                   help="profiling driver: three block-MM sweeps and three J-CoMM iterations of the Tucker "
                        "400^3 workload, three J-CoMM iterations of the sparse 3.3M-nonzero workload, or "
                        "the 4-way CP / Tucker or 5-way Tucker measurements with one timed call per "
                        "configuration")
    return p.parse_args()


# DRAM bytes (read + write) per tensor entry of the timed tensor-core pass (all numerators +
# objective, TF32 reconstruction, 256-column blocks), from the ncu capture of that instantiation on
# the 512^3 tensor (its summary is kept under profiles/); valid only for the kernel sources it was
# taken on
TC_CAPTURE = {
    "sources": {"paper_2602_14683_gb300/csrc/cp3_tc.cuh": "e7d64d56509031efacb862ebb419d899e607b342b9663c7d5addf1319bc96905",
                "paper_2602_14683_gb300/csrc/cp3_tc.cu": "cf38de9d49feace9f689089806412e437781214911db66c94f805ac94a11a98f"},
    "bytes_per_entry": (541.148672e6 + 4.848640e6) / 512 ** 3,
}


def tc_traffic(entries):
    import hashlib
    here = os.path.dirname(os.path.abspath(__file__))
    for rel, digest in TC_CAPTURE["sources"].items():
        with open(os.path.join(here, rel), "rb") as f:
            if hashlib.sha256(f.read()).hexdigest() != digest:
                return None  # the kernel changed since the counters were taken
    return TC_CAPTURE["bytes_per_entry"] * entries


def profile_case(n, prec):
    """Small, fixed launch sequence for ncu captures (one GPU, a few hundred MB)."""
    import torch
    import paper_2602_14683_gb300 as ntf
    g = torch.Generator(device="cuda").manual_seed(0)
    X = torch.rand((n, n, n), device="cuda", generator=g) * 10 + 0.1
    A = [torch.rand((n, 32), device="cuda", generator=g) * 0.9 + 0.1 for _ in range(3)]
    obj = torch.zeros(1, dtype=torch.float64, device="cuda")
    for _ in range(3):
        ntf.jcomm_outer(X, 1.0, A, objective=obj, precision=prec)
        ntf.cp_mu_sweep(X, 1.0, A, objective=obj, precision=prec)
    torch.cuda.synchronize()
    ntf.default_context().device_status()
    print("profile case n=%d precision=%s objective %.6e" % (n, prec, obj.item()))
    return 0


def profile_jcache(ntf, n=512, beta=1.5, L=3, iters=3):
    """Small fixed launch sequence for ncu: J-CoMM outer iterations at beta = 3/2 with three inner
    sweeps and the P~ / Q~ cache on a 512^3, R = 32 tensor (one cache-writing pass and eight
    contraction-only passes per iteration)."""
    import torch
    g = torch.Generator(device="cuda").manual_seed(0)
    X = torch.rand((n, n, n), device="cuda", generator=g) * 10 + 0.1
    A = [torch.rand((n, 32), device="cuda", generator=g) * 0.9 + 0.1 for _ in range(3)]
    obj = torch.zeros(1, dtype=torch.float64, device="cuda")
    for _ in range(iters):
        ntf.jcomm_outer(X, beta, A, objective=obj, precision="tf32", inner_L=L, cache="bf16")
    torch.cuda.synchronize()
    ntf.default_context().device_status()
    print("profile case jcache n=%d objective %.6e" % (n, obj.item()))
    return 0


def run_serving(ntf, n_jobs, slots, seed=0, max_iters=200, rtol=1e-6, sweep=(0.5, 1.0, 1.2), sweep_jobs=None):
    """Serving mix (dense 3-way CP / Tucker jobs, dims log-uniform 16..256, rank / core dims
    4..32, beta in {1/2, 1, 3/2}, J-CoMM L = 1, stop at a 1e-6 relative objective change or
    200 iterations).  Every job's data and init are drawn on the device BEFORE any timed
    phase, so the arrival loop only submits.  Phases: an untimed warm-up set (kernel loading,
    first workspace sizes); a burst submitted at once to measure the saturation throughput;
    the main run of n_jobs Poisson arrivals at 0.8 x saturation; then a load sweep at
    0.5 / 1.0 / 1.2 x saturation (sweep_jobs each).  Latency = completion - SCHEDULED arrival
    (host monotonic clock, the server's own clock), so a submit loop that falls behind its
    schedule shows up as queueing.  No device-wide synchronisation happens while jobs run
    (a slot stream may be capturing its graph)."""
    import torch
    import synth
    stream = torch.cuda.current_stream()
    sweep_jobs = sweep_jobs or max(slots * 4, n_jobs // 5)

    def gen(jobs):
        data = [synth.job_data_torch(j) for j in jobs]
        stream.synchronize()
        return data

    def drain(srv, expect):
        out = []
        while len(out) < expect:
            got = srv.poll(wait_all=True, max_results=4096)
            if not got:
                break
            out += got
        return out

    def submit(srv, j, d):
        X, G, A = d
        return srv.submit(X, j["beta"], A, core=G, rtol=rtol, max_iters=max_iters)

    n_sat = max(slots * 4, n_jobs // 8)
    warm = synth.serving_jobs(2 * slots, seed=seed + 7)
    burst = synth.serving_jobs(n_sat, seed=seed + 11)
    main_jobs = synth.serving_jobs(n_jobs, seed=seed)
    sweeps = {f: synth.serving_jobs(sweep_jobs, seed=seed + 100 + k) for k, f in enumerate(sweep)}
    d_warm, d_burst, d_main = gen(warm), gen(burst), gen(main_jobs)
    d_sweep = {f: gen(js) for f, js in sweeps.items()}
    srv = ntf.Server(slots=slots)
    for j, d in zip(warm, d_warm):
        submit(srv, j, d)
    drain(srv, len(warm))
    del d_warm
    # saturation: every job of the burst submitted at once
    t0 = time.monotonic()
    for j, d in zip(burst, d_burst):
        submit(srv, j, d)
    res_b = drain(srv, len(burst))
    sat = len(burst) / (max(r["t_done"] for r in res_b) - t0)
    del d_burst

    def poisson_run(jobs, data, rate, rng_seed):
        gaps = np.random.default_rng(rng_seed).exponential(1.0 / rate, size=len(jobs))
        sched = {}
        start = time.monotonic()
        due = start
        lag = 0.0
        for j, d, gap in zip(jobs, data, gaps):
            due += gap
            delay = due - time.monotonic()
            if delay > 0:
                time.sleep(delay)
            lag = max(lag, time.monotonic() - due)
            sched[submit(srv, j, d)] = due
        res = drain(srv, len(jobs))
        lat = np.array([r["t_done"] - sched[r["id"]] for r in res])
        span = max(r["t_done"] for r in res) - start
        return res, {"jobs": len(jobs), "offered_per_s": rate, "achieved_per_s": len(res) / span,
                     "p50_latency_s": float(np.percentile(lat, 50)), "p99_latency_s": float(np.percentile(lat, 99)),
                     "max_submit_lag_s": lag, "ok": sum(1 for r in res if r["status"] == 0)}

    res_m, main = poisson_run(main_jobs, d_main, 0.8 * sat, seed + 1)
    del d_main
    sweep_out = {}
    for k, f in enumerate(sweep):
        _, sweep_out["%gx" % f] = poisson_run(sweeps[f], d_sweep[f], f * sat, seed + 200 + k)
        del d_sweep[f]
    srv.close()
    its = np.array([r["iterations"] for r in res_b + res_m])
    return {"jobs": n_jobs, "slots": slots, "saturation_solves_per_s": sat, "saturation_burst_jobs": len(burst),
            "poisson_rate_per_s": main["offered_per_s"], "solves_per_s": main["achieved_per_s"],
            "p50_latency_s": main["p50_latency_s"], "p99_latency_s": main["p99_latency_s"],
            "max_submit_lag_s": main["max_submit_lag_s"], "completed_ok": main["ok"],
            "mean_iterations": float(its.mean()), "load_sweep": sweep_out,
            "latency_from": "scheduled arrival (Poisson), data pre-generated on the device",
            "mix": "dense 3-way CP/Tucker 50/50, dims log-uniform 16..256, rank/core 4..32, beta in {0.5,1,1.5}, "
                   "Poisson-noised low-rank data at mean 10, J-CoMM L=1, stop at 1e-6 rel change or 200 its"}


def c3_data(n=400, J=32, seed=3):
    """C3 inputs: Gamma(2,1) core and factors, model rescaled to mean 10, Poisson noise
    (drawn on the device, seeded); init U(0.1, 1)."""
    import torch
    torch.manual_seed(seed)
    dev = torch.device("cuda", torch.cuda.current_device())
    G = torch.distributions.Gamma(torch.full((J, J, J), 2.0, device=dev), 1.0).sample()
    A = [torch.distributions.Gamma(torch.full((n, J), 2.0, device=dev), 1.0).sample() for _ in range(3)]
    M = torch.einsum("abc,ia,jb,kc->ijk", G, *A)
    M *= 10.0 / M.mean()
    X = torch.poisson(M).float().contiguous()
    del M
    g = torch.Generator(device=dev).manual_seed(seed + 1)
    G0 = torch.rand((J, J, J), device=dev, generator=g) * 0.9 + 0.1
    A0 = [torch.rand((n, J), device=dev, generator=g) * 0.9 + 0.1 for _ in range(3)]
    return X, G0, A0


def c3_vs_oracle(ntf, ctx, T=4, beta=1.5, precisions=("fp32", "tf32", "3xtf32")):
    """C3's accuracy metric: the per-iteration objective error of every precision against the
    FP64 oracle on the 400^3 Tucker problem.  The GPU runs T block-MM sweeps from the shared
    init and records the objective of each incoming iterate; the oracle (FP64, mode-n products
    on the host's cores) runs the same T sweeps from the same FP32 inputs.  Reported:
    |F_gpu(t) - F_ora(t)| / F_ora(t) for t = 0..T-1 (t = 0: the objective of the init only)."""
    import torch
    from oracle import tucker_modeprod as tm
    X, G0, A0 = c3_data()
    traj = {}
    for prec in precisions:
        G, A = G0.clone(), [a.clone() for a in A0]
        F = torch.zeros(T, dtype=torch.float64, device=X.device)
        for t in range(T):
            ntf.tucker_mu_sweep(X, beta, G, A, objective=F[t:t + 1], ctx=ctx, precision=prec)
        traj[prec] = F.cpu().numpy()
    Xh = X.cpu().double()
    Gh, Ah = G0.cpu().double().numpy(), [a.cpu().double().numpy() for a in A0]
    del X
    t0 = time.perf_counter()
    F_ora = []
    for t in range(T):
        Gh, Ah, f = tm.tucker_mu_sweep(Xh, Gh, Ah, beta)
        F_ora.append(f)
    sec = time.perf_counter() - t0
    F_ora = np.array(F_ora)
    out = {"workload": "dense Tucker 400x400x400, core 32x32x32, beta=1.5, block-MM sweeps from the shared init",
           "oracle": "FP64 mode-n products (oracle.tucker_modeprod), %d host threads, %.1f s per sweep"
                     % (torch.get_num_threads(), sec / T),
           "F_oracle": F_ora.tolist()}
    for prec, F in traj.items():
        rel = np.abs(F - F_ora) / F_ora
        out[prec] = {"rel_err_per_iter": rel.tolist(), "max_rel_err": float(rel.max())}
    return out


def run_cp_c1(ntf, ctx, sweeps=100, dims=(60, 50, 40), R=5, seed=0):
    """C1, the latency case: dense CP 60 x 50 x 40, R = 5, beta = 1, plain block-MU; X = CP model
    with U(0.1, 1) factors rescaled to mean 10, Poisson; init U(0.1, 1).  The 100 sweeps are
    enqueued back to back and timed with CUDA events on the stream (the 0.48 MB tensor stays in
    L2, as it would in a user's loop); per precision, microseconds per sweep, eagerly and with one
    sweep captured into a CUDA graph and replayed 100 times (same objective expected)."""
    import torch
    import synth
    dev = torch.device("cuda", torch.cuda.current_device())
    Xn, _ = synth.cp_dense(dims, R, seed=seed, kind="uniform_poisson")
    X = torch.tensor(Xn, dtype=torch.float32, device=dev)
    A0 = [torch.tensor(a, dtype=torch.float32, device=dev) for a in synth.init_factors(dims, R, seed=seed + 1)]
    obj = torch.zeros(1, dtype=torch.float64, device=dev)
    out = {"workload": "dense CP 60x50x40, R=5, beta=1, block-MU, 100 sweeps"}
    for prec in ("fp32", "tf32"):
        A = [a.clone() for a in A0]
        for _ in range(5):
            ntf.cp_mu_sweep(X, 1.0, A, objective=obj, ctx=ctx, precision=prec)
        A = [a.clone() for a in A0]
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(sweeps):
            ntf.cp_mu_sweep(X, 1.0, A, objective=obj, ctx=ctx, precision=prec)
        e1.record()
        torch.cuda.synchronize()
        us = e0.elapsed_time(e1) * 1e3 / sweeps
        out[prec] = {"us_per_sweep": us, "sweeps_per_s": 1e6 / us, "objective_after_100": obj.item()}
        # the same calls captured once into a CUDA graph (the calls are stream-ordered, with no
        # host synchronisation or allocation once the workspaces exist) and the graph replayed
        # once per sweep: the launch and call overhead of the small kernels leaves the loop
        A = [a.clone() for a in A0]
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            ntf.cp_mu_sweep(X, 1.0, A, objective=obj, ctx=ctx, precision=prec)
        for a, a0 in zip(A, A0):
            a.copy_(a0)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(sweeps):
            g.replay()
        e1.record()
        torch.cuda.synchronize()
        usg = e0.elapsed_time(e1) * 1e3 / sweeps
        out[prec].update({"graph_us_per_sweep": usg, "graph_objective_after_100": obj.item()})
        del g
    return out


def run_until(ntf, ctx, X, A0, beta, fn, prec, n_max, target, inner_L=1):
    """Runs fn (a sweep or an outer iteration) from A0 until its objective first reaches
    `target` (checked every 100 iterations on the device record) or n_max iterations.
    Returns (objective per iteration, seconds per iteration, [min, max] ms per 100)."""
    import torch
    stream = torch.cuda.current_stream()
    kw = {"inner_L": inner_L} if inner_L != 1 else {}
    Fr = torch.zeros(n_max, dtype=torch.float64, device=X.device)
    W_ = [a.clone() for a in A0]
    for _ in range(3):  # untimed: workspaces sized for this method and precision
        fn(X, beta, W_, objective=Fr[:1], ctx=ctx, precision=prec, autotune=True, **kw)
    float(Fr[:2].min())  # the stopping check's reduction kernel loads here, not in the timed region
    C_ = [a.clone() for a in A0]
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True)]
    ev[0].record(stream)
    t = 0
    while t < n_max:
        for _ in range(min(100, n_max - t)):
            fn(X, beta, C_, objective=Fr[t:t + 1], ctx=ctx, precision=prec, autotune=True, **kw)
            t += 1
        ev.append(torch.cuda.Event(enable_timing=True))
        ev[-1].record(stream)
        if target is not None and float(Fr[:t].min()) <= target:
            break
    torch.cuda.synchronize()
    chunks = [ev[k].elapsed_time(ev[k + 1]) for k in range(len(ev) - 1)]
    return Fr[:t].cpu().numpy(), ev[0].elapsed_time(ev[-1]) / 1e3 / t, [round(min(chunks), 2), round(max(chunks), 2)]


def ttt_summary(runs, fstar):
    """Iterations and seconds to F*(1 + 1e-4), and to a relative objective change <= 1e-4."""
    target = fstar * (1 + 1e-4)
    res = {}
    for name, (F, per, chunk_ms) in runs.items():
        hit = np.nonzero(F <= target)[0]
        rel = np.abs(np.diff(F)) / F[1:]
        conv = np.nonzero(rel <= 1e-4)[0]
        res[name] = {"iters": int(hit[0]) if hit.size else None,
                     "seconds": float(hit[0] * per) if hit.size else None,
                     "s_per_iter": per, "iters_run": int(F.size),
                     "iters_rel_change_1e-4": int(conv[0]) + 1 if conv.size else None,
                     "seconds_rel_change_1e-4": float((conv[0] + 1) * per) if conv.size else None,
                     "final_rel_gap": float(F[-1] / fstar - 1.0), "ms_per_100_iters_min_max": chunk_ms}
    return res


def run_cp_c2(ntf, ctx, peaks, X, A0, prec, iters=10, betas=(0.0, 0.5, 1.0, 1.5), ttt_betas=(), n_ref=1000):
    """C2 as stated: dense CP 512^3, R = 32, beta in {0, 1/2, 1, 3/2}; block-MU vs J-CoMM with 1 and
    3 inner sweeps (at beta != 1 also with every inner pass recomputing X~ instead of contracting
    the cached P~ / Q~).  Per beta and method: ms per iteration (CUDA events over `iters` iterations,
    inputs resident, the 537 MB tensor larger than L2), the HBM fraction of the whole iteration
    (passes over X x 4 bytes per entry; a block-MU sweep makes 3 passes, J-CoMM at beta = 1 one
    per outer iteration whatever L, at beta != 1 3 L), and, with ttt, the time to F*(1 + 1e-4),
    F* = the lowest objective of n_ref FP32 block-MU sweeps from the same init."""
    import torch
    entries = X.numel()
    obj = torch.zeros(1, dtype=torch.float64, device=X.device)
    out = {"workload": "dense CP 512x512x512, R=32, Gamma(2,1) factors x Gamma(10,0.1) noise", "precision": prec}
    for beta in betas:
        res = {}
        runs = [("block_mu", ntf.cp_mu_sweep, 1, None), ("jcomm_L1", ntf.jcomm_outer, 1, "auto"),
                ("jcomm_L3", ntf.jcomm_outer, 3, "auto")]
        if beta != 1.0:  # J-CoMM with every inner pass recomputing X~ (no P~ / Q~ cache)
            runs += [("jcomm_L1_recompute", ntf.jcomm_outer, 1, "none"), ("jcomm_L3_recompute", ntf.jcomm_outer, 3, "none")]
        for name, fn, L, cache in runs:
            kw = {"inner_L": L, "cache": cache} if fn is ntf.jcomm_outer else {}
            A = [a.clone() for a in A0]
            for _ in range(3):
                fn(X, beta, A, objective=obj, ctx=ctx, precision=prec, autotune=True, **kw)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(iters):
                fn(X, beta, A, objective=obj, ctx=ctx, precision=prec, autotune=True, **kw)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / iters
            passes = 3 if fn is ntf.cp_mu_sweep else (1 if beta == 1.0 else 3 * L)
            gbs = passes * 4 * entries / (ms / 1e3) / 1e9
            res[name] = {"ms": ms, "passes": passes, "hbm_frac_of_iteration": gbs / peaks["hbm_gbs"]}
        if beta in ttt_betas:
            F_ref, per_ref, ch = run_until(ntf, ctx, X, A0, beta, ntf.cp_mu_sweep, "fp32", n_ref, None)
            fstar = float(F_ref.min())
            runs = {"block_mu_fp32": (F_ref, per_ref, ch)}
            for name, fn, L in (("block_mu_" + prec, ntf.cp_mu_sweep, 1), ("jcomm_L1_" + prec, ntf.jcomm_outer, 1),
                                ("jcomm_L3_" + prec, ntf.jcomm_outer, 3)):
                runs[name] = run_until(ntf, ctx, X, A0, beta, fn, prec, 3000, fstar * (1 + 1e-4), inner_L=L)
            res["time_to_target"] = {"F_star": fstar, **ttt_summary(runs, fstar)}
        out["beta%g" % beta] = res
    return out


def run_tucker_c3(ntf, ctx, peaks, iters=10, n=400, J=32, beta=1.5, seed=3, precisions=("fp32", "tf32", "3xtf32")):
    """Dense Tucker 400 x 400 x 400, core 32 x 32 x 32, beta = 3/2: Gamma(2,1) core and
    factors, model rescaled to mean 10, Poisson noise (drawn on the device, seeded); init
    U(0.1, 1).  For each precision, times block-MM sweeps (core, then modes 1..3) and J-CoMM
    outer iterations (L = 1), and reports the objective after the timed sweeps relative to
    the FP32 CUDA-core path's.  Roofline per sweep: four passes over X (4 bytes per entry
    each; FP32 path: 2J flops for Xhat and 2J for each of the P and Q contractions per
    entry, against the derived FP32 FMA peak; tensor-core path: the bytes against the HBM
    copy bandwidth)."""
    import torch
    X, G0, A0 = c3_data(n, J, seed)
    dev = X.device
    obj = torch.zeros(1, dtype=torch.float64, device=dev)
    entries = n ** 3
    fp32_peak = torch.cuda.get_device_properties(dev).multi_processor_count * 128 * 2 * peaks.get("sm_max_mhz", 2070.0) / 1e6
    out = {"workload": "dense Tucker %dx%dx%d, core %dx%dx%d, beta=%g" % (n, n, n, J, J, J, beta)}
    for prec in precisions:
        res = {}
        for name in ("block_mm", "jcomm"):
            Gc, Ac = G0.clone(), [a.clone() for a in A0]

            def step():
                if name == "jcomm":
                    ntf.jcomm_outer(X, beta, Ac, core=Gc, objective=obj, ctx=ctx, precision=prec)
                else:
                    ntf.tucker_mu_sweep(X, beta, Gc, Ac, objective=obj, ctx=ctx, precision=prec)
            for _ in range(3):
                step()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(iters):
                step()
            e1.record()
            torch.cuda.synchronize()
            res[name + "_ms"] = e0.elapsed_time(e1) / max(iters, 1)
            res[name + "_objective"] = obj.item()
        sec = res["block_mm_ms"] / 1e3
        if prec == "fp32":
            flops = 4 * entries * 6 * J
            res["roofline"] = {"bound": "alu", "achieved": flops / sec / 1e12, "peak": fp32_peak, "unit": "TFLOP/s",
                               "frac": flops / sec / 1e12 / fp32_peak,
                               "of": "block-MM sweep: 4 passes x 6J flops per entry over the sweep time, derived FP32 FMA peak"}
        else:
            byt = 4 * entries * 4
            res["roofline"] = {"bound": "hbm", "achieved": byt / sec / 1e9, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                               "frac": byt / sec / 1e9 / peaks["hbm_gbs"],
                               "of": "block-MM sweep: 4 passes x 4 bytes per entry over the sweep time (small GEMMs and "
                                     "W sums included), measured HBM copy bandwidth"}
        out[prec] = res
    if "fp32" in out:
        for prec in precisions:
            if prec != "fp32":
                for name in ("block_mm", "jcomm"):
                    f0 = out["fp32"][name + "_objective"]
                    out[prec][name + "_objective_rel_diff_vs_fp32"] = abs(out[prec][name + "_objective"] - f0) / f0
    return out


def run_coo_c4(ntf, ctx, peaks, iters=20, R=32, seed=0):
    """Sparse 4-way count tensor 183 x 24 x 1140 x 1717 with 3.3M unique nonzeros (first two
    modes periodic, last two Zipf(1.1), values 1 + Geometric(0.3)), CP R = 32, beta = 1,
    J-CoMM outer iterations (L = 1) with the closed-form KL denominators.  Roofline: 20
    bytes streamed per nonzero and pass (4 int32 coordinates + 1 FP32 value), one pass per
    mode."""
    import torch
    import synth
    dims = (183, 24, 1140, 1717)
    idx, vals = synth.coo_counts(dims, 3_300_000, seed=seed)
    dev = torch.device("cuda", torch.cuda.current_device())
    X = ntf.Coo(dims, [torch.tensor(i, device=dev) for i in idx], torch.tensor(vals, dtype=torch.float32, device=dev))
    A0 = [torch.tensor(a, dtype=torch.float32, device=dev) for a in synth.init_factors(dims, R, seed=seed + 1)]
    obj = torch.zeros(1, dtype=torch.float64, device=dev)
    A = [a.clone() for a in A0]
    for _ in range(3):
        ntf.jcomm_outer(X, 1.0, A, objective=obj, ctx=ctx)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(iters):
        ntf.jcomm_outer(X, 1.0, A, objective=obj, ctx=ctx)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / max(iters, 1)
    nnz = X.nnz
    # at beta = 1 every numerator comes from the reference: one pass per mode over that
    # mode's sorted copy of the nonzeros (4 int32 coordinates + 1 FP32 value each)
    byt = len(dims) * 20 * nnz
    sec = ms / 1e3
    N = len(dims)
    # per nonzero and pass: Xhat = sum_r prod of N factor entries (N - 1 multiplies and an add
    # per rank) and the numerator p * prod_{m != n} A^(m) (N - 1 multiplies and an add per rank):
    # 2 N R flops; the N - 1 gathered factor rows are R * 4 bytes each
    flops = N * 2 * N * R * nnz
    gather = N * (N - 1) * R * 4 * nnz
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    fp32_peak = sms * 128 * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
    l2 = l2_copy_gbs()
    # beta = 3/2 on the same tensor (Section 6.3): stored-entry numerators, and every denominator a
    # pass over the whole 8.6e9-entry index space that reads no X (2R flops for Xhat and 2R for the
    # contraction per index entry, one pass per mode), on the tensor cores and on the FP32 pipe
    beta_other = None
    if iters > 0:
        cells = 1
        for d in dims:
            cells *= d
        dflops = N * cells * 4 * R
        beta_other = {"beta": 1.5}
        for prec in ("tf32", "fp32"):
            B = [a.clone() for a in A0]
            ntf.jcomm_outer(X, 1.5, B, objective=obj, ctx=ctx, precision=prec)
            torch.cuda.synchronize()
            e0.record()
            for _ in range(2):
                ntf.jcomm_outer(X, 1.5, B, objective=obj, ctx=ctx, precision=prec)
            e1.record()
            torch.cuda.synchronize()
            ms15 = e0.elapsed_time(e1) / 2
            peak, pname = (peaks["bf16_tflops"], "measured dense bf16 tensor peak (burst)") if prec == "tf32" else \
                (fp32_peak, "derived FP32 FMA-pipe peak")
            beta_other[prec] = {"ms_per_outer": ms15, "objective": obj.item(),
                                "dense_pass": {"achieved_tflops": dflops / (ms15 / 1e3) / 1e12, "peak_tflops": peak,
                                               "frac": dflops / (ms15 / 1e3) / 1e12 / peak,
                                               "of": "N X-free passes over the %d index entries, 4R flops each "
                                                     "(the denominators and the objective's dense part), over the "
                                                     "whole outer iteration (the stored-entry passes included), "
                                                     "against the %s" % (cells, pname)}}
    return {"workload": "sparse COO 183x24x1140x1717, 3.3M nnz, CP R=32, beta=1, J-CoMM L=1",
            "beta_1p5_jcomm": beta_other,
            "us_per_outer": ms * 1e3, "outer_per_s": 1e3 / ms,
            "roofline": {"bound": "hbm", "achieved": byt / sec / 1e9, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                         "frac": byt / sec / 1e9 / peaks["hbm_gbs"],
                         "of": "whole outer iteration (per-mode sorted copies are cached after the first call): "
                               "4 passes x 20 B/nnz streamed; factor-row gathers hit L2"},
            "alu": {"achieved_tflops": flops / sec / 1e12, "peak_tflops": fp32_peak, "frac": flops / sec / 1e12 / fp32_peak,
                    "of": "2NR flops per nonzero and pass (Xhat and the numerator), N passes; FP32 FMA-pipe peak "
                          "derived from %d SMs x 128 lanes x 2 x max clock" % sms},
            "l2_gather": {"achieved_gbs": gather / sec / 1e9, "peak_gbs": l2, "frac": gather / sec / 1e9 / l2,
                          "of": "(N-1) gathered factor rows of R x 4 bytes per nonzero and pass, N passes, against "
                                "the L2-resident copy bandwidth measured in this run (32 MB -> 32 MB, best of 20); "
                                "above 1 when the Zipf-skewed rows are served from L1"}}


def run_batch_cp(ntf, n_jobs=256, alone=16, seed=5):
    """Launches shared by many small jobs (ntf_batch_*): dense CP jobs with dims log-uniform in
    16..64, ranks 4..32, beta in {1/2, 1, 3/2}, J-CoMM L = 1, stop at a 1e-6 relative objective
    change or 200 iterations, FP32 passes.  Every job resident in one batch (one launch per step
    and class for all of them, eight iterations per graph launch) against the first `alone` jobs
    solved one at a time by the same batch; wall time from the first add to the last result,
    data already on the device."""
    import torch
    import synth
    jobs = [j for j in synth.serving_jobs(6 * n_jobs, seed=seed, dim_lo=16, dim_hi=64) if j["model"] == "cp"][:n_jobs]
    data = [synth.job_data_torch(j) for j in jobs]
    torch.cuda.synchronize()
    bt = ntf.Batch(capacity=len(jobs), mem_budget_bytes=2 << 30)

    def solve(sel):
        facs = [[a.clone() for a in data[q][2]] for q in sel]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for q, f in zip(sel, facs):
            if bt.add(data[q][0], jobs[q]["beta"], f) is None:
                raise RuntimeError("batch arena too small")
        res = bt.run(iters=8)
        return res, time.perf_counter() - t0

    solve(list(range(min(8, len(jobs)))))  # warm-up (kernel loading)
    res, sec = solve(list(range(len(jobs))))
    t_alone, its_alone = 0.0, 0
    for q in range(min(alone, len(jobs))):
        r, s = solve([q])
        t_alone += s
        its_alone += r[0]["iterations"]
    bt.close()
    its = sum(r["iterations"] for r in res)
    return {"workload": "%d dense CP jobs, dims log-uniform 16..64, rank 4..32, beta in {0.5,1,1.5}, J-CoMM L=1, "
                        "stop at 1e-6 or 200 its, FP32" % len(jobs),
            "batched": {"jobs": len(res), "seconds": sec, "solves_per_s": len(res) / sec, "iterations": its,
                        "iterations_per_s": its / sec, "ok": sum(1 for r in res if r["status"] == 0)},
            "one_at_a_time": {"jobs": min(alone, len(jobs)), "seconds": t_alone,
                              "solves_per_s": min(alone, len(jobs)) / t_alone, "iterations_per_s": its_alone / t_alone}}


def l2_copy_gbs():
    """Copy bandwidth of a 32 MB -> 32 MB copy that stays in the 129 MB L2 (read + write bytes,
    best of 20 CUDA-event-timed copies): the denominator of the L2-gather fraction."""
    import torch
    a = torch.empty(8 << 20, dtype=torch.float32, device="cuda").fill_(1.0)
    b = torch.empty_like(a)
    for _ in range(5):
        b.copy_(a)
    best = None
    for _ in range(20):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        b.copy_(a)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        best = ms if best is None else min(best, ms)
    return 2 * a.numel() * 4 / (best / 1e3) / 1e9


def flushed_loop_ms(flush, call, iters):
    """Mean device time of `call` over `iters` back-to-back iterations, each preceded by a
    write of `flush` (larger than L2) on the same stream and bracketed by its own CUDA events;
    the host does not wait between iterations, so the intervals hold the call's kernels only
    (the flush is outside them) and host enqueue time overlaps the previous iteration, as in a
    loop that a user runs."""
    import torch
    ev = []
    for _ in range(iters):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        call()
        e1.record()
        ev.append((e0, e1))
    torch.cuda.synchronize()
    return sum(a.elapsed_time(b) for a, b in ev) / max(iters, 1)


def run_cp_4way(ntf, ctx, peaks, iters=20, dims=(80, 70, 60, 50), R=10, seed=5):
    """Dense 4-way CP 80 x 70 x 60 x 50, R = 10 (the shape of the paper's synthetic CP
    experiment): Gamma(2,1) factors x Gamma(10,0.1) noise, init U(0.1, 1).  Times B-CoMM
    sweeps at beta in {1/2, 1, 3/2} and J-CoMM outer iterations (L = 1) at beta = 1, FP32 and
    TF32.  The tensor (67 MB) fits in the 129 MB L2, so a 256 MB buffer is written before
    every timed iteration and each iteration is timed by its own events (flushed_loop_ms).
    Roofline: a B-CoMM sweep makes 4 passes over X (on the 3-way view of the cut the library
    picks), a J-CoMM iteration at beta = 1 one; 4 bytes per entry and pass against the HBM copy
    bandwidth."""
    import torch
    import synth
    dev = torch.device("cuda", torch.cuda.current_device())
    Xn, _ = synth.cp_dense(dims, R, seed=seed, kind="gamma_noise")
    X = torch.tensor(Xn, dtype=torch.float32, device=dev)
    A0 = [torch.tensor(a, dtype=torch.float32, device=dev) for a in synth.init_factors(dims, R, seed=seed + 1)]
    obj = torch.zeros(1, dtype=torch.float64, device=dev)
    flush = torch.empty(64 << 20, dtype=torch.float32, device=dev)
    entries = int(np.prod(dims))
    out = {"workload": "dense 4-way CP %s, R=%d" % ("x".join(map(str, dims)), R),
           "l2": "256 MB write between timed iterations"}
    for prec in ("fp32", "tf32"):
        res = {}
        for name, beta in (("block_mu_b0.5", 0.5), ("block_mu_b1", 1.0), ("block_mu_b1.5", 1.5), ("jcomm_b1", 1.0)):
            A = [a.clone() for a in A0]
            fn = ntf.jcomm_outer if name.startswith("jcomm") else ntf.cp_mu_sweep
            for _ in range(3):
                fn(X, beta, A, objective=obj, ctx=ctx, precision=prec)
            torch.cuda.synchronize()
            ms = flushed_loop_ms(flush, lambda: fn(X, beta, A, objective=obj, ctx=ctx, precision=prec), iters)
            passes = 1 if name.startswith("jcomm") else len(dims)
            gbs = passes * 4 * entries / (ms / 1e3) / 1e9
            res[name] = {"ms": ms, "objective": obj.item(), "hbm_gbs_algorithmic": gbs,
                         "frac_of_measured_hbm": gbs / peaks["hbm_gbs"]}
        out[prec] = res
    return out


def run_tucker_4way(ntf, ctx, peaks, iters=10, dims=(80, 70, 60, 50), J=(10, 9, 8, 7), seed=7):
    """Dense 4-way Tucker 80 x 70 x 60 x 50, core 10 x 9 x 8 x 7 (the shape of the paper's
    synthetic Tucker experiment): Gamma(2,1) core and factors, model rescaled to mean 10,
    Poisson noise, init U(0.1, 1).  Times block-MM sweeps (core, then the four factors) and
    J-CoMM outer iterations (L = 1) at beta in {1/2, 1, 3/2} on the cut the library picks,
    with a 256 MB write before every timed call (the 67 MB tensor fits in L2; flushed_loop_ms)."""
    import torch
    import synth
    dev = torch.device("cuda", torch.cuda.current_device())
    Xn, _, _ = synth.tucker_dense(dims, J, seed=seed)
    X = torch.tensor(Xn, dtype=torch.float32, device=dev)
    G0n, A0n = synth.init_tucker(dims, J, seed=seed + 1)
    G0 = torch.tensor(G0n, dtype=torch.float32, device=dev)
    A0 = [torch.tensor(a, dtype=torch.float32, device=dev) for a in A0n]
    obj = torch.zeros(1, dtype=torch.float64, device=dev)
    flush = torch.empty(64 << 20, dtype=torch.float32, device=dev)
    out = {"workload": "dense 4-way Tucker %s, core %s" % ("x".join(map(str, dims)), "x".join(map(str, J))),
           "l2": "256 MB write between timed iterations", "precision": "fp32"}
    for beta in (0.5, 1.0, 1.5):
        for name in ("block_mm", "jcomm"):
            G, A = G0.clone(), [a.clone() for a in A0]

            def step():
                if name == "jcomm":
                    ntf.jcomm_outer(X, beta, A, core=G, objective=obj, ctx=ctx)
                else:
                    ntf.tucker_mu_sweep(X, beta, G, A, objective=obj, ctx=ctx)
            for _ in range(3):
                step()
            torch.cuda.synchronize()
            out["%s_b%g_ms" % (name, beta)] = flushed_loop_ms(flush, step, iters)
            out["%s_b%g_objective" % (name, beta)] = obj.item()
    return out


def run_tucker_5way(ntf, ctx, peaks, iters=10, dims=(27, 24, 7, 100, 100), J=(10, 10, 5, 10, 10), seed=9):
    """Dense 5-way Tucker 27 x 24 x 7 x 100 x 100, ranks (10, 10, 5, 10, 10): the shape and ranks of
    the paper's real-data Tucker fit, on a synthetic stand-in for its count tensor (the dataset is
    not here): a Tucker intensity with Gamma(0.5, 1) factors and a Gamma(2, 1) core, rescaled so
    that about 99.4% of the Poisson counts are zero, drawn on the device (seeded); init
    U(0.1, 1).  Dense contractions, as in the paper.  Times block-MM sweeps and J-CoMM outer
    iterations (L = 1) at beta in {1/2, 1, 3/2} with precision tf32 (tensor-core passes where
    beta != 1, FP32 passes at beta = 1) on the cut the library picks; the 181 MB tensor is
    larger than L2, no flush."""
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    g = torch.Generator(device=dev).manual_seed(seed)
    torch.manual_seed(seed)
    Gt = torch.distributions.Gamma(torch.full(J, 2.0, device=dev), 1.0).sample()
    At = [torch.distributions.Gamma(torch.full((d, j), 0.5, device=dev), 1.0).sample() for d, j in zip(dims, J)]
    M = torch.einsum("abcde,ia,jb,kc,ld,me->ijklm", Gt, *At)
    M *= 0.0062 / M.mean()
    X = torch.poisson(M).float().contiguous()
    del M
    zeros = float((X == 0).float().mean())
    G0 = torch.rand(J, device=dev, generator=g) * 0.9 + 0.1
    A0 = [torch.rand((d, j), device=dev, generator=g) * 0.9 + 0.1 for d, j in zip(dims, J)]
    obj = torch.zeros(1, dtype=torch.float64, device=dev)
    out = {"workload": "dense 5-way Tucker %s, ranks %s, synthetic counts" % ("x".join(map(str, dims)),
                                                                            ",".join(map(str, J))),
           "zero_fraction": zeros, "precision": "tf32", "l2": "inputs larger than L2 (181 MB), no flush"}
    for beta in (0.5, 1.0, 1.5):
        for name in ("block_mm", "jcomm"):
            G, A = G0.clone(), [a.clone() for a in A0]

            def step():
                if name == "jcomm":
                    ntf.jcomm_outer(X, beta, A, core=G, objective=obj, ctx=ctx, precision="tf32")
                else:
                    ntf.tucker_mu_sweep(X, beta, G, A, objective=obj, ctx=ctx, precision="tf32")
            for _ in range(3):
                step()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(iters):
                step()
            e1.record()
            torch.cuda.synchronize()
            out["%s_b%g_ms" % (name, beta)] = e0.elapsed_time(e1) / max(iters, 1)
            out["%s_b%g_mean_objective" % (name, beta)] = obj.item() / X.numel()
    return out


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                "sm_max_mhz": 2070.0}, "fallback"


# --------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for k, v in zip(names, f[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(k)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------------ CPU oracle
def oracle_step_sample(X, A, cores, budget_s):
    """Times the FP64 oracle on a bounded sample of one J-CoMM outer iteration at beta = 1:
    the numerator/denominator rows of a set of evenly spaced row indices per mode, scaled to
    the full iteration (I_n rows per mode).  The row count is calibrated on a few rows so
    that the sample takes about `budget_s` seconds of CPU time (at most every row, i.e. the
    whole iteration).  Returns (seconds per full step estimate, description)."""
    import oracle
    probe = min(min(DIMS), 2 * cores)  # rows run in parallel: probe with every core busy
    t0 = time.perf_counter()
    for n in range(3):
        oracle.cp_numden_rows(X, A, A, A, n, np.arange(probe, dtype=np.int64), BETA)
    per_row = (time.perf_counter() - t0) / (3 * probe)
    rows_per_mode = int(min(min(DIMS), max(probe, budget_s / (3 * per_row))))
    # when every row fits the budget, the whole iteration is repeated (at most five times)
    reps = max(1, min(5, int(budget_s / (3 * per_row * rows_per_mode))))
    total = 0.0
    spent = 0.0
    for _ in range(reps):
        for n in range(3):
            rows = np.linspace(0, DIMS[n] - 1, rows_per_mode).astype(np.int64)
            t0 = time.perf_counter()
            oracle.cp_numden_rows(X, A, A, A, n, rows, BETA)
            dt = time.perf_counter() - t0
            spent += dt
            total += dt * DIMS[n] / rows_per_mode / reps
    desc = ("FP64 oracle (ntfo_cp_numden_rows, OpenMP) on %d evenly spaced rows per mode (of %s) of one J-CoMM "
            "outer iteration (all three numerator/denominator row sets from the reference factors), %d time(s), "
            "scaled by I_n/rows; %.1f s of CPU work" % (rows_per_mode, "x".join(map(str, DIMS)), reps, spent))
    return total, desc


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import synth
    cores = os.cpu_count() or 1
    os.environ.setdefault("OMP_NUM_THREADS", str(cores))
    X, _ = synth.cp_dense(DIMS, RANK, seed=0, kind="gamma_noise")
    X = X.astype(np.float64)  # the oracle's input type, converted once outside the timed samples
    A = synth.init_factors(DIMS, RANK, seed=1)
    per = []
    desc = ""
    # each step a bounded sample, so that the whole run stays within about three minutes
    budget = min(10.0, 180.0 / max(1, args.warmup + args.steps))
    for s in range(args.warmup + args.steps):
        sec, desc = oracle_step_sample(X, A, cores, budget)
        if s >= args.warmup:
            per.append(sec)
    sec = sum(per) / len(per)
    v = 1.0 / sec
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "sweeps/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": "bounded row sample, see cpu_baseline"},
            "cpu_baseline": {"value": v, "unit": "sweeps/s", "cores": cores, "kind": "oracle", "sample": desc},
            "e2e": {"value": v, "unit": "sweeps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ----------------------------------------------------------------- replicas (N > 1)
def max_over_ranks(x, world, device):
    """The largest of every rank's x (one all-reduce; x itself at world = 1).  Every rank
    solves its own replica, so the job's time is the slowest rank's."""
    if world == 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(steps, world, seconds_max):
    """Whole-job throughput: the steps of all ranks over the slowest rank's time."""
    return world * steps / seconds_max


# ------------------------------------------------------------------------ GPU arm
def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.profile_n > 0:
        return profile_case(args.profile_n, args.precision)
    if args.profile_case:
        import torch
        import paper_2602_14683_gb300 as ntf
        ctx, peaks = ntf.default_context(), load_peaks()[0]
        if args.profile_case == "jcache":
            return profile_jcache(ntf)
        if args.profile_case == "tucker":
            r = run_tucker_c3(ntf, ctx, peaks, iters=0, precisions=(args.precision,))
        elif args.profile_case == "cp4":
            r = run_cp_4way(ntf, ctx, peaks, iters=1)
        elif args.profile_case == "tucker4":
            r = run_tucker_4way(ntf, ctx, peaks, iters=1)
        elif args.profile_case == "tucker5":
            r = run_tucker_5way(ntf, ctx, peaks, iters=1)
        else:
            r = run_coo_c4(ntf, ctx, peaks, iters=0)
        print("profile case", args.profile_case, "done")
        return 0

    import torch
    import torch.distributed as dist
    import paper_2602_14683_gb300 as ntf
    import synth

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    ctx = ntf.default_context(local)
    peaks, peak_src = load_peaks()
    if args.serve:
        line = {"metric": "served p99", "impl": "ntf", **run_serving(ntf, args.serve_jobs, args.slots)}
        if rank == 0:
            print(json.dumps(line))
        return 0

    # inputs: every rank solves its own replica (independent problems: weak scaling)
    X_np, _ = synth.cp_dense(DIMS, RANK, seed=rank, kind="gamma_noise")
    A_np = synth.init_factors(DIMS, RANK, seed=1000 + rank)
    X = torch.tensor(X_np, dtype=torch.float32, device=dev)
    A0 = [torch.tensor(a, dtype=torch.float32, device=dev) for a in A_np]
    stream = torch.cuda.current_stream(dev)
    prec = args.precision

    def barrier():
        if world > 1:
            dist.barrier()

    def timed(fn, steps, warmup):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        return max_over_ranks(e0.elapsed_time(e1) / 1e3, world, dev)

    # ---------------- headline: J-CoMM outer iterations, inputs resident in HBM -------------
    A = [a.clone() for a in A0]
    obj = torch.zeros(1, dtype=torch.float64, device=dev)

    def jstep():
        ntf.jcomm_outer(X, BETA, A, objective=obj, ctx=ctx, precision=prec, autotune=True)

    for _ in range(args.warmup):
        jstep()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    ctx.set_pass_timing(True)
    ctx.pass_timing()
    l0 = ctx.launches
    t_j = timed(jstep, args.steps, 0)
    launches = ctx.launches - l0
    pass_ms, pass_n = ctx.pass_timing()
    ctx.set_pass_timing(False)

    # ---------------- B-CoMM sweeps on the same tensor ----------------
    B = [a.clone() for a in A0]

    def bstep():
        ntf.cp_mu_sweep(X, BETA, B, objective=obj, ctx=ctx, precision=prec, autotune=True)

    t_b = timed(bstep, max(5, args.steps // 2), args.warmup)
    b_rate = job_rate(max(5, args.steps // 2), world, t_b)

    # ---------------- end to end: host buffers, copies inside the timed region -------------
    Xh = torch.empty(X.shape, dtype=torch.float32).pin_memory()
    Xh.copy_(X)
    Ah = [a.cpu().pin_memory() for a in A0]
    Ahost_out = [torch.empty_like(a).pin_memory() for a in Ah]
    obj_h = torch.zeros(1, dtype=torch.float64).pin_memory()
    Xe = torch.empty_like(X)
    Ae = [torch.empty_like(a) for a in A0]

    def estep():
        Xe.copy_(Xh, non_blocking=True)
        for d, h in zip(Ae, Ah):
            d.copy_(h, non_blocking=True)
        ntf.jcomm_outer(Xe, BETA, Ae, objective=obj, ctx=ctx, precision=prec, autotune=True)
        for h, d in zip(Ahost_out, Ae):
            h.copy_(d, non_blocking=True)
        obj_h.copy_(obj, non_blocking=True)

    e_steps = max(5, args.steps // 5)
    t_e = timed(estep, e_steps, min(args.warmup, 3))
    # clocks sampled from before the headline region through the B-CoMM and end-to-end ones
    clk = clocks.stop()
    h2d = X.numel() * 4 + sum(a.numel() * 4 for a in A0)
    d2h = sum(a.numel() * 4 for a in A0) + 8

    # ---------------- time to F*(1 + 1e-4) at beta = 1, every method ----------------
    ttt = None
    if not args.no_ttt:
        # F* = lowest FP64 objective of 1000 FP32 block-MU sweeps from the shared init; every
        # other method runs from the same init until its objective first reaches F*(1+1e-4)
        # or an iteration cap, recording the objective of each incoming iterate on the device
        # (checked every 100 iterations)
        class Extrap:
            # extrapolated sweeps / outer iterations with the Nesterov-type weights, one state
            # per factor list
            def __init__(self, fn):
                self.fn, self.prev, self.w = fn, {}, {}

            def __call__(self, X, beta, A, objective=None, ctx=None, precision="tf32", autotune=False):
                k = id(A)
                if k not in self.prev:
                    self.prev[k] = [a.clone() for a in A]
                    self.w[k] = ntf.nesterov_weights()
                self.fn(X, beta, A, self.prev[k], next(self.w[k]), objective=objective, ctx=ctx,
                        precision=precision, autotune=autotune)

        F_ref, per_ref, ch = run_until(ntf, ctx, X, A0, BETA, ntf.cp_mu_sweep, "fp32", 1000, None)
        fstar = float(F_ref.min())
        runs = {"block_mu_fp32": (F_ref, per_ref, ch)}
        for name, fn, p, cap in (("jcomm_" + prec, ntf.jcomm_outer, prec, 5000),
                                 ("jcomm_3xtf32", ntf.jcomm_outer, "3xtf32", 5000),
                                 ("block_mu_" + prec, ntf.cp_mu_sweep, prec, 2000),
                                 ("block_mu_extrap_" + prec, Extrap(ntf.cp_mu_sweep_extrap), prec, 2000),
                                 ("jcomm_extrap_" + prec, Extrap(ntf.cp_jcomm_outer_extrap), prec, 2000),
                                 ("jcomm_fp32", ntf.jcomm_outer, "fp32", 2000)):
            if name not in runs:
                runs[name] = run_until(ntf, ctx, X, A0, BETA, fn, p, cap, fstar * (1 + 1e-4))
        ttt = {"target": "F*(1+1e-4)", "F_star": fstar,
               "F_star_from": "lowest objective of 1000 FP32 block-MU sweeps", **ttt_summary(runs, fstar)}

    # ---------------- C2 as stated: every beta, block-MU vs J-CoMM L = 1, 3 ----------------
    c2_betas = tuple(float(b) for b in args.c2_betas.split(",")) if args.c2_betas else ()
    # beta = 1's time to target is the every-method run above
    c2 = run_cp_c2(ntf, ctx, peaks, X, A0, prec, betas=c2_betas,
                   ttt_betas=() if args.no_ttt else tuple(b for b in c2_betas if b != BETA))
    c1 = run_cp_c1(ntf, ctx)

    # ---------------- roofline of the dominant kernel (the fused pass) ----------------
    entries = DIMS[0] * DIMS[1] * DIMS[2]
    # J-CoMM at beta = 1: one fused pass per outer iteration; per entry 2R flops rebuild
    # Xtilde, 2R contract P against the last factor (modes 1 and 2), 2R against the
    # row Khatri-Rao product (mode 3); 4 bytes of X read.
    flops_per_launch = entries * 6 * RANK
    bytes_per_launch = entries * 4
    avg_pass = pass_ms / 1e3 / max(pass_n, 1)
    if prec == "fp32":
        sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
        peak = sm_count * 128 * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
        roof = {"bound": "alu", "achieved": flops_per_launch / avg_pass / 1e12, "peak": peak, "unit": "TFLOP/s",
                "peak_source": "FP32 FMA pipe: %d SMs x 128 lanes x 2 flop x %.0f MHz (derived)" %
                               (sm_count, peaks.get("sm_max_mhz", 2070.0)),
                "hbm_achieved_gbs": bytes_per_launch / avg_pass / 1e9}
    else:
        # tensor-core pass: the contractions run far below the tensor peak, so the bound
        # is the HBM stream of X (4 bytes per entry, read once per launch)
        roof = {"bound": "hbm", "achieved": bytes_per_launch / avg_pass / 1e9, "peak": peaks["hbm_gbs"],
                "unit": "GB/s", "peak_source": "%s HBM copy bandwidth" % peak_src,
                "tensor_tflops_algorithmic": flops_per_launch / avg_pass / 1e12}
    roof["frac"] = roof["achieved"] / roof["peak"]
    roof["traffic"] = tc_traffic(entries) if prec == "tf32" else None
    roof["pass_ms_avg"] = avg_pass * 1e3
    roof["pass_launches"] = pass_n

    # ---------------- CPU oracle baseline (rank 0, N = 1 only) ----------------
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cores = os.cpu_count() or 1
        sec, desc = oracle_step_sample(X_np.astype(np.float64), A_np, cores, 12.0)
        cpu = {"value": 1.0 / sec, "unit": "sweeps/s", "cores": cores, "kind": "oracle", "sample": desc}
    # C3's metric needs the oracle too: the per-iteration objective error of each precision
    # against FP64 (same leg: rank 0, N = 1)
    c3_ora = None
    if rank == 0 and world == 1 and not args.no_cpu and not args.no_other:
        c3_ora = c3_vs_oracle(ntf, ctx)

    other = None
    if not args.no_other:
        other = {"tucker_c3": run_tucker_c3(ntf, ctx, peaks), "coo_c4": run_coo_c4(ntf, ctx, peaks),
                 "cp_4way": run_cp_4way(ntf, ctx, peaks), "tucker_4way": run_tucker_4way(ntf, ctx, peaks),
                 "tucker_5way": run_tucker_5way(ntf, ctx, peaks), "batch_cp": run_batch_cp(ntf)}

    serving = None
    if args.serve_jobs > 0:
        serving = run_serving(ntf, args.serve_jobs, args.slots)

    value = job_rate(args.steps, world, t_j)
    line = {
        "metric": METRIC, "value": value, "unit": "sweeps/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_j / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": DTYPES[prec], "data": "synthetic",
        "config": {"workload": WORKLOAD, "precision": prec, "method": "J-CoMM L=1", "plan": "autotuned slab split",
                   "l2": "inputs larger than L2 (537 MB tensor), no flush", "parallelism": "replicas"},
        "block_mu_sweeps_per_s": b_rate,
        "time_to_target": ttt,
        "c1_latency": c1,
        "c2_table": c2,
        "c3_objective_error_vs_oracle": c3_ora,
        "serving": serving,
        "other_configs": other,
        "roofline": roof,
        "cpu_baseline": cpu,
        "e2e": {"value": job_rate(e_steps, world, t_e), "unit": "sweeps/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": launches,
        "clocks": clk,
    }
    if rank == 0:
        print(json.dumps(line))
        sys.stdout.flush()
        sys.stderr.write(summary(line) + "\n")
    if world > 1:
        dist.destroy_process_group()
    return 0


def summary(line):
    """Compact text of the figures beyond the headline, for readers of the log's tail."""
    out = ["SUMMARY %s %.1f %s, pass frac %.3f of HBM (%s)" % (line["config"]["precision"], line["value"], line["unit"],
           line["roofline"]["frac"], line["roofline"]["unit"])]
    t = line.get("time_to_target")
    if t:
        out.append("TTT beta=1 F*(1+1e-4): " + ", ".join(
            "%s %s s (%s it)" % (k, None if v["seconds"] is None else round(v["seconds"], 3), v["iters"])
            for k, v in t.items() if isinstance(v, dict)))
    c2 = line.get("c2_table") or {}
    for b, r in c2.items():
        if not isinstance(r, dict) or "block_mu" not in r:
            continue
        row = "C2 %s ms: block %.3f, J L1 %.3f, J L3 %.3f" % (b, r["block_mu"]["ms"], r["jcomm_L1"]["ms"], r["jcomm_L3"]["ms"])
        if "time_to_target" in r:
            row += "; TTT s: " + ", ".join("%s %s" % (k, None if v["seconds"] is None else round(v["seconds"], 3))
                                           for k, v in r["time_to_target"].items() if isinstance(v, dict))
        out.append(row)
    c1 = line.get("c1_latency")
    if c1:
        out.append("C1 us/sweep: fp32 %.1f, tf32 %.1f; replayed as a CUDA graph: fp32 %.1f, tf32 %.1f" % (
            c1["fp32"]["us_per_sweep"], c1["tf32"]["us_per_sweep"], c1["fp32"].get("graph_us_per_sweep", 0.0),
            c1["tf32"].get("graph_us_per_sweep", 0.0)))
    c3 = line.get("c3_objective_error_vs_oracle")
    if c3:
        out.append("C3 max rel obj err vs FP64 oracle: " + ", ".join(
            "%s %.2e" % (k, v["max_rel_err"]) for k, v in c3.items() if isinstance(v, dict)))
    o = line.get("other_configs") or {}
    if o.get("tucker_c3"):
        tc = o["tucker_c3"]
        out.append("C3 ms block/jcomm: " + ", ".join("%s %.3f/%.3f" % (p, tc[p]["block_mm_ms"], tc[p]["jcomm_ms"])
                                                  for p in ("fp32", "tf32", "3xtf32") if p in tc))
    if o.get("coo_c4"):
        c4 = o["coo_c4"]
        out.append("C4 us/outer %.1f; frac hbm %.3f alu %.3f l2 %.3f" % (c4["us_per_outer"], c4["roofline"]["frac"],
                                                                        c4["alu"]["frac"], c4["l2_gather"]["frac"]))
        if c4.get("beta_1p5_jcomm"):
            b15 = c4["beta_1p5_jcomm"]
            out.append("C4 shape at beta=1.5: %.1f ms/outer on tensor cores, %.1f ms on the FP32 pipe" % (
                b15["tf32"]["ms_per_outer"], b15["fp32"]["ms_per_outer"]))
    if o.get("batch_cp"):
        bc = o["batch_cp"]
        out.append("batched small CP jobs: %.1f solves/s (%d jobs), one at a time %.1f solves/s" % (
            bc["batched"]["solves_per_s"], bc["batched"]["jobs"], bc["one_at_a_time"]["solves_per_s"]))
    sv = line.get("serving")
    if sv:
        out.append("C5 %d jobs: sat %.1f/s, at 0.8x: %.1f/s p50 %.3f s p99 %.3f s; sweep " % (
            sv["jobs"], sv["saturation_solves_per_s"], sv["solves_per_s"], sv["p50_latency_s"], sv["p99_latency_s"]) +
            ", ".join("%s %.1f/%.1f p99 %.3f" % (k, v["achieved_per_s"], v["offered_per_s"], v["p99_latency_s"])
                      for k, v in sv["load_sweep"].items()))
    return "\n".join(out)


if __name__ == "__main__":
    sys.exit(main())
