#!/usr/bin/env python3
"""Benchmark: batched mixed-precision ODWF D^dag D solves on one GB300.

One step solves the 16^3 x 32 x Ns=16 workload's three systems (m_q = 0.002, 0.04, 0.5,
one Gaussian right-hand side each) to a true residual of 1e-10 with the batched mixed-
precision CG (FP16 storage with per-site scales, FP32 links of 12 reals, FP32 arithmetic,
float-float reliable updates), as one odwf_cg_solve_batched call.  Prints one JSON line.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--prec f16|bf16|f32]

--impl reference times the FP64 CPU oracle (a bounded sample per step, see cpu_baseline).
Under torchrun (N > 1) every rank runs an independent replica of the workload (the solve
does not shard); value = all ranks' solves / the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import signal
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "ODWF D†D solves/s & Dslash HBM GB/s vs FP64 CG; p50/p99 served latency"
DIMS = (16, 16, 16, 32)
NS = 16
M0 = 1.3
MASSES = (0.002, 0.04, 0.5)
EPS = 0.25
GAUGE_SEED = 2
RHS_SEED = 100
LRANGE = (0.05, 6.2)
TOL = 1e-10
WORKLOAD = "odwf_dagd_16x16x16x32_ns16_3mass"
ORACLE_COUNTS = os.path.join(ROOT, "tests", "golden", "oracle_cg_16x16x16x32_ns16.json")
NCU_TRAFFIC = os.path.join(ROOT, "profiles", "ncu_traffic.txt")
L2_FLUSH_BYTES = 512 << 20


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def workload_inputs(lib_omega=True):
    """Gauge field, weights and right-hand sides of the workload.  The GPU arm takes the weights
    from the library (odwf_zolotarev_omega); the oracle arm from the oracle's own generator
    (the two agree to 1e-7, tests/test_abi_host.py)."""
    import odwf_synth as syn

    U = syn.gauge_field(DIMS, EPS, GAUGE_SEED)
    if lib_omega:
        import paper_1811_08095_gb300 as odwf

        w, _ = odwf.odwf_zolotarev_omega(NS, LRANGE[0], LRANGE[1])
    else:
        from oracle import zolotarev

        w, _ = zolotarev.omega(NS, LRANGE[0], LRANGE[1], True)
    bs = [syn.gaussian_spinor_even(NS, DIMS, RHS_SEED + k) for k in range(len(MASSES))]
    return U, w, bs


def oracle_iteration_counts():
    """The oracle's own CG iteration counts on this workload (tests/golden, oracle-only script)."""
    if not os.path.exists(ORACLE_COUNTS):
        return None
    d = json.load(open(ORACLE_COUNTS))
    by = {s["mq"]: s for s in d["systems"]}
    if not all(m in by for m in MASSES):
        return None
    # iterations to the 1e-10 residual of this workload (the golden runs go on to 1e-13)
    return [by[m].get("iters_1e10", by[m]["iters"]) for m in MASSES], any(by[m]["capped"] for m in MASSES)


def solution_errors(xs):
    """Per-system error of the solutions against the oracle's own solutions (run to 1e-13), on
    the components sampled in tests/golden: |x - x_oracle| / |x_oracle| over the sample, with the
    bound kappa * tol (kappa from the oracle's Lanczos coefficients)."""
    import numpy as np
    import torch

    if not os.path.exists(ORACLE_COUNTS):
        return None
    by = {s["mq"]: s for s in json.load(open(ORACLE_COUNTS))["systems"]}
    out = []
    for x, mq in zip(xs, MASSES):
        rec = by.get(mq)
        if not rec or "sample_index" not in rec or "kappa" not in rec:
            out.append(None)
            continue
        idx = torch.as_tensor(rec["sample_index"], device=x.device)
        got = x.reshape(-1)[idx].cpu().numpy()
        ref = np.asarray(rec["sample_re"]) + 1j * np.asarray(rec["sample_im"])
        out.append({"mq": mq, "sampled_rel_error": float(np.linalg.norm(got - ref) / np.linalg.norm(ref)),
                    "kappa": rec["kappa"], "bound_kappa_tol": rec["kappa"] * TOL, "samples": len(idx)})
    return out


def oracle_seconds_per_iteration(U, w, b, mq):
    """Bounded sample: one oracle CG iteration (its initial residual, one iteration and the
    final true residual are three S^dag S applications; the time is divided by three)."""
    import oracle

    t = time.perf_counter()
    oracle.cg(U, b, M0, mq, w, tol=1e-30, max_iter=1)
    return (time.perf_counter() - t) / 3.0, oracle.num_threads()


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.send_signal(signal.SIGTERM)
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        rows = []
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        if not rows:
            return None
        sm = sorted(float(r[1]) for r in rows if r[1].replace(".", "").isdigit())
        mx = max(float(r[2]) for r in rows if r[2].replace(".", "").isdigit())
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if "Active" in r[5 + i] and "Not" not in r[5 + i]})
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": mx, "reasons": reasons,
                "samples": len(rows)}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


FLOW_TRAFFIC = os.path.join(ROOT, "profiles", "ncu_traffic_flow.txt")


def ncu_traffic_file(path, kernel_class):
    """DRAM bytes per launch of a kernel class from a committed ncu summary (class bytes ...)."""
    if not os.path.exists(path):
        return None
    for line in open(path):
        parts = line.split()
        if len(parts) >= 2 and not line.startswith("#") and parts[0] == kernel_class:
            return float(parts[1])
    return None


# Kernel classes whose source changed after the committed ncu captures: the block partial of their
# final reduction moved to a fixed per-system stride (one 8-byte store per block, nothing else).
# Their captured DRAM bytes are reported as prior-capture values, `traffic` itself is null.
TRAFFIC_CHANGED_SINCE_CAPTURE = ("K2_schur_norm_mdinv", "K4_normal_cg")
TRAFFIC_NOTE = ("captured before the final reduction's block partial moved to a fixed per-system stride "
                "(the only change to this kernel since; one 8-byte store per block)")


def traffic_fields(kernel_class, tr):
    """{'traffic': tr} when the capture matches the current kernel, else null with the prior value."""
    if tr is not None and kernel_class.endswith(TRAFFIC_CHANGED_SINCE_CAPTURE):
        return {"traffic": None, "traffic_prior_capture": tr, "traffic_note": TRAFFIC_NOTE}
    return {"traffic": tr}


def ncu_traffic(kernel_class):
    """(dram bytes per launch, running systems in that launch) for a kernel class from the
    committed ncu summary, if present."""
    if not os.path.exists(NCU_TRAFFIC):
        return None
    for line in open(NCU_TRAFFIC):
        parts = line.split()
        if len(parts) >= 3 and not line.startswith("#") and parts[0] == kernel_class:
            try:
                return float(parts[1]), int(parts[2])
            except ValueError:
                return None
    return None


def update_arith_name(updates):
    """The reliable-update arithmetic of a mixed solve (AUTO is float-float)."""
    return "FP64" if updates == "f64" else "float-float"


def aggregate(t_local_s: float, solves_local: int, dist=None, device=None):
    """Whole-job throughput of independent replicas: every rank's solves over the slowest rank's
    timed region (max over ranks), as the replicas-only multi-GPU contract asks."""
    if dist is None:
        return solves_local / t_local_s, t_local_s, solves_local
    import torch

    t = torch.tensor([t_local_s, float(solves_local)], dtype=torch.float64, device=device)
    tmax = t[:1].clone()
    dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
    n = t[1:].clone()
    dist.all_reduce(n, op=dist.ReduceOp.SUM)
    return float(n.item()) / float(tmax.item()), float(tmax.item()), int(n.item())


def read_profile(lib):
    import ctypes

    from paper_1811_08095_gb300 import _lib

    arr = (_lib.odwf_kernel_prof * 64)()
    n = ctypes.c_int(0)
    _lib.check(lib.odwf_profile_read(ctypes.cast(arr, ctypes.c_void_p), 64, ctypes.byref(n)))
    out = []
    for i in range(n.value):
        e = arr[i]
        out.append({"name": e.name.decode(), "launches": e.launches, "system_launches": e.system_launches,
                    "total_ms": e.total_ms, "bytes_per_system": e.bytes_per_system,
                    "bytes_per_launch": e.bytes_per_launch})
    return out


DSLASH_DIMS = (32, 32, 32, 32)
DSLASH_TRAFFIC = os.path.join(ROOT, "profiles", "ncu_traffic_dslash.txt")


def dslash_roofline(args, dev, reps=20):
    """Standalone hop kernels on 32^4 x 16 (odwf_time_kernel: one warm-up launch, then `reps`
    launches between two CUDA events on the launching stream).  Per kernel: average launch time,
    algorithmic bytes per launch (each field once per system plus the links once), GB/s and the
    fraction of the measured HBM peak; ncu DRAM traffic where profiles/ holds a capture."""
    import torch

    import odwf_synth as syn
    import paper_1811_08095_gb300 as odwf

    peak, peak_kind = measured_peaks()
    dims = DSLASH_DIMS
    vh = dims[0] * dims[1] * dims[2] * dims[3] // 2
    w, _ = odwf.odwf_zolotarev_omega(NS, LRANGE[0], LRANGE[1])
    U = syn.gauge_field_torch(dims, EPS, 3, device=dev)
    h = odwf.Handle(dims, NS, M0, MASSES[1], w)
    h.set_gauge(U)
    del U
    g = torch.Generator(device=dev)
    g.manual_seed(1)
    fill = torch.randn((NS, vh, 4, 3), dtype=torch.complex128, device=dev, generator=g)
    traffic = {}  # (class, systems) -> DRAM bytes per launch from the committed ncu capture
    if os.path.exists(DSLASH_TRAFFIC):
        for line in open(DSLASH_TRAFFIC):
            parts = line.split()
            if len(parts) >= 3 and not line.startswith("#"):
                traffic[(parts[0], int(parts[1]))] = float(parts[2])
    out = {"lattice": "32^4", "Ns": NS, "spinors": "f16 (per-site FP32 scale)", "reps": reps,
           "timing": "CUDA events around %d launches on the launching stream, after one warm-up launch" % reps,
           "peak": peak, "peak_source": peak_kind + " (MEASURED_PEAKS hbm_gbs)", "kernels": []}
    for link_prec in ("f32", "f16"):
        for nsys in (1, 3):
            for kind in (1, 2, 3, 4):
                if link_prec == "f16" and kind != 1:
                    continue
                r = h.time_kernel(kind, fill, prec="f16", link_prec=link_prec, nsys=nsys, reps=reps)
                per_launch = nsys * r["bytes_per_system"] + r["bytes_per_launch"]
                avg_s = r["total_ms"] / r["launches"] / 1e3
                gbs = per_launch / avg_s / 1e9
                tr = traffic.get((r["name"], nsys))
                rec = {"kernel": r["name"], "links": link_prec, "systems": nsys, "avg_us": round(avg_s * 1e6, 1),
                       "algorithmic_bytes": per_launch, "gbs": round(gbs, 1), "frac": round(gbs / peak, 4)}
                rec.update(traffic_fields(r["name"], tr))
                out["kernels"].append(rec)
    h.close()
    del fill
    torch.cuda.empty_cache()
    k1 = [k for k in out["kernels"] if k["kernel"].endswith("K1_chi_minv")]
    best = max(k1, key=lambda k: k["frac"])
    out["dslash_k1_best"] = {"kernel": best["kernel"], "links": best["links"], "systems": best["systems"],
                             "gbs": best["gbs"], "frac": best["frac"]}
    return out


def run_ours(args, world, rank, local):
    import numpy as np
    import torch

    import paper_1811_08095_gb300 as odwf

    dist = None
    if world > 1:
        import torch.distributed as dist_mod

        dist = dist_mod
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    lib = odwf.load()
    stream = torch.cuda.current_stream()

    U, w, bs_host = workload_inputs()
    h = odwf.Handle(DIMS, NS, M0, MASSES[0], w)
    h.set_gauge(torch.from_numpy(U).to(dev))
    bs = [torch.from_numpy(b).to(dev) for b in bs_host]
    xs = [torch.zeros_like(b) for b in bs]
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def step(prec):
        return h.cg_solve_batched(xs, bs, list(MASSES), tol=TOL, max_iter=200000, prec=prec, delta=args.delta,
                                  link_recon=args.link_recon, check_every=args.check_every, stream=stream,
                                  updates=args.updates)

    for _ in range(args.warmup):
        stats = step(args.prec)
    torch.cuda.synchronize()

    # ---- timed region: K steps, L2 flushed between steps, CUDA events on the solve's stream.
    # The library runs as a user runs it (iteration chunks replayed as CUDA graphs).
    launches0 = lib.odwf_launch_count()
    clocks = ClockSampler(local)
    clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    step_ms = []
    all_stats = []
    t_wall = time.perf_counter()
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st = step(args.prec)
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        all_stats.append(st)
    torch.cuda.synchronize()
    wall_s = time.perf_counter() - t_wall
    if dist:
        dist.barrier()
    clk = clocks.stop()
    launches = lib.odwf_launch_count() - launches0

    # ---- the same K steps again with the library's per-launch CUDA events (kernel durations
    # for the roofline; per-launch events rule out graph replay, so this pass is not timed)
    lib.odwf_profile_enable(1)
    torch.cuda.synchronize()
    prof_step_ms = []
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step(args.prec)
        e1.record(stream)
        e1.synchronize()
        prof_step_ms.append(e0.elapsed_time(e1))
    torch.cuda.synchronize()
    prof = read_profile(lib)
    lib.odwf_profile_enable(0)

    sol_err = solution_errors(xs)  # the solutions of the last profiled step
    value, t_total, nsolves = aggregate(sum(step_ms) / 1e3, len(MASSES) * args.steps, dist, dev)
    for st in all_stats:
        for s in st:
            assert s["status"] == 0 and s["true_resid"] <= TOL, s

    # ---- roofline of the dominant kernel (largest total time) from the in-library events
    peak, peak_kind = measured_peaks()
    dom = max(prof, key=lambda e: e["total_ms"]) if prof else None
    roof = None
    hops = {}
    for e in prof:
        tot_bytes = e["system_launches"] * e["bytes_per_system"] + e["launches"] * e["bytes_per_launch"]
        gbs = tot_bytes / (e["total_ms"] / 1e3) / 1e9 if e["total_ms"] > 0 else 0.0
        hops[e["name"]] = {"launches": e["launches"], "avg_us": 1e3 * e["total_ms"] / max(1, e["launches"]),
                           "gbs": round(gbs, 1), "share_of_step": round(e["total_ms"] / sum(prof_step_ms), 4)}
    if dom:
        per_launch = (dom["system_launches"] * dom["bytes_per_system"] + dom["launches"] * dom["bytes_per_launch"]) \
            / dom["launches"]
        avg_s = dom["total_ms"] / dom["launches"] / 1e3
        achieved = per_launch / avg_s / 1e9
        # ncu traffic of a captured launch, scaled to this run's average launch by algorithmic bytes
        tr = None
        cap = ncu_traffic(dom["name"])
        if cap:
            cap_bytes, cap_sys = cap
            cap_alg = cap_sys * dom["bytes_per_system"] + dom["bytes_per_launch"]
            tr = round(cap_bytes * per_launch / cap_alg)
        roof = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "kernel": dom["name"],
                "timing": "per-launch CUDA events on the launching stream over a second pass of the K timed "
                          "steps (%.1f ms per step with the events vs %.1f without)" % (
                              sum(prof_step_ms) / len(prof_step_ms), sum(step_ms) / len(step_ms)),
                "algorithmic_bytes_per_launch": per_launch, "peak_source": peak_kind + " (MEASURED_PEAKS hbm_gbs)"}
        roof.update(traffic_fields(dom["name"], tr))

    # ---- end to end through the C ABI with pinned host buffers (copies inside the timed region)
    bh = [torch.from_numpy(b).pin_memory() for b in bs_host]
    xh = [torch.zeros_like(b).pin_memory() for b in bh]
    h2d = sum(b.numel() * b.element_size() for b in bh)
    d2h = sum(x.numel() * x.element_size() for x in xh)
    h.cg_solve_batched([x.numpy() for x in xh], [b.numpy() for b in bh], list(MASSES), tol=TOL, max_iter=200000,
                       prec=args.prec, delta=args.delta, link_recon=args.link_recon, stream=stream,
                       updates=args.updates)  # warm
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        h.cg_solve_batched([x.numpy() for x in xh], [b.numpy() for b in bh], list(MASSES), tol=TOL,
                           max_iter=200000, prec=args.prec, delta=args.delta, link_recon=args.link_recon,
                           stream=stream, updates=args.updates)
    e2e_s = time.perf_counter() - t0
    e2e = {"value": round(len(MASSES) * args.steps * world / e2e_s, 4), "unit": "solves/s",
           "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}

    # ---- the FP64 GPU CG on the same systems (the comparison baseline of the metric): one
    # untimed warm-up solve (graph capture, workspaces), then the same K steps as the mixed arm,
    # L2 flushed between steps, CUDA events on the solve's stream
    fp64 = None
    if not args.skip_fp64:
        step("f64")
        torch.cuda.synchronize()
        t64s = []
        for _ in range(max(3, args.steps)):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            st64 = step("f64")
            e1.record(stream)
            e1.synchronize()
            t64s.append(e0.elapsed_time(e1) / 1e3)
        t64 = sum(t64s) / len(t64s)
        fp64 = {"value": round(len(MASSES) / t64, 4), "unit": "solves/s", "steps": len(t64s), "warmup": 1,
                "s_per_step": [round(t, 3) for t in t64s], "iters": [s["iters"] for s in st64],
                "true_resid": [s["true_resid"] for s in st64],
                "speedup_mixed_vs_fp64": round(value / world / (len(MASSES) / t64), 2)}

    # ---- the Dslash proper on a working set far larger than L2: the K1 hop
    # (chi_t = B M^-1 (-1/2 W chi_p)) and the other three hops of the iteration, alone, on
    # 32^4 x 16 with FP16 spinors (436 MB per field and system), one and three systems
    dslash = None if args.skip_dslash else dslash_roofline(args, dev)

    cpu = None
    if rank == 0 and not args.skip_cpu:
        counts = oracle_iteration_counts()
        spi, cores = oracle_seconds_per_iteration(U, w, bs_host[1], MASSES[1])
        if counts:
            iters, capped = counts
            src = "the oracle's own CG iteration counts %s (tests/golden, %s)" % (
                iters, "lower bounds: capped runs" if capped else "converged runs")
        else:
            iters = [s["iters"] for s in (fp64 and st64 or all_stats[-1])]
            src = "the FP64 CG iteration counts measured on the GPU in this run %s" % iters
        cpu = {"value": round(len(MASSES) / (spi * sum(iters)), 8), "unit": "solves/s", "cores": cores,
               "kind": "oracle",
               "sample": "one FP64 oracle CG iteration on the same 16^3x32x16 workload (m_q=0.04; %.1f s per "
                         "iteration on %d threads), scaled by %s" % (spi, cores, src)}

    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 4), "unit": "solves/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(sum(step_ms) / len(step_ms), 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "lattice": "16^3x32", "Ns": NS, "m0": M0, "masses": list(MASSES),
                       "rhs": "one unit-Gaussian right-hand side per mass (seeds 100-102)",
                       "gauge": "U = exp(0.25 i H), H Gaussian traceless Hermitian (seed 2)",
                       "omega": "shifted (R5) Zolotarev on [0.05, 6.2]", "tol": TOL,
                       "precision": "%s storage (per-site FP32 scale), FP32 links (%d reals), FP32 arithmetic, "
                                    "%s reliable updates (delta %g), FP64 reductions" % (
                                        args.prec, args.link_recon, update_arith_name(args.updates),
                                        args.delta),
                       "solver": "batched even-odd CG on S^dag S, 3 systems per launch",
                       "l2": "flushed between steps (512 MB write); per-system working set > 1 GB",
                       "parallelism": "replicas only" if world > 1 else "single GPU",
                       "iters": [s["iters"] for s in all_stats[-1]],
                       "reliable_updates": [s["n_reliable"] for s in all_stats[-1]],
                       "true_resid": [s["true_resid"] for s in all_stats[-1]],
                       "solution_error": sol_err,
                       "wall_s_timed_region": round(wall_s, 3)},
            "roofline": roof, "kernels": hops, "dslash": dslash, "fp64_cg": fp64, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": int(launches), "clocks": clk,
        }
        print(json.dumps(line), flush=True)
    h.close()
    if dist:
        dist.destroy_process_group()


FLOW_DIMS = (64, 64, 64, 64)
FLOW_EPS = 0.01
FLOW_SEGMENT = 10  # Runge-Kutta steps per bench step; one measurement closes each segment
FLOW_GAUGE_EPS = 0.2
FLOW_WORKLOAD = "wilson_flow_64x64x64x64_eps0.01"


def run_flow(args, world, rank, local):
    """Gradient flow on the paper's 64^4 lattice (Sec. 2-3: step 0.01, E(t) for t0, clover Q and
    the admissibility minimum).  A bench step is FLOW_SEGMENT Runge-Kutta steps followed by one
    measurement; the metric is flow steps per second.  Every rank flows its own field (replicas)."""
    import numpy as np
    import torch

    import odwf_synth as syn
    import paper_1811_08095_gb300 as odwf

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    lib = odwf.load()
    stream = torch.cuda.current_stream()
    dims = tuple(args.flow_dims)
    V = math.prod(dims)
    U = syn.gauge_field_torch(dims, FLOW_GAUGE_EPS, 3, device=dev)
    f = odwf.Flow(dims)
    f.set_gauge(U, stream=stream)
    t = 0.0
    obs = [f.measure(t, stream=stream)]

    def segment(t):
        f.run(FLOW_EPS, FLOW_SEGMENT, measure_every=0, t_start=t, stream=stream)
        t += FLOW_SEGMENT * FLOW_EPS
        return t, f.measure(t, stream=stream)

    for _ in range(args.warmup):
        t, o = segment(t)
        obs.append(o)
    torch.cuda.synchronize()
    launches0 = lib.odwf_launch_count()
    clocks = ClockSampler(local)
    clocks.start()
    torch.cuda.synchronize()
    seg_ms = []
    for _ in range(args.steps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        t, o = segment(t)
        e1.record(stream)
        e1.synchronize()
        seg_ms.append(e0.elapsed_time(e1))
        obs.append(o)
    torch.cuda.synchronize()
    clk = clocks.stop()
    launches = lib.odwf_launch_count() - launches0

    # per-launch events over one more segment (the roofline's kernel durations)
    lib.odwf_profile_enable(1)
    t, o = segment(t)
    obs.append(o)
    torch.cuda.synchronize()
    prof = read_profile(lib)
    lib.odwf_profile_enable(0)
    peak, peak_kind = measured_peaks()
    kernels = {}
    for e in prof:
        tot = e["launches"] * e["bytes_per_launch"]
        kernels[e["name"]] = {"launches": e["launches"], "avg_us": round(1e3 * e["total_ms"] / max(1, e["launches"]), 1),
                              "algorithmic_bytes_per_launch": e["bytes_per_launch"],
                              "gbs": round(tot / (e["total_ms"] / 1e3) / 1e9, 1) if e["total_ms"] > 0 else 0.0}
    dom = max(prof, key=lambda e: e["total_ms"])
    avg_s = dom["total_ms"] / dom["launches"] / 1e3
    achieved = dom["bytes_per_launch"] / avg_s / 1e9
    tr = None
    cap = ncu_traffic_file(FLOW_TRAFFIC, dom["name"])
    if cap:
        tr = round(cap)
    roof = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
            "frac": round(achieved / peak, 4), "traffic": tr, "kernel": dom["name"],
            "algorithmic_bytes_per_launch": dom["bytes_per_launch"],
            "timing": "per-launch CUDA events on the launching stream over one extra segment",
            "peak_source": peak_kind + " (MEASURED_PEAKS hbm_gbs)"}

    # end to end: the field from pinned host memory, one segment, the observables back
    Uh = U.cpu().pin_memory()
    del U
    torch.cuda.empty_cache()
    f.set_gauge(Uh.numpy(), stream=stream)
    torch.cuda.synchronize()
    t_e = time.perf_counter()
    for _ in range(args.steps):
        f.set_gauge(Uh.numpy(), stream=stream)
        segment(0.0)
    e2e_s = time.perf_counter() - t_e
    e2e = {"value": round(args.steps * FLOW_SEGMENT * world / e2e_s, 3), "unit": "flow steps/s",
           "h2d_bytes_per_step": Uh.numel() * Uh.element_size(), "d2h_bytes_per_step": 48}
    f.close()

    cpu = None
    if rank == 0 and not args.skip_cpu:
        from oracle import flow as ofl

        sample = (8, 8, 8, 8)
        Us = syn.gauge_field(sample, FLOW_GAUGE_EPS, 3)
        t_c = time.perf_counter()
        ofl.rk3_step(Us, FLOW_EPS)
        sec = time.perf_counter() - t_c
        per_site = sec / math.prod(sample)
        cpu = {"value": round(1.0 / (per_site * V), 8), "unit": "flow steps/s", "cores": 1, "kind": "oracle",
               "sample": "one oracle Runge-Kutta step on an 8^4 field of the same recipe (%.2f s, numpy in one "
                         "thread), scaled by the site count to %s" % (sec, "x".join(map(str, dims)))}

    full = None
    if args.flow_to > 0:
        # the paper's protocol (Sec. 2-3): flow from t = 0 to t_end in steps of 0.01, E(t) for
        # t0, then the admissibility bound and the clover charge
        Uf = syn.gauge_field_torch(dims, args.flow_to_eps, 4, device=dev)
        f2 = odwf.Flow(dims)
        f2.set_gauge(Uf, stream=stream)
        del Uf
        nsteps = int(round(args.flow_to / FLOW_EPS))
        torch.cuda.synchronize()
        t_f = time.perf_counter()
        rec = f2.run(FLOW_EPS, nsteps, measure_every=10, stream=stream)
        wall = time.perf_counter() - t_f
        f2.close()
        adm = next((o["t"] for o in rec if o["plaq_min"] > 44.0 / 45.0), None)
        t0 = odwf.odwf_flow_t0(rec, 0.3)
        qs = [o["q_clover"] for o in rec]
        full = {"field": "U = exp(%g i H), H Gaussian traceless Hermitian (seed 4)" % args.flow_to_eps,
                "t_end": round(nsteps * FLOW_EPS, 4), "steps": nsteps, "measurements": len(rec),
                "wall_s": round(wall, 2), "t0_from_t2E_0.3": t0,
                "t2E_max": round(max(o["t"] ** 2 * o["e_clover"] for o in rec), 6),
                "first_admissible_t": adm, "q_clover_end": round(qs[-1], 6),
                "q_clover_at": {str(round(o["t"], 2)): round(o["q_clover"], 5)
                                for o in rec if round(o["t"], 2) in (0.0, 1.0, 4.0, 16.0, 32.0, 48.0, 64.0)},
                "plaq_min_end": round(rec[-1]["plaq_min"], 8), "e_clover_end": rec[-1]["e_clover"]}

    seg = sum(seg_ms) / len(seg_ms)
    value = world * FLOW_SEGMENT / (seg / 1e3)
    if rank == 0:
        line = {
            "metric": "gradient-flow Runge-Kutta steps/s on %s (eps 0.01), E / Q_clover / admissibility measured "
                      "every 10 steps" % "x".join(map(str, dims)),
            "value": round(value, 3), "unit": "flow steps/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(seg, 3), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32 (links as float-float pairs)", "data": "synthetic",
            "config": {"workload": FLOW_WORKLOAD if dims == FLOW_DIMS else "wilson_flow_%s_eps0.01" % "x".join(
                           map(str, dims)), "lattice": "x".join(map(str, dims)), "eps": FLOW_EPS,
                       "step": "%d Runge-Kutta steps + one measurement" % FLOW_SEGMENT,
                       "gauge": "U = exp(0.2 i H), H Gaussian traceless Hermitian (seed 3)",
                       "site_steps_per_s": round(value * V, 1),
                       "l2": "not flushed: the flow's working set (%.1f GB) exceeds L2" % (1088 * V / 1e9),
                       "parallelism": "replicas only" if world > 1 else "single GPU",
                       "observables": [{k: (round(v, 8) if isinstance(v, float) else v) for k, v in o.items()}
                                       for o in (obs[0], obs[-1])]},
            "roofline": roof, "kernels": kernels, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches),
            "clocks": clk, "flow_protocol": full,
        }
        print(json.dumps(line), flush=True)


HMC_DIMS = (16, 16, 16, 32)
HMC_BETA = 6.2
HMC_CHAIN = (0.00125, 0.01, 0.1, 2 * M0)  # m_ud -> m_H1 -> m_H2 -> m_PV (Sec. 2 mass preconditioning)
HMC_TAU = 0.1
HMC_NSTEPS = 2
HMC_INNER = 4  # gauge steps per outer drift (Sexton-Weingarten)
HMC_WORKLOAD = "hmc_md_omelyan_16x16x16x32_ns16_2f_hasenbusch3"
FP64_ALU_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12  # SMs x FP64 FMA/clk/SM x 2 flops x max SM clock


def run_hmc(args, world, rank, local):
    """Molecular dynamics of the two-flavour HMC (Sec. 2: Omelyan integrator with Sexton-Weingarten
    time scales, HMC_INNER gauge steps per outer drift; Wilson gauge action at beta = 6.2; the u/d
    factor with two levels of mass preconditioning m_ud = 0.00125 -> m_H1 = 0.01 -> m_H2 = 0.1 ->
    m_PV = 2.6) on 16^3 x 32 x 16, the lattice of the paper's first two-flavour DWF HMC (Sec. 5).  A bench step is one trajectory segment of HMC_NSTEPS Omelyan steps
    (tau = HMC_TAU) from the same (U, P, phi): H at the start with the forces, two force evaluations
    per step, H at the end; every pseudofermion solve mixed precision to 1e-10.  The metric is MD
    steps per second; the sustained rate counts 4 x 1420 flops per 5D site per inner CG iteration
    (the four hops of S^dag S, level-1 work and the FP64 force parts not counted)."""
    import numpy as np
    import torch

    import odwf_synth as syn
    import paper_1811_08095_gb300 as odwf

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    lib = odwf.load()
    stream = torch.cuda.current_stream()
    dims, ns = HMC_DIMS, NS
    V = math.prod(dims)
    w, _ = odwf.odwf_zolotarev_omega(ns, LRANGE[0], LRANGE[1])
    h = odwf.Handle(dims, ns, M0, HMC_CHAIN[0], w)
    U0 = syn.gauge_field_torch(dims, EPS, 21 + rank, device=dev)
    P0 = torch.from_numpy(syn.gaussian_momenta(dims, 22 + rank)).to(dev)
    terms = [(torch.from_numpy(syn.gaussian_spinor_even(ns, dims, 23 + k + 10 * rank)).to(dev), HMC_CHAIN[k],
              HMC_CHAIN[k + 1]) for k in range(3)]
    U = torch.empty_like(U0)
    P = torch.empty_like(P0)

    def traj():
        U.copy_(U0)
        P.copy_(P0)
        return h.md_trajectory(U, P, terms, HMC_BETA, HMC_TAU, HMC_NSTEPS, "omelyan", n_inner=HMC_INNER, tol=TOL,
                               prec=args.prec, stream=stream)

    for _ in range(args.warmup):
        traj()
    torch.cuda.synchronize()
    launches0 = lib.odwf_launch_count()
    clocks = ClockSampler(local)
    clocks.start()
    ms, iters, dH, res = [], [], [], []
    for _ in range(args.steps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        H0, H1, st = traj()
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
        iters.append(st["iters"])
        dH.append(H1 - H0)
        res.append(st["true_resid"])
    torch.cuda.synchronize()
    clk = clocks.stop()
    launches = lib.odwf_launch_count() - launches0
    t_local = sum(ms) / 1e3
    dist = None
    if world > 1:
        import torch.distributed as dist
    value, t_max, n_all = aggregate(t_local, HMC_NSTEPS * args.steps, dist, dev)

    # per-launch events over one more trajectory: the kernels' shares and the roofline
    lib.odwf_profile_enable(1)
    traj()
    torch.cuda.synchronize()
    prof = read_profile(lib)
    lib.odwf_profile_enable(0)
    peak, peak_kind = measured_peaks()
    kernels = {}
    prof_total = sum(e["total_ms"] for e in prof) or 1.0
    for e in prof:
        tot = e["system_launches"] * e["bytes_per_system"] + e["launches"] * e["bytes_per_launch"]
        kernels[e["name"]] = {"launches": e["launches"], "ms": round(e["total_ms"], 3),
                              "share_of_profiled": round(e["total_ms"] / prof_total, 4),
                              "gbs": round(tot / (e["total_ms"] / 1e3) / 1e9, 1) if e["total_ms"] > 0 else 0.0}
    dom = max(prof, key=lambda e: e["total_ms"])
    per_launch = (dom["system_launches"] * dom["bytes_per_system"] + dom["launches"] * dom["bytes_per_launch"]) \
        / dom["launches"]
    achieved = per_launch / (dom["total_ms"] / dom["launches"] / 1e3) / 1e9
    roof = {"bound": "hbm", "kernel": dom["name"], "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
            "frac": round(achieved / peak, 4), "traffic": None,
            "share_of_profiled": round(dom["total_ms"] / prof_total, 4),
            "timing": "the library's per-launch CUDA events over one extra trajectory segment",
            "peak_source": peak_kind + " (MEASURED_PEAKS hbm_gbs)"}
    fc = next((e for e in prof if e["name"] == "pf.force_contract"), None)
    force_alu = None
    if fc:
        links = 4 * V
        flops = links * (672.0 * ns + 432.0)
        ach = flops / (fc["total_ms"] / fc["launches"] / 1e3) / 1e12
        force_alu = {"bound": "alu", "kernel": "pf.force_contract", "achieved": round(ach, 4),
                     "peak": round(FP64_ALU_TFLOPS, 3), "unit": "TFLOP/s (FP64)",
                     "frac": round(ach / FP64_ALU_TFLOPS, 4), "flops_per_link": 672 * ns + 432,
                     "peak_source": "152 SMs x 2 FP64 FMA/clk x 2 flops x 2.07 GHz (nominal FP64 1.25 TFLOP/s)"}
    h.close()

    cpu = None
    if rank == 0 and not args.skip_cpu:
        spi, cores = oracle_seconds_per_iteration(U0.cpu().numpy(), w, terms[1][0].cpu().numpy(), HMC_CHAIN[1])
        it = float(np.mean(iters))
        cpu = {"value": round(HMC_NSTEPS / (spi * it), 6), "unit": "MD steps/s", "cores": cores, "kind": "oracle",
               "sample": "one FP64 oracle S^dag S CG iteration on this 16^3x32x16 field (m = 0.01; %.2f s on %d "
                         "threads), times the %d inner iterations of one GPU trajectory segment (the oracle's "
                         "force contractions, operator pieces and gauge force not counted)" % (spi, cores, it)}

    ms_avg = sum(ms) / len(ms)
    flops = float(np.mean(iters)) * (V // 2) * ns * 4 * 1420
    if rank == 0:
        line = {
            "metric": "two-flavour HMC molecular-dynamics steps/s (Omelyan + Sexton-Weingarten, Wilson gauge + 3 "
                      "mass-preconditioned pseudofermion ratios) on 16^3x32x16",
            "value": round(value, 4), "unit": "MD steps/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms_avg, 2), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "%s solves (%s reliable updates), FP64 forces and MD updates" % (
                args.prec, update_arith_name(args.updates)), "data": "synthetic",
            "config": {"workload": HMC_WORKLOAD, "lattice": "16^3x32", "Ns": ns, "m0": M0, "beta": HMC_BETA,
                       "mass_chain": list(HMC_CHAIN), "tau": HMC_TAU, "md_steps_per_bench_step": HMC_NSTEPS,
                       "integrator": "Omelyan, Sexton-Weingarten with %d gauge steps per outer drift" % HMC_INNER,
                       "solves_per_bench_step": 3 * (2 + 2 * HMC_NSTEPS), "tol": TOL,
                       "gauge": "U = exp(%g i H), H Gaussian traceless Hermitian (seed %d)" % (EPS, 21 + rank),
                       "phi": "Gaussian even-site fields (seeds 23-25)", "P": "Gaussian momenta (seed 22)",
                       "l2": "not flushed: every solve streams the 5D fields (%.0f MB each in FP16) many times "
                             "over" % (V // 2 * ns * 52 / 1e6),
                       "parallelism": "replicas only" if world > 1 else "single GPU"},
            "cg_iters_per_step": iters, "dH": dH, "worst_true_resid": max(res),
            "sustained_gflops": round(flops / (ms_avg / 1e3) / 1e9, 1),
            "context": "the paper's first two-flavour DWF HMC on this lattice sustained ~150 GFLOP/s on one "
                       "GTX-280 (Sec. 5; another machine and flop convention)",
            "roofline": roof, "force_roofline": force_alu, "kernels": kernels, "cpu_baseline": cpu,
            "gpu_launches": int(launches), "clocks": clk,
        }
        print(json.dumps(line), flush=True)


SERVE_LATTICES = [(8, 8, 8, 8), (16, 16, 16, 16), (24, 24, 24, 48), (32, 32, 32, 32)]


def run_serve(args, world, rank, local):
    """Serving stream: Poisson arrivals of D^dag D solve requests over four resident fields
    (8^4, 16^4, 24^3x48, 32^4; links exp(0.25 i H), seeds 11-14), Ns in {8, 16}, m_q uniform
    in [0.002, 0.5], 1-12 right-hand sides each, mixed precision to 1e-10.  Reports p50 / p99
    latency of the completed requests, throughput, and how many were still pending at the end.
    The load generator reuses pools of right-hand sides and output buffers (results of this
    timing run are not kept; served results are checked by tests/test_gpu_serving.py)."""
    import numpy as np
    import torch

    import odwf_synth as syn
    import paper_1811_08095_gb300 as odwf

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    rng = np.random.default_rng(21)
    vols = [d[0] * d[1] * d[2] * d[3] for d in SERVE_LATTICES]
    omegas = {ns: odwf.odwf_zolotarev_omega(ns, LRANGE[0], LRANGE[1])[0] for ns in (8, 16)}
    # the client's buffers first, so that the server's budget (90% of the free memory at
    # serve_create) counts only what is left for it
    pool = {}
    g = torch.Generator(device=dev)
    g.manual_seed(1234)
    for k in range(len(SERVE_LATTICES)):
        for ns in (8, 16):
            shape = (ns, vols[k] // 2, 4, 3)
            bs = [torch.randn(shape, dtype=torch.complex128, device=dev, generator=g) for _ in range(12)]
            xs = [torch.zeros(shape, dtype=torch.complex128, device=dev) for _ in range(12)]
            pool[(k, ns)] = (bs, xs)
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    srv = odwf.Server(0)
    srv.set_policy(admit_deadline_ms=args.admit_deadline_ms, fair=args.fair)
    for k, dims in enumerate(SERVE_LATTICES):
        U = syn.gauge_field_torch(dims, EPS, 11 + k, device=dev)
        srv.register_gauge(k, dims, U)
        del U
        torch.cuda.empty_cache()
    torch.cuda.synchronize()
    rate, duration, drain = args.rate, args.duration, args.drain
    t0 = time.perf_counter()
    next_t = t0 + rng.exponential(1.0 / rate)
    pending, done, submitted, solves_done = {}, [], 0, 0
    while True:
        now = time.perf_counter()
        if now - t0 < duration and now >= next_t:
            k = int(rng.integers(0, len(SERVE_LATTICES)))
            ns = int(rng.choice([8, 16]))
            mq = float(rng.uniform(0.002, 0.5))
            nrhs = int(rng.integers(1, 13))
            bs, xs = pool[(k, ns)]
            t = srv.submit(k, ns, M0, mq, omegas[ns], bs[:nrhs], xs[:nrhs], tol=TOL, prec=args.prec)
            pending[t] = (nrhs, k, ns)
            submitted += 1
            next_t += rng.exponential(1.0 / rate)
            continue
        for t in list(pending):
            rc, res = srv.poll(t, 0)
            if rc != odwf._lib.ODWF_PENDING:
                nrhs, k, ns = pending.pop(t)
                done.append((res["latency_ms"], res["queue_ms"], rc, nrhs, k, ns, res["true_resid"]))
                if rc == 0:
                    solves_done += nrhs
        if now - t0 >= duration and (not pending or now - t0 >= duration + drain):
            break
        time.sleep(0.0005)
    wall = time.perf_counter() - t0
    # every request that has ended: solved (status 0), shed at admission (ODWF_ETIMEOUT: waited
    # past the deadline) or failed otherwise; latency = submit -> end
    ok = [d for d in done if d[2] == 0]
    shed = [d for d in done if d[2] == odwf._lib.ODWF_ETIMEOUT]
    bad = [d for d in done if d[2] not in (0, odwf._lib.ODWF_ETIMEOUT)]
    codes = {}
    for d in bad:
        codes[str(d[2])] = codes.get(str(d[2]), 0) + 1

    def pct(v, q):
        return round(float(np.percentile(v, q)), 1) if len(v) else None

    per_lat = {}
    for d in done:
        key = "x".join(str(v) for v in SERVE_LATTICES[d[4]]) + "/Ns%d" % d[5]
        e = per_lat.setdefault(key, {"ended": 0, "solved": 0, "shed": 0, "solves": 0, "_ok": [], "_all": []})
        e["ended"] += 1
        e["_all"].append(d[0])
        if d[2] == 0:
            e["solved"] += 1
            e["solves"] += d[3]
            e["_ok"].append(d[0])
        elif d[2] == odwf._lib.ODWF_ETIMEOUT:
            e["shed"] += 1
    for e in per_lat.values():
        e["p50_solved_ms"], e["p99_solved_ms"] = pct(e["_ok"], 50), pct(e["_ok"], 99)
        e["p50_all_ms"], e["p99_all_ms"] = pct(e["_all"], 50), pct(e["_all"], 99)
        del e["_ok"], e["_all"]
    lat_ok = [d[0] for d in ok]
    lat_all = [d[0] for d in done]
    line = {"metric": "served ODWF D\u2020D solve latency (p50/p99) and throughput", "workload": "serve_poisson",
            "rate_req_s": rate, "duration_s": duration, "admit_deadline_ms": args.admit_deadline_ms,
            "scheduling": "fair (equal stream priorities)" if args.fair else "smaller lattices first (stream priority)",
            "submitted": submitted, "ended": len(done), "solved": len(ok), "shed_at_admission": len(shed),
            "pending_at_end": len(pending), "failed": len(bad), "failed_codes": codes, "per_class": per_lat,
            "wall_s": round(wall, 2),
            "p50_solved_ms": pct(lat_ok, 50), "p99_solved_ms": pct(lat_ok, 99),
            "p50_all_ms": pct(lat_all, 50), "p99_all_ms": pct(lat_all, 99),
            "throughput_req_s": round(len(ok) / wall, 3), "throughput_solves_s": round(solves_done / wall, 3),
            "max_true_resid": max([d[6] for d in ok], default=None),
            "config": {"lattices": SERVE_LATTICES, "Ns": [8, 16], "mq": [0.002, 0.5], "nrhs": [1, 12],
                       "prec": args.prec, "tol": TOL, "arrivals": "Poisson, seed 21",
                       "shedding": "requests waiting longer than admit_deadline_ms for admission end with "
                                   "ODWF_ETIMEOUT (their latency is submit -> shed)"}}
    print(json.dumps(line), flush=True)
    srv.close()


C3_DIMS = (24, 24, 24, 48)
C5_DIMS = (64, 64, 64, 64)


def _solve_stats_line(stats):
    return {"iters": [s["iters"] for s in stats], "reliable_updates": [s["n_reliable"] for s in stats],
            "max_true_resid": max(s["true_resid"] for s in stats)}


def run_batched_c3(args, world, rank, local):
    """24^3 x 48 x Ns=16: 12 point sources (every spin-colour component at one seeded even
    site, wall placement) x 3 masses = 36 systems in one batched mixed-precision call; links
    exp(0.25 i H) seed 3.  The right-hand sides are shared by the three masses of a source.
    Prints solves/s of the batched call, the per-system iteration counts, and the FP64 GPU CG
    on one source's three systems for comparison."""
    import torch

    import odwf_synth as syn
    import paper_1811_08095_gb300 as odwf

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    dims = C3_DIMS
    vh = dims[0] * dims[1] * dims[2] * dims[3] // 2
    w, _ = odwf.odwf_zolotarev_omega(NS, LRANGE[0], LRANGE[1])
    U = syn.gauge_field_torch(dims, EPS, 3, device=dev)
    h = odwf.Handle(dims, NS, M0, MASSES[0], w)
    h.set_gauge(U)
    del U
    site, idx = syn.random_even_site(dims, 7)
    srcs = []
    for sc in range(12):
        spin, col = divmod(sc, 3)
        b = torch.zeros((NS, vh, 4, 3), dtype=torch.complex128, device=dev)
        b[NS - 1 if spin < 2 else 0, idx, spin, col] = 1.0
        srcs.append(b)
    bs = [srcs[k] for k in range(12) for _ in MASSES]
    mqs = [m for _ in range(12) for m in MASSES]
    xs = [torch.zeros_like(srcs[0]) for _ in bs]
    torch.cuda.synchronize()

    def step(prec, xs_, bs_, mqs_):
        return h.cg_solve_batched(xs_, bs_, mqs_, tol=TOL, max_iter=200000, prec=prec, delta=args.delta,
                                  link_recon=args.link_recon, stream=stream, updates=args.updates)

    for _ in range(args.warmup):
        step(args.prec, xs, bs, mqs)
    torch.cuda.synchronize()
    launches0 = odwf.load().odwf_launch_count()
    clocks = ClockSampler(local)
    clocks.start()
    times, stats = [], None
    for _ in range(args.steps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        stats = step(args.prec, xs, bs, mqs)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1) / 1e3)
    clk = clocks.stop()
    launches = odwf.load().odwf_launch_count() - launches0
    for s in stats:
        assert s["status"] == 0 and s["true_resid"] <= TOL, s
    mem = torch.cuda.max_memory_allocated(dev)
    free, total = torch.cuda.mem_get_info(dev)
    fp64 = None
    if not args.skip_fp64:
        x3 = xs[:3]
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st64 = step("f64", x3, bs[:3], mqs[:3])
        e1.record(stream)
        e1.synchronize()
        t64 = e0.elapsed_time(e1) / 1e3
        fp64 = {"value": round(3 / t64, 4), "unit": "solves/s", "systems": "source 0 x 3 masses",
                **_solve_stats_line(st64)}
    value = len(bs) / (sum(times) / len(times))
    line = {"metric": METRIC, "workload": "odwf_dagd_24x24x24x48_ns16_12src_3mass_batched", "value": round(value, 4),
            "unit": "solves/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "s_per_step": round(sum(times) / len(times), 3), "systems": len(bs), "dtype": "f32",
            "data": "synthetic", **_solve_stats_line(stats), "fp64_cg_subset": fp64,
            "gpu_launches": int(launches), "clocks": clk,
            "device_memory": {"torch_allocated_peak_gb": round(mem / 1e9, 2),
                              "used_gb_at_end": round((total - free) / 1e9, 2), "total_gb": round(total / 1e9, 2)},
            "config": {"lattice": "24^3x48", "Ns": NS, "m0": M0, "masses": list(MASSES),
                       "sources": "12 spin-colour point sources at even site %s, wall placement" % (site,),
                       "gauge": "U = exp(0.25 i H) (seed 3)", "prec": args.prec, "link_recon": args.link_recon,
                       "delta": args.delta, "updates": update_arith_name(args.updates), "tol": TOL,
                       "omega": "shifted (R5) Zolotarev on [0.05, 6.2]"}}
    print(json.dumps(line), flush=True)
    h.close()


def run_paper_scale_c5(args, world, rank, local):
    """64^4 x Ns=16, m_q = 0.002, links exp(0.2 i H) seed 5 stored as FP32 12-real, BF16 inner
    solve with float-float reliable updates, one Gaussian right-hand side (seed 5), one solve per
    step.  Reports the solve time, iterations, true residual and the device memory used."""
    import torch

    import odwf_synth as syn
    import paper_1811_08095_gb300 as odwf

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    dims = C5_DIMS
    vh = dims[0] * dims[1] * dims[2] * dims[3] // 2
    mq = 0.002
    w, _ = odwf.odwf_zolotarev_omega(NS, LRANGE[0], LRANGE[1])
    U = syn.gauge_field_torch(dims, 0.2, 5, device=dev)
    h = odwf.Handle(dims, NS, M0, mq, w)
    h.set_gauge(U)
    del U
    torch.cuda.empty_cache()
    g = torch.Generator(device=dev)
    g.manual_seed(5)
    b = torch.randn((NS, vh, 4, 3), dtype=torch.complex128, device=dev, generator=g)
    x = torch.zeros_like(b)
    torch.cuda.synchronize()
    prec = "bf16" if args.prec == "f16" else args.prec
    times, st = [], None
    for i in range(args.warmup + args.steps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        clocks = ClockSampler(local)
        if i >= args.warmup:
            clocks.start()
        e0.record(stream)
        st = h.cg_solve(x, b, tol=TOL, max_iter=200000, prec=prec, delta=args.delta, link_recon=12, stream=stream,
                        updates=args.updates)
        e1.record(stream)
        e1.synchronize()
        if i >= args.warmup:
            times.append(e0.elapsed_time(e1) / 1e3)
            clk = clocks.stop()
    assert st["status"] == 0 and st["true_resid"] <= TOL, st
    free, total = torch.cuda.mem_get_info(dev)
    line = {"metric": METRIC, "workload": "odwf_dagd_64x64x64x64_ns16_single", "value": round(1 / (sum(times) /
            len(times)), 5), "unit": "solves/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "s_per_solve": round(sum(times) / len(times), 2), "iters": st["iters"], "reliable_updates":
            st["n_reliable"], "true_resid": st["true_resid"], "dtype": "f32", "data": "synthetic", "clocks": clk,
            "device_memory": {"used_gb": round((total - free) / 1e9, 2), "total_gb": round(total / 1e9, 2)},
            "config": {"lattice": "64^4", "Ns": NS, "m0": M0, "mq": mq, "gauge": "U = exp(0.2 i H) (seed 5)",
                       "links": "FP32, 12 reals", "prec": prec, "delta": args.delta,
                       "updates": update_arith_name(args.updates), "tol": TOL,
                       "rhs": "unit Gaussian (torch seed 5)"}}
    print(json.dumps(line), flush=True)
    h.close()


def run_profile_case(args, world, rank, local):
    """A short, fixed solver run for kernel profiling (e.g. under ncu): the batched mixed-precision
    CG stops at --iters iterations, so the launch sequence is fixed and the run is short.  Lattice
    --dims, --ns, --nsys systems (masses 0.002, 0.04, 0.5, ...), links exp(0.25 i H) seed 2."""
    import torch

    import odwf_synth as syn
    import paper_1811_08095_gb300 as odwf

    torch.cuda.set_device(local)
    dims = tuple(args.dims)
    w, _ = odwf.odwf_zolotarev_omega(args.ns, LRANGE[0], LRANGE[1])
    U = syn.gauge_field(dims, EPS, GAUGE_SEED)
    h = odwf.Handle(dims, args.ns, M0, 0.04, w)
    h.set_gauge(torch.from_numpy(U).cuda())
    masses = [0.002, 0.04, 0.5, 0.1, 0.01, 0.2][: args.nsys] + [0.05] * max(0, args.nsys - 6)
    bs = [torch.from_numpy(syn.gaussian_spinor_even(args.ns, dims, RHS_SEED + k)).cuda() for k in range(args.nsys)]
    xs = [torch.zeros_like(b) for b in bs]
    st = h.cg_solve_batched(xs, bs, masses, tol=TOL, max_iter=args.iters, prec=args.prec, link_recon=args.link_recon,
                            check_every=args.iters, raise_on_error=False)
    torch.cuda.synchronize()
    print("profile case: iters %s" % [s["iters"] for s in st])
    h.close()


def run_residual_mass(args, world, rank, local):
    """Residual mass and pseudoscalar correlator of the effective 4D operator (Sec. 3, Table 1's
    quantity) on a synthetic field: 16^4 x 16 (links exp(0.25 i H), seed 13), point source at
    the origin, twelve effective solves per mass (FULL_DIRAC through the mixed-precision Schur
    CG, tolerance 1e-10).  Reports m_res per mass, the solve time and iteration counts, the
    dominant kernel's roofline from the library's per-launch events, and the oracle's time for the
    same inner iterations (one oracle S^dag S CG iteration on this field, timed on the host cores,
    times the GPU's iteration count)."""
    import torch

    import odwf_synth as syn
    import oracle
    import paper_1811_08095_gb300 as odwf

    torch.cuda.set_device(local)
    lib = odwf.load()
    dims = tuple(args.dims) if args.dims != list(DIMS) else (16, 16, 16, 16)
    w, _ = odwf.odwf_zolotarev_omega(args.ns, LRANGE[0], LRANGE[1])
    h = odwf.Handle(dims, args.ns, M0, 0.04, w)
    Ud = syn.gauge_field_torch(dims, EPS, 13, device="cuda")
    h.set_gauge(Ud)
    out = []
    lib.odwf_profile_enable(1)
    gpu_s = 0.0
    iters_total = 0
    for mq in (0.04, 0.5):
        t = time.perf_counter()
        mres, corr, st = h.residual_mass((0, 0, 0, 0), tol=TOL, prec=args.prec, mq=mq)
        dt = time.perf_counter() - t
        gpu_s += dt
        iters_total += st["iters"]
        out.append({"mq": mq, "m_res": mres, "m_res_over_mq": mres / mq, "seconds": round(dt, 2),
                    "inner_iters_12_solves": st["iters"], "worst_true_resid": st["true_resid"],
                    "corr_t0_t1_tmid": [corr[0], corr[1], corr[len(corr) // 2]]})
    torch.cuda.synchronize()
    prof = read_profile(lib)
    lib.odwf_profile_enable(0)
    h.close()
    peak, peak_kind = measured_peaks()
    roof = None
    if prof:
        dom = max(prof, key=lambda e: e["total_ms"])
        per_launch = (dom["system_launches"] * dom["bytes_per_system"] + dom["launches"] * dom["bytes_per_launch"]) \
            / dom["launches"]
        achieved = per_launch / (dom["total_ms"] / dom["launches"] / 1e3) / 1e9
        roof = {"bound": "hbm", "kernel": dom["name"], "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "share_of_gpu_time": round(dom["total_ms"] / sum(
                    e["total_ms"] for e in prof), 4), "peak_source": peak_kind + " (MEASURED_PEAKS hbm_gbs)",
                "timing": "the library's per-launch CUDA events during the 24 solves"}
    cpu = None
    if rank == 0 and not args.skip_cpu:
        U = Ud.cpu().numpy()
        b = syn.gaussian_spinor_even(args.ns, dims, 5)
        t = time.perf_counter()
        oracle.cg(U, b, M0, 0.04, w, tol=1e-30, max_iter=1)
        spi = (time.perf_counter() - t) / 3.0  # initial residual, one iteration, final residual
        cpu = {"seconds_for_the_same_inner_iterations": round(spi * iters_total, 1), "cores": oracle.num_threads(),
               "kind": "oracle", "gpu_seconds": round(gpu_s, 2), "ratio": round(spi * iters_total / gpu_s, 1),
               "sample": "one FP64 oracle S^dag S CG iteration on this 16^4 x 16 field (%.2f s on %d threads), "
                         "times the %d inner iterations of the GPU's 24 solves (the FP64 reconstruction and "
                         "refinement steps not counted)" % (spi, oracle.num_threads(), iters_total)}
    del Ud
    print(json.dumps({"workload": "residual_mass_%s_ns%d" % ("x".join(map(str, dims)), args.ns),
                      "metric": "residual mass of the effective operator (point source, 12 solves per mass)",
                      "prec": args.prec, "omega": "shifted (R5) Zolotarev on [0.05, 6.2]", "results": out,
                      "roofline": roof, "cpu_baseline": cpu,
                      "reading": "m_res = tr G_00 / sum_x tr(G_x0^dag G_x0) - m_q, G = (D_eff^-1 - 1)/(2 m0 - m_q)"}),
          flush=True)


def run_reference(args, world, rank, local):
    """The oracle (FP64 CPU program) on host cores: each step is one oracle CG iteration on the
    workload, scaled to solves/s by the oracle's own iteration counts (tests/golden)."""
    if rank != 0:
        return
    U, w, bs = workload_inputs(lib_omega=False)
    counts = oracle_iteration_counts()
    if counts is None:
        print(json.dumps({"impl": "reference", "unavailable": "oracle iteration counts for this workload not "
                                                              "recorded (tests/golden/make_oracle_counts.py)"}))
        return
    iters, capped = counts
    times = []
    cores = 1
    for i in range(args.warmup + args.steps):
        spi, cores = oracle_seconds_per_iteration(U, w, bs[1], MASSES[1])
        if i >= args.warmup:
            times.append(spi)
    spi = sum(times) / len(times)
    value = len(MASSES) / (spi * sum(iters))
    sample = ("per step one FP64 oracle CG iteration on the 16^3x32x16 workload (m_q=0.04), scaled by the "
              "oracle's CG iteration counts %s%s" % (iters, " (lower bounds: capped runs)" if capped else ""))
    line = {"metric": METRIC, "value": round(value, 8), "unit": "solves/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(spi * 1e3, 1), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD, "lattice": "16^3x32", "Ns": NS, "masses": list(MASSES), "tol": TOL},
            "cpu_baseline": {"value": round(value, 8), "unit": "solves/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": round(value, 8), "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="f16", choices=["f16", "bf16", "f32"])
    ap.add_argument("--delta", type=float, default=0.01, help="reliable-update threshold")
    ap.add_argument("--link-recon", type=int, default=12, choices=[12, 18])
    ap.add_argument("--updates", default="auto", choices=["auto", "f64", "ff"],
                    help="arithmetic of the reliable updates (auto: the library's choice)")
    ap.add_argument("--check-every", type=int, default=8, help="iterations between host polls of the solver state")
    ap.add_argument("--workload", default="c2", choices=["c2", "c3", "c5", "serve", "profile", "mres", "dslash", "flow", "hmc"],
                    help="c2: the default line; c3: 36-system batch on 24^3x48; c5: one 64^4 solve; serve; "
                         "profile: a fixed short solver run for ncu; flow: gradient flow on 64^4; hmc: two-flavour "
                         "HMC molecular dynamics on 16^3x32x16")
    ap.add_argument("--dims", type=int, nargs=4, default=list(DIMS), help="profile: lattice")
    ap.add_argument("--ns", type=int, default=NS, help="profile: Ns")
    ap.add_argument("--nsys", type=int, default=3, help="profile: systems")
    ap.add_argument("--flow-dims", type=int, nargs=4, default=list(FLOW_DIMS), help="flow: lattice")
    ap.add_argument("--flow-to", type=float, default=0.0,
                    help="flow: also integrate a fresh field from t = 0 to this flow time (the paper: 64), "
                         "measuring every 10 steps, and report t0, the admissibility time and Q")
    ap.add_argument("--flow-to-eps", type=float, default=1.0,
                    help="flow --flow-to: strength of the random field it flows (1.0: disordered enough that "
                         "t^2 E reaches 0.3 and the field carries topology)")
    ap.add_argument("--iters", type=int, default=4, help="profile: CG iterations")
    ap.add_argument("--rate", type=float, default=50.0, help="serve: arrivals per second")
    ap.add_argument("--duration", type=float, default=60.0, help="serve: seconds of arrivals")
    ap.add_argument("--drain", type=float, default=60.0, help="serve: extra seconds to finish pending requests")
    ap.add_argument("--admit-deadline-ms", type=float, default=10000.0,
                    help="serve: requests not admitted within this time are shed (ODWF_ETIMEOUT); 0 = never")
    ap.add_argument("--fair", action="store_true", help="serve: every batch at the same stream priority")
    ap.add_argument("--skip-fp64", action="store_true")
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--skip-dslash", action="store_true")
    args = ap.parse_args()
    world, rank, local = dist_env()
    if args.impl == "reference":
        run_reference(args, world, rank, local)
    elif args.workload == "serve":
        run_serve(args, world, rank, local)
    elif args.workload == "c3":
        run_batched_c3(args, world, rank, local)
    elif args.workload == "c5":
        run_paper_scale_c5(args, world, rank, local)
    elif args.workload == "profile":
        run_profile_case(args, world, rank, local)
    elif args.workload == "mres":
        run_residual_mass(args, world, rank, local)
    elif args.workload == "flow":
        run_flow(args, world, rank, local)
    elif args.workload == "hmc":
        run_hmc(args, world, rank, local)
    elif args.workload == "dslash":
        import torch

        torch.cuda.set_device(local)
        print(json.dumps({"workload": "dslash_32x32x32x32_ns16",
                          "dslash": dslash_roofline(args, torch.device("cuda", local))}), flush=True)
    else:
        run_ours(args, world, rank, local)


if __name__ == "__main__":
    main()
