"""Benchmark of the Dirac quantum-walk hot path on GB300.

Default workload: the BCC box N = 512 (33,554,432 sites, 1.07 GB complex64 field,
larger than L2), m = 0.1, a Gaussian packet of width 32 sites.  One bench step =
S = 100 stencil steps of the walk (qw_step, complex64) followed by the
observables (qw_observables: norm and <x> in position space, particle weights
through a forward DFT; FP64 accumulation).  `value` = site-steps/s over the
timed steps; the roofline object reports the stencil kernel's achieved HBM
bandwidth (algorithmic bytes: one read + one write of the field per launch)
against the measured copy bandwidth.  The spectral form (qw_evolve_spectral)
and the FP64 plain form are timed on the same box and reported in "extra".

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

--impl reference times the FP64 CPU oracle (the slow plain program) on a
bounded sample of the same workload, on the host cores.
Multi-GPU (torchrun): replicas only -- every rank runs the same workload on its
own GPU with no collective on the data path; value = all ranks' site-steps over
the slowest rank's time.
"""

import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOAD = {"name": "bcc_N512_stencil_c64", "dim": 3, "N": 512, "mass": 0.1, "sigma": 32.0,
            "k0": (0.3, 0.2, 0.1), "substeps": 100}
FALLBACK_HBM_GBS = 6800.0
# DRAM bytes (read + write) per launch of a stencil kernel from one ncu capture of it at BCC N=384
# (14,155,776 sites), per site.  Traffic grows in proportion to the sites, so bench.py reports
# sites x this figure; kernels without a capture get null.
NCU_TRAFFIC_BYTES_PER_SITE = {"step3d_c64_tma_kernel": (469785600 + 409331968) / 14155776,
                              "step3d_c64_tma2_kernel": (476398848 + 408239360) / 14155776}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true")
    ap.add_argument("--N", type=int, default=None, help="override the box side (profiling runs)")
    ap.add_argument("--stencil", default=None, help="force a stencil variant (plain, vec, tma)")
    ap.add_argument("--only", default=None, choices=["spectral", "batched", "served", "projection", "lattices"],
                    help="run one secondary workload alone and print its JSON (profiling runs)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="batched / lattices: keep the default tiling or variant instead of autotuning (profiling runs)")
    ap.add_argument("--lattice-scale", type=int, default=1,
                    help="lattices: divide the chain's N by this and the square lattice's N by its square root")
    ap.add_argument("--requests", type=int, default=2000, help="served workload: number of requests")
    ap.add_argument("--walks", type=int, default=256, help="batched workload: number of walks")
    ap.add_argument("--substeps", type=int, default=None, help="override stencil steps per bench step")
    args = ap.parse_args()
    if args.N is not None:
        WORKLOAD["N"] = args.N
        WORKLOAD["name"] = "bcc_N%d_stencil_c64" % args.N
    if args.substeps is not None:
        WORKLOAD["substeps"] = args.substeps
    return args


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(ms, world, device):
    """Slowest rank's time: all-reduce MAX over the process group (no data-path collective)."""
    if world == 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(sites, substeps, steps, world, ms):
    """Whole-job site-steps/s: every rank advances its own replica by steps x substeps updates."""
    return sites * substeps * steps * world / (ms / 1e3)


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join("/tmp", "qw_clocks_%d_%d.csv" % (os.getpid(), gpu_index))

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, r in rows for i, v in enumerate(r) if v.lower() == "active"})
        return {"sm_mhz": float(np.median([r[0] for r in rows])), "sm_max_mhz": rows[0][1],
                "reasons": reasons, "samples": len(rows)}


def oracle_cpu_baseline(seconds=12.0):
    """FP64 oracle (numpy) stencil on a bounded BCC sample: site-steps/s on the host."""
    from oracle import walk
    from paper_1603_06442_gb300 import inputs
    N = 64
    m = WORKLOAD["mass"]
    a = inputs.gaussian_packet(3, N, (N / 2,) * 3, N / 16, WORKLOAD["k0"], [0.5, 0.5, 0.5, 0.5])
    psi = walk.from_device(3, N, a)
    mats = walk.transition_matrices(3, m)
    sites = N ** 3 // 4
    steps = 0
    t0 = time.perf_counter()
    while time.perf_counter() - t0 < seconds:
        psi = walk.step(3, m, psi, 1, mats=mats)
        steps += 1
    dt = time.perf_counter() - t0
    return {"value": sites * steps / dt, "unit": "site-steps/s", "cores": 1, "kind": "oracle", "seconds": dt,
            "sample": "BCC N=64 box (%d sites), %d oracle update steps in FP64 numpy, %.1f s" % (sites, steps, dt)}


def _oracle_worker(seconds):
    return oracle_cpu_baseline(seconds)


def _single_thread_env():
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[k] = "1"


def oracle_cpu_baseline_all_cores(seconds=12.0):
    """The same oracle sample in one process per host core at once (spawned: the parent may
    hold a CUDA context), summed: the oracle's all-core throughput on this host."""
    import multiprocessing as mp
    n = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    ctx = mp.get_context("spawn")
    pool = ctx.Pool(n, initializer=_single_thread_env)
    try:
        res = pool.map_async(_oracle_worker, [seconds] * n).get(timeout=4 * seconds + 120)
    except mp.TimeoutError:
        pool.terminate()
        return {"value": None, "unit": "site-steps/s", "cores": n, "sample": "timed out"}
    finally:
        pool.close()
        pool.join()
    return {"value": float(sum(r["value"] for r in res)), "unit": "site-steps/s", "cores": n,
            "sample": "%d processes, each the single-core sample for %.1f s" % (n, seconds)}


def run_reference(args, rank, world):
    if rank != 0:
        return
    t_steps = []
    base = None
    for i in range(args.warmup + args.steps):
        r = oracle_cpu_baseline(seconds=3.0)
        if i >= args.warmup:
            t_steps.append(r)
        base = r
    vals = [r["value"] for r in t_steps]
    v = float(np.mean(vals))
    line = {"impl": "reference", "metric": "site-steps/s", "value": v, "unit": "site-steps/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * float(np.mean([r["seconds"] for r in t_steps])), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "c128", "data": "synthetic",
            "config": {"workload": WORKLOAD["name"], "note": "oracle timed on a bounded BCC N=64 sample"},
            "cpu_baseline": {"value": v, "unit": "site-steps/s", "cores": 1, "kind": "oracle",
                             "sample": base["sample"]},
            "e2e": {"value": v, "unit": "site-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args, rank, world, local):
    import torch
    from paper_1603_06442_gb300 import binding as qb, inputs

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    W = WORKLOAD
    dim, N, S = W["dim"], W["N"], W["substeps"]
    plan = qb.Plan(dim, N, W["mass"], "c64")
    if args.stencil:
        plan.set_stencil(args.stencil)
    kernel_name = {1: "step3d_kernel<float>", 2: "step3d_c64_vec_kernel", 3: "step3d_c64_tma_kernel",
                   4: "step3d_c64_tma2_kernel"}[plan.stencil]
    fused = 2 if plan.stencil == 4 else 1   # steps per stencil launch
    a = inputs.gaussian_packet(dim, N, (N / 2,) * 3, W["sigma"], W["k0"], [0.5, 0.5j, 0.5, -0.5j])
    host = torch.from_numpy(a.astype(np.complex64)).pin_memory()
    psi = host.to(dev)
    stream = torch.cuda.current_stream(dev)
    sites = plan.sites
    field_bytes = plan.elems * 8

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)

    # warm-up (the first qw_run_host call also allocates the plan's three host-run device fields;
    # three fields pass through all of them)
    for _ in range(args.warmup):
        plan.step(psi, S, stream)
        plan.observables(psi, stream)
    plan.run_host([host, host, host], S, stream=stream)
    barrier()

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    with ClockSampler(local) as clocks:
        barrier()
        t_start = torch.cuda.Event(enable_timing=True)
        t_end = torch.cuda.Event(enable_timing=True)
        t_start.record(stream)
        for i in range(args.steps):
            ev[i][0].record(stream)
            plan.step(psi, S, stream)
            ev[i][1].record(stream)
            obs = plan.observables(psi, stream)
            ev[i][2].record(stream)
        t_end.record(stream)
        barrier()
    total_ms = t_start.elapsed_time(t_end)
    stencil_ms = sum(e[0].elapsed_time(e[1]) for e in ev)
    ms = max_over_ranks(total_ms, world, dev)
    value = job_value(sites, S, args.steps, world, ms)
    # stencil launches (S / fused, S even) + the observables: the z FFT pass (which also takes norm
    # and <x>) and its two-stage fold, the y pass, the x-pass weights kernel (the x transform happens
    # inside it) and its two-stage fold
    stencil_launches = (S + fused - 1) // fused
    launches_per_step = stencil_launches + 3 + 1 + 3

    # end-to-end through the C ABI with host buffers: qw_run_host copies every step's field
    # from pinned host memory, runs S steps and reads the observables back to the host; the
    # library copies the next step's field on its own copy stream while this one computes.
    e2e_steps = max(2, args.steps)
    # warm-up of the end-to-end path right before it is timed: a pinned buffer left idle (here
    # through the device-timed steps) copies several times slower on its first transfer
    # (measured 7-65 ms against 5.1 ms for the 1.07 GB field), and a run's first copy has
    # nothing to overlap with
    for _ in range(args.warmup):
        plan.run_host([host, host, host], S, stream=stream)
    barrier()
    t0 = time.perf_counter()
    plan.run_host([host] * e2e_steps, S, stream=stream)
    torch.cuda.synchronize(dev)
    e2e_ms = (time.perf_counter() - t0) * 1e3 / e2e_steps
    # the same run again with per-field CUDA events on both streams (not the timed number):
    # how long each copy took and how long each step waited for its field
    plan.set_host_timing(True)
    plan.run_host([host] * e2e_steps, S, stream=stream)
    tl = plan.host_timing(e2e_steps)
    plan.set_host_timing(False)
    copy_ms = [c1 - c0 for c0, c1, _, _, _ in tl]
    # field j's step could start when field j-1's observables ended; it waited for its copy
    waits = [max(0.0, tl[j][2] - tl[j - 1][4]) for j in range(1, len(tl))]
    overlap = {"copy_ms_median": float(np.median(copy_ms)), "copy_ms_max": float(max(copy_ms)),
               "copy_ms_per_field": [round(c, 3) for c in copy_ms],
               "step_wait_for_copy_ms_mean": float(np.mean(waits)), "step_wait_for_copy_ms_max": float(max(waits)),
               "copy_hidden_frac": float(1.0 - sum(waits) / max(1e-9, sum(copy_ms[1:]))),
               "note": "second, event-instrumented run of the same fields: per field the copy's duration on the "
                       "copy stream and how long its step started after the previous field's observables"}
    # the host-to-device copy alone (pinned field), for the e2e bound
    h0, h1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    h0.record(stream)
    psi.copy_(host, non_blocking=True)
    h1.record(stream)
    torch.cuda.synchronize(dev)
    h2d_GBps = field_bytes / (h0.elapsed_time(h1) / 1e3) / 1e9

    extra = {}
    if not args.no_extra and rank == 0:
        extra = extra_measurements(qb, dev, stream)

    if rank != 0:
        plan.close()
        return
    peak, peak_kind = measured_peaks()
    per_launch_ms = stencil_ms / (args.steps * stencil_launches)
    # algorithmic bytes per launch: 64 B per site-step (one read + one write of 4 complex64, the
    # unfused minimum) x the site-steps one launch advances; a fused launch moves one read + one
    # write of the field for `fused` steps, so its own HBM rate is reported beside it
    alg_bytes = 2 * field_bytes * fused
    achieved = alg_bytes / (per_launch_ms / 1e3) / 1e9
    fused_hbm = 2 * field_bytes / (per_launch_ms / 1e3) / 1e9
    line = {
        "metric": "site-steps/s", "value": value, "unit": "site-steps/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c64",
        "data": "synthetic",
        "config": {"workload": W["name"], "dim": dim, "N": N, "sites": sites, "mass": W["mass"],
                   "stencil_steps_per_step": S, "parallelism": "replicas" if world > 1 else "single",
                   "l2": "no flush: the %.2f GB field is larger than L2 (129 MB)" % (field_bytes / 1e9),
                   "input": "Gaussian packet sigma=%g sites, k0=%s" % (W["sigma"], list(W["k0"]))},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak,
                     "traffic": (NCU_TRAFFIC_BYTES_PER_SITE[kernel_name] * sites
                                 if kernel_name in NCU_TRAFFIC_BYTES_PER_SITE else None),
                     "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum of this kernel at "
                                       "BCC N=384, scaled by sites (profiles/%s_bcc_N384.txt)" % kernel_name,
                     "kernel": kernel_name, "peak_kind": peak_kind,
                     "algorithmic_bytes_per_launch": alg_bytes,
                     "steps_per_launch": fused,
                     "kernel_hbm_GBps": fused_hbm,
                     "kernel_hbm_frac": fused_hbm / peak,
                     "avg_launch_ms": per_launch_ms,
                     "site_steps_per_s_at_roofline": peak * 1e9 / (2 * field_bytes) * sites},
        "e2e": {"value": sites * S / (e2e_ms / 1e3), "unit": "site-steps/s",
                "h2d_bytes_per_step": field_bytes, "d2h_bytes_per_step": 48, "ms_per_step": e2e_ms,
                "h2d_GBps": h2d_GBps, "api": "qw_run_host", "overlap": overlap,
                "note": "pinned host field copied every step inside qw_run_host; the library copies the next "
                        "fields' copies on its copy stream while this one computes (three device buffers)"},
        "gpu_launches": args.steps * launches_per_step,
        "clocks": clocks.summary(),
        "final_obs": obs,
    }
    if not args.no_cpu_baseline and world == 1:
        # the oracle on every host core (one process per core, the same bounded sample each);
        # the single-core figure rides along
        single = oracle_cpu_baseline()
        allc = oracle_cpu_baseline_all_cores()
        if allc.get("value"):
            line["cpu_baseline"] = {"value": allc["value"], "unit": "site-steps/s", "cores": allc["cores"],
                                    "kind": "oracle", "sample": "BCC N=64 box, FP64 numpy update steps: " + allc["sample"],
                                    "single_core": single}
        else:
            line["cpu_baseline"] = single
    if extra:
        line["extra"] = extra
    plan.close()
    print(json.dumps(line), flush=True)


def extra_measurements(qb, dev, stream):
    """Secondary numbers of the metric: FP64 plain stencil on the same box."""
    import torch
    out = {}
    W = WORKLOAD
    plan = qb.Plan(3, W["N"], W["mass"], "c128")
    psi = torch.zeros(plan.elems, dtype=torch.complex128, device=dev)
    psi[::7] = 1e-3
    plan.step(psi, 2, stream)
    torch.cuda.synchronize(dev)
    s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    n = 6
    s0.record(stream)
    plan.step(psi, n, stream)
    s1.record(stream)
    torch.cuda.synchronize(dev)
    ms = s0.elapsed_time(s1) / n
    out["fp64_stencil"] = {"site_steps_per_s": plan.sites / (ms / 1e3), "ms_per_step": ms,
                           "hbm_GBps": 2 * plan.elems * 16 / (ms / 1e3) / 1e9}
    plan.close()
    # every complex64 stencil variant on the same box (A/B of the data movement)
    plan = qb.Plan(3, W["N"], W["mass"], "c64")
    psi = torch.zeros(plan.elems, dtype=torch.complex64, device=dev)
    psi[::7] = 1e-3
    variants = {}
    for name in ("plain", "vec", "tma", "tma2", "fused"):
        try:
            plan.set_stencil(name)
        except qb.QwError:
            continue
        plan.step(psi, 2, stream)
        torch.cuda.synchronize(dev)
        n = 10
        s0.record(stream)
        plan.step(psi, n, stream)
        s1.record(stream)
        plan.sync(stream)
        ms = s0.elapsed_time(s1) / n
        variants[name] = {"ms_per_step": ms, "site_steps_per_s": plan.sites / (ms / 1e3),
                          "equiv_GBps_at_64B_per_site_step": 2 * plan.elems * 8 / (ms / 1e3) / 1e9}
    out["c64_stencil_variants"] = variants
    plan.close()
    out["fp32_error_vs_fp64"] = fp32_error_measurement(qb, dev, stream)
    out["lattices"] = lattice_stencil_measurement(qb, dev, stream)
    out["spectral"] = spectral_measurement(qb, dev, stream)
    out["projection"] = projection_measurement(qb, dev, stream)
    out["batched"] = batched_measurement(qb, dev, stream)
    out["served"] = served_measurement(qb, dev, stream)
    return out


def fp32_error_measurement(qb, dev, stream):
    """The bench workload's complex64 result against the complex128 path on the same initial
    field (the complex128 path is the one held to 1e-11 of the FP64 oracle): relative L2 and
    norm drift after the bench step's 100 stencil steps, and after a spectral evolution to
    t = 10^4 (the spectral complex64 error does not grow with t)."""
    import torch
    from paper_1603_06442_gb300 import inputs
    W = WORKLOAD
    dim, N = W["dim"], W["N"]
    a = inputs.gaussian_packet(dim, N, (N / 2,) * 3, W["sigma"], W["k0"], [0.5, 0.5j, 0.5, -0.5j])
    out = {}
    for mode, t in (("stencil", W["substeps"]), ("spectral", 10000)):
        res = {}
        for dt in ("c64", "c128"):
            plan = qb.Plan(dim, N, W["mass"], dt)
            x = torch.from_numpy(a.astype(np.complex64 if dt == "c64" else np.complex128)).to(dev)
            if mode == "stencil":
                plan.step(x, t, stream)
            else:
                plan.evolve_spectral(x, t, stream)
            plan.sync(stream)
            res[dt] = x.to(torch.complex128)
            plan.close()
            del x
        diff = torch.linalg.vector_norm(res["c64"] - res["c128"]).item()
        ref = torch.linalg.vector_norm(res["c128"]).item()
        n64 = torch.linalg.vector_norm(res["c64"]).item() ** 2
        n0 = float(np.sum(np.abs(a.astype(np.complex64).astype(np.complex128)) ** 2))
        out[mode] = {"t": t, "rel_l2_c64_vs_c128": diff / ref, "norm_drift_c64": abs(n64 - n0) / n0}
        del res
        torch.cuda.empty_cache()
    return out


def lattice_stencil_measurement(qb, dev, stream, autotune=True, scale=1):
    """complex64 stencil on the square lattice (N = 8192, 4-spinor, 2.1 GB) and the chain
    (N = 2^28, 2-spinor, 2.1 GB), both larger than L2: every variant the plan supports, the
    FUSED one at the depth and tile the autotuner picks; roofline fraction at the unfused
    bytes per site-step (64 B square lattice, 32 B chain) against the measured copy rate."""
    import torch
    peak, kind = measured_peaks()
    out = {}
    for dim, N in ((2, 8192 // int(round(scale ** 0.5))), (1, (1 << 28) // scale)):
        plan = qb.Plan(dim, N, 0.1, "c64")
        psi = torch.zeros(plan.elems, dtype=torch.complex64, device=dev)
        psi[::7] = 1e-3
        bps = 2 * plan.elems * 8 / plan.sites   # unfused algorithmic bytes per site-step
        if autotune:
            rate_tuned = plan.autotune(stream)
        else:   # the default FUSED depth and tile for this lattice
            plan.set_stencil("fused")
            rate_tuned = None
        tuned = {"variant": [k for k, v in qb.STENCILS.items() if v == plan.stencil][0],
                 "fusion": plan.fusion(), "autotune_rate": rate_tuned}
        res = {}
        for name in ("plain", "fused"):
            if name == "fused" and tuned["variant"] != "fused":
                continue
            plan.set_stencil(name)
            plan.step(psi, 4, stream)
            s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            n = 24
            s0.record(stream)
            plan.step(psi, n, stream)
            s1.record(stream)
            plan.sync(stream)
            ms = s0.elapsed_time(s1) / n
            r = plan.sites / (ms / 1e3)
            res[name] = {"ms_per_step": ms, "site_steps_per_s": r, "frac_of_hbm_unfused": r * bps / 1e9 / peak}
        out["%dd_N%d" % (dim, N)] = {"sites": plan.sites, "bytes_per_site_step_unfused": bps, "variants": res,
                                     "autotuned": tuned, "peak_kind": kind}
        plan.close()
        del psi
        torch.cuda.empty_cache()
    return out


def spectral_measurement(qb, dev, stream):
    """Spectral form on the bench box (complex64 at t = 1e4 and 1e6, complex128 at 1e4): flat in t."""
    import torch
    W = WORKLOAD
    s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    spec = {}
    for dt, tag in (("c64", "c64"), ("c128", "c128")):
        plan = qb.Plan(3, W["N"], W["mass"], dt)
        plan.prepare_spectral()
        psi = torch.zeros(plan.elems, dtype=plan.torch_dtype, device=dev)
        psi[::5] = 1e-3
        for t in ((10 ** 4, 10 ** 6) if dt == "c64" else (10 ** 4,)):
            plan.evolve_spectral(psi, t, stream)
            torch.cuda.synchronize(dev)
            reps = 5
            s0.record(stream)
            for _ in range(reps):
                plan.evolve_spectral(psi, t, stream)
            s1.record(stream)
            plan.sync(stream)
            ms = s0.elapsed_time(s1) / reps
            bytes_min = 4 * plan.elems * (8 if dt == "c64" else 16)   # read+write field, forward and inverse
            spec["%s_t%d" % (tag, t)] = {"ms_per_evolution": ms, "t": t,
                                         "equivalent_site_steps_per_s": plan.sites * t / (ms / 1e3),
                                         "effective_GBps_vs_4_field_passes": bytes_min / (ms / 1e3) / 1e9}
        plan.close()
    return spec


def projection_measurement(qb, dev, stream):
    """Probability projections of the bench field (complex64 BCC N=512): one read of the field
    per call, so HBM-bound; GB/s against the measured copy peak."""
    import torch
    W = WORKLOAD
    plan = qb.Plan(3, W["N"], W["mass"], "c64")
    psi = torch.zeros(plan.elems, dtype=torch.complex64, device=dev)
    psi[::5] = 1e-3
    peak, kind = measured_peaks()
    field_bytes = plan.elems * 8
    s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    res = {}
    for name, keep in (("x", {0}), ("xy_plane", {0, 1}), ("yz_plane", {1, 2}), ("density", {0, 1, 2})):
        out = plan.projection(psi, keep, stream)
        torch.cuda.synchronize(dev)
        reps = 10
        s0.record(stream)
        for _ in range(reps):
            plan.projection(psi, keep, stream)
        s1.record(stream)
        torch.cuda.synchronize(dev)
        ms = s0.elapsed_time(s1) / reps
        written = out.numel() * 8
        gbps = (field_bytes + written) / (ms / 1e3) / 1e9
        res[name] = {"ms": ms, "algorithmic_GBps": gbps, "frac_of_hbm": gbps / peak,
                     "bytes": field_bytes + written}
        del out
    # position moments up to second order (one read of the field; blocking call: the events
    # bracket the kernels, the fold and the 80-byte read-back)
    plan.position_moments(psi, stream)
    reps = 10
    s0.record(stream)
    for _ in range(reps):
        plan.position_moments(psi, stream)
    s1.record(stream)
    torch.cuda.synchronize(dev)
    ms = s0.elapsed_time(s1) / reps
    res["position_moments"] = {"ms": ms, "algorithmic_GBps": field_bytes / (ms / 1e3) / 1e9,
                               "frac_of_hbm": field_bytes / (ms / 1e3) / 1e9 / peak, "bytes": field_bytes}
    # Foldy-Wouthuysen field (Newton-Wigner position): copy, forward FFT, per-k eigenvector
    # projection, inverse FFT; algorithmic bytes 4 field passes like the spectral evolution
    f = torch.empty_like(psi)
    plan.fw_transform(psi, out=f, stream=stream)
    s0.record(stream)
    for _ in range(reps):
        plan.fw_transform(psi, out=f, stream=stream)
    s1.record(stream)
    torch.cuda.synchronize(dev)
    ms = s0.elapsed_time(s1) / reps
    res["fw_transform"] = {"ms": ms, "effective_GBps_vs_4_field_passes": 4 * field_bytes / (ms / 1e3) / 1e9}
    del f
    res["note"] = ("algorithmic bytes = one read of the field + the FP64 output; the output "
                   "tensor is allocated by the binding per call; peak %s" % kind)
    plan.close()
    return res


def served_measurement(qb, dev, stream, n_req=2000, rate=200.0, budget_gb=150, slots=8):
    """Poisson arrivals (200/s) of walk requests: dim U{1,2,3}, sites log-U[1e4, 1e8] snapped to
    2^a 3^b boxes, m U[0, 0.5], t log-U[10, 1e5]; packets of width N/16 at the box centre; each asks
    for norm, <x> and particle weight.  Spectral path, complex64 with FP64 phase and reductions."""
    import time as _t
    from paper_1603_06442_gb300 import inputs
    stream_reqs = inputs.sample_served_stream(n_req, rate, seed=0)
    srv = qb.qw_server_create(int(budget_gb) << 30, slots=slots, max_pending=1 << 16)
    chi = {1: [1, 0], 2: [0.5, 0.5, 0.5j, -0.5j], 3: [0.5, 0.5, 0.5j, -0.5j]}
    reqs = []
    for r in stream_reqs:
        d, N = r["dim"], r["N"]
        reqs.append(qb.make_request(d, N, r["mass"], r["t"], x0=[N / 2] * d, sigma=max(N / 16, 1.0),
                                    k0=[0.2] * d, chi=chi[d]))
    # no warm-up of the per-size FFT plans: a box size seen for the first time builds its
    # tables on the device inside its request (reported apart below)
    seen, first = set(), []
    for r in stream_reqs:
        key = (r["dim"], r["N"])
        first.append(key not in seen)
        seen.add(key)
    lat, out, pend = [], [], {}
    lat_of = {}
    t0 = _t.perf_counter()
    i = 0
    while i < len(reqs) or pend:
        now = _t.perf_counter() - t0
        while i < len(reqs) and stream_reqs[i]["arrival"] <= now:
            tk = qb.qw_submit(srv, reqs[i])
            if tk is None:
                break
            pend[tk] = i
            i += 1
        for tk in list(pend):
            done, obs, l = qb.qw_poll(srv, tk)
            if done:
                lat.append(l)
                lat_of[pend[tk]] = l
                out.append(obs)
                del pend[tk]
        _t.sleep(0.0002)
    wall = _t.perf_counter() - t0
    st = qb.qw_server_stats(srv)
    qb.qw_server_destroy(srv)
    site_t = 0.0
    fp64 = fp64_plain_sample(qb, dev, stream, stream_reqs)
    est = []
    for r in stream_reqs:
        d, N = r["dim"], r["N"]
        sites = N if d == 1 else (N * N if d == 2 else N ** 3 // 4)
        site_t += sites * r["t"]
        est.append(fp64["fit"][d]["fixed_s"] + sites * r["t"] / fp64["fit"][d]["site_steps_per_s"])
    lat_first = np.array([lat_of[i] for i in lat_of if first[i]])
    lat_rest = np.array([lat_of[i] for i in lat_of if not first[i]])
    lat = np.array(lat)
    est = np.array(est)
    pct = lambda a, q: float(np.percentile(a, q) * 1e3) if len(a) else None
    return {"requests": len(reqs), "arrival_rate_per_s": rate, "slots": slots, "budget_GB": budget_gb,
            "latency_p50_ms": pct(lat, 50), "latency_p99_ms": pct(lat, 99),
            "latency_mean_ms": float(lat.mean() * 1e3), "wall_s": wall, "completed_per_s": len(lat) / wall,
            "first_seen_sizes": {"requests": int(len(lat_first)), "latency_p50_ms": pct(lat_first, 50),
                                 "latency_p99_ms": pct(lat_first, 99)},
            "repeat_sizes": {"requests": int(len(lat_rest)), "latency_p50_ms": pct(lat_rest, 50),
                             "latency_p99_ms": pct(lat_rest, 99)},
            "equivalent_site_steps_per_s": site_t / wall, "peak_pool_GB": st["peak_bytes"] / 2 ** 30,
            "max_norm_drift": float(max(abs(o["norm"] - 1) for o in out)),
            "fp64_plain_unbatched": {"service_p50_ms": float(np.percentile(est, 50) * 1e3),
                                     "service_p99_ms": float(np.percentile(est, 99) * 1e3),
                                     "measured_sample": fp64["sample"],
                                     "fit": {str(k): v for k, v in fp64["fit"].items()},
                                     "note": "every request of a seeded sample with sites*t <= %.0e run end to end "
                                             "in the FP64 plain form (plan, copy in, t stencil steps, observables); "
                                             "per-dimension cost model fixed_s + sites*t/rate fitted to it and "
                                             "applied to every request of the stream, no queueing"
                                             % fp64["max_site_steps"]}}


def fp64_plain_sample(qb, dev, stream, stream_reqs, per_dim=4, max_site_steps=2e9):
    """The unbatched FP64 plain form, measured: the first `per_dim` requests of each dimension
    with sites*t <= max_site_steps run alone (complex128 plan, host field copied in, t stencil
    steps, observables read back), timed end to end; a per-dimension model fixed + sites*t/rate
    is fitted by least squares to these samples and to one long run per dimension."""
    import time as _t
    import torch
    from paper_1603_06442_gb300 import inputs
    chi = {1: [1, 0], 2: [0.5, 0.5, 0.5j, -0.5j], 3: [0.5, 0.5, 0.5j, -0.5j]}
    sample, fit = [], {}
    for d in (1, 2, 3):
        picked = []
        for r in stream_reqs:
            N = r["N"]
            sites = N if d == 1 else (N * N if d == 2 else N ** 3 // 4)
            if r["dim"] == d and sites * r["t"] <= max_site_steps:
                picked.append((N, r["mass"], r["t"], sites))
            if len(picked) == per_dim:
                break
        # one long run per dimension anchors the rate
        picked.append({1: (1 << 22, 0.1, 400, 1 << 22), 2: (1024, 0.1, 1500, 1 << 20),
                       3: (256, 0.1, 300, 256 ** 3 // 4)}[d])
        xs, ys = [], []
        for N, m, t, sites in picked:
            a = inputs.gaussian_packet(d, N, [N / 2] * d, max(N / 16, 1.0), [0.2] * d, chi[d])
            host = torch.from_numpy(a.astype(np.complex128)).pin_memory()
            torch.cuda.synchronize(dev)
            t0 = _t.perf_counter()
            plan = qb.Plan(d, N, m, "c128")
            x = host.to(dev, non_blocking=True)
            plan.step(x, t, stream)
            plan.observables(x, stream)
            torch.cuda.synchronize(dev)
            el = _t.perf_counter() - t0
            plan.close()
            sample.append({"dim": d, "N": N, "t": t, "site_steps": sites * t, "seconds": el})
            xs.append(sites * t)
            ys.append(el)
        A = np.vstack([np.ones(len(xs)), np.array(xs, dtype=float)]).T
        (c0, c1), *_ = np.linalg.lstsq(A, np.array(ys), rcond=None)
        fit[d] = {"fixed_s": max(float(c0), 0.0), "site_steps_per_s": 1.0 / float(c1) if c1 > 0 else float("inf")}
    return {"sample": sample, "fit": fit, "max_site_steps": max_site_steps}


def _drain(qb, srv, tickets):
    import time as _t
    left = set(t for t in tickets if t is not None)
    while left:
        for t in list(left):
            if qb.qw_poll(srv, t)[0]:
                left.discard(t)
        _t.sleep(0.0005)


def batched_measurement(qb, dev, stream, runs=3, n_walks=256, autotune=True):
    """256 uneven walks (2D N log-U[64,1024], BCC N log-U[32,128], m U[0,0.5], t U{100..5000},
    packets of width N/16) in one persistent launch replayed from a CUDA graph; tiling autotuned."""
    import torch
    from paper_1603_06442_gb300 import inputs
    mix = inputs.sample_batch_mix(n_walks, seed=0)
    fields = []
    for w in mix:
        N = w["N"]
        a = inputs.gaussian_packet(w["dim"], N, [N / 2] * w["dim"], w["sigma"], [0.0] * w["dim"],
                                   [0.5, 0.5, 0.5j, -0.5j])
        fields.append(torch.from_numpy(a.astype(np.complex64)).to(dev))
    b = qb.Batch([(w["dim"], w["N"], w["mass"], w["t"], x) for w, x in zip(mix, fields)])
    if autotune:
        best, tuned_rate = b.autotune(rounds_cap=256, stream=stream)
    else:
        best, tuned_rate = b.tiling()[0], None
    site_steps = 0
    for w in mix:
        sites = w["N"] ** 2 if w["dim"] == 2 else w["N"] ** 3 // 4
        site_steps += sites * w["t"]
    b.run(stream)
    b.sync(stream)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(runs):
        b.run(stream)
    e1.record(stream)
    b.sync(stream)
    ms = e0.elapsed_time(e1) / runs
    obs = b.observables(stream)
    worst_norm = max(abs(o["norm"] - 1.0) for o in obs)
    b.close()
    rate = site_steps / (ms / 1e3)
    peak, _ = measured_peaks()
    return {"walks": len(mix), "site_steps_per_run": site_steps, "ms_per_run": ms,
            "site_steps_per_s": rate, "algorithmic_GBps_at_64B": rate * 64 / 1e9,
            "frac_of_hbm_at_64B": rate * 64 / 1e9 / peak,
            "note": "one persistent launch; a round advances a tile by the autotuned fusion depth of its "
                    "lattice (1: per-site update from HBM; >= 2: tile + halo in shared memory, one HBM read "
                    "and write per round); algorithmic bytes are the unfused 64 B per site-step",
            "autotuned_fusion_depth": {"1d": best["depth"][0], "2d": best["depth"][1], "bcc": best["depth"][2]},
            "autotuned_box": {"2d": best["box"][1][:2], "bcc": best["box"][2]},
            "autotuned_tile_sites": best["tile_sites"], "autotuned_l2_budget_MiB": best["l2_budget_bytes"] / 2 ** 20,
            "autotune_rate_at_256_steps": tuned_rate,
            "max_norm_drift_after_%d_runs" % (runs + 1): worst_norm,
            "launches_per_run": 1, "graph": True}


def run_only(args, local):
    import torch
    from paper_1603_06442_gb300 import binding as qb
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    if args.only == "served":
        out = served_measurement(qb, dev, stream, n_req=args.requests)
    elif args.only == "batched":
        out = batched_measurement(qb, dev, stream, n_walks=args.walks, autotune=not args.no_autotune)
    elif args.only == "lattices":
        out = lattice_stencil_measurement(qb, dev, stream, autotune=not args.no_autotune, scale=args.lattice_scale)
    elif args.only == "projection":
        out = projection_measurement(qb, dev, stream)
    else:
        out = spectral_measurement(qb, dev, stream)
    print(json.dumps({"only": args.only, "config": {"workload": WORKLOAD["name"], "N": WORKLOAD["N"]},
                      "result": out}), flush=True)


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.only:
        if rank == 0:
            run_only(args, local)
        return
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    run_ours(args, rank, world, local)


if __name__ == "__main__":
    main()
