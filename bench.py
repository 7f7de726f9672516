"""Benchmark: Parareal time-to-1e-6 on one GB300, stencil GLUP/s and %HBM.

One step = one full Parareal solve of the 256^3 FP32-stencil / FP64-
correction workload (N = 32 slices, T = 1, dt_F = 1/8192, coarse RK4 on 32^3
at 1/256, k^-2 random initial field): the coarse start-up chain, then
iterations (batched fine sweep of all open slices, serial coarse sweep with
the correction and norms) until the defect d^k against the serial fine
solution is <= 1e-6.

Reported ``value``: fine-stencil point updates executed in the solve per
second (GLUP/s), inputs resident in HBM.  Beside it: the solve time
(time-to-1e-6), the serial fine time on the same GPU, the roofline of the
fused RK4 kernel from CUDA-event timing of its launches inside the timed
region, the end-to-end number through the C ABI with host buffers, and the
FP64 CPU oracle timed on this host.

The default line also carries three comparisons, each with its own clock
record: the 128^3 learned-vs-stencil propagator (c4_learned_128), the 64
uneven instances (c3_batch64) and the 32^3 FP64 plain method, the
latency-bound regime in which the slices batched on one GPU can beat serial
fine stepping (c1_fp64_32).

``--impl reference`` times the CPU oracle instead (the only reference this
method has), on a bounded sample of the same workload.
"""
import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("time-to-1e-6-error Parareal vs serial fine on 1 GB300; stencil GLUP/s, % HBM peak")
UNIT = "GLUP/s"
TOL = 1e-6
# ncu summary and kernel source of the batched fine sweep, per launch path
PROFILE_SUMMARY = {0: (os.path.join(ROOT, "profiles", "rk4_fused_256.md"), "stencil.cu"),
                   2: (os.path.join(ROOT, "profiles", "rk4_fused_rows2_256.md"), "stencil.cu")}
TUNE_CACHE = os.path.join(ROOT, "paper_1409_8563_gb300", "tune_cache.jsonl")


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def stencil_hash(src="stencil.cu"):
    h = hashlib.sha1()
    with open(os.path.join(ROOT, "paper_1409_8563_gb300", "csrc", src), "rb") as f:
        h.update(f.read())
    return h.hexdigest()[:12]


def ncu_traffic(path):
    """DRAM bytes per launch of the fine-sweep kernel of launch path `path`
    from the committed ncu summary, or None when the summary is missing or the
    kernel source changed since."""
    if path not in PROFILE_SUMMARY or not os.path.exists(PROFILE_SUMMARY[path][0]):
        return None
    summary, src = PROFILE_SUMMARY[path]
    text = open(summary).read()
    m = re.search(r"stencil_sha1:\s*([0-9a-f]+)", text)
    t = re.search(r"traffic_bytes_per_launch_full:\s*([0-9.eE+]+)", text)
    if not m or not t or m.group(1) != stencil_hash(src):
        return None
    return float(t.group(1))


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def power_w(self):
        """Mean board power (W) over the samples, or None."""
        pw = []
        for l in getattr(self, "lines", []):
            f = [x.strip() for x in l.split(",")]
            try:
                pw.append(float(f[2]))
            except (ValueError, IndexError):
                continue
        return statistics.mean(pw) if pw else None

    def summary(self):
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            f = [x.strip() for x in l.split(",")]
            if len(f) < 7:
                continue
            try:
                sm.append(float(f[0]))
                mx = max(mx, float(f[1]))
            except ValueError:
                continue
            for nm, v in zip(names, f[3:7]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx or None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_init(n_gpus):
    if n_gpus <= 1 or "RANK" not in os.environ:
        return 0, 1, None
    import torch.distributed as dist
    dist.init_process_group("nccl")
    return dist.get_rank(), dist.get_world_size(), dist


def barrier(dist):
    if dist is not None:
        dist.barrier()


def _reduce_device(dist):
    """NCCL reduces device tensors; gloo (CPU ranks) host tensors."""
    return "cuda" if dist.get_backend() == "nccl" else "cpu"


def max_over_ranks(dist, x):
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=_reduce_device(dist))
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(dist, x):
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=_reduce_device(dist))
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


# FP32 instructions of one RK4 point-step of the fused kernel's arithmetic,
# halo excluded: four 7-term stencil FMA chains, y4 = u + 2 h, and the step's
# base b = u + ((y2 - u) + 2 (y3 - u) + (y4 - u)) / 3 (three subtractions, one
# addition, two FMAs).
FP32_OPS_PER_POINT_STEP = 4 * 7 + 1 + 6
FP32_LANES_PER_SM = 128        # four sub-partitions of 32 FP32 lanes


def alu_roof(point_steps_per_s, clocks):
    """The fused step against the FP32 issue rate: one FP32 instruction per
    lane per clock at the maximum SM clock (an FMA counts once)."""
    import torch
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    mhz = (clocks or {}).get("sm_max_mhz") or 2070.0
    peak = sms * FP32_LANES_PER_SM * mhz * 1e6
    ach = point_steps_per_s * FP32_OPS_PER_POINT_STEP
    return {"achieved": ach / 1e12, "peak": peak / 1e12, "unit": "T FP32 instr/s",
            "frac": ach / peak, "ops_per_point_step": FP32_OPS_PER_POINT_STEP,
            "peak_from": f"{sms} SMs x {FP32_LANES_PER_SM} FP32 lanes x {mhz:.0f} MHz"}


def s_bound(n_p, k, nc_over_nf, tauc_over_tauf):
    """Speedup bound of Eq. (speedup): 1 / ((1 + K/N_p) (N_c/N_f)(tau_c/tau_f) + K/N_p)."""
    return 1.0 / ((1.0 + k / n_p) * nc_over_nf * tauc_over_tauf + k / n_p)


def gamma_terms(n_p, k, n_f, n_c, tau_f_serial, tau_f_batched, tau_c, t_p, t_s):
    """Energy overhead models (Sec. 2.2.3).  gamma_bound = N_p / S_bound with
    the paper's speedup bound (one node per slice), from the step costs
    measured here.  On one GPU all slices share the device, so the same cost
    model is also evaluated for one device at constant power: the start-up
    chain and every iteration's serial G chain (Eq. cost_parareal's coarse
    terms, one G per open slice), the batched fine sweeps of the open slices
    at the batched per-slice step cost, over N_p N_f serial fine steps."""
    sb = s_bound(n_p, k, n_c / n_f, tau_c / tau_f_serial)
    coarse = (n_p + sum(n_p - j - 1 for j in range(k))) * n_c * tau_c
    fine = sum(n_p - j for j in range(k)) * n_f * tau_f_batched
    return {"gamma_bound_paper": n_p / sb, "s_bound_paper": sb,
            "gamma_bound_one_gpu": (coarse + fine) / (n_p * n_f * tau_f_serial),
            "t_ratio_measured": t_p / t_s,
            "tau_f_serial_us": tau_f_serial * 1e6, "tau_f_batched_us": tau_f_batched * 1e6,
            "tau_c_us": tau_c * 1e6, "K": k, "N_p": n_p, "N_f": n_f, "N_c": n_c}


# ------------------------------------------------------------ CPU oracle leg

def oracle_sample(n_steps, n=256):
    """Time n_steps FP64 RK4 steps of the oracle on one 256^3 field (1 thread)."""
    from oracle import core
    from paper_1409_8563_gb300 import configs
    cfg, u0 = configs.fp32_256()
    P = core.Problem(n, a=tuple(cfg.a), nu0=cfg.nu0, nu_amp=cfg.nu_amp, nu_omega=cfg.nu_omega)
    t0 = time.perf_counter()
    P.rk4(u0, 0, cfg.dt_fine, n_steps)
    dt = time.perf_counter() - t0
    return n ** 3 * n_steps / dt / 1e9, dt


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from oracle import build as obuild
    obuild.build()
    for _ in range(args.warmup):
        oracle_sample(1)
    vals, total = [], 0.0
    for _ in range(args.steps):
        v, dt = oracle_sample(1)
        vals.append(v)
        total += dt
    value = statistics.median(vals)
    sample = "1 RK4 step of one 256^3 field per step (FP64 C oracle, 1 thread)"
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": "fp32_256 Parareal (oracle: fine RK4 steps of the same field)",
                       "n": 256, "n_slices": 32},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ------------------------------------------------------------------- GPU leg

def run(args):
    import numpy as np
    import torch

    rank, world, dist = dist_init(args.gpus)
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    import __graft_entry__
    if rank == 0:
        __graft_entry__.build()
    barrier(dist)
    from paper_1409_8563_gb300 import configs, native

    if args.workload == "fp32_128":
        cfg, u0 = configs.fp32_128(seed=rank)
        desc = ("fp32_128: Parareal to d^k <= 1e-6, 128^3, N=32, dt_F=1/2048, "
                "coarse RK4 on 32^3 at 1/256, k^-2 field to k=32")
    else:
        cfg, u0 = configs.fp32_256(seed=rank)
        desc = ("fp32_256: Parareal to d^k <= 1e-6, 256^3, N=32, dt_F=1/8192, "
                "coarse RK4 on 32^3 at 1/256, k^-2 field to k=32")
    # the stencil G is linear: Eq. (parareal) evaluated as F(U^k[n]) + G(U^{k+1}[n] - U^k[n])
    # (the same iteration, with G's FP32 rounding scaled by the change of its input)
    cfg.correction_form = (native.CORRECTION_DIFFERENCE if args.correction == "difference"
                           else native.CORRECTION_STANDARD)
    cfg.coarse_transfer = (native.TRANSFER_SPECTRAL if args.transfer == "spectral"
                           else native.TRANSFER_BOX)
    cfg.pipeline_blocks = args.pipeline
    n, N = cfg.n, cfg.n_slices
    P = n ** 3
    nf = round(cfg.T / N / cfg.dt_fine)
    stream = torch.cuda.Stream()
    ctx = native.Parareal(cfg, stream=stream)
    # launch shapes from the autotuner (cached per grid, dtype, batch and SM count)
    ctx.autotune(TUNE_CACHE)
    fine_shape, coarse_shape, serial_shape = ctx.launch_shape()
    kernel = {0: f"rk4_fused_kernel<float,{fine_shape[1]},{fine_shape[2]},1> zchunk {fine_shape[3]}",
              2: f"rk4_fused_kernel<float,{fine_shape[1]},{fine_shape[2]},2> zchunk {fine_shape[3]}"}.get(
                  fine_shape[0], "rk4_stage_kernel<float>")
    u0_dev = torch.from_numpy(u0).to("cuda")
    u0_host = torch.from_numpy(u0).pin_memory()
    out_host = torch.empty((n, n, n), dtype=torch.float32).pin_memory()

    # serial fine reference u_fine(T) on the same GPU (also the time to beat)
    ctx.set_problem(u0_dev)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ctx.serial_fine(None, as_reference=True)          # warm-up of the serial path
    with torch.cuda.stream(stream):
        ev0.record(stream)
        ctx.serial_fine(None, as_reference=True)
        ev1.record(stream)
    ev1.synchronize()
    serial_ms = ev0.elapsed_time(ev1)

    def solve():
        ctx.set_problem(u0_dev)
        return ctx.iterate(N, TOL, native.STOP_DEFECT)

    ks = []
    for _ in range(args.warmup):
        k, h = solve()
        ks.append(k)
    torch.cuda.synchronize()
    barrier(dist)

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    launches0 = ctx.launch_count()
    ctx.profile(True)
    updates = 0
    hists = []
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        barrier(dist)
        torch.cuda.nvtx.range_push("timed")     # lets a profiler select the timed steps
        for i in range(args.steps):
            starts[i].record(stream)
            k, h = solve()
            ends[i].record(stream)
            hists.append(h)
            updates += sum((N - j) for j in range(k)) * P * nf
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        barrier(dist)
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    fine_ms, fine_launches, fine_bytes = ctx.profile_read()
    ctx.profile(False)
    launches = ctx.launch_count() - launches0
    # energy of the serial fine run for comparison: board power sampled over
    # enough repetitions to span a few seconds
    reps = max(1, int(round(3000.0 / max(serial_ms, 1.0))))
    with ClockSampler(local) as clk_s:
        with torch.cuda.stream(stream):
            ev0.record(stream)
            for _ in range(reps):
                ctx.serial_fine(None, as_reference=True)
            ev1.record(stream)
        ev1.synchronize()
    serial_rep_ms = ev0.elapsed_time(ev1) / reps
    # one application of the coarse propagator alone (restriction, N_c coarse
    # steps, prolongation), for the energy model's coarse step cost
    g_src = u0_dev.float()
    g_dst = torch.empty_like(g_src)
    torch.cuda.synchronize()
    ctx.propagate(1, g_src, g_dst, 1, 1)
    with torch.cuda.stream(stream):
        ev0.record(stream)
        for _ in range(10):
            ctx.propagate(1, g_src, g_dst, 1, 1)
        ev1.record(stream)
    ev1.synchronize()
    g_apply_ms = ev0.elapsed_time(ev1) / 10
    del g_src, g_dst
    total_ms = max_over_ranks(dist, sum(step_ms))
    updates = sum_over_ranks(dist, updates)
    value = updates / (total_ms / 1000.0) / 1e9

    # the same solve as one CUDA graph launch with the stopping test on the
    # device (parareal_iterate_device): one warm-up (builds the graph), one timed
    ctx.set_problem(u0_dev)
    ctx.iterate(N, TOL, native.STOP_DEFECT, device=True)
    with torch.cuda.stream(stream):
        ctx.set_problem(u0_dev)
        ev0.record(stream)
        k_dev, h_dev = ctx.iterate(N, TOL, native.STOP_DEFECT, device=True)
        ev1.record(stream)
    ev1.synchronize()
    device_loop_ms = ev0.elapsed_time(ev1)

    # end to end through the C ABI with host buffers: H2D of u0 and D2H of
    # the final slice inside every timed step
    e2e_ms = []
    for i in range(max(1, args.steps)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx.set_problem(u0_host.numpy())
        k, _ = ctx.iterate(N, TOL, native.STOP_DEFECT)
        ctx.get_slice(N, out_host.numpy())
        e2e_ms.append(1000 * (time.perf_counter() - t0))
    e2e_upd = updates / args.steps
    e2e_value = e2e_upd / (statistics.mean(e2e_ms) / 1000.0) / 1e9

    peak, peak_kind = peaks()
    avg_launch_ms = fine_ms / max(fine_launches, 1)
    bytes_per_launch = fine_bytes / max(fine_launches, 1)
    achieved = bytes_per_launch / (avg_launch_ms / 1000.0) / 1e9
    # ncu DRAM traffic of a full N-field launch, scaled to the average launch
    # of the solve (traffic grows in proportion to the fields per launch)
    traffic = ncu_traffic(fine_shape[0]) if args.workload == "fp32_256" else None
    fields_per_launch = bytes_per_launch / (2.0 * 4.0 * P)
    if traffic is not None:
        traffic *= fields_per_launch / N
    k_star = max(len(h) for h in hists)
    final_defect = float(hists[-1][-1, 2])

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        from oracle import build as obuild
        obuild.build()
        v, dt = oracle_sample(args.cpu_steps)
        cpu = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"{args.cpu_steps} FP64 RK4 steps of one 256^3 field (C oracle, 1 thread, "
                         f"{dt:.1f} s)"}

    clocks = clk.summary()
    p_par, p_ser = clk.power_w(), clk_s.power_w()
    energy = None
    if p_par is not None and p_ser is not None:
        e_par = p_par * total_ms / args.steps / 1000.0
        e_ser = p_ser * serial_rep_ms / 1000.0
        n_c = round(cfg.T / N / cfg.dt_coarse)
        gam = gamma_terms(N, k_star, nf, n_c, serial_ms / 1000.0 / (N * nf),
                          avg_launch_ms / 1000.0 / fields_per_launch,
                          g_apply_ms / 1000.0 / n_c, total_ms / args.steps, serial_ms)
        energy = {"parareal_j": e_par, "serial_fine_j": e_ser, "ratio": e_par / e_ser,
                  "gamma_measured": e_par / e_ser, **gam,
                  "power_w_parareal": p_par, "power_w_serial_fine": p_ser,
                  "what": "GPU board power (nvidia-smi, every 200 ms) x CUDA-event time per "
                          "solve; gamma_measured = Q_p / Q_s (Sec. 3.4.2); gamma_bound_paper = "
                          "N_p / S_bound (Eq. gamma_expected) for one node per slice; "
                          "gamma_bound_one_gpu = the same cost model for all slices on one GPU "
                          "at constant power; the paper's node, network and cooling terms are "
                          "not measurable here"}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "precision": "FP32 stencil; FP64 correction, norms and nu(t)",
        "data": "synthetic",
        "config": {"workload": desc, "correction_form": args.correction,
                   "coarse_transfer": args.transfer, "pipeline_blocks": args.pipeline,
                   "n": n, "n_slices": N, "fine_steps_per_slice": nf,
                   "l2": ("inputs larger than L2 (%.2f GB per field set)" % (4.0 * N * P / 1e9)),
                   "parallelism": "replicas" if world > 1 else "single GPU",
                   "launch_shapes": {"fine_sweep": list(fine_shape), "coarse": list(coarse_shape),
                                     "serial_fine": list(serial_shape)}},
        "time_to_1e-6_ms": total_ms / args.steps,
        "time_to_1e-6_device_loop_ms": device_loop_ms, "k_star_device_loop": k_dev,
        "serial_fine_ms": serial_ms,
        "parareal_over_serial": (total_ms / args.steps) / serial_ms,
        "k_star": k_star, "final_defect": final_defect,
        "roofline": {"kernel": kernel, "bound": "hbm", "achieved": achieved, "peak": peak,
                     "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": traffic, "algorithmic_bytes_per_launch": bytes_per_launch,
                     "fields_per_launch": fields_per_launch,
                     "avg_launch_ms": avg_launch_ms, "timed_launches": fine_launches,
                     "kernel_glups": bytes_per_launch / 8.0 / (avg_launch_ms / 1000.0) / 1e9,
                     "alu": alu_roof(bytes_per_launch / 8.0 / (avg_launch_ms / 1000.0), clocks)},
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": UNIT, "ms_per_step": statistics.mean(e2e_ms),
                "h2d_bytes_per_step": int(u0.nbytes), "d2h_bytes_per_step": int(out_host.numel() * 4)},
        "gpu_launches": launches,
        "clocks": clocks,
        "energy_to_solution": energy,
    }
    ctx.close()
    del u0_dev
    torch.cuda.empty_cache()
    if rank == 0 and world == 1 and args.workload == "fp32_256" and not args.no_c4:
        line["c4_learned_128"] = c4_learned_128(local, pipeline=args.pipeline)
    if rank == 0 and world == 1 and args.workload == "fp32_256" and not args.no_c3:
        line["c3_batch64"] = {m: batch64(args.correction, m == "queue", 1, 1, local)
                              for m in ("graph", "queue")}
    if rank == 0 and world == 1 and args.workload == "fp32_256" and not args.no_c1:
        line["c1_fp64_32"] = fp64_32(local, steps=20, warmup=3)
    if rank == 0:
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()
    return 0


# ------------------------------------------ the learned-propagator comparison

def c4_learned_128(dev_index, steps=3, n_ics=63, epochs=20, batch=8, lr=1e-3, pipeline=0):
    """The learned-coarse-propagator configuration at 128^3, N = 32: the linear
    learned propagator (stencil skip, nu as a factor), trained here on the
    pairs the fine solver generates (n_ics seeded k^-2 fields plus white noise,
    x 32 slices = 2016 pairs, `epochs` epochs on the tensor-core training
    kernels), evaluated as phase kernels on the coarse grid (and, as
    learned_composed, as one 9^3 kernel per slice), against Parareal with the
    stencil propagator alone and the serial fine run; the stencil and the
    phase-kernel learned G once more with pipelined iterations (two blocks).
    All Parareal runs use the difference form of the correction and run as
    one graph launch each (parareal_iterate_device).  Times are CUDA events on
    the contexts' stream; clocks are sampled over the whole
    comparison, training included."""
    import torch
    from paper_1409_8563_gb300 import configs, inputs, native
    base, u0 = configs.fp32_128()
    n, N = base.n, base.n_slices
    nf = round(base.T / N / base.dt_fine)
    mk = lambda kind, ev, pb=pipeline: native.Config.make(
        n, N, base.T, base.dt_fine, base.dt_coarse, base.coarse_factor, fine_dtype=native.F32,
        coarse_kind=kind, nu0=base.nu0, nu_amp=base.nu_amp, nu_omega=base.nu_omega,
        learned_skip=native.SKIP_STENCIL, learned_act=native.ACT_LINEAR,
        correction_form=native.CORRECTION_DIFFERENCE, learned_eval=ev, pipeline_blocks=pb)
    stream = torch.cuda.Stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn, reps):
        with torch.cuda.stream(stream):
            e0.record(stream)
            r = None
            for _ in range(reps):
                r = fn()
            e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1) / reps, r

    out = {"workload": "learned_128: 128^3, N=32, dt_F=1/2048, stencil G = RK4 on 32^3 at 1/256; "
                       "linear learned G folded with the prolongation into phase kernels on the "
                       "coarse grid (and, as learned_composed, one 9^3 kernel per slice)",
           "steps": steps, "pipeline_blocks": pipeline}
    with ClockSampler(dev_index) as clk:
        trainer = native.Parareal(mk(native.COARSE_LEARNED, native.EVAL_LAYERS), stream=stream)
        t0 = time.perf_counter()
        ics = torch.stack([torch.from_numpy(inputs.spectral_ic(n, seed=1000 + i, kmax=32)
                                            + 0.2 * inputs.random_field(n, seed=2000 + i)).float()
                           for i in range(n_ics)]).cuda()
        pu = torch.empty((n_ics * N, n, n, n), dtype=torch.float32, device="cuda")
        pf = torch.empty_like(pu)
        torch.cuda.synchronize()          # tensors made on the default stream, used on `stream`
        sl = trainer.make_pairs(ics, pu, pf)
        torch.cuda.synchronize()
        pairs_s = time.perf_counter() - t0
        del ics
        trainer.set_coarse_model(inputs.initial_weights(seed=0))
        t0 = time.perf_counter()
        hist = trainer.train_coarse(pu, pf, sl, epochs=epochs, batch=batch, lr=lr, seed=1)
        torch.cuda.synchronize()
        out["train"] = {"pairs": int(len(sl)), "pairs_s": pairs_s, "epochs": epochs,
                        "batch": batch, "lr": lr, "train_s": time.perf_counter() - t0,
                        "loss_first_last": [float(hist[0]), float(hist[-1])]}
        w = trainer.get_coarse_model()
        trainer.close()
        del pu, pf
        torch.cuda.empty_cache()
        u = torch.from_numpy(u0).cuda()
        torch.cuda.synchronize()
        # "learned": the phase-kernel evaluation; "learned_composed": the same
        # operator as one 9^3 kernel on the fine grid; "*_pipelined": the next
        # iteration's fine sweep started in two blocks of slices while the
        # coarse chain runs (pipeline_blocks = 2), the same iterates
        for name, kind, ev, pb in (("stencil", native.COARSE_STENCIL, native.EVAL_LAYERS, pipeline),
                                   ("learned", native.COARSE_LEARNED, native.EVAL_POLYPHASE, pipeline),
                                   ("learned_composed", native.COARSE_LEARNED, native.EVAL_COMPOSED, pipeline),
                                   ("stencil_pipelined", native.COARSE_STENCIL, native.EVAL_LAYERS, 2),
                                   ("learned_pipelined", native.COARSE_LEARNED, native.EVAL_POLYPHASE, 2)):
            if pb == pipeline and name.endswith("_pipelined"):
                continue
            c = native.Parareal(mk(kind, ev, pb), stream=stream)
            c.autotune(TUNE_CACHE)
            if kind == native.COARSE_LEARNED:
                c.set_coarse_model(w)
            c.set_problem(u)
            c.serial_fine(None, as_reference=True)
            if "serial_fine_ms" not in out:
                out["serial_fine_ms"], _ = timed(lambda: c.serial_fine(None, as_reference=True), steps)

            def solve(c=c):
                c.set_problem(u)
                return c.iterate(N, TOL, native.STOP_DEFECT, device=True)
            solve()
            ms, (k, h) = timed(solve, steps)
            src = u.float()
            dst = torch.empty_like(src)
            torch.cuda.synchronize()
            g_ms, _ = timed(lambda: c.propagate(1, src, dst, 1, 1), 10)
            out[name] = {"k_star": int(k), "time_to_1e-6_ms": ms, "g_apply_ms": g_ms,
                         "glups_in_solve": sum(N - j for j in range(k)) * n ** 3 * nf / ms / 1e6,
                         "final_defect": float(h[-1, 2]), "defects": [float(x) for x in h[:, 2]],
                         "pipeline_blocks": pb}
            c.close()
    out["learned_over_stencil"] = out["learned"]["time_to_1e-6_ms"] / out["stencil"]["time_to_1e-6_ms"]
    out["learned_over_serial_fine"] = out["learned"]["time_to_1e-6_ms"] / out["serial_fine_ms"]
    out["clocks"] = clk.summary()
    return out


# ------------------------------------------------- the other configurations

def _timed(fn, reps=1):
    import torch
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    out = None
    for _ in range(reps):
        out = fn()
    torch.cuda.synchronize()
    return (time.perf_counter() - t0) * 1000 / reps, out


def fp64_32(dev_index, steps=5, warmup=3):
    """32^3 FP64, N = 8 (the paper-scale plain method): time-to-1e-6 of
    Parareal (host and device iteration loops) against serial fine, the
    latency-bound regime where one GPU's batched slices can win."""
    import torch
    from paper_1409_8563_gb300 import configs, native
    cfg, u0 = configs.plain_fp64_32()
    ctx = native.Parareal(cfg)
    u = torch.from_numpy(u0).cuda()
    ctx.set_problem(u)
    ctx.serial_fine(None, as_reference=True)

    def solve(device=False):
        ctx.set_problem(u)
        return ctx.iterate(cfg.n_slices, TOL, native.STOP_DEFECT, device=device)
    for _ in range(warmup):
        solve()
        solve(True)
    with ClockSampler(dev_index) as clk:
        serial_ms, _ = _timed(lambda: ctx.serial_fine(None, as_reference=True), steps)
        ms, (k, h) = _timed(solve, steps)
        ms_dev, (k_dev, _) = _timed(lambda: solve(True), steps)
    P, N, nf = 32 ** 3, cfg.n_slices, round(cfg.T / cfg.n_slices / cfg.dt_fine)
    ups = sum(N - j for j in range(k)) * P * nf
    out = {"workload": "fp64_32: 32^3 FP64, N=8, dt_F=1/1024, G = same grid at 1/64, 8 Fourier modes",
           "time_to_1e-6_ms": ms, "serial_fine_ms": serial_ms,
           "time_to_1e-6_device_loop_ms": ms_dev, "k_star_device_loop": int(k_dev),
           "parareal_over_serial": ms / serial_ms,
           "parareal_device_loop_over_serial": ms_dev / serial_ms, "k_star": int(k),
           "defects": [float(x) for x in h[:, 2]], "glups_in_solve": ups / ms / 1e6,
           "dtype": "f64", "steps": steps, "warmup": warmup, "clocks": clk.summary()}
    ctx.close()
    return out


def run_fp64_32(args):
    import __graft_entry__
    __graft_entry__.build()
    print(json.dumps(fp64_32(0, args.steps, args.warmup)))
    return 0


def paper_exact(n, t, nu0, nu_amp, nu_omega):
    """u(x, t) = a(t) u0(x - t (1, 1, 1)) with u0 = sin sin sin and
    a(t) = exp(-12 pi^2 int_0^t nu), the closed-form solution of Sec. 3."""
    import numpy as np
    integral = nu0 * t if nu_omega == 0.0 else nu0 * t + nu0 * nu_amp * (1.0 - np.cos(nu_omega * t)) / nu_omega
    s = np.sin(2 * np.pi * (np.arange(n) / n - t))
    return np.exp(-12.0 * np.pi ** 2 * integral) * s[:, None, None] * s[None, :, None] * s[None, None, :]


def run_paper_faithful(args):
    """The paper's own configuration (Sec. 3.1) at its size: 128^3 FP64, F = RK4
    with fourth-order differences at T/2^15, G = forward Euler / upwind at
    T/2^11, nu frozen: eps_fine, eps_coarse, d^k for k <= 4 with N_p = --slices,
    times of the serial fine run and of each Parareal iteration count."""
    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1409_8563_gb300 import configs, native
    out = {"workload": "paper_faithful", "n": 128, "n_slices": args.slices, "runs": {}}
    for omega in (0.0, 100.0):
        cfg, u0 = configs.paper_faithful(n=128, n_slices=args.slices, omega=omega)
        ctx = native.Parareal(cfg)
        u = torch.from_numpy(u0).cuda()
        exact = paper_exact(128, cfg.T, cfg.nu0, cfg.nu_amp, cfg.nu_omega)
        err = lambda f: float(np.max(np.abs(f - exact)) / np.max(np.abs(exact)))
        res = torch.empty_like(u)
        ctx.set_problem(u)
        serial_ms, _ = _timed(lambda: ctx.serial_fine(res, as_reference=True))
        eps_fine = err(res.cpu().numpy())
        ctx.set_problem(u)
        coarse_ms, _ = _timed(lambda: ctx.coarse_sweep(0, cfg.n_slices, chain=True))
        ctx.get_slice(cfg.n_slices, res)
        eps_coarse = err(res.cpu().numpy())
        ctx.set_problem(u)
        k_max = min(4, cfg.n_slices)
        par_ms, (k, h) = _timed(lambda: ctx.iterate(k_max, 0.0, native.STOP_NONE))
        out["runs"][f"omega={omega:g}"] = {
            "eps_fine": eps_fine, "eps_coarse": eps_coarse, "defects": [float(x) for x in h[:, 2]],
            "serial_fine_ms": serial_ms, "coarse_chain_ms": coarse_ms,
            f"parareal_{k_max}_iterations_ms": par_ms,
            "fine_glups_serial": 128 ** 3 * 2 ** 15 / serial_ms / 1e6}
        ctx.close()
    print(json.dumps(out))
    return 0


def run_learned_128(args):
    """128^3, N = 32: learned coarse propagators (trained here on pairs the
    fine solver generates) vs the stencil coarse propagator vs shift only vs
    serial fine: iterations and time to d^k <= 1e-6.  Two nets correct the
    stencil propagator: the GELU network as specified, and the linear one
    (nu as a factor) with the correction applied to U^{k+1}[n] - U^k[n]; the
    linear one is timed layer by layer (BF16, tensor cores) and composed into
    one 9^3 kernel per slice (FP32)."""
    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1409_8563_gb300 import configs, inputs, native
    base, u0 = configs.fp32_128()
    n, N = base.n, base.n_slices
    mk = lambda kind, r, dtg, skip=native.SKIP_SHIFT, act=native.ACT_GELU, \
        form=native.CORRECTION_STANDARD, ev=native.EVAL_LAYERS: native.Config.make(
            n, N, base.T, base.dt_fine, dtg, r, fine_dtype=native.F32, coarse_kind=kind,
            nu0=base.nu0, nu_amp=base.nu_amp, nu_omega=base.nu_omega, learned_skip=skip,
            learned_act=act, correction_form=form, learned_eval=ev)
    # the nets correct the stencil propagator (RK4 on 32^3 at 1/256)
    learned = native.Parareal(mk(native.COARSE_LEARNED, base.coarse_factor, base.dt_coarse,
                                 native.SKIP_STENCIL))
    linear = native.Parareal(mk(native.COARSE_LEARNED, base.coarse_factor, base.dt_coarse,
                                native.SKIP_STENCIL, native.ACT_LINEAR,
                                native.CORRECTION_DIFFERENCE))
    n_ics = args.n_ics
    t0 = time.perf_counter()
    # k^-2 fields to k = 32 plus white noise: broadband inputs, so the net sees
    # (and learns F's damping of) the high modes Parareal's iterates contain
    ics = torch.stack([torch.from_numpy(inputs.spectral_ic(n, seed=1000 + i, kmax=32)
                                        + 0.2 * inputs.random_field(n, seed=2000 + i)).float()
                       for i in range(n_ics)]).cuda()
    pu = torch.empty((n_ics * N, n, n, n), dtype=torch.float32, device="cuda")
    pf = torch.empty_like(pu)
    sl = learned.make_pairs(ics, pu, pf)
    torch.cuda.synchronize()
    pairs_s = time.perf_counter() - t0
    del ics
    train = {}
    for name, c in (("learned_gelu", learned), ("learned_linear", linear)):
        c.set_coarse_model(inputs.initial_weights(seed=0))
        t0 = time.perf_counter()
        hist = c.train_coarse(pu, pf, sl, epochs=args.epochs, batch=args.batch, lr=args.lr, seed=1)
        torch.cuda.synchronize()
        train[name] = {"loss_first_last": [float(hist[0]), float(hist[-1])],
                       "train_s": time.perf_counter() - t0}
    del pu, pf
    torch.cuda.empty_cache()
    # the trained linear net evaluated as one 9^3 kernel per slice
    composed = native.Parareal(mk(native.COARSE_LEARNED, base.coarse_factor, base.dt_coarse,
                                  native.SKIP_STENCIL, native.ACT_LINEAR,
                                  native.CORRECTION_DIFFERENCE, native.EVAL_COMPOSED))
    composed.set_coarse_model(linear.get_coarse_model())
    u = torch.from_numpy(u0).cuda()
    res = {}
    # ... and folded with the prolongation into phase kernels on the coarse grid
    poly = native.Parareal(mk(native.COARSE_LEARNED, base.coarse_factor, base.dt_coarse,
                              native.SKIP_STENCIL, native.ACT_LINEAR,
                              native.CORRECTION_DIFFERENCE, native.EVAL_POLYPHASE))
    poly.set_coarse_model(linear.get_coarse_model())
    ctxs = {"learned_linear_polyphase": poly,
            "learned_linear_composed": composed,
            "learned_linear": linear,
            "learned_gelu": learned,
            "stencil": native.Parareal(base),
            "stencil_difference_form": native.Parareal(
                mk(native.COARSE_STENCIL, base.coarse_factor, base.dt_coarse,
                   form=native.CORRECTION_DIFFERENCE)),
            "shift": native.Parareal(mk(native.COARSE_SHIFT, 1, base.T / N))}
    serial_ms = None
    for name, c in ctxs.items():
        c.set_problem(u)
        c.serial_fine(None, as_reference=True)
        if serial_ms is None:
            serial_ms, _ = _timed(lambda: c.serial_fine(None, as_reference=True), 2)

        def solve(c=c):
            c.set_problem(u)
            return c.iterate(N, TOL, native.STOP_DEFECT)
        solve()
        torch.cuda.nvtx.range_push("solve_" + name)     # lets a profiler select this solve
        ms, (k, h) = _timed(solve, args.steps)
        torch.cuda.nvtx.range_pop()
        # one application of G (slice 1) on its own
        src = u.float() if c.cfg.fine_dtype == native.F32 else u
        dst = torch.empty_like(src)
        g_ms, _ = _timed(lambda: c.propagate(1, src, dst, 1, 1), 5)
        res[name] = {"k_star": k, "time_to_1e-6_ms": ms, "g_apply_ms": g_ms,
                     "defects": [float(x) for x in h[:, 2]]}
    print(json.dumps({"workload": "learned_128", "serial_fine_ms": serial_ms, "runs": res,
                      "train": {"pairs": int(len(sl)), "epochs": args.epochs, "batch": args.batch,
                                "lr": args.lr, "pairs_s": pairs_s, **train}}))
    for c in ctxs.values():
        c.close()
    return 0


def run_learned_512(args):
    """512^3, N = 16 (dt_F = 1/32768, stencil G on 64^3 at 1/512): Parareal with
    the linear learned propagator (stencil skip, phase kernels on the coarse
    grid, difference-form correction), trained here on the pairs the fine
    solver generates from --n-ics seeded fields (16 pairs each), against
    stencil-G Parareal and the serial fine run: iterations and time to
    d^k <= 1e-6, fine GLUP/s inside each solve, clocks sampled over the
    solves.  One solve each (a solve takes about a minute at this size);
    contexts are built one after another to bound the device memory
    (~160 GB at the peak, during training)."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1409_8563_gb300 import configs, inputs, native
    base, u0 = configs.fp32_512()
    n, N = base.n, base.n_slices
    P, nf = n ** 3, round(base.T / N / base.dt_fine)
    mk = lambda kind, ev: native.Config.make(
        n, N, base.T, base.dt_fine, base.dt_coarse, base.coarse_factor, fine_dtype=native.F32,
        coarse_kind=kind, nu0=base.nu0, nu_amp=base.nu_amp, nu_omega=base.nu_omega,
        learned_skip=native.SKIP_STENCIL, learned_act=native.ACT_LINEAR,
        correction_form=native.CORRECTION_DIFFERENCE, learned_eval=ev)
    out = {"workload": "learned_512", "n": n, "n_slices": N, "fine_steps_per_slice": nf}
    # training (layer by layer, BF16, tensor cores)
    t0 = time.perf_counter()
    trainer = native.Parareal(mk(native.COARSE_LEARNED, native.EVAL_LAYERS))
    n_ics = args.n_ics
    ics = torch.stack([torch.from_numpy(inputs.spectral_ic(n, seed=1000 + i, kmax=32)
                                        + 0.2 * inputs.random_field(n, seed=2000 + i)).float()
                       for i in range(n_ics)]).cuda()
    pu = torch.empty((n_ics * N, n, n, n), dtype=torch.float32, device="cuda")
    pf = torch.empty_like(pu)
    sl = trainer.make_pairs(ics, pu, pf)
    torch.cuda.synchronize()
    out["pairs"] = int(len(sl))
    out["pairs_s"] = time.perf_counter() - t0
    del ics
    trainer.set_coarse_model(inputs.initial_weights(seed=0))
    t0 = time.perf_counter()
    hist = trainer.train_coarse(pu, pf, sl, epochs=args.epochs, batch=1, lr=args.lr, seed=1)
    torch.cuda.synchronize()
    out["train"] = {"epochs": args.epochs, "batch": 1, "lr": args.lr,
                    "loss_first_last": [float(hist[0]), float(hist[-1])],
                    "train_s": time.perf_counter() - t0}
    w = trainer.get_coarse_model()
    trainer.close()
    del pu, pf
    torch.cuda.empty_cache()
    u = torch.from_numpy(u0).cuda()
    ref = torch.empty((n,) * 3, dtype=torch.float64, device="cuda")
    runs = {}
    with ClockSampler(0) as clk:
        for name, kind in (("stencil_difference_form", native.COARSE_STENCIL),
                           ("learned_linear_polyphase", native.COARSE_LEARNED)):
            # the trained linear net folded with the prolongation into phase kernels
            c = native.Parareal(mk(kind, native.EVAL_POLYPHASE if kind == native.COARSE_LEARNED
                                   else native.EVAL_LAYERS))
            c.autotune(TUNE_CACHE)
            if kind == native.COARSE_LEARNED:
                c.set_coarse_model(w)
            c.set_problem(u)
            if "serial_fine_ms" not in out:
                ms, _ = _timed(lambda: c.serial_fine(ref, as_reference=True))
                out["serial_fine_ms"] = ms
                out["serial_fine_glups"] = P * N * nf / ms / 1e6
            else:
                c.set_reference(ref)
            ms, (k, h) = _timed(lambda: c.iterate(N, TOL, native.STOP_DEFECT))
            ups = sum(N - j for j in range(k)) * P * nf
            runs[name] = {"k_star": k, "time_to_1e-6_ms": ms, "glups_in_solve": ups / ms / 1e6,
                          "defects": [float(x) for x in h[:, 2]],
                          "launch_shape_fine": list(c.launch_shape()[0])}
            c.close()
    out["runs"] = runs
    out["clocks"] = clk.summary()
    print(json.dumps(out))
    return 0


def run_learned_g(args):
    """One application of the learned coarse propagator (128^3, N = 32,
    stencil skip, linear network) per evaluation: layer by layer (BF16,
    tensor cores), composed into one 9^3 kernel (FP32), and folded with the
    prolongation into phase kernels on the coarse grid (FP32), with perturbed
    initial weights (the cost does not depend on their values); the stencil
    propagator alone beside them.  A small, self-contained target for ncu."""
    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1409_8563_gb300 import configs, inputs, native
    base, u0 = configs.fp32_128()
    mk = lambda kind, ev: native.Config.make(
        128, 32, base.T, base.dt_fine, base.dt_coarse, base.coarse_factor, fine_dtype=native.F32,
        coarse_kind=kind, nu0=base.nu0, nu_amp=base.nu_amp, nu_omega=base.nu_omega,
        learned_skip=native.SKIP_STENCIL, learned_act=native.ACT_LINEAR,
        correction_form=native.CORRECTION_DIFFERENCE, learned_eval=ev)
    w = inputs.initial_weights(seed=0)
    w = (w + 0.01 * np.random.default_rng(1).standard_normal(w.shape)).astype(np.float32)
    src = torch.from_numpy(u0).cuda()
    dst = torch.empty_like(src)
    out = {"workload": "learned_g", "n": 128, "n_slices": 32}
    for name, kind, ev in (("polyphase", native.COARSE_LEARNED, native.EVAL_POLYPHASE),
                           ("composed", native.COARSE_LEARNED, native.EVAL_COMPOSED),
                           ("layers", native.COARSE_LEARNED, native.EVAL_LAYERS),
                           ("stencil", native.COARSE_STENCIL, native.EVAL_LAYERS)):
        c = native.Parareal(mk(kind, ev))
        if kind == native.COARSE_LEARNED:
            c.set_coarse_model(w)
        for _ in range(args.warmup):
            c.propagate(1, src, dst, 1, 1)
        ms, _ = _timed(lambda: c.propagate(1, src, dst, 1, 1), max(args.steps, 1))
        out[name + "_g_apply_ms"] = ms
        c.close()
    print(json.dumps(out))
    return 0


def batch64(correction="difference", queue=False, steps=1, warmup=1, dev_index=0):
    """64 uneven instances (sizes from {32,48,64,96,128}, nu0 in [0.002, 0.02],
    N = 8, T = 1) solved to a defect of 1e-6: one CUDA graph per round, the
    fine sweeps as each instance's own launches (graph mode) or as one
    persistent launch over a queue of every instance's tile steps (queue
    mode); autotuned launch shapes.  serial_fine_ms: every instance's serial
    fine run, all instances concurrently."""
    import torch
    from paper_1409_8563_gb300 import configs, inputs, native
    ns, nus = inputs.batch_instances(seed=0)
    cfgs, u0s = [], []
    for i, (n, nu0) in enumerate(zip(ns, nus)):
        cfg, u0 = configs.batch_instance(n, nu0, seed=i)
        cfg.correction_form = (native.CORRECTION_DIFFERENCE if correction == "difference"
                               else native.CORRECTION_STANDARD)
        cfgs.append(cfg)
        u0s.append(torch.from_numpy(u0).cuda())
    b = native.Batch(cfgs)
    if queue:
        b.set_fine_mode(1)
    tune_ms, _ = _timed(lambda: b.autotune(os.path.join(ROOT, "paper_1409_8563_gb300", "tune_cache.jsonl")))
    for i, u in enumerate(u0s):
        b.set_problem(i, u)
    b.serial_fine(True)

    def solve():
        for i, u in enumerate(u0s):
            b.set_problem(i, u)
        return b.iterate(8, TOL, native.STOP_DEFECT)
    for _ in range(max(warmup, 1)):
        solve()
    with ClockSampler(dev_index) as clk:
        serial_ms, _ = _timed(lambda: b.serial_fine(True), 1)
        ms, (k, d) = _timed(solve, max(steps, 1))
    ups = 0
    for cfg, kk in zip(cfgs, k):
        nf = round(cfg.T / cfg.n_slices / cfg.dt_fine)
        ups += sum(cfg.n_slices - j for j in range(int(kk))) * cfg.n ** 3 * nf
    out = {"workload": "batch64", "fine_mode": "queue" if queue else "graph",
           "time_to_1e-6_ms": ms, "serial_fine_ms": serial_ms,
           "parareal_over_serial": ms / serial_ms,
           "k_star": [int(x) for x in k], "max_defect": float(max(d)),
           "glups_in_solve": ups / ms / 1e6, "autotune_ms": tune_ms,
           "correction_form": correction, "fine_shape": list(b.fine_mode()),
           "graph_launches": b.graph_launches(), "clocks": clk.summary()}
    b.close()
    del u0s
    torch.cuda.empty_cache()
    return out


def run_train_128(args):
    """Training throughput of the learned propagator at 128^3 (batch 8 of
    synthetic pairs, Adam): one warm-up epoch, then `steps` timed epochs of
    8 batches; per batch: forward with pre-activations, loss, all gradients,
    Adam and the operand copies.  The ncu target of the training kernels."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1409_8563_gb300 import configs, inputs, native
    base, _ = configs.fp32_128()
    n, N = base.n, base.n_slices
    act = native.ACT_GELU if args.act == "gelu" else native.ACT_LINEAR
    cfg = native.Config.make(n, N, base.T, base.dt_fine, base.dt_coarse, base.coarse_factor,
                             fine_dtype=native.F32, coarse_kind=native.COARSE_LEARNED, nu0=base.nu0,
                             nu_amp=base.nu_amp, nu_omega=base.nu_omega,
                             learned_skip=native.SKIP_STENCIL, learned_act=act,
                             correction_form=(native.CORRECTION_DIFFERENCE if act == native.ACT_LINEAR
                                              else native.CORRECTION_STANDARD),
                             learned_eval=native.EVAL_LAYERS)
    ctx = native.Parareal(cfg)
    npairs, batch = 64, 8
    g = torch.Generator(device="cuda").manual_seed(0)
    pu = torch.randn((npairs, n, n, n), device="cuda", generator=g)
    pf = 0.9 * pu
    sl = [i % N for i in range(npairs)]
    ctx.set_coarse_model(inputs.initial_weights(seed=0))
    ctx.train_coarse(pu, pf, sl, epochs=1, batch=batch, lr=1e-3, seed=1)
    ms, _ = _timed(lambda: ctx.train_coarse(pu, pf, sl, epochs=args.steps, batch=batch, lr=1e-3, seed=2))
    nb = args.steps * (npairs // batch)
    print(json.dumps({"workload": f"train_128: learned propagator training at {n}^3, batch {batch}, "
                                  f"{args.act} activations", "ms_per_batch": ms / nb,
                      "points_per_s": batch * n ** 3 / (ms / nb / 1000.0), "batches": nb}))
    ctx.close()
    return 0


def run_batch64(args):
    import __graft_entry__
    __graft_entry__.build()
    print(json.dumps(batch64(args.correction, args.queue, args.steps, args.warmup)))
    return 0


def run_fine_sweep(args):
    """One batched fine sweep (4 RK4 steps) of --slices fields of 256^3 FP32 in
    the autotuned launch shape: a small, self-contained target for ncu."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1409_8563_gb300 import inputs, native
    n, S, steps = 256, args.slices, 4
    cfg = native.Config.make(n, S, S * steps / 8192, 1 / 8192, steps / 8192, 8, fine_dtype=native.F32)
    if args.tile:
        # "tx,ty,zchunk" (fused kernel, one row per thread) or "path,tx,ty,zchunk"
        t = args.tile.split(",")
        os.environ["PARAREAL_FINE_TILE"] = ",".join(t if len(t) == 4 else ["0"] + t)
    ctx = native.Parareal(cfg)
    if not args.tile:
        ctx.autotune(TUNE_CACHE)
    u = torch.from_numpy(inputs.spectral_ic(n, seed=1, kmax=32)).cuda()
    ctx.set_problem(u)
    for s in range(1, S + 1):
        ctx.set_slice(s, u)
    ctx.fine_sweep(0, S)   # warm-up launches; the next sweep is the one to capture
    ctx.profile(True)
    for _ in range(max(args.steps, 1)):
        ctx.fine_sweep(0, S)
    fine_ms, launches, nbytes = ctx.profile_read()
    ctx.profile(False)
    per_launch = fine_ms / max(launches, 1)
    print(json.dumps({"workload": "fine_sweep", "slices": S, "rk4_steps_per_sweep": steps,
                      "sweeps": max(args.steps, 1), "launch_ms": per_launch,
                      "glups": S * n ** 3 / per_launch / 1e6,
                      "gbs_algorithmic": nbytes / launches / per_launch / 1e6,
                      "launch_shape": ctx.launch_shape()[0]}))
    ctx.close()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-steps", type=int, default=8)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--pipeline", type=int, default=0,
                    help="pipelined iterations: the next iteration's fine sweep in this many "
                         "blocks on a second stream while the coarse chain runs (0: off)")
    ap.add_argument("--no-c3", action="store_true",
                    help="fp32_256: leave out the 64-instance batch comparison (graph and queue modes)")
    ap.add_argument("--no-c1", action="store_true",
                    help="fp32_256: leave out the 32^3 FP64 comparison (Parareal vs serial fine)")
    ap.add_argument("--no-c4", action="store_true",
                    help="skip the 128^3 learned-propagator comparison of the default line")
    ap.add_argument("--workload", default="fp32_256",
                    choices=["fp32_256", "fp32_128", "fp64_32", "learned_128", "learned_512",
                             "learned_g", "batch64", "fine_sweep", "paper_faithful", "c4",
                             "train_128"])
    ap.add_argument("--slices", type=int, default=8)
    ap.add_argument("--correction", default="difference", choices=["difference", "standard"],
                    help="evaluation of the Parareal correction (fp32_256 / fp32_128 / batch64)")
    ap.add_argument("--queue", action="store_true",
                    help="batch64: the fine sweeps of a round as one persistent launch over a "
                         "queue of every instance's tile steps")
    ap.add_argument("--transfer", default="box", choices=["box", "spectral"],
                    help="fp32_256 / fp32_128: restriction and prolongation of the coarse "
                         "propagator (box + trilinear, or spectral)")
    ap.add_argument("--tile", default=None,
                    help="fine_sweep: launch shape 'tx,ty,zchunk' (fused kernel, one row per "
                         "thread) or 'path,tx,ty,zchunk' (path 2: two rows per thread) instead of "
                         "autotuning")
    ap.add_argument("--n-ics", type=int, default=None,
                    help="learned workloads: seeded training fields (default 63 at 128^3, 2 at 512^3)")
    ap.add_argument("--epochs", type=int, default=None,
                    help="default 20 for c4 (the default line's comparison), 10 for learned_128, 16 at 512^3")
    ap.add_argument("--batch", type=int, default=8)
    ap.add_argument("--act", default="linear", choices=["linear", "gelu"],
                    help="train_128: activations of the trained network")
    ap.add_argument("--lr", type=float, default=None, help="default 1e-3 at 128^3, 2e-3 at 512^3")
    args = ap.parse_args()
    big = args.workload == "learned_512"
    args.n_ics = args.n_ics if args.n_ics is not None else (2 if big else 63)
    # the 128^3 comparison of the default line (c4) trains 20 epochs, learned_128 10
    args.epochs = args.epochs if args.epochs is not None else (16 if big else (20 if args.workload == "c4" else 10))
    args.lr = args.lr if args.lr is not None else (2e-3 if big else 1e-3)
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "fp64_32":
        return run_fp64_32(args)
    if args.workload == "learned_128":
        return run_learned_128(args)
    if args.workload == "learned_g":
        return run_learned_g(args)
    if args.workload == "learned_512":
        return run_learned_512(args)
    if args.workload == "batch64":
        return run_batch64(args)
    if args.workload == "c4":
        # the 128^3 learned-vs-stencil comparison of the headline line, alone
        import __graft_entry__
        __graft_entry__.build()
        print(json.dumps(c4_learned_128(0, epochs=args.epochs, lr=args.lr, pipeline=args.pipeline)))
        return 0
    if args.workload == "fine_sweep":
        return run_fine_sweep(args)
    if args.workload == "train_128":
        return run_train_128(args)
    if args.workload == "paper_faithful":
        return run_paper_faithful(args)
    return run(args)


if __name__ == "__main__":
    sys.exit(main())
