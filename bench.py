"""Benchmark of the semi-Lagrangian Gauss-Newton-Krylov registration hot path.

One step = one full registration (Eq. (5)) of the 256^3 clinical-size
synthetic workload from v = 0 to ||g|| / ||g0|| <= 5e-2: four nested smoothed
label regions (0.2/0.5/0.8/1.0, Gaussian blur sigma = 1 voxel, N(0, 0.02^2)
noise), reference made by a random band-limited velocity (|k| <= 8,
max |v| = 1.0), nt = 4 RK2 steps, cubic Lagrange interpolation, H1
regularisation beta_v = 1e-2 (middle of the 1e-1 / 1e-2 / 1e-3 sweep;
--beta selects another), beta_w = 1e-4.

value = SL interpolation throughput of the whole job: grid points x scalar
fields interpolated by all gather kernels of the registration, divided by the
wall time of the registration (Gpts/s); ms_per_step is the time to tolerance.
roofline = the dominant kernel of the step, algorithmic bytes per launch over
its CUDA-event time per launch, against the measured HBM copy bandwidth.

--impl reference times the FP64 CPU oracle on the host cores on a bounded
sample of the same workload (one gradient evaluation per step).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "SL interp Gpts/s (256^3 Gauss-Newton registration to gtol 5e-2, FP32, tricubic, nt=4)"
UNIT = "Gpts/s"
GATHER_KINDS = ("sl_interp", "sl_backtrace_rk2", "sl_adjoint_step", "sl_incremental_step",
                "sl_incremental_last", "sl_map_step")


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=256, help="grid points per axis")
    ap.add_argument("--beta", type=float, default=1e-2)
    ap.add_argument("--storage", default="f32", choices=["f32", "f16", "bf16"],
                    help="storage precision of the solver's scalar fields (arithmetic is FP32)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--mixed-report", action="store_true",
                    help="FP32 vs FP16 vs BF16 storage on the blob workload at --n (default 512): "
                         "time, throughput and each result's error against the FP64 oracle")
    ap.add_argument("--warmstart-report", action="store_true",
                    help="time to tolerance at --n: plain FP32 from v=0 vs FP16 storage + learned warm start "
                         "(network trained at n/2 on pairs the method generates)")
    ap.add_argument("--ws-steps", type=int, default=2000, help="training steps of the warm-start network")
    ap.add_argument("--large-report", action="store_true",
                    help="largest single-GPU case (--large-n, default 1024): FP32 from v=0 vs FP16 storage + "
                         "learned warm start, both without stored state gradients; Dice on 3 labels; the same "
                         "registration on images sampled to 256^3 and 512^3; sampled oracle parity")
    ap.add_argument("--large-n", type=int, default=1024)
    ap.add_argument("--large-precond", default="spectral", choices=["spectral", "two-level", "both"],
                    help="preconditioner of the mixed + learned run of --large-report (both: the spectral run, "
                         "then the same learned registration with the two-level preconditioner)")
    ap.add_argument("--large-pc-coarse", type=int, default=4,
                    help="fine-to-coarse ratio of the two-level preconditioner in --large-report")
    ap.add_argument("--large-vmax", type=float, default=0.5,
                    help="max |v*| of the large case (0.5: CFL 20 at 1024^3, nt=4)")
    ap.add_argument("--net-report", action="store_true",
                    help="timing of the warm-start network kernels (every conv shape of the U-Net at 128^3, "
                         "batch 4), one training step, and the SL reverse-mode transport at 256^3")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--interp-report", action="store_true",
                    help="SL interpolation micro-benchmark: Gpts/s and roofline fractions of the gather kernel "
                         "for tricubic / trilinear, 256^3..1024^3, realistic / zero / random displacements, "
                         "1 and 4 fields")
    ap.add_argument("--interp-sizes", default="256,512,1024")
    ap.add_argument("--syn-report", action="store_true",
                    help="the paper's SYN pairs (spherical-harmonic template, trigonometric velocity of K modes): "
                         "regularisation-parameter search per K at 128^3 (nt 4) and 256^3 (nt 8)")
    ap.add_argument("--syn-sizes", default="128,256")
    ap.add_argument("--vjp-report", action="store_true",
                    help="reverse-mode transport at --vjp-n (default 1024^3) with time-step checkpointing: "
                         "time, device memory, adjoint identity")
    ap.add_argument("--vjp-n", type=int, default=1024)
    ap.add_argument("--no-mixed-learned", action="store_true",
                    help="skip the FP16 storage + learned warm start registration of the default line")
    ap.add_argument("--weights", default=None,
                    help="warm-start network weights (default: the network with the preconditioner head, "
                         "weights/unet_warmstart_pc_128.npz, if present, else weights/unet_warmstart_128.npz)")
    ap.add_argument("--spectral-iterate", type=int, default=1, choices=[0, 1],
                    help="claire_opts.spectral_iterate of the solver contexts (1: S v from the carried spectrum)")
    ap.add_argument("--precond", default="spectral", choices=["spectral", "two-level"],
                    help="PCG preconditioner of the timed registration")
    ap.add_argument("--no-other-precond", action="store_true",
                    help="skip the registration with the other preconditioner after the timed loop")
    ap.add_argument("--pc-weight-report", action="store_true",
                    help="the coarse preconditioner correction at 256^3: FP16 + warm start + two-level with the "
                         "network's weight, least-squares fitted weights and constant weights")
    ap.add_argument("--precond-report", action="store_true",
                    help="time to tolerance at --n with the spectral and the two-level zero-velocity preconditioner")
    return ap.parse_args()


def workload(n):
    """Seeded inputs of the 256^3 clinical-size case (no transport here)."""
    from paper_2209_08189_gb300 import synth
    grid = (n, n, n)
    base = synth.label_template(grid, seed=0)
    vstar = synth.bandlimited_velocity(grid, seed=0, kmax=8, vmax=1.0)
    return grid, base, vstar


def config_dict(args, n_gpus):
    return {"workload": "clinical-size synthetic: %d^3 nested-label template, band-limited v* "
                        "|k|<=8 max|v|=1, Gauss-Newton-Krylov to gtol 5e-2 from v=0" % args.n,
            "grid": [args.n] * 3, "nt": 4, "interp": "cubic Lagrange", "beta_v": args.beta,
            "beta_w": 1e-4, "reg": "H1 seminorm", "gtol": 5e-2, "max_pcg": 50,
            "storage": args.storage, "precond": args.precond, "spectral_iterate": args.spectral_iterate,
            "l2_policy": "inputs larger than L2 (working set %.1f GB > 129 MB L2)"
                         % (args.n ** 3 * 4 * 60 / 1e9),
            "parallelism": "replicas" if n_gpus > 1 else "single GPU"}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs)"
    return 6800.0, "fallback 6.8 TB/s"


def kernel_source_hash():
    h = hashlib.sha1()
    # the files that define and launch the SL gather kernels
    for f in ("sl_tiled.cuh", "common.cuh", "storage.cuh", "sl_kernels.cu"):
        with open(os.path.join(ROOT, "paper_2209_08189_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:12]


def ncu_traffic(kernel, src_hash):
    """DRAM bytes per launch of `kernel` from the committed ncu summaries, if
    they were taken on the current kernel source; else None."""
    pdir = os.path.join(ROOT, "profiles")
    if not os.path.isdir(pdir):
        return None
    pat = re.compile(r"^traffic_bytes_per_launch:\s+(\S+)\s+(\S+)\s+source=(\S+)", re.M)
    for fn in sorted(os.listdir(pdir)):
        if not fn.endswith((".md", ".txt")):
            continue
        with open(os.path.join(pdir, fn)) as f:
            for k, val, hsh in pat.findall(f.read()):
                if k == kernel and hsh == src_hash:
                    return float(val)
    return None


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        # the raw samples go to $CLAIRE_CLOCKS_DIR when set, else the temporary directory
        import tempfile
        self.path = os.path.join(os.environ.get("CLAIRE_CLOCKS_DIR") or tempfile.gettempdir(),
                                 "claire_clocks_rank%d.csv" % index)

    def start(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.fh,
                stderr=subprocess.DEVNULL)
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
        self.fh.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx.append(float(parts[2]))
                except ValueError:
                    continue
                for name, val in zip(names, parts[5:9]):
                    if val.lower().startswith("active"):
                        reasons.add(name)
        if not sm:
            return None
        loaded = [s for s in sm if s > 0.5 * max(sm)] or sm
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


def aggregate_ranks(secs, pts, dist=None, device=None):
    """Whole-job figures over replica ranks: the slowest rank's time and the
    work of all ranks (no data-path collective; one reduction per figure)."""
    if dist is None:
        return secs, pts
    import torch
    t = torch.tensor([secs], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    q = torch.tensor([pts], dtype=torch.float64, device=device)
    dist.all_reduce(q, op=dist.ReduceOp.SUM)
    return float(t.item()), float(q.item())


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


# ---------------------------------------------------------------------------
# reference arm: the FP64 oracle on the host cores
# ---------------------------------------------------------------------------

def oracle_sample(grid, m0, m1, beta):
    """One gradient evaluation of the oracle (state, characteristics, adjoint)
    on the workload; returns (seconds, interpolated point-fields)."""
    import oracle
    p = oracle.Params(nt=4, beta_v=beta, beta_w=1e-4)
    v = np.zeros((3,) + grid)
    t0 = time.perf_counter()
    st = oracle.State(v, m0, m1, p)
    oracle.gradient(st)
    dt = time.perf_counter() - t0
    N = float(np.prod(grid))
    # backtraces (2 x 3 fields), div v at X+, nt state steps, nt adjoint steps
    pts = N * (6 + 1 + 4 + 4)
    return dt, pts


def cpu_model():
    """CPU model string of this host (for the CPU baseline's record)."""
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                key = line.split(":")[0].strip().lower()
                if key in ("model name", "cpu model", "hardware"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    try:  # Arm hosts list no model name in /proc/cpuinfo; lscpu decodes the part number
        import subprocess
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    import platform
    return platform.processor() or platform.machine()


def run_reference(args):
    world, rank, _ = dist_setup(args)
    if rank != 0:
        return
    import oracle
    grid, base, vstar = workload(args.n)
    from paper_2209_08189_gb300 import synth
    p = oracle.Params(nt=4, beta_v=args.beta, beta_w=1e-4)
    m1 = synth.add_noise(oracle.transport(base, vstar, p), 0.02, seed=1)
    m0 = synth.add_noise(base, 0.02, seed=0)
    for _ in range(args.warmup):
        oracle_sample(grid, m0, m1, args.beta)
    secs, pts = 0.0, 0.0
    for _ in range(args.steps):
        s, q = oracle_sample(grid, m0, m1, args.beta)
        secs += s
        pts += q
    val = pts / secs / 1e9
    cores = oracle.num_threads()
    sample = "one oracle gradient evaluation (state + adjoint solve, nt=4) of the %d^3 workload per step" % args.n
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": config_dict(args, args.gpus),
        "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "cpu_model": cpu_model(), "sample": sample},
        "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------

def run_ours(args):
    import torch
    world, rank, local = dist_setup(args)
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU (no CPU fallback)")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
        pg = dist
    import __graft_entry__ as entry
    if rank == 0:
        entry.build()
    if pg:
        pg.barrier()
    entry.build()
    from paper_2209_08189_gb300 import claire, synth

    grid, base, vstar = workload(args.n)
    N = int(np.prod(grid))
    stream = torch.cuda.current_stream(dev)
    storage = {"f32": claire.STORAGE_F32, "f16": claire.STORAGE_F16, "bf16": claire.STORAGE_BF16}[args.storage]
    precond = claire.PRECOND_TWO_LEVEL if args.precond == "two-level" else claire.PRECOND_SPECTRAL
    ctx = claire.Context(grid, args.beta, 4, stream=stream.cuda_stream, beta_w=1e-4, gtol=5e-2,
                         max_gn=50, max_pcg=50, storage=storage, precond=precond,
                         spectral_iterate=args.spectral_iterate)
    # reference image by our own transport of the clean template, then noise
    base_d = torch.from_numpy(base.astype(np.float32)).to(dev)
    vstar_d = torch.from_numpy(vstar.astype(np.float32)).to(dev)
    m1c = torch.empty(grid, device=dev)
    ctx.transport(vstar_d, base_d, m1c, claire.TRANSPORT_FWD)
    m1 = (m1c.cpu().numpy().astype(np.float64))
    m1 = synth.add_noise(m1, 0.02, seed=1).astype(np.float32)
    m0 = synth.add_noise(base, 0.02, seed=0).astype(np.float32)
    m0_d = torch.from_numpy(m0).to(dev)
    m1_d = torch.from_numpy(m1).to(dev)
    ctx.set_images(m0_d, m1_d)
    v = torch.zeros((3,) + grid, device=dev)

    def step():
        v.zero_()
        st, rep = ctx.register(v)
        if st < 0:
            raise RuntimeError("registration failed: %s" % rep["status"])
        return rep

    for _ in range(args.warmup):
        step()
    ctx.set_timing(True)
    ctx.kernel_stats(reset=True)
    clocks = ClockSampler(local)
    clocks.start()
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    reps = [step() for _ in range(args.steps)]
    e1.record(stream)
    torch.cuda.synchronize()
    if pg:
        pg.barrier()
    ck = clocks.stop()
    secs = e0.elapsed_time(e1) * 1e-3
    stats = ctx.kernel_stats(reset=True)
    ctx.set_timing(False)
    pts = sum(r["interp_points"] for r in reps)
    tmax, pts_all = aggregate_ranks(secs, pts, pg, dev)
    value = pts_all / tmax / 1e9

    # dominant kernel of ours (cuFFT is a library call, not counted)
    mine = [s for s in stats if s["name"] != "cufft" and s["launches"] > 0]
    launches = int(sum(s["launches"] for s in mine))
    top = max(mine, key=lambda s: s["seconds"])
    peak, peak_src = measured_peaks()
    per_launch_bytes = top["bytes"] / top["launches"]
    per_launch_s = top["seconds"] / top["launches"]
    achieved = per_launch_bytes / per_launch_s / 1e9
    gathers = [s for s in stats if s["name"] in GATHER_KINDS and s["launches"] > 0]
    g_bytes = sum(s["bytes"] for s in gathers)
    g_secs = sum(s["seconds"] for s in gathers)
    g_pts = sum(s["points"] for s in gathers)
    total_kernel_s = sum(s["seconds"] for s in stats)
    # shared-memory (LSU) ceiling of the gathers: 128 B/clk/SM x SMs x max SM
    # clock; a tricubic point needs 64 x 4 B of shared-memory reads
    props = torch.cuda.get_device_properties(dev)
    sm_mhz = ck["sm_max_mhz"] if ck else 2070.0
    lsu_bytes_s = 128.0 * props.multi_processor_count * sm_mhz * 1e6
    top_pts = top["points"] / top["launches"] if top["points"] else 0.0
    roofline = {"bound": "hbm", "kernel": top["name"], "achieved": achieved, "peak": peak,
                "unit": "GB/s", "frac": achieved / peak, "peak_source": peak_src,
                "traffic": ncu_traffic(top["name"], kernel_source_hash()),
                "algorithmic_bytes_per_launch": per_launch_bytes,
                "launch_ms": per_launch_s * 1e3,
                "share_of_kernel_time": top["seconds"] / total_kernel_s if total_kernel_s else None,
                "lsu": {"achieved_gpts": top_pts / per_launch_s / 1e9,
                        "peak_gpts": lsu_bytes_s / 256.0 / 1e9,
                        "frac": (top_pts / per_launch_s) / (lsu_bytes_s / 256.0),
                        "note": "shared-memory read ceiling of a tricubic gather (64 x 4 B per point)"},
                "all_gathers": {"gpts_s": g_pts / g_secs / 1e9 if g_secs else None,
                                "achieved_GBs": g_bytes / g_secs / 1e9 if g_secs else None,
                                "frac": (g_bytes / g_secs / 1e9) / peak if g_secs else None}}

    # end to end through the C ABI with host buffers (pinned), copies timed
    e2e = None
    if not args.no_e2e:
        m0_h = torch.from_numpy(m0).pin_memory()
        m1_h = torch.from_numpy(m1).pin_memory()
        v_h = torch.zeros((3,) + grid).pin_memory()
        ctx2 = ctx
        if pg:
            pg.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        pts_e = 0.0
        for _ in range(args.steps):
            v_h.zero_()
            ctx2.set_images(m0_h.numpy(), m1_h.numpy())
            st, rep = ctx2.register(v_h.numpy())
            pts_e += rep["interp_points"]
        torch.cuda.synchronize()
        te = time.perf_counter() - t0
        te, pts_e = aggregate_ranks(te, pts_e, pg, dev)
        e2e = {"value": pts_e / te / 1e9, "unit": UNIT, "h2d_bytes_per_step": 4 * N * 5,
               "d2h_bytes_per_step": 4 * N * 3, "ms_per_step": 1e3 * te / args.steps}

    # the same registration with the other preconditioner (not timed with the
    # headline: one warm-up and one timed solve, device-synchronised wall clock)
    other = None
    if rank == 0 and world == 1 and not args.no_other_precond:
        alt = "spectral" if args.precond == "two-level" else "two-level"
        ctx.set_images(m0_d, m1_d)
        ctx.set_opts(precond=claire.PRECOND_TWO_LEVEL if alt == "two-level" else claire.PRECOND_SPECTRAL)
        for _ in range(2):
            v.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st_a, rep_a = ctx.register(v)
            torch.cuda.synchronize()
            ta = time.perf_counter() - t0
        ctx.set_opts(precond=claire.PRECOND_TWO_LEVEL if args.precond == "two-level" else claire.PRECOND_SPECTRAL)
        other = {"precond": alt, "time_to_tol_s": ta, "gn_iters": rep_a["gn_iters"],
                 "pcg_iters_total": rep_a["pcg_iters_total"], "inner_pcg_iters": rep_a["pc_inner_iters_total"],
                 "gnorm_rel": rep_a["gnorm_rel"], "J": rep_a["J"], "r": rep_a["r"], "status": rep_a["status"]}

    # the metric's second form: FP16 storage + learned warm start on the same
    # workload, stopped at the plain run's absolute gradient (outside the
    # headline's timed region; its own warm-up, CUDA events per solve)
    mixed = None
    if rank == 0 and world == 1 and not args.no_mixed_learned:
        mixed = mixed_learned_leg(args, ctx, claire, grid, dev, stream, m0, m1, m0_d, m1_d)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        m0_64 = m0.astype(np.float64)
        m1_64 = m1.astype(np.float64)
        runs = [oracle_sample(grid, m0_64, m1_64, args.beta) for _ in range(3)]
        s, q = sorted(runs)[1]  # median of three runs
        cpu = {"value": q / s / 1e9, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
               "cpu_model": cpu_model(), "runs_s": [r[0] for r in runs],
               "sample": "one oracle gradient evaluation (state + adjoint solve, nt=4) of the "
                         "same %d^3 workload, median of 3 runs (%.1f s)" % (args.n, s)}

    r0 = reps[0]
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * tmax / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if args.storage == "f32" else "f32 math, %s storage" % args.storage,
            "data": "synthetic", "config": config_dict(args, world),
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": ck,
            "gpu_launches": launches,
            "registration": {"gn_iters": r0["gn_iters"], "pcg_iters_total": r0["pcg_iters_total"],
                             "gnorm_rel": r0["gnorm_rel"], "r": r0["r"], "J": r0["J"],
                             "detj_min": r0["detj_min"], "detj_max": r0["detj_max"],
                             "cfl": r0["cfl"], "status": r0["status"],
                             "time_to_tol_s": tmax / args.steps,
                             "precond": args.precond},
            "registration_other_precond": other,
            "registration_mixed_learned": mixed,
            "kernels": {s["name"]: {"launches": s["launches"], "ms": 1e3 * s["seconds"],
                                    "GBs": (s["bytes"] / s["seconds"] / 1e9) if s["seconds"] else None}
                        for s in stats if s["launches"] > 0},
        }
        print(json.dumps(line))
    ctx.close()
    if pg:
        pg.destroy_process_group()


def mixed_learned_leg(args, ctx32, claire, grid, dev, stream, m0, m1, m0_d, m1_d):
    """Time to tolerance of FP16 storage + the learned warm start against the
    plain FP32 registration from v = 0 on the same images.  The network
    (weights written by paper_2209_08189_gb300/train_warmstart.py) sees the
    images sampled to its grid; its velocity is prolonged spectrally.  Both
    solves stop at the same absolute gradient, gtol |g(v = 0)| of the FP32
    context.  Timed with CUDA events from the prediction to the returned
    velocity, after one warm-up solve; final J and mismatch are also evaluated
    by the FP64 oracle at every returned velocity (outside the timing).  A
    third arm runs FP16 + warm start with the two-level zero-velocity
    preconditioner instead of S^-1; with a network that has the
    preconditioner head, a fourth adds its coarse preconditioner weight
    (claire_set_pc_weight) to the third."""
    import torch
    import oracle
    if args.weights is None:
        wdir = os.path.join(ROOT, "paper_2209_08189_gb300", "weights")
        pcf = os.path.join(wdir, "unet_warmstart_pc_128.npz")
        args.weights = pcf if os.path.exists(pcf) else os.path.join(wdir, "unet_warmstart_128.npz")
    if not os.path.exists(args.weights):
        return {"unavailable": "no trained weights at %s (python -m paper_2209_08189_gb300.train_warmstart)"
                               % os.path.relpath(args.weights, ROOT)}
    from paper_2209_08189_gb300 import net, warmstart
    st = stream.cuda_stream
    N = int(np.prod(grid))
    zero = torch.zeros((3,) + grid, device=dev)
    g = torch.empty((3,) + grid, device=dev)
    ctx32.set_opts(g0_ref=0.0)
    ctx32.gradient(zero, g)
    g0 = math.sqrt(claire.claire_dot(ctx32.handle, g, g, 3 * N))
    # plain FP32 from zero (the headline's solve, timed the same way here)
    v32 = torch.zeros((3,) + grid, device=dev)

    def timed(fn):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        rep = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) * 1e-3, rep

    def plain():
        v32.zero_()
        return ctx32.register(v32, check=False)[1]

    u = net.UNet.from_file(args.weights, stream=st)
    ws = warmstart.WarmStart(u, int(u.meta["n_net"]))
    ctx16 = claire.Context(grid, args.beta, 4, stream=st, beta_w=1e-4, gtol=5e-2, max_gn=50, max_pcg=50,
                           storage=claire.STORAGE_F16, g0_ref=g0, spectral_iterate=args.spectral_iterate)
    ctx16.set_images(m0_d, m1_d)
    v16 = torch.zeros((3,) + grid, device=dev)

    pc_net = bool(u.pc_head)
    wc = torch.empty(tuple(s // 2 for s in grid), device=dev) if pc_net else None  # coarse grid (pc_coarse 2)
    use_pcw = [False]

    def learned():
        ws.predict(m0_d, m1_d, v16)
        if use_pcw[0]:
            ctx16.set_pc_weight(ws.pc_weight(wc))
        return ctx16.register(v16, check=False)[1]

    reps = max(1, min(args.steps, 3))
    res = {}
    p = oracle.Params(nt=4, beta_v=args.beta, beta_w=1e-4)
    m0_64, m1_64 = m0.astype(np.float64), m1.astype(np.float64)
    # the third arm adds the paper's two-level zero-velocity preconditioner to
    # FP16 storage + the warm start (the fastest combination to the same tolerance)
    arms = [("plain_fp32", plain, None, False), ("fp16_learned", learned, claire.PRECOND_SPECTRAL, False),
            ("fp16_learned_two_level", learned, claire.PRECOND_TWO_LEVEL, False)]
    if pc_net:  # the network's coarse preconditioner correction on top of the two-level preconditioner
        arms.append(("fp16_learned_two_level_pcw", learned, claire.PRECOND_TWO_LEVEL, True))
    for name, fn, pc, pcw in arms:
        use_pcw[0] = pcw
        if pc is not None:
            ctx16.set_opts(precond=pc)
            ctx16.set_pc_weight(None)
        fn()  # warm-up
        times, rep = [], None
        for _ in range(reps):
            t, rep = timed(fn)
            times.append(t)
        res[name] = {"time_to_tol_s": float(np.mean(times)), "runs": reps, "status": rep["status"],
                     "gn_iters": rep["gn_iters"], "pcg_iters_total": rep["pcg_iters_total"],
                     "gnorm_rel_to_plain_g0": rep["gnorm_rel"], "J": rep["J"], "mismatch": rep["mismatch"]}
        if pc == claire.PRECOND_TWO_LEVEL:
            res[name]["inner_pcg_iters"] = rep["pc_inner_iters_total"]
        vv = v32 if fn is plain else v16
        J_o, mis_o, _ = oracle.objective(vv.cpu().numpy().astype(np.float64), m0_64, m1_64, p)
        res[name]["oracle_J"] = J_o
        res[name]["oracle_mismatch"] = mis_o
    vg = torch.empty_like(v16)
    ws.predict(m0_d, m1_d, vg)
    res["fp16_learned"]["mismatch_at_guess"] = ctx32.objective(vg)[1]
    res["plain_fp32"]["mismatch_at_zero"] = ctx32.objective(zero)[1]
    res["speedup"] = res["plain_fp32"]["time_to_tol_s"] / res["fp16_learned"]["time_to_tol_s"]
    res["speedup_two_level"] = res["plain_fp32"]["time_to_tol_s"] / res["fp16_learned_two_level"]["time_to_tol_s"]
    if pc_net:
        res["speedup_two_level_pcw"] = (res["plain_fp32"]["time_to_tol_s"] /
                                        res["fp16_learned_two_level_pcw"]["time_to_tol_s"])
        wstat = wc.cpu().numpy()
        res["fp16_learned_two_level_pcw"]["weight_stats"] = {
            "min": float(wstat.min()), "mean": float(wstat.mean()), "max": float(wstat.max())}
    res["network"] = {"weights": os.path.relpath(args.weights, ROOT), "n_net": u.meta["n_net"],
                      "params": u.num_params(), "training": u.meta.get("training")}
    res["stop"] = "both at |g| <= 5e-2 |g(v=0)| of the FP32 context (%.6g)" % g0
    ctx16.close()
    return res


def run_mixed_report(args):
    """Blob template (8 Gaussian blobs + sine, clipped) with a velocity of 6
    random modes |k| <= 16 per component, max |v| = 0.5, at n^3; one
    registration per storage type; errors against the FP64 oracle evaluated
    at each returned velocity on the same FP32 images."""
    import torch
    import oracle
    from paper_2209_08189_gb300 import claire, synth
    import __graft_entry__ as entry
    entry.build()
    n = args.n if args.n != 256 else 512
    grid = (n, n, n)
    dev = torch.device("cuda", 0)
    m0 = synth.blob_template(grid, seed=0).astype(np.float32)
    vstar = synth.mode_velocity(grid, seed=0, nmodes=6, kmax=16, vmax=0.5).astype(np.float32)
    ctx = claire.Context(grid, args.beta, 4, stream=torch.cuda.current_stream().cuda_stream)
    m1d = torch.empty(grid, device=dev)
    ctx.transport(torch.from_numpy(vstar).to(dev), torch.from_numpy(m0).to(dev), m1d, claire.TRANSPORT_FWD)
    m1 = m1d.cpu().numpy()
    ctx.close()
    p = oracle.Params(nt=4, beta_v=args.beta, beta_w=1e-4)
    m0_64, m1_64 = m0.astype(np.float64), m1.astype(np.float64)
    out = {"workload": "blob template, 6 modes |k|<=16 per component, max|v|=0.5, %d^3, nt=4, "
                       "tricubic, beta_v=%g, gtol 5e-2" % (n, args.beta), "runs": {}}
    vel = {}
    for name, sto in (("f32", claire.STORAGE_F32), ("f16", claire.STORAGE_F16), ("bf16", claire.STORAGE_BF16)):
        ctx = claire.Context(grid, args.beta, 4, stream=torch.cuda.current_stream().cuda_stream, beta_w=1e-4,
                             gtol=5e-2, max_gn=50, max_pcg=50, storage=sto)
        ctx.set_images(torch.from_numpy(m0).to(dev), torch.from_numpy(m1).to(dev))
        v = torch.zeros((3,) + grid, device=dev)
        ctx.register(v)  # warm-up
        v.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st, rep = ctx.register(v)
        torch.cuda.synchronize()
        secs = time.perf_counter() - t0
        vh = v.cpu().numpy()
        vel[name] = vh
        ctx.close()
        v64 = vh.astype(np.float64)
        J_o, mis_o, _ = oracle.objective(v64, m0_64, m1_64, p)
        dj = oracle.detj(v64, p)
        out["runs"][name] = {
            "time_to_tol_s": secs, "gn_iters": rep["gn_iters"], "pcg_iters": rep["pcg_iters_total"],
            "gnorm_rel": rep["gnorm_rel"], "interp_gpts_s": rep["interp_points"] / secs / 1e9,
            "mismatch_rel_err_vs_oracle": abs(rep["mismatch"] - mis_o) / mis_o,
            "J_rel_err_vs_oracle": abs(rep["J"] - J_o) / J_o,
            "detj_min": rep["detj_min"], "detj_max": rep["detj_max"],
            "detj_rel_err_vs_oracle": max(abs(rep["detj_min"] - dj.min()) / dj.min(),
                                          abs(rep["detj_max"] - dj.max()) / dj.max()),
            "r": rep["r"]}
        del dj
    ref = vel["f32"].astype(np.float64)
    for name in ("f16", "bf16"):
        out["runs"][name]["velocity_rel_l2_vs_f32"] = float(
            np.linalg.norm(vel[name] - ref) / np.linalg.norm(ref))
    # transport of m0 by the mixed velocity: GPU FP32 kernel vs oracle
    ctx = claire.Context(grid, args.beta, 4, stream=torch.cuda.current_stream().cuda_stream)
    mt = torch.empty(grid, device=dev)
    ctx.transport(torch.from_numpy(vel["f16"]).to(dev), torch.from_numpy(m0).to(dev), mt, claire.TRANSPORT_FWD)
    mo = oracle.transport(m0_64, vel["f16"].astype(np.float64), p)
    out["transport_rel_l2_vs_oracle"] = float(np.linalg.norm(mt.cpu().numpy() - mo) / np.linalg.norm(mo))
    ctx.close()
    print(json.dumps(out))


def run_warmstart_report(args):
    """Time to tolerance on the clinical-size workload: plain FP32 from v = 0
    against FP16 storage + learned warm start.  The network (4-level U-Net,
    BF16) is trained at n/2 on pairs the method generates (label and blob
    templates advected by band-limited velocities |k| <= 8, max|v| in
    [0.3, 1.2], noise sigma 0.02); at n the images are sampled to n/2, the
    prediction is prolonged spectrally.  Both solves stop at the same absolute
    gradient, 5e-2 |g(v=0)|; the warm-started timing includes the prediction
    and the gradient at v = 0.  Final J and mismatch are re-evaluated by the
    FP64 oracle at each returned velocity."""
    import torch
    import oracle
    import __graft_entry__ as entry
    entry.build()
    from paper_2209_08189_gb300 import claire, synth, net, warmstart
    n = args.n
    nn_ = n // 2
    dev = torch.device("cuda", 0)
    st = torch.cuda.current_stream().cuda_stream
    out = {"workload": "%d^3 nested-label template, band-limited v* |k|<=8 max|v|=1, noise 0.02, nt=4, "
                       "tricubic, beta_v=%g, beta_w=1e-4, gtol 5e-2 of |g(v=0)|" % (n, args.beta)}
    t0 = time.perf_counter()
    src = warmstart.PairSource(nn_, n_templates=24, n_velocities=48, kmax=(4, 8), vmax=(0.3, 1.2), noise=0.02,
                               seed=0)
    out["pair_pool_s"] = time.perf_counter() - t0
    u = net.UNet(seed=0, stream=st)
    t0 = time.perf_counter()
    hist = warmstart.train(u, src, steps=args.ws_steps, batch=4, lr=1e-3, lr_final=1e-4, wv=1.0, wm=1.0,
                           log_every=max(1, args.ws_steps // 10))
    out["training"] = {"grid": nn_, "steps": args.ws_steps, "batch": 4, "pairs": 4 * args.ws_steps,
                       "params": u.num_params(), "seconds": time.perf_counter() - t0,
                       "history": [{"step": h[0], "Lv": h[1], "mismatch_rel": h[2]} for h in hist]}
    src.ctx.close()
    grid, base, vstar = workload(n)
    N = int(np.prod(grid))
    ctx32 = claire.Context(grid, args.beta, 4, stream=st, beta_w=1e-4, gtol=5e-2, max_gn=50, max_pcg=50)
    ctx16 = claire.Context(grid, args.beta, 4, stream=st, beta_w=1e-4, gtol=5e-2, max_gn=50, max_pcg=50,
                           storage=claire.STORAGE_F16)
    base_d = torch.from_numpy(base.astype(np.float32)).to(dev)
    m1c = torch.empty(grid, device=dev)
    ctx32.transport(torch.from_numpy(vstar.astype(np.float32)).to(dev), base_d, m1c, claire.TRANSPORT_FWD)
    m1 = synth.add_noise(m1c.cpu().numpy().astype(np.float64), 0.02, seed=1).astype(np.float32)
    m0 = synth.add_noise(base, 0.02, seed=0).astype(np.float32)
    m0_d = torch.from_numpy(m0).to(dev)
    m1_d = torch.from_numpy(m1).to(dev)
    ctx32.set_images(m0_d, m1_d)
    ctx16.set_images(m0_d, m1_d)
    ws = warmstart.WarmStart(u, nn_)
    zero = torch.zeros((3,) + grid, device=dev)
    g = torch.empty((3,) + grid, device=dev)

    def solve(ctx, learned, pc=claire.PRECOND_SPECTRAL):
        v = torch.zeros((3,) + grid, device=dev)
        ctx.set_opts(precond=pc)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        split = {}
        if learned:
            ws.predict(m0_d, m1_d, v)
            torch.cuda.synchronize()
            split["predict_s"] = time.perf_counter() - t0
            ctx.gradient(zero, g)
            g0 = math.sqrt(claire.claire_dot(ctx.handle, g, g, 3 * N))
            ctx.set_opts(g0_ref=g0)
            split["g0_s"] = time.perf_counter() - t0 - split["predict_s"]
        else:
            ctx.set_opts(g0_ref=0.0)
        status, rep = ctx.register(v)
        torch.cuda.synchronize()
        secs = time.perf_counter() - t0
        return secs, rep, v, split

    runs = {}
    TL = claire.PRECOND_TWO_LEVEL
    for name, ctx, learned, pc in (("fp32_zero", ctx32, False, 0), ("fp16_zero", ctx16, False, 0),
                                   ("fp32_learned", ctx32, True, 0), ("fp16_learned", ctx16, True, 0),
                                   ("fp32_zero_two_level", ctx32, False, TL),
                                   ("fp16_learned_two_level", ctx16, True, TL)):
        solve(ctx, learned, pc)  # warm-up
        secs, rep, v, split = solve(ctx, learned, pc)
        runs[name] = {"time_to_tol_s": secs, "gn_iters": rep["gn_iters"], "pcg_iters": rep["pcg_iters_total"],
                      "inner_pcg_iters": rep["pc_inner_iters_total"],
                      "J": rep["J"], "mismatch": rep["mismatch"], "r": rep["r"], "gnorm_rel_to_own_g0":
                      rep["gnorm_rel"], "detj_min": rep["detj_min"], "detj_max": rep["detj_max"], **split}
        runs[name]["_v"] = v.cpu().numpy()
    vw = torch.empty((3,) + grid, device=dev)
    ws.predict(m0_d, m1_d, vw)
    out["guess"] = {"mismatch_at_guess": ctx32.objective(vw)[1], "mismatch_at_zero": ctx32.objective(zero)[1]}
    p = oracle.Params(nt=4, beta_v=args.beta, beta_w=1e-4)
    m0_64, m1_64 = m0.astype(np.float64), m1.astype(np.float64)
    for name in ("fp32_zero", "fp16_learned", "fp16_learned_two_level"):
        J_o, mis_o, _ = oracle.objective(runs[name]["_v"].astype(np.float64), m0_64, m1_64, p)
        runs[name]["oracle_J"] = J_o
        runs[name]["oracle_mismatch"] = mis_o
    for r in runs.values():
        r.pop("_v")
    out["runs"] = runs
    a, b = runs["fp32_zero"], runs["fp16_learned"]
    out["speedup_fp16_learned_vs_fp32_zero"] = a["time_to_tol_s"] / b["time_to_tol_s"]
    out["oracle_J_rel_diff_learned_vs_plain"] = (b["oracle_J"] - a["oracle_J"]) / a["oracle_J"]
    out["oracle_mismatch_rel_diff_learned_vs_plain"] = (b["oracle_mismatch"] - a["oracle_mismatch"]) / \
        a["oracle_mismatch"]
    c2 = runs["fp16_learned_two_level"]
    out["speedup_fp16_learned_two_level_vs_fp32_zero"] = a["time_to_tol_s"] / c2["time_to_tol_s"]
    out["oracle_J_rel_diff_learned_two_level_vs_plain"] = (c2["oracle_J"] - a["oracle_J"]) / a["oracle_J"]
    out["oracle_mismatch_rel_diff_learned_two_level_vs_plain"] = (c2["oracle_mismatch"] - a["oracle_mismatch"]) / \
        a["oracle_mismatch"]
    print(json.dumps(out))


def run_precond_report(args):
    """Time to tolerance of the bench workload at --n with the spectral
    preconditioner S^{-1} and the paper's two-level zero-velocity one
    (coarse grid n/2, inner PCG to 1e-1, flexible outer PCG), FP32 and FP16
    storage, from v = 0 (one warm-up solve each).  J and the mismatch at every
    returned velocity are re-evaluated by the FP64 oracle."""
    import torch
    import oracle
    import __graft_entry__ as entry
    entry.build()
    from paper_2209_08189_gb300 import claire, synth
    dev = torch.device("cuda", 0)
    st = torch.cuda.current_stream().cuda_stream
    grid, base, vstar = workload(args.n)
    out = {"workload": "%d^3 nested-label template, band-limited v* |k|<=8 max|v|=1, noise 0.02, nt=4, "
                       "tricubic, beta_v=%g, beta_w=1e-4, gtol 5e-2" % (args.n, args.beta)}
    ctxs = {}
    for sto in ("f32", "f16"):
        ctxs[sto] = claire.Context(grid, args.beta, 4, stream=st, beta_w=1e-4, gtol=5e-2, max_gn=50, max_pcg=50,
                                   storage=claire.STORAGE_F32 if sto == "f32" else claire.STORAGE_F16)
    base_d = torch.from_numpy(base.astype(np.float32)).to(dev)
    m1c = torch.empty(grid, device=dev)
    ctxs["f32"].transport(torch.from_numpy(vstar.astype(np.float32)).to(dev), base_d, m1c, claire.TRANSPORT_FWD)
    m1 = synth.add_noise(m1c.cpu().numpy().astype(np.float64), 0.02, seed=1).astype(np.float32)
    m0 = synth.add_noise(base, 0.02, seed=0).astype(np.float32)
    m0_d = torch.from_numpy(m0).to(dev)
    m1_d = torch.from_numpy(m1).to(dev)
    for c in ctxs.values():
        c.set_images(m0_d, m1_d)
    p = oracle.Params(nt=4, beta_v=args.beta, beta_w=1e-4)
    m0_64, m1_64 = m0.astype(np.float64), m1.astype(np.float64)
    def solve(ctx, timing=0):
        for _ in range(2):  # warm-up, then timed
            v = torch.zeros((3,) + grid, device=dev)
            ctx.set_opts(timing=timing)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            status, rep = ctx.register(v)
            torch.cuda.synchronize()
            secs = time.perf_counter() - t0
        ctx.set_opts(timing=0)
        return secs, rep, v

    runs = {}
    # (storage, preconditioner, coarse ratio, inner tolerance)
    for sto, pc, coarse, tol in (("f32", "spectral", 2, 0.1), ("f32", "two-level", 2, 0.1),
                                 ("f16", "two-level", 2, 0.1), ("f32", "two-level", 4, 0.1),
                                 ("f32", "two-level", 2, 0.2)):
        ctx = ctxs[sto]
        ctx.set_opts(precond=claire.PRECOND_TWO_LEVEL if pc == "two-level" else claire.PRECOND_SPECTRAL,
                     pc_coarse=coarse, pc_tol=tol)
        secs, rep, v = solve(ctx)
        J_o, mis_o, _ = oracle.objective(v.cpu().numpy().astype(np.float64), m0_64, m1_64, p)
        name = "%s_%s" % (sto, pc) + ("" if (coarse, tol) == (2, 0.1) else "_coarse%d_tol%g" % (coarse, tol))
        runs[name] = {
            "time_to_tol_s": secs, "status": rep["status"], "gn_iters": rep["gn_iters"],
            "pcg_iters": rep["pcg_iters_total"], "pcg_per_gn": rep["pcg_iters"],
            "inner_pcg_iters": rep["pc_inner_iters_total"], "gnorm_rel": rep["gnorm_rel"], "J": rep["J"],
            "r": rep["r"], "detj_min": rep["detj_min"], "detj_max": rep["detj_max"], "oracle_J": J_o,
            "oracle_mismatch": mis_o}
    out["runs"] = runs
    # phase split with per-launch CUDA-event timing (adds launch overhead)
    phases = {}
    for pc in ("spectral", "two-level"):
        ctx = ctxs["f32"]
        ctx.set_opts(precond=claire.PRECOND_TWO_LEVEL if pc == "two-level" else claire.PRECOND_SPECTRAL,
                     pc_coarse=2, pc_tol=0.1)
        secs, rep, _ = solve(ctx, timing=2)
        phases[pc] = {"total_s": secs, **{k: v for k, v in rep["t_phase_s"].items()}}
    out["phases_timed"] = phases
    a = runs["f32_spectral"]
    for k in ("f32_two-level", "f16_two-level"):
        b = runs[k]
        out["speedup_%s_vs_f32_spectral" % k] = a["time_to_tol_s"] / b["time_to_tol_s"]
        out["oracle_J_rel_diff_%s" % k] = (b["oracle_J"] - a["oracle_J"]) / a["oracle_J"]
        out["oracle_mismatch_rel_diff_%s" % k] = (b["oracle_mismatch"] - a["oracle_mismatch"]) / a["oracle_mismatch"]
    print(json.dumps(out))


def run_pc_weight_report(args):
    """Coarse preconditioner correction on the clinical-size 256^3 workload:
    FP16 storage, the two-level zero-velocity preconditioner (coarse 128^3)
    and the warm start of the network with the preconditioner head, with the
    coarse weight w of its data term set to: none (w = 1, the paper's
    operator); the network's prediction; the least-squares fit of the data
    term (claire_net_pcw_stats, 8 band-limited probes |k| <= 6, pooled over
    2^3 cells) at v* and at the warm start; and constants.  Constants also
    from v = 0 and at beta_v 1e-3.  Each run: one warm-up solve, then one timed
    (host wall clock around synchronised calls); all stop at 5e-2 |g(v = 0)|."""
    import torch
    from paper_2209_08189_gb300 import claire, synth, net, warmstart
    import __graft_entry__ as entry
    entry.build()
    dev = torch.device("cuda", 0)
    st = torch.cuda.current_stream(dev).cuda_stream
    grid, base, vstar = workload(256)
    N = int(np.prod(grid))
    nc = tuple(s // 2 for s in grid)
    f = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(dev)
    ctx32 = claire.Context(grid, 1e-2, 4, stream=st, beta_w=1e-4, gtol=5e-2, max_gn=50, max_pcg=50)
    base_d, vstar_d = f(base), f(vstar)
    m1c = torch.empty(grid, device=dev)
    ctx32.transport(vstar_d, base_d, m1c, claire.TRANSPORT_FWD)
    m1 = synth.add_noise(m1c.cpu().numpy().astype(np.float64), 0.02, seed=1)
    m0 = synth.add_noise(base, 0.02, seed=0)
    m0_d, m1_d = f(m0), f(m1)
    ctx32.set_images(m0_d, m1_d)
    zero = torch.zeros((3,) + grid, device=dev)
    gt = torch.empty_like(zero)
    ctx32.gradient(zero, gt)
    g0 = math.sqrt(claire.claire_dot(ctx32.handle, gt, gt, 3 * N))
    ctx16 = claire.Context(grid, 1e-2, 4, stream=st, beta_w=1e-4, gtol=5e-2, max_gn=50, max_pcg=50,
                           storage=claire.STORAGE_F16, g0_ref=g0, precond=claire.PRECOND_TWO_LEVEL)
    ctx16.set_images(m0_d, m1_d)
    wfile = os.path.join(ROOT, "paper_2209_08189_gb300", "weights", "unet_warmstart_pc_128.npz")
    u = net.UNet.from_file(args.weights or wfile, stream=st)
    ws = warmstart.WarmStart(u, int(u.meta["n_net"]))
    v0 = torch.empty_like(zero)
    ws.predict(m0_d, m1_d, v0)
    wl = torch.empty(nc, device=dev)
    ws.pc_weight(wl)
    L = net.lib()

    def fit(vlin, probes):
        num, den = torch.zeros(grid, device=dev), torch.zeros(grid, device=dev)
        gb, hp, sp = torch.empty_like(zero), torch.empty_like(zero), torch.empty_like(zero)
        ctx32.gradient(vlin, gt)
        ctx32.mean_state_gradient(gb)
        for q in probes:
            ctx32.hessian_matvec(q, hp)
            ctx32.spectral(q, sp, claire.SPECTRAL_REG)
            net._check(L.claire_net_pcw_stats(gb.data_ptr(), q.data_ptr(), hp.data_ptr(), sp.data_ptr(), N,
                                              num.data_ptr(), den.data_ptr(), st), "pcw_stats")
        pool = lambda x: x.reshape(nc[0], 2, nc[1], 2, nc[2], 2).sum(dim=(1, 3, 5))
        A, B = pool(den), pool(num)
        one = torch.ones_like(A)
        return torch.where(A > 0, torch.clamp(B / torch.where(A > 0, A, one), min=0.0), one).contiguous()

    def run(w, start):
        ctx16.set_pc_weight(w)
        out = None
        for _ in range(2):
            v = start.clone()
            torch.cuda.synchronize()
            t = time.perf_counter()
            _, r = ctx16.register(v, check=False)
            torch.cuda.synchronize()
            out = (time.perf_counter() - t, r, v)
        t, r, v = out
        row = {"ms": 1e3 * t, "gn": r["gn_iters"], "pcg": r["pcg_iters_total"],
               "inner": r["pc_inner_iters_total"], "gnorm_rel": r["gnorm_rel"], "J": ctx32.objective(v)[0]}
        if w is not None:
            row["w_min_mean_max"] = [float(w.min()), float(w.mean()), float(w.max())]
        return row

    probes = [f(synth.mode_velocity(grid, seed=9000 + i, nmodes=8, kmax=6, vmax=0.3)) for i in range(8)]
    out = {"workload": "256^3 clinical-size pair (bench.py default), FP16 storage, two-level (coarse 128^3), "
                       "warm start of " + os.path.relpath(args.weights or wfile, ROOT),
           "runs": {}}
    R = out["runs"]
    R["b1e-2 v0 none"] = run(None, v0)
    R["b1e-2 v0 learned"] = run(wl, v0)
    R["b1e-2 v0 fit at v*"] = run(fit(vstar_d, probes), v0)
    R["b1e-2 v0 fit at v0"] = run(fit(v0, probes), v0)
    for beta in (1e-2, 1e-3):
        claire.claire_set_beta(ctx16.handle, beta, 1e-4)
        claire.claire_set_beta(ctx32.handle, beta, 1e-4)
        for sname, start in (("v0", v0), ("zero", zero)):
            for c in (1.0, 1.5, 2.0, 3.0, 4.0, 6.0):
                R["b%g %s const %g" % (beta, sname, c)] = run(torch.full(nc, c, device=dev), start)
    print(json.dumps(out))


def run_net_report(args):
    """CUDA-event timing (mean of 10 after a warm-up) of the network kernels
    and the reverse-mode transport.  Convolution TFLOP/s count 2 * voxels *
    27 * Cin * Cout flops; bytes count each input and output activation once
    (BF16).  Peak for the fraction: the measured dense BF16 rate."""
    import torch
    import __graft_entry__ as entry
    entry.build()
    from paper_2209_08189_gb300 import claire, net, warmstart, synth
    st = torch.cuda.current_stream().cuda_stream
    peaks = {}
    pp = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pp):
        with open(pp) as f:
            peaks = json.load(f)
    bf16_peak = float(peaks.get("bf16_tflops", 1900.0))

    def timeit(fn, reps=10):
        fn()
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            fn()
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    out = {"bf16_peak_tflops": bf16_peak, "conv": {}}
    B, n = 4, 128
    for lvl, ci, co in [(0, 16, 16), (0, 48, 16), (1, 16, 32), (1, 32, 32), (1, 96, 32), (2, 32, 64), (2, 64, 64),
                        (2, 192, 64), (3, 64, 128), (3, 128, 128)]:
        D = n >> lvl
        x = (torch.randn((B, D, D, D, ci), device="cuda")).to(torch.bfloat16)
        w = (torch.randn((co, 27, ci), device="cuda") / math.sqrt(27 * ci)).to(torch.bfloat16)
        y = torch.empty((B, D, D, D, co), device="cuda", dtype=torch.bfloat16)
        X, Y = net.Act(x, 0, ci), net.Act(y, 0, co)
        t = timeit(lambda: net.conv3d(X, w, None, Y, 0.1, 1, st))
        chunks = net.wgrad_chunks(ci, co, (B, D, D, D))
        part = torch.empty(chunks * co * 27 * ci, device="cuda")
        pb = torch.empty(chunks * co, device="cuda")
        dw = torch.empty((co, 27, ci), device="cuda")
        db = torch.empty(co, device="cuda")
        tw = timeit(lambda: net.conv3d_wgrad(X, Y, chunks, part, pb, dw, db, st))
        P = B * D ** 3
        fl = 2.0 * P * 27 * ci * co
        out["conv"]["l%d_%dx%d" % (lvl, ci, co)] = {
            "voxels": P, "fwd_ms": t, "fwd_tflops": fl / t / 1e9, "fwd_frac_bf16_peak": fl / t / 1e9 / bf16_peak,
            "fwd_gbs": P * (ci + co) * 2 / t / 1e6, "wgrad_ms": tw, "wgrad_tflops": fl / tw / 1e9}
        del x, w, y, part, pb, dw, db
    src = warmstart.PairSource(128, n_templates=4, n_velocities=4, noise=0.0, seed=0)
    u = net.UNet(seed=0, stream=st)
    warmstart.train(u, src, steps=3, batch=4)
    m0, m1, vs = src.batch(4)
    out["unet_forward_ms"] = timeit(lambda: u.forward(m0, m1), 5)
    v = u.forward(m0, m1)
    dv = torch.zeros_like(v)
    out["unet_backward_ms"] = timeit(lambda: u.backward(dv), 5)
    gv = torch.empty((3, 128, 128, 128), device="cuda")
    out["vjp_128_ms"] = timeit(lambda: src.ctx.transport_vjp(v[0], m0[0], m1[0], None, gv), 5)
    t0 = time.perf_counter()
    warmstart.train(u, src, steps=10, batch=4)
    out["train_step_ms"] = (time.perf_counter() - t0) / 10 * 1e3
    src.ctx.close()
    g = (256,) * 3
    ctx = claire.Context(g, 1e-2, 4, stream=st)
    m = torch.from_numpy(synth.blob_template(g, seed=1).astype(np.float32)).cuda()
    vv = torch.from_numpy(synth.bandlimited_velocity(g, seed=2, kmax=8, vmax=1.0).astype(np.float32)).cuda()
    gb = torch.randn(g, device="cuda")
    gm = torch.empty(g, device="cuda")
    gvv = torch.empty((3,) + g, device="cuda")
    out["transport_256_ms"] = timeit(lambda: ctx.transport(vv, m, gm), 5)
    out["vjp_256_ms"] = timeit(lambda: ctx.transport_vjp(vv, m, gb, gm, gvv), 3)
    out["vjp_256_recompute_ms"] = timeit(lambda: ctx.transport_vjp(vv, m, gb, gm, gvv, recompute=True), 3)
    print(json.dumps(out))


def run_interp_report(args):
    """Micro-benchmark of the SL interpolation kernel (a2) alone.

    Fields: n^3 FP32 values (seeded uniform, the values do not change the
    work).  Displacements (grid units): (a) realistic, the RK2 characteristic
    X of the clinical-size velocity v* (band-limited |k| <= 8, max |v| = 1,
    drawn at 64^3 and prolonged spectrally; nt = 4, so CFL = 10 n / 256);
    (b) zero; (c) uniform random in +-CFL per component (no spatial
    coherence: every tile takes the global-memory path).  1 field
    (claire_interp, 20 B/pt) and 4 fields sharing the displacement
    (claire_interp_fields, (8*4 + 12) / 4 = 11 B/pt per field).  Each case:
    3 warm-up launches, then the mean of 10 launches timed with CUDA events on
    the launching stream; the inputs (>= 256 MB) exceed the 129 MB L2.
    Gpts/s counts grid points x fields; HBM fraction = algorithmic bytes / time
    / measured copy bandwidth; LSU fraction = Gpts/s / the shared-memory read
    ceiling (128 B/clk/SM x SMs x clock / (4 B x stencil size))."""
    import torch
    import __graft_entry__ as entry
    entry.build()
    from paper_2209_08189_gb300 import claire, synth
    dev = torch.device("cuda", 0)
    st = torch.cuda.current_stream(dev)
    peak, peak_src = measured_peaks()
    props = torch.cuda.get_device_properties(dev)
    sizes = [int(x) for x in args.interp_sizes.split(",") if x]
    gen = torch.Generator(device=dev)
    gen.manual_seed(0)
    v64 = torch.from_numpy(synth.bandlimited_velocity((64, 64, 64), seed=0, kmax=8, vmax=1.0).astype(np.float32)).to(dev)
    clocks = ClockSampler(0)
    clocks.start()
    rows = []
    for n in sizes:
        grid = (n, n, n)
        N = n ** 3
        ctx = claire.Context(grid, 1e-2, 4, stream=st.cuda_stream, kernels_only=1)
        f = torch.rand((4,) + grid, device=dev, generator=gen)
        out = torch.empty((4,) + grid, device=dev)
        v = torch.empty((3,) + grid, device=dev)
        claire.claire_resample(v64, (64, 64, 64), v, grid, 3, claire.RESAMPLE_SPECTRAL, st.cuda_stream)
        d_real = torch.empty((3,) + grid, device=dev)
        ctx.backtrace(v, d_real, 1)
        del v
        cfl = 10.0 * n / 256.0
        disps = {"realistic": d_real, "zero": torch.zeros((3,) + grid, device=dev),
                 "random": (torch.rand((3,) + grid, device=dev, generator=gen) * 2.0 - 1.0) * cfl}
        for kind, d in disps.items():
            for order in (3, 1):
                for nf in (1, 4):
                    def call():
                        if nf == 1:
                            claire.claire_interp(ctx.handle, f[0], d, out[0], order)
                        else:
                            claire.claire_interp_fields(ctx.handle, f, nf, d, out, order)
                    for _ in range(3):
                        call()
                    claire.claire_gather_fallback_tiles(reset=True)
                    reps = 10
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    torch.cuda.synchronize()
                    e0.record(st)
                    for _ in range(reps):
                        call()
                    e1.record(st)
                    torch.cuda.synchronize()
                    t = e0.elapsed_time(e1) * 1e-3 / reps
                    glob = claire.claire_gather_fallback_tiles(reset=True) / reps
                    tiles = (-(-n // 4)) * (-(-n // 8)) * (-(-n // 32))
                    bpp = (8.0 * nf + 12.0) / nf
                    gpts = N * nf / t / 1e9
                    m = 64 if order == 3 else 8
                    lsu_gpts = 128.0 * props.multi_processor_count * 2070e6 / (4.0 * m) / 1e9
                    rows.append({"n": n, "displacement": kind, "interp": "tricubic" if order == 3 else "trilinear",
                                 "fields": nf, "ms": t * 1e3, "gpts_s": gpts,
                                 "bytes_per_pt_field": bpp, "hbm_GBs": gpts * bpp,
                                 "hbm_frac": gpts * bpp / peak, "lsu_frac": gpts / lsu_gpts,
                                 "global_tile_frac": glob / tiles})
                    print("n=%4d %-9s %-9s fields=%d  %8.3f ms  %7.1f Gpts/s  HBM %5.1f %%  LSU %5.1f %%  "
                          "global tiles %5.1f %%" % (n, kind, rows[-1]["interp"], nf, t * 1e3, gpts,
                                                      100 * rows[-1]["hbm_frac"], 100 * rows[-1]["lsu_frac"],
                                                      100 * rows[-1]["global_tile_frac"]), flush=True)
        ctx.close()
        del f, out, d_real, disps
        torch.cuda.empty_cache()
    ck = clocks.stop()
    print(json.dumps({"interp_report": rows, "peak_GBs": peak, "peak_source": peak_src, "clocks": ck,
                      "lsu_ceiling_note": "128 B/clk/SM x %d SMs x 2.07 GHz / (4 B x 64 or 8 reads per point)"
                                          % props.multi_processor_count}))


def run_syn_report(args):
    """The paper's SYN experiment (Sec. 4): template = overlap counts of ten
    perturbed |Y_8^6| shapes, velocity = K trigonometric modes with amplitude
    k^-1/2, reference = the template advected by that velocity.  Per K in
    {4, 8, 12, 16}: the two-stage regularisation-parameter search (Sec. 3)
    with linear interpolation, nt = 4 at 128^3 and 8 at 256^3 (the paper's
    choices), gtol 5e-2, Jacobian bounds [0.1, 10].  Times are host wall clock
    around the synchronised search; the paper's own times (one V100) are
    context, not a target."""
    import torch
    import __graft_entry__ as entry
    entry.build()
    from paper_2209_08189_gb300 import claire, synth
    dev = torch.device("cuda", 0)
    st = torch.cuda.current_stream().cuda_stream
    paper_s = {128: {4: 15, 8: 14, 12: 14, 16: 15}, 256: {4: 110, 8: 100, 12: 94, 16: 95}}
    rows = []
    for n in [int(x) for x in args.syn_sizes.split(",") if x]:
        grid = (n, n, n)
        nt = 4 if n <= 128 else 8
        m0 = torch.from_numpy(synth.syn_template(grid, seed=0)).to(dev)
        m0.div_(float(m0.max()))  # overlap counts scaled to [0, 1]
        for K in (4, 8, 12, 16):
            ctx = claire.Context(grid, 1.0, nt, stream=st, interp=claire.INTERP_LINEAR, beta_w=1e-5, gtol=5e-2,
                                 max_gn=50, max_pcg=50, spectral_iterate=args.spectral_iterate)
            vk = torch.from_numpy(synth.syn_velocity(grid, K).astype(np.float32)).to(dev)
            m1 = torch.empty(grid, device=dev)
            ctx.transport(vk, m0, m1)
            ctx.set_images(m0, m1)
            v = torch.zeros((3,) + grid, device=dev)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            stt, rep = ctx.param_search(v)
            torch.cuda.synchronize()
            secs = time.perf_counter() - t0
            last = rep["last"]
            rows.append({"n": n, "nt": nt, "K": K, "search_s": secs, "solves": rep["solves"],
                         "beta_v": rep["beta_v"], "beta_w": rep["beta_w"], "r": last["r"],
                         "detj_min": last["detj_min"], "detj_max": last["detj_max"],
                         "gn_iters_total": int(sum(t["gn_iters"] for t in rep["trace"])),
                         "paper_v100_s": paper_s.get(n, {}).get(K)})
            print("SYN n=%d nt=%d K=%2d: search %.2f s, %d solves, beta_v %.3g beta_w %.3g, r %.3f, det %.2f..%.2f "
                  "(paper, one V100: %s s)" % (n, nt, K, secs, rep["solves"], rep["beta_v"], rep["beta_w"], last["r"],
                                                last["detj_min"], last["detj_max"], paper_s.get(n, {}).get(K)),
                  flush=True)
            ctx.close()
            del vk, m1, v
            torch.cuda.empty_cache()
    print(json.dumps({"syn_report": rows}))


def run_vjp_report(args):
    """claire_transport_vjp with CLAIRE_VJP_RECOMPUTE (states recomputed from m0
    during the backward sweep: 2 N floats instead of (nt + 1) N) at n^3, nt = 4,
    cubic Lagrange, on an FP16 low-memory context.  Inputs: the sphere template,
    a band-limited velocity (|k| <= 8, max|v| 0.5, drawn at 64^3 and prolonged),
    a seeded N(0,1) cotangent.  Checks the adjoint identity <gm0, x> = <gbar, T x>
    for a seeded random x on the full field (FP64 sums on the device), and
    times one call with CUDA events after a warm-up call."""
    import gc
    import torch
    import __graft_entry__ as entry
    entry.build()
    from paper_2209_08189_gb300 import claire, synth
    n = args.vjp_n
    grid = (n,) * 3
    N = n ** 3
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    st = stream.cuda_stream
    ctx = claire.Context(grid, 1e-2, 4, stream=st, storage=claire.STORAGE_F16, lowmem=1)
    m0, _ = synth.sphere_template(grid, seed=0)
    m0 = torch.from_numpy(m0).to(dev)
    v64 = torch.from_numpy(synth.bandlimited_velocity((64,) * 3, seed=0, kmax=8, vmax=0.5).astype(np.float32)).to(dev)
    v = torch.empty((3,) + grid, device=dev)
    claire.claire_resample(v64, (64,) * 3, v, grid, 3, claire.RESAMPLE_SPECTRAL, st)
    claire.lib().claire_resample_release()
    gen = torch.Generator(device=dev)
    gen.manual_seed(0)
    gbar = torch.randn(grid, device=dev, generator=gen)
    x = torch.randn(grid, device=dev, generator=gen)
    gm0 = torch.empty(grid, device=dev)
    gv = torch.empty((3,) + grid, device=dev)
    torch.cuda.synchronize()
    ctx.transport_vjp(v, m0, gbar, gm0, gv, recompute=True)  # warm-up (allocates the scratch)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    ctx.transport_vjp(v, m0, gbar, gm0, gv, recompute=True)
    e1.record(stream)
    torch.cuda.synchronize()
    t_vjp = e0.elapsed_time(e1) * 1e-3
    free, total = torch.cuda.mem_get_info()
    used = (total - free) / 1e9
    tx = torch.empty(grid, device=dev)
    ctx.transport(v, x, tx)
    lhs = claire.claire_dot(ctx.handle, gm0, x, N)
    rhs = claire.claire_dot(ctx.handle, gbar, tx, N)
    nrm = math.sqrt(claire.claire_dot(ctx.handle, gm0, gm0, N) * claire.claire_dot(ctx.handle, x, x, N))
    gvn = math.sqrt(claire.claire_dot(ctx.handle, gv, gv, 3 * N))
    out = {"n": n, "nt": 4, "interp": "cubic Lagrange", "recompute": True, "vjp_s": t_vjp,
           "device_gb_in_use": used, "adjoint_identity_rel": abs(lhs - rhs) / nrm, "lhs": lhs, "rhs": rhs,
           "gv_norm": gvn, "gv_finite": bool(math.isfinite(gvn)),
           "scratch_gb": (2 * N * 4 + N * 8) / 1e9}
    ctx.close()
    print(json.dumps(out))


def run_large_report(args):
    """Largest single-GPU registration.  Workload: three nested spheres with a
    blob texture (synth.sphere_template, labels 1..3) at n^3, advected by a
    band-limited velocity |k| <= 8, max|v| = --large-vmax (drawn at 64^3, prolonged
    spectrally) to give the reference; labels follow the same velocity
    (indicator transport, threshold 1/2).  nt = 4, tricubic, beta_v = 1e-2,
    beta_w = 1e-4, gtol 5e-2 of |g(v=0)|.  Both solves keep no stored state
    gradients (lowmem).  Memory is the device memory in use (cudaMemGetInfo)
    after each context is created.  Oracle parity at n^3 is checked on 10^6
    sampled points of one backtrace and one interpolation (FP64)."""
    import gc
    import torch
    import oracle
    import __graft_entry__ as entry
    entry.build()
    from paper_2209_08189_gb300 import claire, synth, net, warmstart
    n = args.large_n
    grid = (n, n, n)
    N = n ** 3
    dev = torch.device("cuda", 0)
    st = torch.cuda.current_stream().cuda_stream
    out = {"workload": "%d^3 nested spheres + blob texture (3 labels), band-limited v* |k|<=8 max|v|=%g, nt=4, "
                       "tricubic, beta_v=%g, beta_w=1e-4, gtol 5e-2 of |g(v=0)|, at most 50 GN iterations"
                       % (n, args.large_vmax, args.beta)}

    def used_gb():
        free, total = torch.cuda.mem_get_info()
        return (total - free) / 1e9

    def flush():
        gc.collect()
        torch.cuda.empty_cache()
        claire.lib().claire_resample_release()  # cached plans and spectra of the grid transfers

    t0 = time.perf_counter()
    m0, labels = synth.sphere_template(grid, seed=0)
    v64 = synth.bandlimited_velocity((64, 64, 64), seed=0, kmax=8, vmax=args.large_vmax).astype(np.float32)
    out["generate_s"] = time.perf_counter() - t0
    # warm-start network, trained at 128^3 on method-generated pairs (sphere and blob families)
    t0 = time.perf_counter()
    src = warmstart.PairSource(128, n_templates=24, n_velocities=48, kmax=(4, 8), vmax=(0.3, 1.2), noise=0.0,
                               seed=1, families=("label", "blob"))
    u = net.UNet(seed=0, stream=st)
    hist = warmstart.train(u, src, steps=args.ws_steps, batch=4, lr=1e-3, lr_final=1e-4, log_every=0)
    src.ctx.close()
    del src
    flush()
    out["training_s"] = time.perf_counter() - t0

    # ---- FP16 + lowmem context: reference image and labels, learned run, sampled
    # oracle parity, registrations of sampled images; device tensors are kept
    # few because the context takes most of the memory
    ctx = claire.Context(grid, args.beta, 4, stream=st, beta_w=1e-4, gtol=5e-2, max_gn=50, max_pcg=50,
                         storage=claire.STORAGE_F16, lowmem=1, wall_limit_s=1200,
                         spectral_iterate=args.spectral_iterate,
                         precond=claire.PRECOND_TWO_LEVEL if args.large_precond == "two-level"
                         else claire.PRECOND_SPECTRAL, pc_coarse=args.large_pc_coarse)
    out["fp16_lowmem_device_gb"] = used_gb()
    out["learned_run_precond"] = args.large_precond
    vstar = torch.empty((3,) + grid, device=dev)
    claire.claire_resample(torch.from_numpy(v64).to(dev), (64, 64, 64), vstar, grid, 3, claire.RESAMPLE_SPECTRAL,
                           st)
    m0_d = torch.from_numpy(m0).to(dev)
    m1_d = torch.empty(grid, device=dev)
    ctx.transport(vstar, m0_d, m1_d)
    m1 = m1_d.cpu().numpy()

    def carried_labels(v):
        """Indicators of the labels of m0 carried by v (transported), on the host."""
        buf = torch.empty(grid, device=dev)
        tmp = torch.empty(grid, device=dev)
        res = []
        for k in (1, 2, 3):
            buf.copy_(torch.from_numpy((labels == k).astype(np.float32)))
            ctx.transport(v, buf, tmp)
            res.append(tmp.cpu().numpy())
        del buf, tmp
        flush()
        return res

    ref = carried_labels(vstar)

    def dice_of(lab):
        """claire_dice of each label indicator against the reference's (threshold 1/2)."""
        a = torch.empty(grid, device=dev)
        b = torch.empty(grid, device=dev)
        res = []
        for x, y in zip(lab, ref):
            a.copy_(torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)))
            b.copy_(torch.from_numpy(y))
            res.append(ctx.dice(a, b))
        del a, b
        flush()
        return res

    def dice(v):
        return dice_of(carried_labels(v))

    out["dice_before"] = dice_of([(labels == k).astype(np.float32) for k in (1, 2, 3)])
    ctx.set_images(m0_d, m1_d)   # the context keeps its own (FP16) copies
    del vstar, m1_d, m0_d
    flush()

    def sampled(nc):
        """Images sampled by nearest neighbour to nc^3 (every (n/nc)-th node), on the device."""
        r = n // nc
        return (torch.from_numpy(np.ascontiguousarray(m0[::r, ::r, ::r])).to(dev),
                torch.from_numpy(np.ascontiguousarray(m1[::r, ::r, ::r])).to(dev))

    runs = {}
    # learned warm start + FP16 storage
    v = torch.zeros((3,) + grid, device=dev)
    g = torch.empty((3,) + grid, device=dev)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ctx.gradient(v, g)
    g0 = math.sqrt(claire.claire_dot(ctx.handle, g, g, 3 * N))
    del g
    a0, a1 = sampled(128)
    vc = u.forward(a0, a1)
    claire.claire_resample(vc[0], (128,) * 3, v, grid, 3, claire.RESAMPLE_SPECTRAL, st)
    torch.cuda.synchronize()
    t_pred = time.perf_counter() - t0
    _, mis_guess = ctx.objective(v)
    flush()
    ctx.set_opts(g0_ref=g0)
    torch.cuda.synchronize()
    stt, rep = ctx.register(v, check=False)
    torch.cuda.synchronize()
    runs["fp16_learned"] = {"time_to_tol_s": time.perf_counter() - t0, "predict_and_g0_s": t_pred,
                            "status": rep["status"], "gn_iters": rep["gn_iters"], "pcg_iters": rep["pcg_iters_total"],
                            "inner_pcg_iters": rep["pc_inner_iters_total"], "pc_fallbacks": rep["pc_fallbacks"],
                            "gnorm_rel": rep["gnorm_rel"],
                            "J": rep["J"], "mismatch": rep["mismatch"], "r": rep["r"], "detj_min": rep["detj_min"],
                            "detj_max": rep["detj_max"], "cfl": rep["cfl"], "mismatch_at_guess": mis_guess,
                            "peak_device_gb": used_gb()}
    ctx.set_opts(g0_ref=0.0)
    runs["fp16_learned"]["dice"] = dice(v)
    # sampled oracle parity of one backtrace and one interpolation at n^3
    flush()
    d = torch.empty((3,) + grid, device=dev)
    ctx.backtrace(v, d, 1)
    m0_d = torch.from_numpy(m0).to(dev)
    mo = torch.empty(grid, device=dev)
    ctx.interp(m0_d, d, mo)
    rng = np.random.default_rng(0)
    S = 1000000
    idx = torch.from_numpy(rng.integers(0, N, size=S)).to(dev)
    d_s = d.view(3, -1)[:, idx].double().cpu().numpy()
    out_s = mo.view(-1)[idx].double().cpu().numpy()
    v_s = v.view(3, -1)[:, idx].double().cpu().numpy()
    vh = v.cpu().numpy()
    del d, mo, m0_d, v
    flush()
    ii = idx.cpu().numpy()
    x = np.stack([ii // (n * n), (ii // n) % n, ii % n]).astype(np.float64)
    h = 2.0 * math.pi / n
    dt = 0.25
    u0 = v_s / h
    yp = x - dt * u0
    U = np.stack([oracle.interp_points(vh[c].astype(np.float64), yp, 3) for c in range(3)]) / h
    d_ref = -0.5 * dt * (u0 + U)
    m_ref = oracle.interp_points(m0.astype(np.float64), x + d_s, 3)
    del vh
    out["sampled_parity"] = {"points": S, "velocity": "the learned run's result",
                             "backtrace_rel_linf": float(np.max(np.abs(d_s - d_ref)) / np.max(np.abs(d_ref))),
                             "interp_rel_linf": float(np.max(np.abs(out_s - m_ref)) / np.max(np.abs(m_ref)))}
    # the same registration on images sampled to 256^3 and 512^3, velocity prolonged back
    for nc in (256, 512):
        if nc >= n:
            continue
        g_c = (nc,) * 3
        c_ctx = claire.Context(g_c, args.beta, 4, stream=st, beta_w=1e-4, gtol=5e-2, max_gn=50, max_pcg=50,
                               lowmem=1)
        a0, a1 = sampled(nc)
        c_ctx.set_images(a0, a1)
        vc = torch.zeros((3,) + g_c, device=dev)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, rep = c_ctx.register(vc)
        torch.cuda.synchronize()
        secs = time.perf_counter() - t0
        c_ctx.close()
        del c_ctx, a0, a1
        flush()
        vf = torch.empty((3,) + grid, device=dev)
        claire.claire_resample(vc, g_c, vf, grid, 3, claire.RESAMPLE_SPECTRAL, st)
        _, mis_f = ctx.objective(vf)
        runs["fp32_at_%d" % nc] = {"time_to_tol_s": secs, "gn_iters": rep["gn_iters"],
                                   "pcg_iters": rep["pcg_iters_total"], "r_at_%d" % nc: rep["r"],
                                   "mismatch_at_%d_after_prolongation" % n: mis_f, "dice": dice(vf)}
        del vf, vc
        flush()
    if args.large_precond == "both":
        # the same learned registration with the two-level zero-velocity
        # preconditioner (timed from the prediction; g(v = 0) is reused)
        ctx.set_opts(precond=claire.PRECOND_TWO_LEVEL, g0_ref=g0)
        v = torch.empty((3,) + grid, device=dev)
        a0, a1 = sampled(128)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        vc = u.forward(a0, a1)
        claire.claire_resample(vc[0], (128,) * 3, v, grid, 3, claire.RESAMPLE_SPECTRAL, st)
        stt, rep = ctx.register(v, check=False)
        torch.cuda.synchronize()
        runs["fp16_learned_two_level"] = {
            "time_to_tol_s": time.perf_counter() - t0, "pc_coarse": args.large_pc_coarse,
            "status": rep["status"], "gn_iters": rep["gn_iters"], "pcg_iters": rep["pcg_iters_total"],
            "inner_pcg_iters": rep["pc_inner_iters_total"], "pc_fallbacks": rep["pc_fallbacks"],
            "gnorm_rel": rep["gnorm_rel"], "J": rep["J"], "mismatch": rep["mismatch"], "r": rep["r"],
            "peak_device_gb": used_gb()}
        del a0, a1
        runs["fp16_learned_two_level"]["dice"] = dice(v)
        del v
        flush()
        ctx.set_opts(precond=claire.PRECOND_SPECTRAL, g0_ref=0.0)
    _, mis_zero = ctx.objective(torch.zeros((3,) + grid, device=dev))
    runs["fp16_learned"]["mismatch_at_zero"] = mis_zero
    ctx.close()
    del ctx
    u._bufs = {}  # the network's activation buffers are not needed any more
    flush()
    out["runs"] = runs
    print(json.dumps(out), flush=True)  # the FP16 part, in case the FP32 context does not fit
    # ---- plain FP32 (lowmem) from zero
    out["device_gb_before_fp32_context"] = used_gb()
    try:
        ctx = claire.Context(grid, args.beta, 4, stream=st, beta_w=1e-4, gtol=5e-2, max_gn=50, max_pcg=50,
                             lowmem=1, wall_limit_s=1200, spectral_iterate=args.spectral_iterate)
    except claire.ClaireError as e:
        runs["fp32_zero"] = {"error": str(e)}
        print(json.dumps(out))
        return
    out["fp32_lowmem_device_gb"] = used_gb()
    m0_d = torch.from_numpy(m0).to(dev)
    m1_d = torch.from_numpy(m1).to(dev)
    ctx.set_images(m0_d, m1_d)
    del m0_d, m1_d
    flush()
    v = torch.zeros((3,) + grid, device=dev)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    stt, rep = ctx.register(v)
    torch.cuda.synchronize()
    runs["fp32_zero"] = {"time_to_tol_s": time.perf_counter() - t0, "status": rep["status"],
                         "gn_iters": rep["gn_iters"], "pcg_iters": rep["pcg_iters_total"], "J": rep["J"],
                         "mismatch": rep["mismatch"], "r": rep["r"], "detj_min": rep["detj_min"],
                         "detj_max": rep["detj_max"], "cfl": rep["cfl"], "peak_device_gb": used_gb()}
    runs["fp32_zero"]["dice"] = dice(v)
    del v
    ctx.close()
    flush()
    out["runs"] = runs
    a, b = runs["fp32_zero"], runs["fp16_learned"]
    out["speedup_fp16_learned_vs_fp32_zero"] = a["time_to_tol_s"] / b["time_to_tol_s"]
    print(json.dumps(out))


def main():
    args = parse_args()
    if args.pc_weight_report:
        run_pc_weight_report(args)
        return
    if args.precond_report:
        run_precond_report(args)
        return
    if args.net_report:
        run_net_report(args)
        return
    if args.large_report:
        run_large_report(args)
        return
    if args.interp_report:
        run_interp_report(args)
        return
    if args.syn_report:
        run_syn_report(args)
        return
    if args.vjp_report:
        run_vjp_report(args)
        return
    if args.warmstart_report:
        run_warmstart_report(args)
        return
    if args.mixed_report:
        run_mixed_report(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
