"""VMC throughput benchmark of the GB300 GCF-PEPS library.

Workload: pure Z2 gauge theory, 8x8 open lattice, GCF PEPS with D = 4
(D_k = 2) and i.i.d. N(0,1) Z2-symmetric tensors, boundary cutoff chi = 16,
coupling h = 0.5 (electric; paper form h_p = 1, g = 0.5), 4096 Markov chains
x 64 sweeps per step in one persistent launch, FP32 contraction.  One step =
one VMC iteration: sample_batch (sweeps + amplitude, E_loc and d ln psi/dA
measured after every sweep) followed by the FP64 SR step (reductions + CG
solve + parameter update).  Metric: VMC samples/s (one sample = one measured
configuration).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Under torchrun (N > 1) every rank runs the workload on its own chains with
the same tensors (chains are independent; no collective on the data path);
the slowest rank's time sets the whole-job rate.
"""

from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = dict(workload="z2_8x8_D4_chi16_4096chains_x64sweeps", N=2, Lx=8, Ly=8, D=4, chi=16, h_p=1.0,
                g=0.5, chains=4096, sweeps=64)
METRIC = "VMC samples/sec (amp+E_loc+grad) per GB300 at D,chi"
SR_ARGS = dict(diag_shift=1e-4, lr=0.01, max_iter=100, tol=1e-6)


def flops_per_sample(Lx, Ly, Dk, chi, cplx=False):
    """Algorithmic work per sample: ~4 boundary passes x Lx*Ly sites x
    U = 2 (D_k^5 chi^2 + D_k^4 chi^2 + D_k^3 chi^3) (cost scaling of the
    paper's main text), x4 for complex arithmetic."""
    U = 2.0 * (Dk ** 5 * chi ** 2 + Dk ** 4 * chi ** 2 + Dk ** 3 * chi ** 3)
    return 4.0 * Lx * Ly * U * (4.0 if cplx else 1.0)


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
            "sm_max_mhz": 2070.0}, "fallback"


# the files the FP32 sampling kernel is compiled from (its translation unit and
# every header it includes)
KERNEL_SOURCES = ("vmc_f32.cu", "launch.h", "common.cuh", "envsteps.cuh", "linalg.cuh", "mma.cuh",
                  "peps_dev.cuh", "vmc_kernel.cuh")


def source_hash():
    """sha256 (first 16 hex) of the sampling kernel's sources, in sorted order."""
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2503_20566_gb300", "csrc")
    for name in sorted(KERNEL_SOURCES):
        with open(os.path.join(d, name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


PROFILE = os.path.join(ROOT, "profiles", "vmc_kernel_grouped4_f32_z2_8x8_D4_chi16.md")


def profiled_traffic(samples_per_launch, kernel, smem_level):
    """DRAM bytes per launch scaled from the committed ncu capture, or None if
    the kernel's sources changed since the counters were taken or the launch
    runs another kernel form (kernel and shared-memory level)."""
    try:
        txt = open(PROFILE).read()
    except OSError:
        return None
    m1 = re.search(r"source_sha256: ([0-9a-f]+)", txt)
    m2 = re.search(r"traffic_bytes_per_sample: ([0-9.eE+]+)", txt)
    m3 = re.search(r"kernel_form: (\S+) level (\d+)", txt)
    if not (m1 and m2 and m3) or m1.group(1) != source_hash():
        return None
    if m3.group(1) != kernel or int(m3.group(2)) != smem_level:
        return None
    return float(m2.group(1)) * samples_per_launch


def fp32_alu_peak_tflops(sm_count=152, sm_mhz=2070.0):
    """FP32 FMA peak from unit counts: SMs x 128 FP32 lanes x 2 flop x clock."""
    return sm_count * 128 * 2 * sm_mhz * 1e6 / 1e12


# ---------------------------------------------------------------------------
# CPU oracle baseline (bounded sample)
# ---------------------------------------------------------------------------
def _oracle_chain(args):
    seed, chain, n_sweeps = args
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    import synth
    from oracle import peps as P
    from oracle import vmc
    from oracle.lattice import Lattice

    w = WORKLOAD
    lat = Lattice(w["Lx"], w["Ly"], w["N"])
    Dk = w["D"] // w["N"]
    _, n = P.layout(lat, Dk)
    pe = P.GIPEPS(lat, Dk, synth.round_to(synth.tensor_entries(2, n, False), "f32"))
    powers = synth.plaquette_powers(102, chain + 1, lat.n_plaquettes, w["N"])[chain]
    cfg = lat.config_from_powers(np.zeros((lat.Ly, lat.Lx)), powers)
    recs = vmc.run_chain(pe, vmc.Model(h=w["h_p"], g=w["g"]), cfg, w["chi"], seed, chain, n_sweeps)
    return len(recs)


def cpu_oracle_rate(n_procs, chains_per_proc=1, sweeps=1):
    import multiprocessing as mp

    ctx = mp.get_context("spawn")
    jobs = [(7, c, sweeps) for c in range(n_procs * chains_per_proc)]
    t0 = time.perf_counter()
    with ctx.Pool(n_procs) as pool:
        done = sum(pool.map(_oracle_chain, jobs))
    dt = time.perf_counter() - t0
    return done / dt, done, dt


# ---------------------------------------------------------------------------
def err_vs_fp64(ctx, configs, w, n_check=64):
    """Error of the benchmarked precision against the library's FP64 form on
    the same tensors (the FP64 form matches the FP64 oracle to ~1e-10 in the
    parity tests), on the first n_check final configurations: amplitude error
    |exp(d log|psi| + i d phase) - 1| and E_loc error |dE| / max(1, |E|)."""
    import torch

    import paper_2503_20566_gb300 as G

    sub = configs[:n_check].contiguous()
    ref = G.Context(w["N"], w["Lx"], w["Ly"], w["D"], w["chi"], h=w["h_p"], g=w["g"], precision="fp64", seed=0)
    try:
        ref.set_tensors(ctx.get_tensors())
        la, ph = ctx.amplitude(sub)
        la64, ph64 = ref.amplitude(sub)
        e, e64 = ctx.local_energy(sub), ref.local_energy(sub)
    finally:
        ref.close()
    amp = (torch.exp(torch.complex(la - la64, ph - ph64)) - 1).abs().cpu().numpy()
    ee = ((e - e64).abs() / torch.clamp(e64.abs(), min=1.0)).cpu().numpy()
    return {"configs": int(sub.shape[0]), "reference": "FP64 form of the library on the same tensors",
            "amp_max": float(amp.max()), "amp_median": float(np.median(amp)),
            "eloc_max": float(ee.max()), "eloc_median": float(np.median(ee))}


# ---------------------------------------------------------------------------
def clocks_sampler_start(path):
    q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    try:
        f = open(path, "w")
        p = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits", "-lms", "200"],
                             stdout=f, stderr=subprocess.DEVNULL)
        return p, f
    except (OSError, FileNotFoundError):
        return None, None


def clocks_sampler_stop(p, f, path, gpu_index):
    if p is None:
        return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
    p.terminate()
    try:
        p.wait(timeout=5)
    except subprocess.TimeoutExpired:
        p.kill()
    f.close()
    sm, smax, reasons = [], None, set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in open(path):
        parts = [x.strip() for x in line.split(",")]
        if len(parts) < 9 or not parts[0].isdigit() or int(parts[0]) != gpu_index:
            continue
        try:
            sm.append(float(parts[1]))
            smax = float(parts[2])
        except ValueError:
            continue
        for nm, v in zip(names, parts[5:9]):
            if v.lower() == "active":
                reasons.add(nm)
    return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": smax, "reasons": sorted(reasons),
            "samples": len(sm)}


# ---------------------------------------------------------------------------
def run_reference(args):
    """Reference arm: the FP64 oracle on the host cores, bounded samples."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    cores = max(1, min(os.cpu_count() or 1, 16))
    for _ in range(max(0, args.warmup)):
        cpu_oracle_rate(cores, 1, 1)
    t0 = time.perf_counter()
    done = 0
    for _ in range(args.steps):
        _, d, _ = cpu_oracle_rate(cores, 1, 1)
        done += d
    dt = time.perf_counter() - t0
    v = done / dt
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "samples/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * dt / max(1, args.steps),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD["workload"], "sample_per_step":
                                             f"{cores} chains x 1 sweep (of 4096 x 64)"},
            "cpu_baseline": {"value": v, "unit": "samples/s", "cores": cores, "kind": "oracle",
                             "sample": f"{cores} chains x 1 sweep per step, FP64 NumPy, one process per core"},
            "e2e": {"value": v, "unit": "samples/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gcf", choices=["gcf", "reference"])
    ap.add_argument("--chains", type=int, default=WORKLOAD["chains"])
    ap.add_argument("--sweeps", type=int, default=WORKLOAD["sweeps"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "tf32", "bf16"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--clocks-log", default=None,
                    help="keep the nvidia-smi clock samples of the timed region here ({rank} is replaced)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="keep the planner's kernel form")
    ap.add_argument("--no-forms", action="store_true", help="skip the precision-form comparison")
    args = ap.parse_args()
    if args.warmup < 3:
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        return run_reference(args)

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    # CPU baseline first (spawned workers, before any CUDA initialisation)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cores = max(1, min(os.cpu_count() or 1, 16))
        rate, done, dt = cpu_oracle_rate(cores, 1, 2)
        cpu = {"value": rate, "unit": "samples/s", "cores": cores, "kind": "oracle",
               "sample": f"{done} samples = {cores} chains x 2 sweeps of the same workload "
                         f"(FP64 NumPy, one process per core), {dt:.1f} s"}

    import torch

    import paper_2503_20566_gb300 as G
    import synth
    from paper_2503_20566_gb300 import replicas

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    w = WORKLOAD
    n_chains, n_sweeps = args.chains, args.sweeps
    seeds = replicas.rank_seeds(rank)
    ctx = G.Context(w["N"], w["Lx"], w["Ly"], w["D"], w["chi"], h=w["h_p"], g=w["g"], precision=args.precision,
                    seed=seeds["tensors"])
    powers = torch.from_numpy(synth.plaquette_powers(seeds["chains"], n_chains, (w["Lx"] - 1) * (w["Ly"] - 1),
                                                     w["N"]))
    configs = ctx.init_configs(n_chains, powers=powers)
    # the library's autotuner picks the kernel form (executor x shared-memory level) on this workload
    tune_ms = [] if args.no_autotune else ctx.autotune(configs, n_sweeps=4)
    kernel_name = ctx.kernel_name + "<float>"
    samples = ctx.alloc_samples(n_chains, n_sweeps, grad=True)
    stream = ctx.stream
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def step(i):
        ctx.sample_batch(configs, n_sweeps, seed=1000 * i + rank, out=samples)
        return ctx.sr_step(samples, n_chains, **SR_ARGS)

    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    launches0 = ctx.launch_count
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clk_path = (args.clocks_log.format(rank=rank) if args.clocks_log
                else os.path.join(tempfile.gettempdir(), f"gcfvmc_clocks_{os.getpid()}_rank{rank}.csv"))
    sampler, sf = clocks_sampler_start(clk_path)
    time.sleep(0.3)
    torch.cuda.synchronize()
    stats = None
    for i in range(args.steps):
        flush.fill_(float(i))  # 256 MiB write evicts L2 between steps (outside the events)
        with torch.cuda.stream(stream):
            ev[i][0].record(stream)
            ctx.sample_batch(configs, n_sweeps, seed=seeds["step"](i), out=samples)
            ev[i][1].record(stream)
            stats = ctx.sr_step(samples, n_chains, **SR_ARGS)
            ev[i][2].record(stream)
    torch.cuda.synchronize()
    clocks = clocks_sampler_stop(sampler, sf, clk_path, torch.cuda.current_device())
    launches = ctx.launch_count - launches0
    t_steps = [ev[i][0].elapsed_time(ev[i][2]) for i in range(args.steps)]
    t_kernel = [ev[i][0].elapsed_time(ev[i][1]) for i in range(args.steps)]
    group = dist.group.WORLD if dist else None
    total_ms = replicas.max_over_ranks(float(sum(t_steps)), group, "cuda")
    samples_per_step = n_chains * n_sweeps
    value = replicas.whole_job_rate(samples_per_step, args.steps, world, total_ms)

    # the contraction forms side by side (kernel only, same tensors and chains):
    # plain FP32 on CUDA cores, TF32x3 and BF16 on tensor cores
    forms = None
    if rank == 0 and world == 1 and not args.no_forms:
        forms = {"sweeps": 8, "chains": n_chains, "unit": "samples/s (sampling kernel only)"}
        for prec in ("fp32", "tf32", "bf16"):
            fctx = G.Context(w["N"], w["Lx"], w["Ly"], w["D"], w["chi"], h=w["h_p"], g=w["g"], precision=prec,
                             seed=seeds["tensors"])
            fcfg = fctx.init_configs(n_chains, powers=powers)
            fout = fctx.alloc_samples(n_chains, 8, grad=True)
            fctx.sample_batch(fcfg, 8, seed=1, out=fout)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(fctx.stream):
                e0.record(fctx.stream)
                fctx.sample_batch(fcfg, 8, seed=2, out=fout)
                e1.record(fctx.stream)
            torch.cuda.synchronize()
            forms[{"fp32": "fp32", "tf32": "tf32x3", "bf16": "bf16"}[prec]] = n_chains * 8 / (e0.elapsed_time(e1) / 1e3)
            del fctx, fcfg, fout

    # end to end through the host-buffer C call
    e2e = None
    if not args.no_e2e:
        host_cfg = np.ascontiguousarray(configs.cpu().numpy())
        cfg_bytes = host_cfg.nbytes
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        for i in range(args.steps):
            ctx.vmc_step_host(host_cfg, n_sweeps, 50_000 + 1000 * i + rank, **SR_ARGS)
        torch.cuda.synchronize()
        e2e_s = replicas.max_over_ranks(time.perf_counter() - t0, group, "cuda")
        e2e = {"value": replicas.whole_job_rate(samples_per_step, args.steps, world, 1000.0 * e2e_s),
               "unit": "samples/s",
               "h2d_bytes_per_step": cfg_bytes, "d2h_bytes_per_step": cfg_bytes + 8 * 8}

    if rank == 0:
        try:
            err = err_vs_fp64(ctx, configs, w)
        except Exception as exc:  # the JSON line is printed whatever happens here
            err = {"error": f"{type(exc).__name__}: {exc}"[:300]}
        peaks, src = load_peaks()
        kern_s = float(np.mean(t_kernel)) / 1000.0
        fl = flops_per_sample(w["Lx"], w["Ly"], w["D"] // w["N"], w["chi"]) * samples_per_step
        peak = fp32_alu_peak_tflops()
        achieved = fl / kern_s / 1e12
        line = {
            "metric": METRIC, "value": value, "unit": "samples/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": w["workload"], "lattice": "8x8 open", "gauge": "Z2", "D": w["D"],
                       "chi": w["chi"], "chains": n_chains, "sweeps_per_step": n_sweeps, "h": w["g"],
                       "precision": args.precision, "sr": SR_ARGS, "parallelism": f"replicas{world}",
                       "l2": "256 MiB buffer written between timed steps (outside the events)",
                       "kernel_form": {"kernel": kernel_name, "smem_level": ctx.smem_level,
                                       "autotune_ms_per_form": [round(t, 3) if t < 1e299 else None
                                                                for t in tune_ms]}},
            "gpu_launches": launches,
            "kernel_ms": float(np.mean(t_kernel)),
            "sr_ms": float(np.mean([a - b for a, b in zip(t_steps, t_kernel)])),
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak, "traffic": profiled_traffic(samples_per_step, kernel_name, ctx.smem_level),
                         "kernel": kernel_name,
                         "algorithmic_flop_per_launch": fl,
                         "peak_source": "FP32 FMA units x max SM clock (152 x 128 x 2 x 2070 MHz)",
                         "tensor_peak_tf32_of_" + src: peaks.get("bf16_tflops", 0) / 2.0},
            "clocks": clocks,
            "sr_stats": {"e_mean": stats[0], "e_err": stats[2], "cg_iters": stats[3], "residual": stats[4]},
            "err_vs_fp64": err,
        }
        if e2e:
            line["e2e"] = e2e
        if forms:
            line["precision_forms"] = forms
        if cpu:
            line["cpu_baseline"] = cpu
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
