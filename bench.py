"""VMC throughput benchmark of the GB300 GCF-PEPS library.

One step = one VMC iteration over one batch of chains: the sampling launch
(sweeps, then amplitude, E_loc and d ln psi/dA measured on every sample)
followed by the FP64 reductions, CG solve and parameter update of each
context (SR; for the tVMC workload the two TDVP stages, each with its own
sampling launch).  Metric: VMC samples/s (one sample = one measured
configuration).  Workloads (--config):

  z2b_32x32_mixed (default): Z2 gauge + hard-core bosons at half filling,
      D = 4 (D_k = 2), chi = 24, (h, g, J) = (1, 0.33, 0.5), 16384 chains over
      three lattices 16x16 / 24x24 / 32x32 (5462 / 5461 / 5461 chains) in one
      persistent launch (gcf_sample_multi), one sweep per step, SR on each;
  z3_16x16 / z4_16x16: pure Z3 D = 6 / Z4 D = 8 on 16x16, chi = 32, complex64
      tensors, g = 0.375 / 0.33, 8192 chains x 1 sweep, full SR step
      (FP64 CG, diagonal shift 1e-4);
  z2_10x10_tvmc: pure Z2 10x10, D = 6 (D_k = 3), chi = 36, complex64,
      g = 0.2, two-stage tVMC step with dt = 0.01, 8192 samples per stage;
  z2_8x8: pure Z2 8x8, D = 4, chi = 16 (exact), h = 0.5, 4096 chains x 64
      sweeps, SR.

Usage: python bench.py [--config C] [--gpus N] [--steps K] [--warmup W]
                       [--impl reference] [--precision fp32|tf32|bf16]
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

METRIC = "VMC samples/sec (amp+E_loc+grad) per GB300 at D,chi"


def _lattice(N, L, D, chi, chains, g, h=1.0, J=0.0, matter=False, cplx=False):
    return dict(N=N, Lx=L, Ly=L, D=D, chi=chi, h_p=h, g=g, J=J, matter=matter, cplx=cplx, chains=chains)


WORKLOADS = {
    "z2b_32x32_mixed": dict(
        workload="z2_hardcore_bosons_16x16+24x24+32x32_D4_chi24_16384chains_half_filling",
        lattices=[_lattice(2, 16, 4, 24, 5462, 0.33, J=0.5, matter=True),
                  _lattice(2, 24, 4, 24, 5461, 0.33, J=0.5, matter=True),
                  _lattice(2, 32, 4, 24, 5461, 0.33, J=0.5, matter=True)],
        sweeps=1, batches=16, mode="sr", dt=0.0),
    "z3_16x16": dict(workload="z3_16x16_D6_chi32_c64_8192chains", lattices=[_lattice(3, 16, 6, 32, 8192, 0.375, cplx=True)],
                     sweeps=1, batches=8, mode="sr", dt=0.0),
    "z4_16x16": dict(workload="z4_16x16_D8_chi32_c64_8192chains", lattices=[_lattice(4, 16, 8, 32, 8192, 0.33, cplx=True)],
                     sweeps=1, batches=8, mode="sr", dt=0.0),
    "z2_10x10_tvmc": dict(workload="z2_10x10_D6_chi36_c64_tvmc_dt0.01_8192samples", lattices=[_lattice(2, 10, 6, 36, 8192, 0.2, cplx=True)],
                          sweeps=1, batches=8, mode="tvmc", dt=0.01),
    "z2_8x8": dict(workload="z2_8x8_D4_chi16_4096chains_x64sweeps", lattices=[_lattice(2, 8, 4, 16, 4096, 0.5)],
                   sweeps=64, batches=1, mode="sr", dt=0.0),
}
DEFAULT_CONFIG = "z2b_32x32_mixed"
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
                  "peps_dev.cuh", "tcgen05.cuh", "vmc_kernel.cuh")


def source_hash():
    """sha256 (first 16 hex) of the sampling kernel's sources, in sorted order."""
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2503_20566_gb300", "csrc")
    for name in sorted(KERNEL_SOURCES):
        with open(os.path.join(d, name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic(samples_per_launch, kernel, smem_level, workload, pdir=None):
    """DRAM bytes per launch scaled from a committed ncu capture of this
    workload (profiles/*.md carrying `workload: <name>`), or None if there is
    none, the kernel's sources changed since the counters were taken, or the
    launch runs another kernel form (kernel and shared-memory level)."""
    pdir = pdir or os.path.join(ROOT, "profiles")
    for name in sorted(os.listdir(pdir)) if os.path.isdir(pdir) else []:
        try:
            txt = open(os.path.join(pdir, name)).read()
        except OSError:
            continue
        m0 = re.search(r"workload: ([^\s`]+)", txt)
        m1 = re.search(r"source_sha256: ([0-9a-f]+)", txt)
        m2 = re.search(r"traffic_bytes_per_sample: ([0-9.eE+]+)", txt)
        m3 = re.search(r"kernel_form: (\S+) level (\d+)", txt)
        if not (m0 and m1 and m2 and m3) or m0.group(1) != workload:
            continue
        if m1.group(1) != source_hash() or m3.group(1) != kernel or int(m3.group(2)) != smem_level:
            return None
        return float(m2.group(1)) * samples_per_launch
    return None


def fp32_alu_peak_tflops(sm_count, sm_mhz=2070.0):
    """FP32 FMA peak from unit counts: SMs x 128 FP32 lanes x 2 flop x clock."""
    return sm_count * 128 * 2 * sm_mhz * 1e6 / 1e12


# ---------------------------------------------------------------------------
# CPU oracle baseline (bounded sample)
# ---------------------------------------------------------------------------
def _oracle_chain(args):
    config, li, seed, chain, n_sweeps = args
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    import synth
    from oracle import peps as P
    from oracle import vmc
    from oracle.lattice import Lattice

    w = WORKLOADS[config]["lattices"][li]
    lat = Lattice(w["Lx"], w["Ly"], w["N"], matter=w["matter"])
    Dk = w["D"] // w["N"]
    _, n = P.layout(lat, Dk)
    pe = P.GIPEPS(lat, Dk, synth.round_to(synth.tensor_entries(2 + li, n, w["cplx"]), "c64" if w["cplx"] else "f32"))
    powers = synth.plaquette_powers(102 + li, chain + 1, lat.n_plaquettes, w["N"])[chain]
    occ = np.zeros((lat.Ly, lat.Lx))
    if w["matter"]:
        occ = synth.occupations(102 + li, chain + 1, lat.n_s, lat.n_s // 2)[chain].reshape(lat.Ly, lat.Lx)
    cfg = lat.config_from_powers(occ, powers)
    recs = vmc.run_chain(pe, vmc.Model(h=w["h_p"], g=w["g"], J=w["J"]), cfg, w["chi"], seed, chain, n_sweeps)
    return len(recs)


def cpu_oracle_rate(config, n_procs, sweeps=1):
    """The oracle on n_procs host processes, one chain each, the chains spread
    over the workload's lattices in proportion to their chain counts."""
    import multiprocessing as mp

    lats = WORKLOADS[config]["lattices"]
    tot = sum(l["chains"] for l in lats)
    jobs = []
    for c in range(n_procs):
        li = min(len(lats) - 1, int(c * tot / n_procs) * len(lats) // tot) if len(lats) > 1 else 0
        jobs.append((config, li, 7, c, sweeps))
    ctx = mp.get_context("spawn")
    # one thread per process: the spawned workers inherit these before NumPy loads
    keep = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    os.environ.update({k: "1" for k in keep})
    t0 = time.perf_counter()
    try:
        with ctx.Pool(n_procs) as pool:
            done = sum(pool.map(_oracle_chain, jobs))
    finally:
        for k, v in keep.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    dt = time.perf_counter() - t0
    mix = "/".join(str(sum(1 for j in jobs if j[1] == i)) for i in range(len(lats)))
    return done / dt, done, dt, mix


# ---------------------------------------------------------------------------
def err_vs_fp64(ctxs, configs, lats, n_check=16):
    """Error of the benchmarked precision against the library's FP64 form on
    the same tensors (the FP64 form matches the FP64 oracle to ~1e-10 in the
    parity tests), on the first n_check final configurations of each lattice:
    amplitude error |exp(d log|psi| + i d phase) - 1| and E_loc error
    |dE| / max(1, |E|)."""
    import torch

    import paper_2503_20566_gb300 as G

    amp, ee = [], []
    for ctx, cfg, w in zip(ctxs, configs, lats):
        sub = cfg[:n_check].contiguous()
        ref = G.Context(w["N"], w["Lx"], w["Ly"], w["D"], w["chi"], matter=w["matter"], h=w["h_p"], g=w["g"],
                        J=w["J"], complex_=w["cplx"], precision="fp64", seed=0)
        try:
            ref.set_tensors(ctx.get_tensors())
            la, ph = ctx.amplitude(sub)
            la64, ph64 = ref.amplitude(sub)
            e, e64 = ctx.local_energy(sub), ref.local_energy(sub)
        finally:
            ref.close()
        amp.append((torch.exp(torch.complex(la - la64, ph - ph64)) - 1).abs().cpu().numpy())
        ee.append(((e - e64).abs() / torch.clamp(e64.abs(), min=1.0)).cpu().numpy())
    amp, ee = np.concatenate(amp), np.concatenate(ee)
    return {"configs": int(amp.size), "reference": "FP64 form of the library on the same tensors",
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
REFERENCE_BUDGET_S = 150.0


def run_reference(args):
    """Reference arm: the FP64 oracle on the host cores.  A step is one
    bounded sample of the workload: one chain per host core (one sweep,
    measured), spread over the workload's lattices in proportion to their
    chains.  The CPU needs no warm-up, and the run stops after the step that
    passes REFERENCE_BUDGET_S (at least one step), so that the arm ends within
    a few minutes whatever --steps asks; the line reports the steps run."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    wl = WORKLOADS[args.config]
    cores = max(1, min(os.cpu_count() or 1, 16))
    t0 = time.perf_counter()
    done = 0
    mix = ""
    steps = 0
    while steps < max(1, args.steps):
        _, d, _, mix = cpu_oracle_rate(args.config, cores, 1)
        done += d
        steps += 1
        if time.perf_counter() - t0 > REFERENCE_BUDGET_S:
            break
    dt = time.perf_counter() - t0
    v = done / dt
    sample = (f"{cores} chains x 1 sweep per step (lattice mix {mix}), FP64 NumPy, one process per core; "
              f"{steps} of {args.steps} steps run (time cap {REFERENCE_BUDGET_S:.0f} s), no warm-up")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "samples/s", "n_gpus": args.gpus,
            "steps": steps, "warmup": 0, "ms_per_step": 1000 * dt / steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": wl["workload"], "sample_per_step": sample},
            "cpu_baseline": {"value": v, "unit": "samples/s", "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": "samples/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


class Workload:
    """The workload's contexts, chains and sample buffers on this rank.

    The chains of the truncated workloads are advanced in `batches` equal
    shares, one share per step in turn (one persistent launch per step), so
    that a step takes seconds; every chain of the workload is kept and
    advances once every `batches` steps, and the SR / tVMC update of a step
    uses that step's samples."""

    def __init__(self, config, precision, seeds, chains_scale=1.0):
        import torch

        import paper_2503_20566_gb300 as G
        import synth

        self.wl = WORKLOADS[config]
        self.lats = [dict(l, chains=max(1, int(round(l["chains"] * chains_scale)))) for l in self.wl["lattices"]]
        self.sweeps = self.wl["sweeps"]
        self.mode = self.wl["mode"]
        self.batches = max(1, int(self.wl.get("batches", 1)))
        self.batch = 0
        self.per_batch = [-(-w["chains"] // self.batches) for w in self.lats]
        self.ctxs, self.configs, self.samples = [], [], []
        for li, w in enumerate(self.lats):
            ctx = G.Context(w["N"], w["Lx"], w["Ly"], w["D"], w["chi"], matter=w["matter"], h=w["h_p"], g=w["g"],
                            J=w["J"], complex_=w["cplx"], precision=precision, seed=seeds["tensors"] + li)
            n = w["chains"]
            powers = torch.from_numpy(synth.plaquette_powers(seeds["chains"] + li, n, (w["Lx"] - 1) * (w["Ly"] - 1),
                                                             w["N"]))
            occ = None
            if w["matter"]:
                occ = torch.from_numpy(synth.occupations(seeds["chains"] + li, n, w["Lx"] * w["Ly"],
                                                         (w["Lx"] * w["Ly"]) // 2))
            self.configs.append(ctx.init_configs(n, occupations=occ, powers=powers))
            self.samples.append(ctx.alloc_samples(self.per_batch[li], self.sweeps, grad=True))
            self.ctxs.append(ctx)
        self.launches_per_step = 2 if self.mode == "tvmc" else 1

    def _slice(self, b):
        """Per lattice: (configs of batch b, its chain count)."""
        out = []
        for li, w in enumerate(self.lats):
            a = b * self.per_batch[li]
            e = min(w["chains"], a + self.per_batch[li])
            out.append((self.configs[li][a:e], max(0, e - a)))
        return out

    def _outs(self, counts):
        """The sample buffers cut to n chains (e_loc holds two values per sample)."""
        per = {"e_loc": 2}
        out = []
        for smp, n in zip(self.samples, counts):
            d = {}
            for k, v in smp.items():
                d[k] = v[:n] if k in ("accepted", "proposed") else v[: n * self.sweeps * per.get(k, 1)]
            out.append(d)
        return out

    def samples_in_batch(self, b):
        return sum(n for _, n in self._slice(b)) * self.sweeps

    @property
    def samples_per_launch(self):
        """Samples of one launch, averaged over the batches."""
        return sum(self.samples_in_batch(b) for b in range(self.batches)) / self.batches

    @property
    def stream(self):
        return self.ctxs[0].stream

    def sample(self, seed, b):
        import paper_2503_20566_gb300 as G

        sl = self._slice(b)
        outs = self._outs([n for _, n in sl])
        if len(self.ctxs) == 1:
            self.ctxs[0].sample_batch(sl[0][0], self.sweeps, seed=seed, out=outs[0])
        else:
            G.sample_multi(self.ctxs, [c for c, _ in sl], self.sweeps, [seed + 7919 * i for i in range(len(self.ctxs))],
                           outs=outs)
        return outs, [n for _, n in sl]

    def update(self, outs, counts, stage=0):
        import paper_2503_20566_gb300 as G

        stats = []
        mode = G.SR if self.mode == "sr" else (G.TDVP_STAGE1 if stage == 0 else G.TDVP_STAGE2)
        for ctx, smp, n in zip(self.ctxs, outs, counts):
            stats.append(ctx.sr_step(smp, n, mode=mode, dt=self.wl["dt"], **SR_ARGS))
        return stats

    def step(self, seed, ev=None, stream=None):
        """One VMC iteration on the next batch of chains; ev: (start,
        after-sampling, end) events of each sampling launch and update,
        recorded on `stream`.  Returns (stats, samples of the step)."""
        stats = None
        b = self.batch
        self.batch = (self.batch + 1) % self.batches
        for stage in range(self.launches_per_step):
            if ev:
                ev[stage][0].record(stream)
            outs, counts = self.sample(seed + 100 * stage, b)
            if ev:
                ev[stage][1].record(stream)
            stats = self.update(outs, counts, stage)
            if ev:
                ev[stage][2].record(stream)
        return stats, self.samples_in_batch(b) * self.launches_per_step

    def flops_per_launch(self):
        """Algorithmic work of one launch, averaged over the batches."""
        return sum(flops_per_sample(w["Lx"], w["Ly"], w["D"] // w["N"], w["chi"], w["cplx"]) * w["chains"] * self.sweeps
                   for w in self.lats) / self.batches

    def kernel_name(self):
        """Name of the sampling kernel the last launch ran."""
        if len(self.ctxs) > 1:
            return "gcf::vmc_kernel_multi4" if self.ctxs[0].multi_chains_per_cta == 4 else "gcf::vmc_kernel_multi"
        return self.ctxs[0].kernel_name

    def scalar(self):
        return "<gcf::cfloat>" if self.lats[0]["cplx"] else "<float>"


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--config", default=DEFAULT_CONFIG, choices=sorted(WORKLOADS))
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gcf", choices=["gcf", "reference"])
    ap.add_argument("--chains-scale", type=float, default=1.0, help="scale every lattice's chain count")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "tf32", "bf16"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--clocks-log", default=None,
                    help="keep the nvidia-smi clock samples of the timed region here ({rank} is replaced)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="keep the planner's kernel form")
    ap.add_argument("--no-forms", action="store_true", help="skip the precision-form comparison")
    ap.add_argument("--no-check", action="store_true", help="skip the FP64 comparison after timing")
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
        rate, done, dt, mix = cpu_oracle_rate(args.config, cores, 1)
        cpu = {"value": rate, "unit": "samples/s", "cores": cores, "kind": "oracle",
               "sample": f"{done} samples = {cores} chains x 1 sweep of the same workload (lattice mix {mix}; "
                         f"FP64 NumPy, one process per core), {dt:.1f} s"}

    import torch

    import paper_2503_20566_gb300 as G
    from paper_2503_20566_gb300 import replicas

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    seeds = replicas.rank_seeds(rank)
    W = Workload(args.config, args.precision, seeds, args.chains_scale)
    # the library's autotuner picks the kernel form of a single-lattice workload
    tune_ms = []
    if len(W.ctxs) == 1 and not args.no_autotune:
        # on a subset of the chains (eight per SM) when the workload is large
        sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
        sub = W.configs[0][: min(W.configs[0].shape[0], 8 * sms)]
        tune_ms = W.ctxs[0].autotune(sub, n_sweeps=min(4, W.sweeps))
    stream = W.stream
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    for i in range(args.warmup):
        W.step(1000 * i + rank)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    launches0 = sum(c.launch_count for c in W.ctxs)
    ev = [[tuple(torch.cuda.Event(enable_timing=True) for _ in range(3)) for _ in range(W.launches_per_step)]
          for _ in range(args.steps)]
    clk_path = (args.clocks_log.format(rank=rank) if args.clocks_log
                else os.path.join(tempfile.gettempdir(), f"gcfvmc_clocks_{os.getpid()}_rank{rank}.csv"))
    sampler, sf = clocks_sampler_start(clk_path)
    time.sleep(0.3)
    torch.cuda.synchronize()
    stats = None
    energies = []
    samples_done = 0
    for i in range(args.steps):
        flush.fill_(float(i))  # 256 MiB write evicts L2 between steps (outside the events)
        with torch.cuda.stream(stream):
            stats, n_smp = W.step(seeds["step"](i), ev[i], stream)
        samples_done += n_smp
        energies.append([s[0] for s in stats])
    torch.cuda.synchronize()
    clocks = clocks_sampler_stop(sampler, sf, clk_path, torch.cuda.current_device())
    kernel_name = W.kernel_name() + W.scalar()
    # the four-chain multi-context kernel keeps its hot buffers in scratch
    smem_level = 0 if "multi4" in kernel_name else W.ctxs[0].smem_level
    launches = sum(c.launch_count for c in W.ctxs) - launches0
    t_steps = [sum(e[0].elapsed_time(e[2]) for e in ev[i]) for i in range(args.steps)]
    t_kernel = [[e[0].elapsed_time(e[1]) for e in ev[i]] for i in range(args.steps)]
    kern_launch_ms = float(np.mean([t for row in t_kernel for t in row]))
    group = dist.group.WORLD if dist else None
    total_ms = replicas.max_over_ranks(float(sum(t_steps)), group, "cuda")
    value = replicas.whole_job_rate(samples_done / args.steps, args.steps, world, total_ms)

    # the contraction forms side by side (sampling launch only, same tensors,
    # a quarter of the chains): plain FP32 on CUDA cores, TF32x3 and BF16
    forms = None
    if rank == 0 and world == 1 and not args.no_forms:
        forms = {"chains": "one batch of the workload (the first), second launch on it",
                 "unit": "samples/s (sampling launch only)"}
        for prec in ("fp32", "tf32", "bf16"):
            F = Workload(args.config, prec, seeds, args.chains_scale)
            F.sample(1, 0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(F.stream):
                e0.record(F.stream)
                F.sample(2, 0)
                e1.record(F.stream)
            torch.cuda.synchronize()
            forms[{"fp32": "fp32", "tf32": "tf32x3", "bf16": "bf16x3"}[prec]] = \
                F.samples_in_batch(0) / (e0.elapsed_time(e1) / 1e3)
            if prec == "bf16":
                forms["bf16x3_on_tcgen05"] = all(c.tensor_core_form for c in F.ctxs)
            for c in F.ctxs:
                c.close()
            del F

    # end to end through the public API from host memory: every step copies
    # the chains' configurations in (pinned host -> device) and the updated
    # configurations and the SR statistics out
    e2e = None
    if not args.no_e2e:
        host_cfg = [c.cpu().pin_memory() for c in W.configs]
        e2e_steps = min(args.steps, 3)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        done, h2d, d2h = 0, 0, 0
        for i in range(e2e_steps):
            b = W.batch
            for li, w in enumerate(W.lats):
                a = b * W.per_batch[li]
                e = min(w["chains"], a + W.per_batch[li])
                W.configs[li][a:e].copy_(host_cfg[li][a:e], non_blocking=True)
                h2d += host_cfg[li][a:e].numel()
            _, n_smp = W.step(50_000 + 1000 * i + rank)
            done += n_smp
            for li, w in enumerate(W.lats):
                a = b * W.per_batch[li]
                e = min(w["chains"], a + W.per_batch[li])
                host_cfg[li][a:e].copy_(W.configs[li][a:e], non_blocking=True)
                d2h += host_cfg[li][a:e].numel()
            d2h += 8 * 8 * len(W.ctxs) * W.launches_per_step  # the SR statistics
            torch.cuda.synchronize()
        e2e_s = replicas.max_over_ranks(time.perf_counter() - t0, group, "cuda")
        e2e = {"value": replicas.whole_job_rate(done / e2e_steps, e2e_steps, world, 1000.0 * e2e_s),
               "unit": "samples/s", "h2d_bytes_per_step": int(h2d // e2e_steps),
               "d2h_bytes_per_step": int(d2h // e2e_steps), "steps": e2e_steps}

    if rank == 0:
        err = None
        if not args.no_check:
            try:
                err = err_vs_fp64(W.ctxs, W.configs, W.lats)
            except Exception as exc:  # the JSON line is printed whatever happens here
                err = {"error": f"{type(exc).__name__}: {exc}"[:300]}
        peaks, src = load_peaks()
        sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
        fl = W.flops_per_launch()
        achieved = fl / (kern_launch_ms / 1000.0) / 1e12
        # TF32 is the tensor-core type of FP32 data (nominal TF32 = BF16 / 2);
        # the sampling launch runs for seconds inside a step: the sustained peak
        tc_peak = peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops", 0.0)) / 2.0
        wl = W.wl
        line = {
            "metric": METRIC, "value": value, "unit": "samples/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "c64" if W.lats[0]["cplx"] else "f32",
            "data": "synthetic",
            "config": {"workload": wl["workload"],
                       "lattices": [f"{w['Lx']}x{w['Ly']} Z{w['N']}{' + hard-core bosons' if w['matter'] else ''} "
                                    f"D={w['D']} chi={w['chi']} chains={w['chains']}" for w in W.lats],
                       "chains_total": sum(w["chains"] for w in W.lats), "batches": W.batches,
                       "chains_per_step": samples_done / args.steps / W.launches_per_step / W.sweeps,
                       "batching": ("all chains every step" if W.batches == 1 else
                                    f"the chains in {W.batches} equal shares, one share per step in turn "
                                    "(one persistent launch per step; every chain kept and advanced once "
                                    f"every {W.batches} steps; the update uses the step's samples)"),
                       "sweeps_per_launch": W.sweeps, "launches_per_step": W.launches_per_step,
                       "couplings": {"h": W.lats[0]["h_p"], "g": W.lats[0]["g"], "J": W.lats[0]["J"]},
                       "update": "two-stage tVMC (dt=%g)" % wl["dt"] if W.mode == "tvmc" else "SR",
                       "precision": args.precision, "sr": SR_ARGS, "parallelism": f"replicas{world}",
                       "l2": "256 MiB buffer written between timed steps (outside the events)",
                       "kernel_form": {"kernel": kernel_name, "smem_level": smem_level,
                                       "autotune_ms_per_form": [round(t, 3) if t < 1e299 else None
                                                                for t in tune_ms]}},
            "gpu_launches": launches,
            "kernel_ms": kern_launch_ms,
            "update_ms": float(np.mean(t_steps)) - kern_launch_ms * W.launches_per_step,
            "roofline": {"bound": "tensor", "achieved": achieved, "peak": tc_peak, "unit": "TFLOP/s",
                         "frac": achieved / tc_peak if tc_peak else None,
                         "traffic": profiled_traffic(W.samples_per_launch, kernel_name, smem_level,
                                                     wl["workload"]),
                         "kernel": kernel_name, "algorithmic_flop_per_launch": fl,
                         "peak_source": f"TF32 tensor peak = 1/2 x bf16 sustained ({src})",
                         "fp32_alu_frac": achieved / fp32_alu_peak_tflops(sms)},
            "clocks": clocks,
            "sr_stats": [{"e_mean": s[0], "e_err": s[2], "cg_iters": s[3], "residual": s[4], "converged": bool(s[6])}
                         for s in stats],
            "energy_per_step": energies,
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
