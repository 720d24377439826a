"""Whole runs over the library's calls: an SR optimisation and a tVMC
trajectory, with per-step metrics and checkpoints.

Each step samples the chains (gcf_sample_batch: amplitudes, E_loc, O per
sample) and hands the samples to gcf_sr_step, which reduces them in FP64,
solves (S + lambda) x = F by CG and updates the parameters on the device:

* SR (Sec. S-3): A <- A - lr x, one sampling pass per step.
* tVMC (Eqs. S6-S8, two-stage scheme): with alpha_dot = -i (S + lambda)^-1 F,
  alpha_1 = alpha + c_1 dt alpha_dot(alpha) and
  alpha(t + dt) = alpha_1 + c_2 dt alpha_dot(alpha_1), c_{1,2} = (1 +- i)/2;
  each stage samples at its own parameters, so a time step is two passes.

Nothing here touches the data: the drivers choose the seeds, call the library
and record what it returns.  Step k of a run draws its Metropolis stream from
seed_of_step(k) (for tVMC, stage s of step k uses seed_of_step(2k + s)), so a
run resumed from a checkpoint at step k samples exactly as the original did.
"""

from __future__ import annotations

import json
import time

from . import checkpoint as ck
from .binding import SR, TDVP_STAGE1, TDVP_STAGE2


def default_seed_of_step(base: int):
    """Seed of sampling pass k: distinct per pass, fixed by (base, k)."""
    return lambda k: (int(base) * 1_000_003 + 10_000 + 1000 * int(k)) % (1 << 63)


def _record(kind, step, stats, out, seconds, n_samples):
    acc = out["accepted"].sum().item()
    prop = out["proposed"].sum().item()
    return {"kind": kind, "step": step, "e_mean": stats[0], "e_mean_im": stats[1], "e_err": stats[2],
            "cg_iters": int(stats[3]), "cg_residual": stats[4], "cg_converged": bool(stats[6]),
            "acceptance": acc / prop if prop else None, "samples": n_samples, "seconds": seconds,
            "samples_per_s": n_samples / seconds if seconds > 0 else None}


class _Run:
    """Shared bookkeeping: the JSONL log, checkpoints and the start step."""

    def __init__(self, ctx, configs, log_path, checkpoint_path, checkpoint_every, seed, resume):
        self.ctx, self.configs = ctx, configs
        self.log = open(log_path, "a") if log_path else None
        self.ck_path, self.ck_every, self.seed = checkpoint_path, int(checkpoint_every or 0), seed
        self.start = 0
        if resume is not None:
            self.configs = ck.restore(ctx, resume, device=configs.device)
            self.start = int(resume.step)

    def emit(self, rec, records, on_step):
        records.append(rec)
        if self.log:
            self.log.write(json.dumps(rec) + "\n")
            self.log.flush()
        if on_step:
            on_step(rec)

    def maybe_checkpoint(self, next_step, extra):
        if self.ck_path and self.ck_every and next_step % self.ck_every == 0:
            ck.save(self.ck_path, self.ctx, self.configs, step=next_step, seed=self.seed, extra=extra)

    def close(self):
        if self.log:
            self.log.close()


def sr_optimize(ctx, configs, n_steps, n_sweeps, seed=0, seed_of_step=None, diag_shift=1e-4, lr=0.01,
                max_iter=100, tol=1e-6, log_path=None, checkpoint_path=None, checkpoint_every=0, resume=None,
                on_step=None):
    """Run SR steps n_start .. n_steps-1 (n_start = 0, or the checkpoint's
    step when `resume` is a checkpoint.Checkpoint).  `configs`: device int8
    (n_chains, cfg_len), updated in place (a resumed run continues from the
    checkpoint's configurations).  Returns (configs, per-step records)."""
    seed_of = seed_of_step or default_seed_of_step(seed)
    run = _Run(ctx, configs, log_path, checkpoint_path, checkpoint_every, seed, resume)
    n_chains = run.configs.shape[0]
    out = ctx.alloc_samples(n_chains, n_sweeps)
    records = []
    try:
        for step in range(run.start, n_steps):
            t0 = time.perf_counter()
            ctx.sample_batch(run.configs, n_sweeps, seed=seed_of(step), out=out)
            stats = ctx.sr_step(out, n_chains, diag_shift=diag_shift, lr=lr, mode=SR, max_iter=max_iter, tol=tol)
            run.emit(_record("sr", step, stats, out, time.perf_counter() - t0, n_chains * n_sweeps), records,
                     on_step)
            run.maybe_checkpoint(step + 1, {"driver": "sr", "lr": lr, "diag_shift": diag_shift})
    finally:
        run.close()
    return run.configs, records


def tvmc_evolve(ctx, configs, n_steps, dt, n_sweeps, seed=0, seed_of_step=None, diag_shift=1e-4, max_iter=100,
                tol=1e-6, log_path=None, checkpoint_path=None, checkpoint_every=0, resume=None, on_step=None):
    """Integrate n_steps tVMC time steps of size dt with the two-stage scheme
    (complex tensors).  The record of step k carries <E> at time k dt (from
    the first stage's samples) and the second stage's CG figures under
    "stage2".  Returns (configs, per-step records)."""
    if not ctx.complex:
        raise ValueError("tVMC needs complex tensors")
    seed_of = seed_of_step or default_seed_of_step(seed)
    run = _Run(ctx, configs, log_path, checkpoint_path, checkpoint_every, seed, resume)
    n_chains = run.configs.shape[0]
    out = ctx.alloc_samples(n_chains, n_sweeps)
    records = []
    try:
        for step in range(run.start, n_steps):
            t0 = time.perf_counter()
            ctx.sample_batch(run.configs, n_sweeps, seed=seed_of(2 * step), out=out)
            s1 = ctx.sr_step(out, n_chains, diag_shift=diag_shift, lr=0.0, mode=TDVP_STAGE1, dt=dt,
                             max_iter=max_iter, tol=tol)
            rec = _record("tvmc", step, s1, out, 0.0, 2 * n_chains * n_sweeps)
            ctx.sample_batch(run.configs, n_sweeps, seed=seed_of(2 * step + 1), out=out)
            s2 = ctx.sr_step(out, n_chains, diag_shift=diag_shift, lr=0.0, mode=TDVP_STAGE2, dt=dt,
                             max_iter=max_iter, tol=tol)
            sec = time.perf_counter() - t0
            rec.update({"time": step * dt, "seconds": sec,
                        "samples_per_s": rec["samples"] / sec if sec > 0 else None,
                        "stage2": {"e_mean": s2[0], "cg_iters": int(s2[3]), "cg_residual": s2[4],
                                   "cg_converged": bool(s2[6])}})
            run.emit(rec, records, on_step)
            run.maybe_checkpoint(step + 1, {"driver": "tvmc", "dt": dt, "diag_shift": diag_shift})
    finally:
        run.close()
    return run.configs, records
