"""Host drivers of whole runs (SR optimisation, tVMC trajectory), checked on
the CPU with a stand-in context that records the library calls: the order of
sampling and solve calls, the modes and step sizes (two-stage tVMC, Eqs.
S6-S8), the seeds per pass, the per-step JSONL records, and that a run resumed
from a periodic checkpoint ends in the same state as an uninterrupted one."""

import json

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2503_20566_gb300 import checkpoint as ck  # noqa: E402
from paper_2503_20566_gb300 import drivers  # noqa: E402
from paper_2503_20566_gb300.binding import SR, TDVP_STAGE1, TDVP_STAGE2  # noqa: E402


class Stand:
    """Records calls; parameters and configurations change deterministically
    with the seed and the update, so runs can be compared exactly."""

    def __init__(self, complex_=False):
        self.N, self.Lx, self.Ly, self.D, self.chi = 2, 3, 3, 4, 2
        self.matter, self.complex, self.precision = False, complex_, "fp32"
        self.h, self.g, self.J, self.m, self.Q = 1.0, 0.3, 0.0, 0.0, None
        self.n_params, self.cfg_len = 10, 21
        self.params = np.linspace(0.1, 1.0, self.n_params) * (1 + 1j if complex_ else 1)
        self.calls = []

    def get_tensors(self):
        return self.params.copy()

    def set_tensors(self, values):
        self.params = np.array(values, copy=True)

    def alloc_samples(self, n_chains, n_sweeps, grad=True):
        return {"accepted": torch.zeros(n_chains, dtype=torch.int32),
                "proposed": torch.zeros(n_chains, dtype=torch.int32), "seed": [None]}

    def sample_batch(self, configs, n_sweeps, seed, out=None):
        self.calls.append(("sample", seed))
        configs.copy_((configs.to(torch.int64) * 3 + seed % 5) % 2)
        out["accepted"].fill_(1)
        out["proposed"].fill_(4)
        out["seed"][0] = seed
        return out

    def sr_step(self, samples, n_chains, diag_shift=1e-4, lr=0.01, mode=SR, dt=0.0, max_iter=100, tol=1e-10):
        self.calls.append(("sr", mode, dt, lr))
        e = float(np.real(self.params.sum()))
        step = (samples["seed"][0] % 7 + 1) * 1e-3
        self.params = self.params - (lr if mode == SR else dt) * step * (1 if mode != TDVP_STAGE2 else 2)
        return [e, 0.0, 0.01, 5.0, 1e-7, 1.0, 1.0, 0.0]


def _configs():
    return torch.from_numpy(np.random.default_rng(0).integers(0, 2, size=(4, 21)).astype(np.int8))


def test_sr_optimize_samples_then_solves_each_step(tmp_path):
    ctx = Stand()
    seed_of = drivers.default_seed_of_step(5)
    log = str(tmp_path / "run.jsonl")
    cfg, recs = drivers.sr_optimize(ctx, _configs(), n_steps=3, n_sweeps=2, seed=5, lr=0.02, log_path=log)
    assert ctx.calls == [("sample", seed_of(0)), ("sr", SR, 0.0, 0.02), ("sample", seed_of(1)),
                         ("sr", SR, 0.0, 0.02), ("sample", seed_of(2)), ("sr", SR, 0.0, 0.02)]
    assert [r["step"] for r in recs] == [0, 1, 2]
    assert all(r["acceptance"] == 0.25 and r["samples"] == 8 and r["cg_converged"] for r in recs)
    lines = [json.loads(x) for x in open(log)]
    assert [x["e_mean"] for x in lines] == [r["e_mean"] for r in recs]


def test_tvmc_runs_two_stages_per_step():
    ctx = Stand(complex_=True)
    seed_of = drivers.default_seed_of_step(1)
    cfg, recs = drivers.tvmc_evolve(ctx, _configs(), n_steps=2, dt=0.01, n_sweeps=1, seed=1)
    assert ctx.calls == [("sample", seed_of(0)), ("sr", TDVP_STAGE1, 0.01, 0.0),
                         ("sample", seed_of(1)), ("sr", TDVP_STAGE2, 0.01, 0.0),
                         ("sample", seed_of(2)), ("sr", TDVP_STAGE1, 0.01, 0.0),
                         ("sample", seed_of(3)), ("sr", TDVP_STAGE2, 0.01, 0.0)]
    assert [r["time"] for r in recs] == [0.0, 0.01]
    assert all("stage2" in r and r["samples"] == 8 for r in recs)
    with pytest.raises(ValueError, match="complex"):
        drivers.tvmc_evolve(Stand(), _configs(), n_steps=1, dt=0.01, n_sweeps=1)


@pytest.mark.parametrize("kind", ["sr", "tvmc"])
def test_resumed_run_ends_where_the_uninterrupted_run_ends(tmp_path, kind):
    def run(ctx, n_steps, **kw):
        if kind == "sr":
            return drivers.sr_optimize(ctx, _configs(), n_steps=n_steps, n_sweeps=2, seed=9, **kw)
        return drivers.tvmc_evolve(ctx, _configs(), n_steps=n_steps, dt=0.02, n_sweeps=2, seed=9, **kw)

    full = Stand(complex_=(kind == "tvmc"))
    cfg_full, recs_full = run(full, 5)
    path = str(tmp_path / "run.ck")
    first = Stand(complex_=(kind == "tvmc"))
    run(first, 3, checkpoint_path=path, checkpoint_every=1)
    saved = ck.load(path)
    assert saved.step == 3 and saved.extra["driver"] == kind
    second = Stand(complex_=(kind == "tvmc"))
    second.params = second.params * 0  # a fresh context: everything comes from the checkpoint
    cfg_res, recs_res = run(second, 5, resume=saved)
    assert [r["step"] for r in recs_res] == [3, 4]
    assert np.array_equal(second.params, full.params)
    assert torch.equal(cfg_res, cfg_full)
    assert [r["e_mean"] for r in recs_res] == [r["e_mean"] for r in recs_full[3:]]
