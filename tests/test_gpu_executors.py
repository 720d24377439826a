"""Both executors of the sampling kernel, at every shared-memory placement
level, give the oracle's results.

The library runs a chain either on a whole CTA or on one of two or four
128-thread groups of a CTA (optionally in lockstep: the groups meet before
every row of a pass), and keeps none, the hot buffers (1), also the staged
B / T rows (2), or also the right environments (3) in shared memory.
GCFVMC_EXEC, GCFVMC_SMEM / GCFVMC_SMEM_CTA and GCFVMC_LOCK force a form at
context creation; each is checked against the FP64 oracle on the same seeded
inputs, with amplitudes and a replayed Markov chain (3 chains, so a
four-group CTA also runs with groups that have no chain).  Forms that do not
fit an SM are skipped.
"""

import numpy as np
import pytest

from oracle import vmc

from gpu_helpers import TOL, amp_err, configs_for, setup

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

CASES = [
    (8, 8, 2, 4, 16, False, False, "fp32"),  # the 8x8 Z2 D=4 chi=16 workload shape
    (3, 7, 3, 6, 4, True, False, "fp32"),    # Z3 complex, ragged, truncated
    (4, 3, 2, 4, 4, False, True, "fp32"),    # Z2 + hard-core bosons
]


def _ids(c):
    return "{}x{}-Z{}-D{}-chi{}{}{}".format(c[0], c[1], c[2], c[3], c[4], "-c" if c[5] else "", "-m" if c[6] else "")


@pytest.mark.parametrize("executor,level,lock", [("cta", 0, 0), ("cta", 1, 0), ("cta", 3, 0), ("group", 1, 0),
                                                 ("group", 2, 0), ("group", 3, 0), ("group", 1, 1),
                                                 ("group4", 1, 0), ("group4", 1, 1), ("group4", 2, 1)])
@pytest.mark.parametrize("case", CASES, ids=_ids)
def test_executor_amplitude_and_chain(case, executor, level, lock, monkeypatch):
    import paper_2503_20566_gb300 as G

    monkeypatch.setenv("GCFVMC_EXEC", executor)
    monkeypatch.setenv("GCFVMC_SMEM" if executor.startswith("group") else "GCFVMC_SMEM_CTA", str(level))
    monkeypatch.setenv("GCFVMC_LOCK", str(lock))
    Lx, Ly, N, D, chi, cplx, matter, prec = case
    h, g, J = 1.0, 0.4, (0.5 if matter else 0.0)
    lat, pe, ctx = setup(Lx, Ly, N, D, chi, seed=61, complex_=cplx, matter=matter, precision=prec, h=h, g=g, J=J)
    nb = (Lx * Ly) // 2 if matter else 0
    # amplitudes of independent configurations
    cfgs, _, _ = configs_for(lat, 12, seed=62, n_bosons=nb)
    try:
        la, ph = ctx.amplitude(torch.from_numpy(cfgs).cuda())
    except G.GcfError as err:
        if "does not fit" in str(err) or "too many resources" in str(err) or "invalid argument" in str(err):
            pytest.skip(f"{executor} level {level} does not fit an SM: {err}")
        raise
    la, ph = la.cpu().numpy(), ph.cpu().numpy()
    for i in range(len(cfgs)):
        ref = vmc.amplitude(pe, cfgs[i], chi)
        assert amp_err(la[i], ph[i], ref[0], ref[1]) < TOL[prec], i
    # a short chain, replayed by the oracle
    n_chains, n_sweeps = 3, 2
    dev = torch.from_numpy(cfgs[:n_chains].copy()).cuda()
    out = ctx.sample_batch(dev, n_sweeps, seed=4242)
    torch.cuda.synchronize()
    la = out["log_abs"].cpu().numpy()
    final = dev.cpu().numpy()
    model = vmc.Model(h=h, g=g, J=J)
    for c in range(n_chains):
        recs = vmc.run_chain(pe, model, cfgs[c], chi, 4242, c, n_sweeps, measure=True)
        assert np.array_equal(final[c], recs[-1]["cfg"].astype(np.int8)), c
        for w, rec in enumerate(recs):
            assert amp_err(la[c * n_sweeps + w], 0.0, rec["log_abs"], 0.0) < TOL[prec] * 10


def test_lockstep_wait_that_runs_out_is_reported_and_results_stay_exact(monkeypatch):
    """A lockstep wait with nobody to meet: the test hook makes one group of a
    four-group CTA never count in, so every wait runs to its iteration limit.
    The kernel must end, report the timeouts through the status the host
    reads, and still produce the oracle's chains; without the hook no wait
    runs out."""
    monkeypatch.setenv("GCFVMC_EXEC", "group4")
    monkeypatch.setenv("GCFVMC_LOCK", "1")
    for fault in (1, 0):
        monkeypatch.setenv("GCFVMC_LOCK_FAULT", str(fault))
        lat, pe, ctx = setup(4, 4, 2, 4, 4, seed=131, precision="fp32", h=1.0, g=0.4)
        cfgs, _, _ = configs_for(lat, 4, seed=132)  # four chains: one CTA, every group busy
        dev = torch.from_numpy(cfgs).cuda()
        out = ctx.sample_batch(dev, 2, seed=77)
        torch.cuda.synchronize()
        if fault:
            assert ctx.phase_timeouts >= 1
        else:
            assert ctx.phase_timeouts == 0
        final = dev.cpu().numpy()
        la = out["log_abs"].cpu().numpy()
        model = vmc.Model(h=1.0, g=0.4)
        for c in range(len(cfgs)):
            recs = vmc.run_chain(pe, model, cfgs[c], 4, 77, c, 2, measure=True)
            assert np.array_equal(final[c], recs[-1]["cfg"].astype(np.int8)), c
            for w, rec in enumerate(recs):
                assert amp_err(la[c * 2 + w], 0.0, rec["log_abs"], 0.0) < TOL["fp32"] * 10
