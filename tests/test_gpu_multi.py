"""gcf_sample_multi: lattices of different sizes advanced in one launch.

Each context's chains must evolve exactly as gcf_sample_batch would evolve
them with that context's seed (same kernel arithmetic: one chain per CTA), and
one chain is replayed by the FP64 oracle.
"""

import numpy as np
import pytest

from oracle import vmc

from gpu_helpers import TOL, amp_err, configs_for, setup

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

SIZES = [(4, 4), (5, 4), (6, 6)]


def _contexts(matter):
    out = []
    for i, (Lx, Ly) in enumerate(SIZES):
        lat, pe, ctx = setup(Lx, Ly, 2, 4, 4, seed=91 + i, matter=matter, precision="fp32", h=1.0, g=0.33,
                             J=0.5 if matter else 0.0)
        nb = (Lx * Ly) // 2 if matter else 0
        cfgs, _, _ = configs_for(lat, 3 + i, seed=95 + i, n_bosons=nb)
        out.append((lat, pe, ctx, cfgs))
    return out


@pytest.mark.parametrize("form", ["cta", "group4"])
@pytest.mark.parametrize("matter", [False, True], ids=["gauge", "matter"])
def test_sample_multi_equals_per_context_sampling(matter, form, monkeypatch):
    """Both forms of the launch (one chain per CTA; four chains per CTA, the
    form taken when a context truncates) against per-context sampling in
    the same executor."""
    import paper_2503_20566_gb300 as G

    monkeypatch.setenv("GCFVMC_EXEC", form)
    monkeypatch.setenv("GCFVMC_MULTI", form)
    items = _contexts(matter)
    seeds = [1001, 2002, 3003]
    n_sweeps = 2
    dev = [torch.from_numpy(c).cuda() for (_, _, _, c) in items]
    outs = G.sample_multi([it[2] for it in items], dev, n_sweeps, seeds)
    torch.cuda.synchronize()
    assert items[0][2].multi_chains_per_cta == (4 if form == "group4" else 1)
    for (lat, pe, ctx, cfgs), d, o, sd in zip(items, dev, outs, seeds):
        ref_cfg = torch.from_numpy(cfgs).cuda()
        ref = ctx.sample_batch(ref_cfg, n_sweeps, seed=sd)
        torch.cuda.synchronize()
        assert torch.equal(d, ref_cfg)
        for key in ("log_abs", "e_loc", "O", "block_ids", "accepted", "proposed"):
            assert torch.equal(o[key], ref[key]), key
    # the first context's first chain against the oracle
    lat, pe, ctx, cfgs = items[0]
    model = vmc.Model(h=1.0, g=0.33, J=0.5 if matter else 0.0)
    recs = vmc.run_chain(pe, model, cfgs[0], 4, seeds[0], 0, n_sweeps, measure=True)
    assert np.array_equal(dev[0][0].cpu().numpy(), recs[-1]["cfg"].astype(np.int8))
    la = outs[0]["log_abs"].cpu().numpy()
    for w, rec in enumerate(recs):
        assert amp_err(la[w], 0.0, rec["log_abs"], 0.0) < TOL["fp32"] * 10


def test_sample_multi_rejects_mixed_scalar_types():
    import paper_2503_20566_gb300 as G

    _, _, a = setup(4, 4, 2, 4, 4, seed=1, precision="fp32")
    _, _, b = setup(4, 4, 2, 4, 4, seed=2, precision="fp64")
    ca, cb = a.init_configs(2), b.init_configs(2)
    with pytest.raises(G.GcfError):
        G.sample_multi([a, b], [ca, cb], 1, [1, 2])
