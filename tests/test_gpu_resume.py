"""Resume from a checkpoint reproduces the chains bit for bit.

Step 0 (sampling + SR update) runs in one context, which is then checkpointed
and runs step 1.  The checkpoint is restored into a fresh context of the same
model, which runs step 1 with the same seed: configurations and every sample
output must be identical to the uninterrupted run's.
"""

import pytest

from gpu_helpers import configs_for, setup

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

KEYS = ("log_abs", "phase", "e_loc", "block_ids", "O", "accepted", "proposed")


def test_resume_reproduces_the_chains(tmp_path):
    import paper_2503_20566_gb300 as G
    from paper_2503_20566_gb300 import checkpoint as ck
    from paper_2503_20566_gb300.replicas import rank_seeds

    lat, pe, ctx = setup(4, 4, 2, 4, 4, seed=181, precision="fp32", h=1.0, g=0.4)
    cfgs, _, _ = configs_for(lat, 16, seed=182)
    dev = torch.from_numpy(cfgs).cuda()
    step_seed = rank_seeds(0)["step"]
    out0 = ctx.sample_batch(dev, 2, seed=step_seed(0))
    ctx.sr_step(out0, n_chains=16, diag_shift=1e-3, lr=0.05, max_iter=50)
    path = str(tmp_path / "run.ck")
    ck.save(path, ctx, dev, step=1, seed=0)
    out1 = ctx.sample_batch(dev, 2, seed=step_seed(1))
    torch.cuda.synchronize()

    got = ck.load(path)
    ctx2 = G.Context(2, 4, 4, 4, 4, precision="fp32", h=1.0, g=0.4, seed=999)
    dev2 = ck.restore(ctx2, got)
    out2 = ctx2.sample_batch(dev2, 2, seed=step_seed(got.step))
    torch.cuda.synchronize()
    assert torch.equal(dev2, dev)
    for key in KEYS:
        assert torch.equal(out2[key], out1[key]), key
