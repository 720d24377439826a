"""The persistent sampling launch recorded in a CUDA graph.

gcf_sample_batch_async enqueues the sampling kernel with no host
synchronisation and no allocation; recorded once with torch.cuda.graph and
replayed from the same starting configurations, it must reproduce the
synchronous gcf_sample_batch bit for bit, replay after replay.
"""

import pytest

from gpu_helpers import configs_for, setup

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

KEYS = ("log_abs", "phase", "e_loc", "block_ids", "O", "accepted", "proposed")


@pytest.mark.parametrize("case", [(4, 4, 2, 4, 4, False), (5, 4, 3, 6, 4, True)], ids=["z2-4x4", "z3-5x4-c"])
def test_sampling_launch_replays_from_a_cuda_graph(case):
    Lx, Ly, N, D, chi, cplx = case
    lat, pe, ctx = setup(Lx, Ly, N, D, chi, seed=111, complex_=cplx, precision="fp32")
    n, n_sweeps, seed = 64, 2, 2024
    cfgs, _, _ = configs_for(lat, n, seed=112)
    host = torch.from_numpy(cfgs)
    # reference (the synchronous call also sizes the scratch)
    ref_cfg = host.cuda()
    ref = ctx.sample_batch(ref_cfg, n_sweeps, seed=seed)
    torch.cuda.synchronize()
    static_cfg = host.cuda()
    out = ctx.alloc_samples(n, n_sweeps)
    ctx.sample_batch_async(static_cfg, n_sweeps, seed, out, stream=torch.cuda.current_stream())
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        ctx.sample_batch_async(static_cfg, n_sweeps, seed, out, stream=torch.cuda.current_stream())
    for _ in range(2):
        static_cfg.copy_(host)
        for key in KEYS:
            out[key].zero_()
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(static_cfg, ref_cfg)
        for key in KEYS:
            assert torch.equal(out[key], ref[key]), key


def test_async_sampling_refuses_unsized_scratch():
    import paper_2503_20566_gb300 as G

    lat, pe, ctx = setup(4, 4, 2, 4, 4, seed=113, precision="fp32")
    cfgs, _, _ = configs_for(lat, 8, seed=114)
    dev = torch.from_numpy(cfgs).cuda()
    out = ctx.alloc_samples(8, 1)
    with pytest.raises(G.GcfError):
        ctx.sample_batch_async(dev, 1, 1, out)
