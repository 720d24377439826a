"""Markov chains at full size replayed by the oracle.

Z2 gauge field + hard-core bosons at half filling, D = 4 (D_k = 2), chi = 24
(every boundary-MPS bond truncated from 48), (h, g, J) = (1, 0.33, 0.5): the
largest lattices of the benchmark workload, 16x16 and 32x32; and pure Z3 on
16x16, D = 6, chi = 32, complex tensors, g = 0.375 (the Z3 workload).  The
library's FP64 form samples the chains with gcf_sample_batch (plaquette pass,
both hop passes with matter, then the measurement) and the oracle replays them from the same
starting configurations with the same SplitMix64 counters (Sec. S-1 sweep,
Eq. S2 E_loc).  In FP64 every Metropolis ratio agrees to ~1e-12, far from any
acceptance threshold, so the configurations after every sweep and the
acceptance counts must be equal bit for bit; log|psi| and E_loc of every
sample agree within the FP64 tolerance of the full-size amplitude tests.
"""

import numpy as np
import pytest

from oracle import vmc

from gpu_helpers import amp_err, configs_for, oracle_net

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

# (L, N, D, chi, matter, complex, g, chains, sweeps)
CASES = [(16, 2, 4, 24, True, False, 0.33, 2, 2), (32, 2, 4, 24, True, False, 0.33, 1, 1),
         (16, 3, 6, 32, False, True, 0.375, 1, 1)]


@pytest.mark.parametrize("L,N,D,chi,matter,cplx,g,n_chains,n_sweeps", CASES,
                         ids=["16x16-Z2-bosons", "32x32-Z2-bosons", "16x16-Z3-complex"])
def test_full_size_chains_replay_the_oracle(L, N, D, chi, matter, cplx, g, n_chains, n_sweeps):
    import paper_2503_20566_gb300 as G

    h, J = 1.0, (0.5 if matter else 0.0)
    lat, pe, vals = oracle_net(L, L, N, D, 5, complex_=cplx, matter=matter, precision="fp64")
    ctx = G.Context(N, L, L, D, chi, matter=matter, h=h, g=g, J=J, complex_=cplx, precision="fp64", seed=5)
    ctx.set_tensors(vals)
    cfgs, _, _ = configs_for(lat, n_chains, seed=6, n_bosons=L * L // 2 if matter else 0)
    dev = torch.from_numpy(cfgs).cuda()
    out = ctx.sample_batch(dev, n_sweeps, seed=77)
    torch.cuda.synchronize()
    assert ctx.svd_unconverged == 0
    la = out["log_abs"].cpu().numpy()
    ph = out["phase"].cpu().numpy()
    e = torch.view_as_complex(out["e_loc"].view(-1, 2)).cpu().numpy()
    acc = out["accepted"].cpu().numpy()
    prop = out["proposed"].cpu().numpy()
    final = dev.cpu().numpy()
    model = vmc.Model(h=h, g=g, J=J)
    worst_amp = worst_e = 0.0
    for c in range(n_chains):
        recs = vmc.run_chain(pe, model, cfgs[c], chi, 77, c, n_sweeps, measure=True)
        assert np.array_equal(final[c], recs[-1]["cfg"].astype(np.int8)), c
        assert acc[c] == sum(r["accepted"] for r in recs), c
        assert prop[c] == sum(r["proposed"] for r in recs), c
        for w, rec in enumerate(recs):
            s = c * n_sweeps + w
            worst_amp = max(worst_amp, amp_err(la[s], ph[s], rec["log_abs"], rec["phase"]))
            worst_e = max(worst_e, abs(e[s] - rec["e_loc"]) / max(1.0, abs(rec["e_loc"])))
    print(f"{L}x{L} Z{N}: {n_chains} chains x {n_sweeps} sweeps, {int(prop.sum())} moves proposed, "
          f"{int(acc.sum())} accepted; amplitude error max {worst_amp:.1e}, E_loc {worst_e:.1e}")
    assert worst_amp < 1e-7 and worst_e < 1e-7, (worst_amp, worst_e)
