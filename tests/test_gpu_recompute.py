"""The checkpointed boundary-MPS store (gcf_model.recompute_env) against the
full store, bit for bit.

With recompute_env = K the sampling kernel keeps only every K-th B[r] / T[r]
of a chain and rebuilds the ones between from the kept one when a pass needs
them (the main text's "environments recomputed instead of stored when chi is
large").  A rebuilt MPS is the same sequence of operations on the same rows,
so every output must equal the full store's exactly: the Markov chains'
configurations, acceptance counts, log|psi|, phase, E_loc, block ids and O,
for sampling (plaquette and both hop passes with matter) and for the fixed-
configuration calls.  The scratch per chain slot shrinks; the figure for the
32x32 Z2 + bosons, D = 4, chi = 24 lattice is printed.
"""

import numpy as np
import pytest

from gpu_helpers import configs_for, setup

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

CASES = [
    (7, 9, 2, 4, 4, False, True, 2),    # Z2 + bosons, every pass, K = 2
    (6, 8, 3, 6, 5, True, False, 3),    # Z3 complex, truncated, K = 3
    (5, 10, 2, 4, 6, False, True, -1),  # K = ceil(sqrt(Ly + 1)) = 4
]


def _ids(c):
    return "{}x{}-Z{}-D{}-chi{}{}{}-K{}".format(c[0], c[1], c[2], c[3], c[4], "-c" if c[5] else "",
                                               "-m" if c[6] else "", c[7])


def _context(case, recompute):
    import paper_2503_20566_gb300 as G

    Lx, Ly, N, D, chi, cplx, matter, K = case
    lat, pe, ref = setup(Lx, Ly, N, D, chi, seed=131, complex_=cplx, matter=matter, h=1.0, g=0.4,
                         J=0.5 if matter else 0.0)
    if not recompute:
        return lat, ref
    ctx = G.Context(N, Lx, Ly, D, chi, matter=matter, h=1.0, g=0.4, J=0.5 if matter else 0.0, complex_=cplx,
                    precision="fp32", seed=131, recompute_env=K)
    ctx.set_tensors(ref.get_tensors())
    return lat, ctx


@pytest.mark.parametrize("case", CASES, ids=_ids)
def test_recomputed_environments_equal_the_full_store(case):
    Lx, Ly, N, D, chi, cplx, matter, K = case
    lat, full = _context(case, False)
    _, ck = _context(case, True)
    assert full.checkpoint_interval == 0
    assert ck.checkpoint_interval == (K if K > 0 else 4)
    nb = (Lx * Ly) // 4 * 2 if matter else 0  # even: sum of occupations = sum of Q = 0 mod 2
    cfgs, _, _ = configs_for(lat, 24, seed=132, n_bosons=nb)
    a = torch.from_numpy(cfgs).cuda()
    b = a.clone()
    oa = full.sample_batch(a, 3, seed=77)
    ob = ck.sample_batch(b, 3, seed=77)
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    for key in ("log_abs", "phase", "e_loc", "block_ids", "O", "accepted", "proposed"):
        assert torch.equal(oa[key], ob[key]), key
    # fixed configurations (bottom-up absorption, then the measurement pass)
    for fa, fb in ((full.amplitude(a), ck.amplitude(a)), ((full.local_energy(a),), (ck.local_energy(a),)),
                   (full.log_grad(a), ck.log_grad(a))):
        for x, y in zip(fa, fb):
            assert torch.equal(x, y)
    assert ck.scratch_bytes_per_chain < full.scratch_bytes_per_chain


def test_scratch_per_chain_of_the_large_lattice():
    import paper_2503_20566_gb300 as G

    sizes = {}
    for K in (0, -1):
        ctx = G.Context(2, 32, 32, 4, 24, matter=True, h=1.0, g=0.33, J=0.5, precision="fp32", seed=1,
                        recompute_env=K)
        sizes[K] = (ctx.scratch_bytes_per_chain, ctx.checkpoint_interval)
        ctx.close()
    print("32x32 Z2 + bosons D=4 chi=24 scratch per chain slot: full store %.2f MB, checkpointed (K=%d) %.2f MB"
          % (sizes[0][0] / 1e6, sizes[-1][1], sizes[-1][0] / 1e6))
    assert sizes[-1][0] < 0.6 * sizes[0][0]
