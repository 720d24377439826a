"""Edge cases of the boundary, against the oracle or the header's stated error
behaviour.

* Empty batches: every batch call with zero configurations succeeds, launches
  no kernel and writes nothing (the VJP of an empty batch is zero).
* Static background charges Q_x (Eq. 1): starting configurations bit-exact,
  amplitudes, E_loc and O, and a replayed chain, with and without matter.
* The narrowest lattices the method has: 2 x L and L x 2 strips (one column or
  one row of plaquettes) and 2 x 2 (a single plaquette).
* chi = 1: the boundary MPS truncated to a product state at every cut.
* Arguments the header rejects: lattice sides outside [2, 64], D not a multiple
  of N, chi < 1, n_sweeps < 1, an SR step without samples.
"""

import numpy as np
import pytest

from oracle import vmc
from oracle.lattice import Lattice

from gpu_helpers import TOL, amp_err, configs_for, setup
from paper_2503_20566_gb300.binding import GCF_EINVAL

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _check_fixed(lat, pe, ctx, cfgs, chi, prec, model):
    """Amplitude, E_loc and O of fixed configurations against the oracle."""
    dev = torch.from_numpy(cfgs).cuda()
    la, ph = (t.cpu().numpy() for t in ctx.amplitude(dev))
    e = ctx.local_energy(dev).cpu().numpy()
    bid, O = (t.cpu().numpy() for t in ctx.log_grad(dev))
    for i, c in enumerate(cfgs):
        ola, oph = vmc.amplitude(pe, c, chi)
        assert amp_err(la[i], ph[i], ola, oph) < TOL[prec], i
        ref = vmc.local_energy(pe, model, c, chi)
        scale = max(1.0, abs(ref - lat.diagonal_energy(c, model.g)))
        assert abs(e[i] - ref) <= TOL[prec] * scale * 10, (i, e[i], ref)
        for v, (rb, rblk) in enumerate(vmc.log_grad(pe, c, chi)):
            assert bid[i, v] == rb
            r = rblk.reshape(-1)
            assert np.abs(O[i, v, : r.size] - r).max() <= TOL[prec] * max(1.0, np.abs(r).max()) * 10, (i, v)


def _check_chain(pe, ctx, cfgs, chi, prec, model, n_sweeps=2, seed=4321):
    """A short Markov chain per configuration, replayed by the oracle."""
    dev = torch.from_numpy(cfgs).cuda()
    out = ctx.sample_batch(dev, n_sweeps, seed=seed)
    torch.cuda.synchronize()
    final = dev.cpu().numpy()
    la = out["log_abs"].cpu().numpy()
    e = torch.view_as_complex(out["e_loc"].view(-1, 2)).cpu().numpy()
    for c in range(len(cfgs)):
        recs = vmc.run_chain(pe, model, cfgs[c], chi, seed, c, n_sweeps, measure=True)
        assert np.array_equal(final[c], recs[-1]["cfg"].astype(np.int8)), c
        for w, rec in enumerate(recs):
            s = c * n_sweeps + w
            assert amp_err(la[s], 0.0, rec["log_abs"], 0.0) < TOL[prec] * 10
            assert abs(e[s] - rec["e_loc"]) <= TOL[prec] * max(1.0, abs(rec["e_loc"])) * 10
        assert int(out["accepted"][c]) == sum(r["accepted"] for r in recs)


def test_empty_batches_launch_nothing():
    lat, pe, ctx = setup(4, 4, 2, 4, 4, seed=141, precision="fp32")
    empty = torch.empty((0, lat.cfg_len), dtype=torch.int8, device="cuda")
    n0 = ctx.launch_count
    la, ph = ctx.amplitude(empty)
    e = ctx.local_energy(empty)
    bid, O = ctx.log_grad(empty)
    out = ctx.sample_batch(empty, 2, seed=1)
    g = ctx.log_grad_vjp(empty, np.zeros(0))
    torch.cuda.synchronize()
    assert ctx.launch_count == n0
    assert la.numel() == ph.numel() == e.numel() == bid.numel() == O.numel() == 0
    assert all(t.numel() == 0 for t in out.values())
    assert g.shape[0] == ctx.n_params and torch.count_nonzero(g) == 0


@pytest.mark.parametrize("case", [
    # (Lx, Ly, N, D, chi, complex, matter, Q, n_bosons)
    (4, 3, 3, 6, 4, True, False, [[1, 0, 0, 0], [0, 0, 0, 0], [0, 0, 0, 2]], 0),
    (4, 3, 2, 4, 4, False, True, [[0, 0, 0, 0], [0, 1, 0, 0], [0, 0, 0, 0]], 5),
], ids=["z3-4x3-c-Q", "z2-4x3-m-Q"])
def test_background_charges(case):
    import paper_2503_20566_gb300 as G

    Lx, Ly, N, D, chi, cplx, matter, Q, nb = case
    h, g, J = 1.0, 0.4, (0.5 if matter else 0.0)
    lat, pe, ctx = setup(Lx, Ly, N, D, chi, seed=151, complex_=cplx, matter=matter, precision="fp64",
                         h=h, g=g, J=J, Q=Q)
    model = vmc.Model(h=h, g=g, J=J)
    cfgs, occ, powers = configs_for(lat, 4, seed=152, n_bosons=nb)
    assert all(lat.is_physical(c) for c in cfgs)
    got = ctx.init_configs(4, occupations=torch.from_numpy(occ) if matter else None,
                           powers=torch.from_numpy(powers)).cpu().numpy()
    assert np.array_equal(got, cfgs)
    # a configuration that is physical for Q = 0 violates this Gauss law
    free = Lattice(Lx, Ly, N, matter=matter)
    cfg0, _, _ = configs_for(free, 1, seed=153, n_bosons=nb + (1 if matter else 0))
    la, _ = ctx.amplitude(torch.from_numpy(cfg0))
    assert np.isneginf(la.cpu().numpy()[0])
    with pytest.raises(G.GcfError):
        ctx.local_energy(torch.from_numpy(cfg0))
    _check_fixed(lat, pe, ctx, cfgs[:3], chi, "fp64", model)
    _check_chain(pe, ctx, cfgs[:2], chi, "fp64", model)


@pytest.mark.parametrize("case", [
    # (Lx, Ly, N, D, chi, complex, matter, precision)
    (2, 5, 2, 4, 2, False, False, "fp32"),
    (6, 2, 3, 6, 4, True, False, "fp64"),
    (2, 2, 2, 4, 2, False, False, "fp64"),
    (2, 4, 2, 4, 2, False, True, "fp32"),
    (5, 4, 2, 4, 1, False, False, "fp64"),   # chi = 1
    (4, 4, 3, 6, 1, True, False, "fp64"),    # chi = 1, complex
], ids=["2x5-z2", "6x2-z3-c", "2x2-z2", "2x4-z2-m", "5x4-chi1", "4x4-z3-c-chi1"])
def test_narrow_lattices_and_chi_one(case):
    Lx, Ly, N, D, chi, cplx, matter, prec = case
    h, g, J = 1.0, 0.35, (0.5 if matter else 0.0)
    lat, pe, ctx = setup(Lx, Ly, N, D, chi, seed=161, complex_=cplx, matter=matter, precision=prec,
                         h=h, g=g, J=J)
    model = vmc.Model(h=h, g=g, J=J)
    nb = (Lx * Ly) // 2 if matter else 0
    cfgs, _, _ = configs_for(lat, 4, seed=162, n_bosons=nb)
    _check_fixed(lat, pe, ctx, cfgs[:3], chi, prec, model)
    _check_chain(pe, ctx, cfgs, chi, prec, model)


@pytest.mark.parametrize("args", [
    dict(N=2, Lx=1, Ly=4, D=4, chi=2), dict(N=2, Lx=4, Ly=1, D=4, chi=2), dict(N=2, Lx=65, Ly=4, D=4, chi=2),
    dict(N=2, Lx=4, Ly=4, D=5, chi=2), dict(N=3, Lx=4, Ly=4, D=2, chi=2), dict(N=2, Lx=4, Ly=4, D=4, chi=0),
    dict(N=1, Lx=4, Ly=4, D=4, chi=2),
], ids=["Lx1", "Ly1", "Lx65", "D-not-multiple", "D-below-N", "chi0", "N1"])
def test_rejected_models(args):
    import paper_2503_20566_gb300 as G

    with pytest.raises(G.GcfError) as ei:
        G.Context(args["N"], args["Lx"], args["Ly"], args["D"], args["chi"], precision="fp32")
    assert ei.value.status == GCF_EINVAL


def test_rejected_calls():
    import paper_2503_20566_gb300 as G

    lat, pe, ctx = setup(4, 4, 2, 4, 4, seed=171, precision="fp32")
    cfgs, _, _ = configs_for(lat, 2, seed=172)
    dev = torch.from_numpy(cfgs).cuda()
    n0 = ctx.launch_count
    with pytest.raises(G.GcfError) as ei:
        ctx.sample_batch(dev, 0, seed=1)
    assert ei.value.status == GCF_EINVAL
    empty = ctx.alloc_samples(0, 1)
    with pytest.raises(G.GcfError) as ei:
        ctx.sr_step(empty, 0)
    assert ei.value.status == GCF_EINVAL
    assert ctx.launch_count == n0
    assert np.array_equal(dev.cpu().numpy(), cfgs)


def test_svd_sweep_limit_is_reported():
    """A truncated-bond SVD that stops at its sweep limit is reported, not
    silent: with one Jacobi sweep a truncating contraction cannot converge,
    so gcf_amplitude returns GCF_ETIMEOUT and counts the SVDs; with the
    default limit the same call converges, reports none and matches the
    oracle."""
    from paper_2503_20566_gb300.binding import GCF_ETIMEOUT, GcfError

    Lx, Ly, N, D, chi = 6, 5, 2, 4, 3
    lat, pe, ctx = setup(Lx, Ly, N, D, chi, seed=151)
    cfgs, _, _ = configs_for(lat, 3, seed=152)
    dev = torch.from_numpy(cfgs).cuda()
    la, ph = (t.cpu().numpy() for t in ctx.amplitude(dev))
    assert ctx.svd_unconverged == 0
    for i, c in enumerate(cfgs):
        assert amp_err(la[i], ph[i], *vmc.amplitude(pe, c, chi)) < TOL["fp32"]
    ctx.set_svd_sweeps(1)
    with pytest.raises(GcfError) as err:
        ctx.amplitude(dev)
    assert err.value.status == GCF_ETIMEOUT
    assert ctx.svd_unconverged > 0
    ctx.set_svd_sweeps(40)
    ctx.amplitude(dev)
    assert ctx.svd_unconverged == 0
    with pytest.raises(GcfError) as err:
        ctx.set_svd_sweeps(0)
    assert err.value.status == GCF_EINVAL
