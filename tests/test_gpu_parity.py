"""GPU parity: the CUDA library (through its C ABI) against the FP64 oracle.

Every comparison uses inputs produced by ``synth`` and the oracle only.  FP32
results must agree within relative error 1e-4 (|delta log|psi|| + phase, per
sample; E_loc and O relative to their size), FP64 within 1e-9.
"""

import numpy as np
import pytest

import synth
from oracle import peps as P
from oracle import vmc
from oracle.lattice import Lattice

from gpu_helpers import TOL, amp_err, configs_for, setup

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import paper_2503_20566_gb300 as G

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    G.load_library()


# (Lx, Ly, N, D, chi, complex, matter, precision): exact and truncated chi,
# real and complex, Z2/Z3/Z4, ragged shapes, D_k = 1, 2, 3.
AMP_CASES = [
    (4, 4, 2, 2, 4, False, False, "fp64"),   # 4x4 Z2 D=2 chi=4 (D_k = 1), FP64
    (8, 8, 2, 4, 16, False, False, "fp32"),  # 8x8 Z2 D=4 chi=16 (exact), FP32
    (6, 5, 2, 4, 4, False, False, "fp32"),   # truncated chi < 2^3
    (7, 3, 2, 4, 4, False, False, "fp32"),   # ragged
    (3, 7, 3, 6, 4, True, False, "fp32"),    # Z3 complex, ragged
    (5, 4, 3, 6, 2, True, False, "fp64"),    # Z3 complex truncated, FP64
    (4, 4, 4, 8, 4, True, False, "fp32"),    # Z4 complex
    (5, 5, 2, 6, 5, False, False, "fp32"),   # D_k = 3 truncated
    (4, 3, 2, 4, 4, False, True, "fp32"),    # Z2 + hard-core bosons
    (3, 3, 2, 6, 3, False, True, "fp64"),    # Z2 + bosons, D_k = 3 (the 3x3 ED check's lattice)
    (3, 3, 2, 6, 3, False, True, "fp32"),
]


def _ids(c):
    return "{}x{}-Z{}-D{}-chi{}-{}{}-{}".format(c[0], c[1], c[2], c[3], c[4], "c" if c[5] else "r",
                                                 "-m" if c[6] else "", c[7])


@pytest.mark.parametrize("case", AMP_CASES, ids=_ids)
def test_amplitude_parity(case):
    Lx, Ly, N, D, chi, cplx, matter, prec = case
    lat, pe, ctx = setup(Lx, Ly, N, D, chi, seed=11, complex_=cplx, matter=matter, precision=prec)
    nb = (Lx * Ly) // 2 if matter else 0
    cfgs, _, _ = configs_for(lat, 6, seed=21, n_bosons=nb)
    la, ph = ctx.amplitude(torch.from_numpy(cfgs))
    la, ph = la.cpu().numpy(), ph.cpu().numpy()
    for i, c in enumerate(cfgs):
        ola, oph = vmc.amplitude(pe, c, chi)
        assert amp_err(la[i], ph[i], ola, oph) < TOL[prec], (i, la[i], ola, ph[i], oph)


@pytest.mark.parametrize("case", AMP_CASES[:6] + AMP_CASES[7:], ids=_ids)
def test_local_energy_parity(case):
    Lx, Ly, N, D, chi, cplx, matter, prec = case
    h, g, J = 1.0, 0.37, (0.5 if matter else 0.0)
    lat, pe, ctx = setup(Lx, Ly, N, D, chi, seed=12, complex_=cplx, matter=matter, precision=prec,
                         h=h, g=g, J=J)
    nb = (Lx * Ly) // 2 if matter else 0
    cfgs, _, _ = configs_for(lat, 3, seed=22, n_bosons=nb)
    e = ctx.local_energy(torch.from_numpy(cfgs)).cpu().numpy()
    model = vmc.Model(h=h, g=g, J=J)
    for i, c in enumerate(cfgs):
        ref = vmc.local_energy(pe, model, c, chi)
        scale_ = max(1.0, abs(ref - lat.diagonal_energy(c, g)))
        assert abs(e[i] - ref) <= TOL[prec] * scale_ * 10, (i, e[i], ref)


@pytest.mark.parametrize("case", [AMP_CASES[0], AMP_CASES[1], AMP_CASES[2], AMP_CASES[4], AMP_CASES[8],
                                  AMP_CASES[9], AMP_CASES[10]],
                         ids=_ids)
def test_log_grad_parity(case):
    Lx, Ly, N, D, chi, cplx, matter, prec = case
    lat, pe, ctx = setup(Lx, Ly, N, D, chi, seed=13, complex_=cplx, matter=matter, precision=prec)
    nb = (Lx * Ly) // 2 if matter else 0
    cfgs, _, _ = configs_for(lat, 2, seed=23, n_bosons=nb)
    bid, O = ctx.log_grad(torch.from_numpy(cfgs))
    bid, O = bid.cpu().numpy(), O.cpu().numpy()
    for i, c in enumerate(cfgs):
        ref = vmc.log_grad(pe, c, chi)
        for v, (rb, rblk) in enumerate(ref):
            assert bid[i, v] == rb
            r = rblk.reshape(-1)
            got = O[i, v, : r.size]
            assert np.abs(got - r).max() <= TOL[prec] * max(1.0, np.abs(r).max()) * 10, (i, v)


def test_init_tensors_follow_the_generator():
    import paper_2503_20566_gb300 as G

    for cplx in (False, True):
        ctx = G.Context(3, 5, 4, 6, 4, complex_=cplx, precision="fp32", seed=99)
        ref = synth.round_to(synth.tensor_entries(99, ctx.n_params, cplx), "c64" if cplx else "f32")
        got = ctx.get_tensors()
        assert np.allclose(got, ref, rtol=1e-6, atol=1e-7)


@pytest.mark.parametrize("N,matter", [(2, False), (3, False), (4, False), (2, True)])
def test_init_configs_bit_exact(N, matter):
    import paper_2503_20566_gb300 as G

    Lx, Ly = 5, 4
    lat = Lattice(Lx, Ly, N, matter=matter)
    ctx = G.Context(N, Lx, Ly, N, 2, matter=matter, precision="fp32")
    nb = 6 if matter else 0
    cfgs, occ, powers = configs_for(lat, 40, seed=31, n_bosons=nb)
    got = ctx.init_configs(40, occupations=torch.from_numpy(occ) if matter else None,
                           powers=torch.from_numpy(powers)).cpu().numpy()
    assert np.array_equal(got, cfgs)


def test_unphysical_configuration_handling():
    import paper_2503_20566_gb300 as G

    lat, pe, ctx = setup(4, 4, 2, 4, 4, seed=5)
    cfgs, _, _ = configs_for(lat, 2, seed=6)
    bad = cfgs.copy()
    bad[1, lat.hi(1, 1)] ^= 1
    la, ph = ctx.amplitude(torch.from_numpy(bad))
    la = la.cpu().numpy()
    assert np.isneginf(la[1]) and np.isfinite(la[0])
    with pytest.raises(G.GcfError) as ei:
        ctx.local_energy(torch.from_numpy(bad))
    assert ei.value.status == 4
    with pytest.raises(G.GcfError):
        ctx.set_tensors(np.full(ctx.n_params, np.nan))


def _replay_chain(pe, model, cfg0, chi, seed, chain, n_sweeps):
    return vmc.run_chain(pe, model, cfg0, chi, seed, chain, n_sweeps, measure=True)


@pytest.mark.parametrize("case", [
    (4, 4, 2, 4, 4, False, False, "fp64", 6, 3),
    (4, 3, 3, 6, 4, True, False, "fp64", 4, 3),
    (4, 3, 2, 4, 4, False, True, "fp64", 4, 2),
    (5, 4, 2, 4, 4, False, False, "fp32", 4, 2),
    (3, 3, 2, 6, 3, False, True, "fp64", 6, 4),
    (3, 3, 2, 6, 3, False, True, "fp32", 6, 4),
], ids=lambda c: "{}x{}-Z{}-{}{}-{}".format(c[0], c[1], c[2], "c" if c[5] else "r", "-m" if c[6] else "", c[7]))
def test_sample_batch_replays_oracle_chain(case):
    """Same starting configurations, seed and SplitMix64 counters: the GPU
    chains equal the oracle's sweep by sweep (configurations bit-exact,
    measurements within tolerance)."""
    Lx, Ly, N, D, chi, cplx, matter, prec, n_chains, n_sweeps = case
    h, g, J = 1.0, 0.4, (0.5 if matter else 0.0)
    lat, pe, ctx = setup(Lx, Ly, N, D, chi, seed=14, complex_=cplx, matter=matter, precision=prec, h=h, g=g, J=J)
    nb = (Lx * Ly) // 2 if matter else 0
    cfgs, _, _ = configs_for(lat, n_chains, seed=24, n_bosons=nb)
    dev = torch.from_numpy(cfgs).cuda()
    out = ctx.sample_batch(dev, n_sweeps, seed=777)
    torch.cuda.synchronize()
    la = out["log_abs"].cpu().numpy()
    e = torch.view_as_complex(out["e_loc"].view(-1, 2)).cpu().numpy()
    model = vmc.Model(h=h, g=g, J=J)
    final = dev.cpu().numpy()
    for c in range(n_chains):
        recs = _replay_chain(pe, model, cfgs[c], chi, 777, c, n_sweeps)
        assert np.array_equal(final[c], recs[-1]["cfg"].astype(np.int8)), c
        for w, rec in enumerate(recs):
            s = c * n_sweeps + w
            assert amp_err(la[s], 0.0, rec["log_abs"], 0.0) < TOL[prec] * 10
            ref = rec["e_loc"]
            assert abs(e[s] - ref) <= TOL[prec] * max(1.0, abs(ref)) * 10
        acc = out["accepted"].cpu().numpy()[c]
        assert acc == sum(r["accepted"] for r in recs)


def test_sr_step_parity_fp64():
    """SR update on the same fixed configurations: GPU (CG, FP64) vs the
    oracle's dense solve, Eqs. S3 and S7."""
    Lx, Ly, N, D, chi = 4, 3, 2, 4, 4
    lat, pe, ctx = setup(Lx, Ly, N, D, chi, seed=15, precision="fp64", h=1.0, g=0.3)
    cfgs, _, _ = configs_for(lat, 24, seed=25)
    dev = torch.from_numpy(cfgs).cuda()
    e = ctx.local_energy(dev)
    bid, O = ctx.log_grad(dev)
    samples = {"e_loc": torch.view_as_real(e).reshape(-1).contiguous(), "block_ids": bid, "O": O}
    p0 = ctx.get_tensors()
    stats = ctx.sr_step(samples, n_chains=24, diag_shift=1e-3, lr=0.1, max_iter=500, tol=1e-12)
    p1 = ctx.get_tensors()
    model = vmc.Model(h=1.0, g=0.3)
    Ed = np.array([vmc.local_energy(pe, model, c, chi) for c in cfgs])
    Od = np.array([vmc.log_grad_dense(pe, c, chi) for c in cfgs])
    S, F, eb = vmc.sr_matrices(Od, Ed, np.full(len(cfgs), 1.0 / len(cfgs)))
    x = vmc.sr_solve(S, F, 1e-3)
    assert abs(stats[0] - eb.real) < 1e-10 * max(1, abs(eb))
    dp = p1 - p0
    ref = -0.1 * x.real
    assert np.linalg.norm(dp - ref) <= 1e-7 * np.linalg.norm(ref), (np.linalg.norm(dp - ref), np.linalg.norm(ref))


def test_tdvp_stage_parity_complex_fp64():
    Lx, Ly, N, D, chi = 3, 3, 2, 4, 2
    lat, pe, ctx = setup(Lx, Ly, N, D, chi, seed=16, complex_=True, precision="fp64", h=1.0, g=0.4)
    cfgs, _, _ = configs_for(lat, 16, seed=26)
    dev = torch.from_numpy(cfgs).cuda()
    e = ctx.local_energy(dev)
    bid, O = ctx.log_grad(dev)
    samples = {"e_loc": torch.view_as_real(e).reshape(-1).contiguous(), "block_ids": bid, "O": O}
    import paper_2503_20566_gb300 as G

    p0 = ctx.get_tensors()
    ctx.sr_step(samples, n_chains=16, diag_shift=1e-2, mode=G.TDVP_STAGE1, dt=0.01, max_iter=500, tol=1e-12)
    p1 = ctx.get_tensors()
    model = vmc.Model(h=1.0, g=0.4)
    Ed = np.array([vmc.local_energy(pe, model, c, chi) for c in cfgs])
    Od = np.array([vmc.log_grad_dense(pe, c, chi) for c in cfgs])
    S, F, _ = vmc.sr_matrices(Od, Ed, np.full(len(cfgs), 1.0 / len(cfgs)))
    ref = vmc.TDVP_C1 * 0.01 * vmc.tdvp_velocity(S, F, 1e-2)
    assert np.linalg.norm((p1 - p0) - ref) <= 1e-7 * np.linalg.norm(ref)


def test_vmc_step_host_end_to_end():
    lat, pe, ctx = setup(4, 4, 2, 4, 4, seed=17, h=1.0, g=0.5)
    cfgs, _, _ = configs_for(lat, 8, seed=27)
    host = np.ascontiguousarray(cfgs.copy())
    stats = ctx.vmc_step_host(host, n_sweeps=2, seed=5, lr=0.01, max_iter=50)
    assert np.isfinite(stats[0]) and stats[3] >= 1
    for c in host:
        assert lat.is_physical(c)


def test_sr_step_parity_fp64_full_rank_preconditioned():
    """More samples than parameters (S of full rank): the CG runs with the
    diagonal preconditioner and still lands on the oracle's dense solve."""
    Lx, Ly, N, D, chi = 3, 3, 2, 2, 2
    lat, pe, ctx = setup(Lx, Ly, N, D, chi, seed=16, precision="fp64", h=1.0, g=0.3)
    n = 8 * ctx.n_params
    cfgs, _, _ = configs_for(lat, n, seed=26)
    dev = torch.from_numpy(cfgs).cuda()
    e = ctx.local_energy(dev)
    bid, O = ctx.log_grad(dev)
    samples = {"e_loc": torch.view_as_real(e).reshape(-1).contiguous(), "block_ids": bid, "O": O}
    p0 = ctx.get_tensors()
    stats = ctx.sr_step(samples, n_chains=n, diag_shift=1e-3, lr=0.1, max_iter=500, tol=1e-12)
    p1 = ctx.get_tensors()
    assert stats[7] == 1.0 and stats[6] == 1.0
    model = vmc.Model(h=1.0, g=0.3)
    Ed = np.array([vmc.local_energy(pe, model, c, chi) for c in cfgs])
    Od = np.array([vmc.log_grad_dense(pe, c, chi) for c in cfgs])
    S, F, eb = vmc.sr_matrices(Od, Ed, np.full(len(cfgs), 1.0 / len(cfgs)))
    x = vmc.sr_solve(S, F, 1e-3)
    ref = -0.1 * x.real
    dp = p1 - p0
    assert np.linalg.norm(dp - ref) <= 1e-7 * np.linalg.norm(ref), (np.linalg.norm(dp - ref), np.linalg.norm(ref))


@pytest.mark.parametrize("case", [(4, 3, 4, 4, 24, 1e-2), (3, 3, 4, 2, None, 10.0)], ids=["plain-cg", "jacobi"])
def test_sr_step_parity_fp32(case):
    """The FP32 storage path of the SR step (O in FP32, FP32 partial products,
    FP64 sums and CG; the path the benchmark runs) against the oracle's dense
    FP64 solve on the same rounded tensors, Eqs. S3 and S7.  The first case has
    fewer samples than parameters (plain CG), the second twice as many
    (Jacobi-preconditioned; the larger shift keeps its condition number where
    CG converges).  Bound: 2e-3 relative, about a hundred times the change of
    the dense solution under 1e-5 relative noise on O and E_loc."""
    Lx, Ly, D, chi, n, shift = case
    lat, pe, ctx = setup(Lx, Ly, 2, D, chi, seed=15, precision="fp32", h=1.0, g=0.3)
    if n is None:
        n = 2 * ctx.n_params
    cfgs, _, _ = configs_for(lat, n, seed=25)
    dev = torch.from_numpy(cfgs).cuda()
    e = ctx.local_energy(dev)
    bid, O = ctx.log_grad(dev)
    samples = {"e_loc": torch.view_as_real(e).reshape(-1).contiguous(), "block_ids": bid, "O": O}
    p0 = ctx.get_tensors()
    stats = ctx.sr_step(samples, n_chains=n, diag_shift=shift, lr=0.1, max_iter=2000, tol=1e-10)
    p1 = ctx.get_tensors()
    assert stats[7] == (1.0 if n >= ctx.n_params else 0.0)
    model = vmc.Model(h=1.0, g=0.3)
    Ed = np.array([vmc.local_energy(pe, model, c, chi) for c in cfgs])
    Od = np.array([vmc.log_grad_dense(pe, c, chi) for c in cfgs])
    S, F, eb = vmc.sr_matrices(Od, Ed, np.full(len(cfgs), 1.0 / len(cfgs)))
    ref = -0.1 * vmc.sr_solve(S, F, shift).real
    assert abs(stats[0] - eb.real) < 1e-4 * max(1, abs(eb))
    dp = p1 - p0
    print("fp32 SR", n, "samples", ctx.n_params, "params: rel dev %.2e" % (np.linalg.norm(dp - ref) / np.linalg.norm(ref)),
          "iters", stats[3])
    assert np.linalg.norm(dp - ref) <= 2e-3 * np.linalg.norm(ref)
