"""Parity at the full workload sizes: amplitudes, E_loc and O against the oracle.

The 8x8 Z2 D=4 chi=16 workload is covered in full by test_gpu_parity.py.  Here
the larger lattices of the hot-path scope run in the library's default kernel
form (the one the benchmark times): Z3 16x16 D=6 chi=32 and Z4 16x16 D=8
chi=32 with complex tensors, Z2 + hard-core bosons 32x32 D=4 chi=24 at half
filling, and Z2 10x10 D=6 chi=36 complex.  Per case: 8 amplitudes against the
FP64 oracle, and for the first two samples E_loc (Eq. S2, every plaquette and
hop term) and O (Eq. S3, every vertex).

Tolerance.  These contractions truncate (chi below the exact bond dimension),
and a truncated boundary MPS is as sensitive to rounding as its cuts are
close to degenerate: an input error of size u sigma_1 turns the kept
subspace by about u sigma_1 / (sigma_chi - sigma_chi+1) (Wedin), at every one
of the tens to hundreds of cuts.  The sensitivity of each sample is measured
independently of the library: the oracle's own steps run once more in single
precision (NumPy's LAPACK), and its distance from the FP64 oracle, d32, is
what any careful FP32 evaluation of this truncated amplitude can be expected
to reach.  Samples with d32 <= 1e-5 (well conditioned) are held to the FP32
bound 1e-4; the others to 10 d32.  The oracle's smallest relative gap and
largest sigma_1 / (sigma_chi - sigma_chi+1) over the sample's cuts are
printed with every sample.  E_loc and O take 10x the amplitude bound of their
sample (relative to the off-diagonal part of E_loc and to the largest entry
of each O block), as in the other FP32 parity tests.
"""

import functools

import numpy as np
import pytest

from oracle import vmc

from gpu_helpers import amp_err, configs_for, oracle_net, setup

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

CASES = [
    (16, 16, 3, 6, 32, True, False),   # Z3, complex
    (16, 16, 4, 8, 32, True, False),   # Z4, complex
    (32, 32, 2, 4, 24, False, True),   # Z2 + hard-core bosons, half filling
    (10, 10, 2, 6, 36, True, False),   # Z2, D_k = 3, complex
]
N_AMP, N_FULL = 8, 2
BOUND = {"fp64": 1e-7, "fp32": 1e-4, "tf32": 1e-4}
WELL_CONDITIONED = 1e-5


def _ids(c):
    return "{}x{}-Z{}-D{}-chi{}{}{}".format(c[0], c[1], c[2], c[3], c[4], "-c" if c[5] else "", "-m" if c[6] else "")


def _model(case):
    return vmc.Model(h=1.0, g=0.33, J=0.5 if case[6] else 0.0)


@functools.lru_cache(maxsize=None)
def _oracle(case, store):
    """FP64 oracle values (and the single-precision sensitivity) of the case's
    samples on the tensors rounded to `store`, computed once per case."""
    Lx, Ly, N, D, chi, cplx, matter = case
    lat, pe, _ = oracle_net(Lx, Ly, N, D, seed=121, complex_=cplx, matter=matter,
                            precision="fp64" if store == "f64" else "fp32")
    nb = (Lx * Ly) // 2 if matter else 0
    cfgs, _, _ = configs_for(lat, N_AMP, seed=122, n_bosons=nb)
    single = np.complex64 if cplx else np.float32
    amps, d32, gaps = [], [], []
    for c in cfgs:
        sp = []
        la, ph = vmc.amplitude(pe, c, chi, spectra=sp)
        la32, ph32 = vmc.amplitude(pe, c, chi, dtype=single)
        amps.append((la, ph))
        d32.append(amp_err(la32, ph32, la, ph))
        rel = [(S[chi - 1] - S[chi]) / S[chi - 1] for (_, _, S) in sp]
        kap = [S[0] / max(S[chi - 1] - S[chi], 1e-300) for (_, _, S) in sp]
        gaps.append((len(sp), min(rel) if rel else 1.0, max(kap) if kap else 1.0))
    model = _model(case)
    eloc = [vmc.local_energy(pe, model, cfgs[i], chi) for i in range(N_FULL)]
    ediag = [lat.diagonal_energy(cfgs[i], model.g, model.m) for i in range(N_FULL)]
    grads = [vmc.log_grad(pe, cfgs[i], chi) for i in range(N_FULL)]
    return cfgs, amps, d32, gaps, eloc, ediag, grads


@pytest.mark.parametrize("prec", ["fp64", "fp32", "tf32"])
@pytest.mark.parametrize("case", CASES, ids=_ids)
def test_full_size_amplitude_energy_gradient(case, prec):
    Lx, Ly, N, D, chi, cplx, matter = case
    store = "f64" if prec == "fp64" else "f32"
    cfgs, amps, d32, gaps, eloc, ediag, grads = _oracle(case, store)
    _, _, ctx = setup(Lx, Ly, N, D, chi, seed=121, complex_=cplx, matter=matter, precision=prec,
                      h=1.0, g=0.33, J=0.5 if matter else 0.0)
    dev = torch.from_numpy(cfgs).cuda()
    la, ph = (t.cpu().numpy() for t in ctx.amplitude(dev))
    assert ctx.svd_unconverged == 0
    e = ctx.local_energy(dev[:N_FULL]).cpu().numpy()
    bid, O = (t.cpu().numpy() for t in ctx.log_grad(dev[:N_FULL]))
    bounds = []
    for i in range(len(cfgs)):
        err = amp_err(la[i], ph[i], *amps[i])
        if prec == "fp64":
            bound = BOUND[prec]
        else:
            bound = BOUND[prec] if d32[i] <= WELL_CONDITIONED else 10.0 * d32[i]
        bounds.append(bound)
        ncut, gap, kap = gaps[i]
        print(f"{prec} {_ids(case)} sample {i}: amp err {err:.2e} bound {bound:.1e} | oracle FP32 {d32[i]:.2e}, "
              f"{ncut} cuts, min rel gap {gap:.1e}, max sigma1/gap {kap:.1e}")
        assert err <= bound, (i, err, bound)
    for i in range(N_FULL):
        scale = max(1.0, abs(eloc[i] - ediag[i]))
        ee = abs(e[i] - eloc[i]) / scale
        ge = 0.0
        for v, (rb, rblk) in enumerate(grads[i]):
            assert bid[i, v] == rb, (i, v)
            ref = rblk.reshape(-1)
            ge = max(ge, np.abs(O[i, v, :ref.size] - ref).max() / max(1.0, np.abs(ref).max()))
        print(f"{prec} {_ids(case)} sample {i}: E_loc err {ee:.2e}, O err {ge:.2e} (bound {10 * bounds[i]:.1e})")
        assert ee <= 10 * bounds[i], (i, ee)
        assert ge <= 10 * bounds[i], (i, ge)
