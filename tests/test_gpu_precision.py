"""Mixed-precision contraction forms against the FP64 oracle.

precision="tf32": the contraction GEMMs run on tensor cores with the 3-pass
TF32 split (about 21 significant bits), held to the FP32 bound 1e-4.
precision="bf16": the strip-environment GEMMs (plaquette and vertical-hop
ratios: Metropolis decisions and E_loc) take BF16 operands with FP32
accumulation, on the fifth-generation tensor cores (tcgen05) for real tensors
and on mma.sync for complex ones; the boundary-MPS absorption and the row
environments (amplitude, O) run in the TF32x3 form.  Held to the BF16 bound
1e-2 on E_loc and to the FP32-class bound on amplitudes and O, whose GEMMs
never see BF16.  Amplitudes are compared as |exp(d log|psi| + i d
phase) - 1|, E_loc relative to its off-diagonal part, O relative to the
largest entry of its block, as in the FP32 parity tests.
"""

import numpy as np
import pytest

from oracle import vmc

from gpu_helpers import amp_err, configs_for, setup

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

# TF32x3 is held to the FP32 bound; the BF16 form to the BF16 bound 1e-2 on
# E_loc (the only output that passes through BF16 GEMMs) and to the TF32x3
# bounds on amplitudes and O.
TOL = {"tf32": {"amp": 1e-4, "eloc": 1e-3, "grad": 1e-3},
       "bf16": {"amp": 1e-4, "eloc": 1e-2, "grad": 1e-3}}

CASES = [
    (8, 8, 2, 4, 16, False, False),  # 8x8 Z2 D=4 chi=16 (exact)
    (6, 5, 2, 4, 4, False, False),   # truncated
    (3, 7, 3, 6, 4, True, False),    # Z3 complex, ragged
    (5, 5, 2, 6, 5, False, False),   # D_k = 3, truncated
    (4, 3, 2, 4, 4, False, True),    # Z2 + hard-core bosons
    (6, 6, 4, 8, 8, True, False),    # Z4 complex
]


def _ids(c):
    return "{}x{}-Z{}-D{}-chi{}{}{}".format(c[0], c[1], c[2], c[3], c[4], "-c" if c[5] else "", "-m" if c[6] else "")


@pytest.mark.parametrize("prec", ["tf32", "bf16"])
@pytest.mark.parametrize("case", CASES, ids=_ids)
def test_mixed_precision_amplitude_energy_gradient(case, prec):
    Lx, Ly, N, D, chi, cplx, matter = case
    h, g, J = 1.0, 0.37, (0.5 if matter else 0.0)
    lat, pe, ctx = setup(Lx, Ly, N, D, chi, seed=71, complex_=cplx, matter=matter, precision=prec, h=h, g=g, J=J)
    nb = (Lx * Ly) // 2 if matter else 0
    cfgs, _, _ = configs_for(lat, 4, seed=72, n_bosons=nb)
    dev = torch.from_numpy(cfgs).cuda()
    tol = TOL[prec]
    la, ph = ctx.amplitude(dev)
    la, ph = la.cpu().numpy(), ph.cpu().numpy()
    e = ctx.local_energy(dev).cpu().numpy()
    bid, O = ctx.log_grad(dev)
    bid, O = bid.cpu().numpy(), O.cpu().numpy()
    model = vmc.Model(h=h, g=g, J=J)
    worst = {"amp": 0.0, "eloc": 0.0, "grad": 0.0, "grad_fro": 0.0}
    for i, c in enumerate(cfgs):
        ola, oph = vmc.amplitude(pe, c, chi)
        worst["amp"] = max(worst["amp"], amp_err(la[i], ph[i], ola, oph))
        ref = vmc.local_energy(pe, model, c, chi)
        scale_ = max(1.0, abs(ref - lat.diagonal_energy(c, g)))
        worst["eloc"] = max(worst["eloc"], abs(e[i] - ref) / scale_)
        for v, (rb, rblk) in enumerate(vmc.log_grad(pe, c, chi)):
            assert bid[i, v] == rb
            r = rblk.reshape(-1)
            d = O[i, v, : r.size] - r
            worst["grad"] = max(worst["grad"], np.abs(d).max() / max(1.0, np.abs(r).max()))
            worst["grad_fro"] = max(worst["grad_fro"], np.linalg.norm(d) / max(1e-300, np.linalg.norm(r)))
    print(prec, _ids(case), {k: float("%.3g" % v) for k, v in worst.items()},
          "tcgen05" if ctx.tensor_core_form else "mma.sync")
    if prec == "bf16" and not cplx:
        assert ctx.tensor_core_form  # real chains of the BF16 form run on tcgen05
    assert ctx.tensor_timeouts == 0
    for key in ("amp", "eloc", "grad"):
        assert worst[key] <= tol[key], (key, worst[key])


@pytest.mark.parametrize("prec", ["tf32", "bf16"])
def test_mixed_precision_chain_replays_oracle(prec):
    """Metropolis decisions depend on ratios; with TF32x3 they match the
    oracle's bit for bit on this case, with BF16 the chain stays physical
    and its amplitudes match the oracle on its own configurations."""
    Lx, Ly, N, D, chi = 5, 4, 2, 4, 4
    lat, pe, ctx = setup(Lx, Ly, N, D, chi, seed=73, precision=prec)
    cfgs, _, _ = configs_for(lat, 4, seed=74)
    dev = torch.from_numpy(cfgs).cuda()
    out = ctx.sample_batch(dev, 2, seed=99)
    torch.cuda.synchronize()
    final = dev.cpu().numpy()
    la = out["log_abs"].cpu().numpy()
    model = vmc.Model(h=1.0, g=0.4)
    for c in range(len(cfgs)):
        assert lat.is_physical(final[c])
        if prec == "tf32":
            recs = vmc.run_chain(pe, model, cfgs[c], chi, 99, c, 2, measure=True)
            assert np.array_equal(final[c], recs[-1]["cfg"].astype(np.int8)), c
            for w, rec in enumerate(recs):
                assert amp_err(la[c * 2 + w], 0.0, rec["log_abs"], 0.0) < TOL[prec]["amp"]
        else:
            ola, _ = vmc.amplitude(pe, final[c], chi)
            assert amp_err(la[c * 2 + 1], 0.0, ola, 0.0) < TOL[prec]["amp"]
