"""Eq. (3) energy convolution (negf_energy_convolution) and the self-consistent
scattering loop (negf_scba, Fig. 2) through the C ABI, against the CPU oracle: the
convolution against the oracle's direct sum, the loop against the oracle's loop (same
mixing and stopping rule), and the conservation of the energy-integrated current at
the GPU's own fixed point."""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import negf_oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2602_03438_gb300 as P
    P.negf.load_library()
    return P


@pytest.fixture(scope="module")
def ctx(P):
    c = P.Context(0, 1 << 30)
    yield c
    c.close()


@pytest.mark.parametrize("ne,M,shape", [(64, 4, (3, 5, 5)), (100, 7, (2, 9)), (13, 6, (40,)), (1000, 3, (8,)),
                                        (1, 2, (4,))])
def test_energy_convolution_matches_direct_sum(P, ctx, ne, M, shape):
    rng = np.random.default_rng(ne + M)
    X = rng.normal(size=(ne,) + shape) + 1j * rng.normal(size=(ne,) + shape)
    w = rng.uniform(0, 1, size=2 * M + 1)
    Xd = torch.from_numpy(X).cuda()
    Yd = torch.empty_like(Xd)
    P.negf.negf_energy_convolution(ctx, Xd, Yd, w)
    assert ctx.sync() == 0
    ref = O.energy_convolution(X, w)
    assert np.abs(Yd.cpu().numpy() - ref).max() <= 1e-13 * np.abs(ref).max()


def _loop(P, ctx, dev, prec, wl, wg, tol, max_iter=80):
    sys_ = P.upload(dev)
    out = P.allocate_outputs(sys_, greater=True)
    P.negf_obc(ctx, sys_, out["sigma_L"], out["sigma_R"], out["iters"], out["obc_status"], prec=P.FP64)
    fL = torch.from_numpy(dev.f_L()).cuda()
    fR = torch.from_numpy(dev.f_R()).cuda()
    n = out["GR_diag"].numel()
    sig = {k: torch.zeros(n, dtype=torch.complex128, device="cuda") for k in ("R", "L", "G")}
    it, ch = P.negf.negf_scba(ctx, sys_, prec, out["sigma_L"], out["sigma_R"], fL, fR, wl, wg, sig["R"], sig["L"],
                              sig["G"], out["GR_diag"], out["GL_diag"], out["GG_diag"], out["GR_up"], out["GR_low"],
                              out["GL_low"], out["GG_low"], out["status"], mixing=0.5, tol=tol, max_iter=max_iter)
    assert ctx.sync() == 0
    w = torch.from_numpy(dev.weights()).cuda()
    P.negf_observables(ctx, sys_, out["sigma_L"], w, out["GR_diag"], out["GR_up"], out["GR_low"], out["GL_diag"],
                       out["GL_low"], None, None, out["current"], None, prec=prec)
    assert ctx.sync() == 0
    ne, nb, b = dev.ne, dev.nb, dev.b
    r = {k: v.cpu().numpy().reshape(ne, nb, b, b) for k, v in sig.items()}
    for k in ("GL_diag", "GG_diag"):
        r[k] = out[k].cpu().numpy().reshape(ne, nb, b, b)
    r["J"] = out["current"].cpu().numpy().reshape(ne, nb - 1)
    r["sigma"] = (out["sigma_L"].cpu().numpy().reshape(ne, b, b), out["sigma_R"].cpu().numpy().reshape(ne, b, b))
    return it, ch, r


@pytest.mark.parametrize("prec", ["FP64", "MIXED"])
def test_scba_loop_matches_oracle_loop(P, ctx, prec):
    dev = W.scba_device(4, 16, 96)
    wl, wg = W.einstein_kernel(dev.energy, 3, 0.05, dev.kT)
    it, ch, r = _loop(P, ctx, dev, getattr(P, prec), wl, wg, tol=1e-9)
    ref = O.scba_loop(dev, wl, wg, sigma=r["sigma"], mixing=0.5, tol=1e-9, max_iter=80)
    assert ch < 1e-9 and ref["change"] < 1e-9
    assert abs(it - ref["iters"]) <= 1
    tol = 1e-9 if prec == "FP64" else 1e-6
    scale = np.abs(ref["sigG"]).max()
    for k, kr in (("L", "sigL"), ("G", "sigG"), ("R", "sigR")):
        assert np.abs(r[k] - ref[kr]).max() <= tol * scale, k
    GLd = np.stack([o["GL_diag"] for o in ref["out"]])
    GGd = np.stack([o["GG_diag"] for o in ref["out"]])
    gscale = max(np.abs(GLd).max(), np.abs(GGd).max())
    assert np.abs(r["GL_diag"] - GLd).max() <= tol * gscale
    assert np.abs(r["GG_diag"] - GGd).max() <= tol * gscale


def test_scba_fixed_point_conserves_the_integrated_current(P, ctx):
    """Checked on the GPU's own outputs: the energy-integrated current is the same at
    every interface (eta = 1e-10, so that the broadening sink is negligible) while the
    energy-resolved current changes along the device."""
    dev = W.scba_device(6, 16, 128)
    dev.eta = 1e-10
    wl, wg = W.einstein_kernel(dev.energy, 4, 0.05, dev.kT)
    it, ch, r = _loop(P, ctx, dev, P.MIXED, wl, wg, tol=1e-10, max_iter=100)
    assert ch < 1e-10
    J = r["J"]
    Jint = J.sum(axis=0)
    assert np.ptp(Jint) <= 1e-6 * np.abs(Jint).max()
    assert np.abs(np.ptp(J, axis=1)).max() >= 1e-2 * np.abs(J).max()
