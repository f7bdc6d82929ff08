"""G^> (negf_rgf_keldysh) through the C ABI against the CPU oracle.

G^> = G^R Sigma^> G^A (Eq. (2) with B^>), computed by the lesser recursion run on
Sigma^> = Sigma^>_scat - i (1 - f) Gamma in the same sweep pair as G^R and G^<.
Errors are measured per energy over the Keldysh blocks (G^< and G^> diagonal and
lower) against the largest of their norms: G^< and G^> share the scale of the
spectral function, and each alone can be many decades smaller than the other
(far below or far above the chemical potentials)."""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import negf_oracle as O
from negf_testutil import TOL_FP64, TOL_MIXED, strong_leads

pytestmark = pytest.mark.gpu

KELDYSH = ("GL_diag", "GL_low", "GG_diag", "GG_low")


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2602_03438_gb300 as P
    P.negf.load_library()
    return P


@pytest.fixture(scope="module")
def ctx(P):
    c = P.Context(0, 2 << 30)
    yield c
    c.close()


def _run(P, ctx, dev, prec, scat=True, sigma=None):
    sys_ = P.upload(dev)
    out = P.allocate_outputs(sys_, greater=True)
    if sigma is None:
        P.negf_obc(ctx, sys_, out["sigma_L"], out["sigma_R"], out["iters"], out["obc_status"], prec=P.FP64)
    else:
        out["sigma_L"].copy_(torch.from_numpy(np.ascontiguousarray(sigma[0]).reshape(-1)))
        out["sigma_R"].copy_(torch.from_numpy(np.ascontiguousarray(sigma[1]).reshape(-1)))
    fL = torch.from_numpy(dev.f_L()).cuda()
    fR = torch.from_numpy(dev.f_R()).cuda()
    sc = P.Scattering.from_devices([dev]) if scat and dev.sigR_scat is not None else None
    P.negf_rgf_keldysh(ctx, sys_, prec, out["sigma_L"], out["sigma_R"], fL, fR, sc, out["GR_diag"],
                       out["GR_up"], out["GR_low"], out["GL_diag"], out["GL_low"], out["GG_diag"],
                       out["GG_low"], out["status"])
    assert ctx.sync() == 0
    nb, b, ne = dev.nb, dev.b, dev.ne
    r = {}
    for k in ("GR_diag", "GL_diag", "GG_diag"):
        r[k] = out[k].cpu().numpy().reshape(ne, nb, b, b)
    for k in ("GR_up", "GR_low", "GL_low", "GG_low"):
        r[k] = out[k].cpu().numpy().reshape(ne, nb - 1, b, b)
    r["sigma_L"] = out["sigma_L"].cpu().numpy().reshape(ne, b, b)
    r["sigma_R"] = out["sigma_R"].cpu().numpy().reshape(ne, b, b)
    r["status"] = out["status"].cpu().numpy()
    return r, out, sys_, sc, fL, fR


def _keldysh_err(r, e, ref):
    num = max(np.linalg.norm(r[k][e][i] - ref[k][i]) for k in KELDYSH for i in range(ref[k].shape[0]))
    den = max(np.linalg.norm(ref[k][i]) for k in KELDYSH for i in range(ref[k].shape[0]))
    return num / max(den, 1e-300)


@pytest.mark.parametrize("prec", ["FP64", "MIXED"])
@pytest.mark.parametrize("nb,b", [(3, 8), (4, 24), (3, 70)])
def test_greater_with_scattering_matches_dense_oracle(P, ctx, prec, nb, b):
    dev = W.small_scattering_device(nb, b, 6, seed=50 + nb + b, overlap=True, strength=0.05)
    strong_leads(dev, seed=5)
    r, *_ = _run(P, ctx, dev, getattr(P, prec))
    assert np.all(r["status"] == 0)
    tol = TOL_FP64 if prec == "FP64" else TOL_MIXED
    for e in range(dev.ne):
        ref = O.solve_energy(dev, e, greater=True, sigma=(r["sigma_L"][e], r["sigma_R"][e]))
        assert _keldysh_err(r, e, ref) <= tol, (prec, e)


def test_greater_ballistic_fluctuation_dissipation(P, ctx):
    """Both leads at one chemical potential: G^> = -((1 - f)/f) G^< exactly (checked on
    the GPU's own outputs, no oracle involved)."""
    dev = strong_leads(W.banded_device(4, 16, 24, seed=8, overlap=True), seed=2)
    dev.mu_R = dev.mu_L
    dev.kT = 0.5
    f = dev.f_L()
    r, *_ = _run(P, ctx, dev, P.FP64, scat=False)
    for e in range(dev.ne):
        if not 0.05 < f[e] < 0.95:
            continue
        ratio = -(1.0 - f[e]) / f[e]
        for kg, kl in (("GG_diag", "GL_diag"), ("GG_low", "GL_low")):
            scale = np.abs(r[kg][e]).max()
            assert np.abs(r[kg][e] - ratio * r[kl][e]).max() <= 1e-10 * scale, (e, kg)


@pytest.mark.parametrize("prec", ["FP64", "MIXED"])
def test_keldysh_call_leaves_retarded_and_lesser_unchanged(P, ctx, prec):
    """G^R and G^< of negf_rgf_keldysh are bit-identical to those of negf_rgf_lesser."""
    dev = W.small_scattering_device(3, 32, 4, seed=77, overlap=True, strength=0.05)
    strong_leads(dev, seed=9)
    p = getattr(P, prec)
    r, out, sys_, sc, fL, fR = _run(P, ctx, dev, p)
    o2 = P.allocate_outputs(sys_)
    P.negf_rgf_lesser(ctx, sys_, p, out["sigma_L"], out["sigma_R"], fL, fR, sc, o2["GR_diag"], o2["GR_up"],
                      o2["GR_low"], o2["GL_diag"], o2["GL_low"], o2["status"])
    assert ctx.sync() == 0
    for k in ("GR_diag", "GR_up", "GR_low", "GL_diag", "GL_low"):
        assert torch.equal(out[k], o2[k]), k
