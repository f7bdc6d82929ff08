"""Selected inversion of the arrowhead BT matrix (negf_rgf_arrowhead) through the C ABI,
against the oracle's dense inverse of the bordered matrix: the device's blocks of G^R,
the tip block and the arrow's row and column blocks, FP64 and mixed precision, with
scattering and S != I, and an uneven two-device batch."""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import negf_oracle as O
from negf_testutil import TOL_FP64, TOL_MIXED, strong_leads

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


def _run(P, ctx, devs, gates, prec):
    sys_ = P.upload(devs)
    out = P.allocate_outputs(sys_, lesser=False)
    P.negf_obc(ctx, sys_, out["sigma_L"], out["sigma_R"], out["iters"], out["obc_status"], prec=P.FP64)
    L = sys_.layout()
    tot = L[-1]
    Ht = torch.from_numpy(np.concatenate([g[0].reshape(-1) for g in gates])).cuda()
    Ha = torch.from_numpy(np.concatenate([g[1].reshape(-1) for g in gates])).cuda()
    Gt = torch.empty(int(tot[3]), dtype=torch.complex128, device="cuda")
    Gr = torch.empty(int(tot[4]), dtype=torch.complex128, device="cuda")
    Gc = torch.empty(int(tot[4]), dtype=torch.complex128, device="cuda")
    sc = P.Scattering.from_devices(devs)
    P.negf.negf_rgf_arrowhead(ctx, sys_, prec, Ht, Ha, out["sigma_L"], out["sigma_R"], sc, out["GR_diag"],
                              out["GR_up"], out["GR_low"], Gt, Gr, Gc, out["status"])
    assert ctx.sync() == 0
    res = []
    for d, dev in enumerate(devs):
        o, nb, b, ne = L[d], dev.nb, dev.b, dev.ne
        bb = b * b
        cut = lambda t, off, n: t[off:off + n].cpu().numpy()
        r = {"sigma_L": cut(out["sigma_L"], o[3], ne * bb).reshape(ne, b, b),
             "sigma_R": cut(out["sigma_R"], o[3], ne * bb).reshape(ne, b, b),
             "GR_diag": cut(out["GR_diag"], o[4], ne * nb * bb).reshape(ne, nb, b, b),
             "GR_up": cut(out["GR_up"], o[5], ne * (nb - 1) * bb).reshape(ne, nb - 1, b, b),
             "GR_low": cut(out["GR_low"], o[5], ne * (nb - 1) * bb).reshape(ne, nb - 1, b, b),
             "G_tip": cut(Gt, o[3], ne * bb).reshape(ne, b, b),
             "G_row": cut(Gr, o[4], ne * nb * bb).reshape(ne, nb, b, b),
             "G_col": cut(Gc, o[4], ne * nb * bb).reshape(ne, nb, b, b),
             "status": cut(out["status"], o[2], ne)}
        res.append(r)
    return res


def _families(r, e):
    return {"GR": [r["GR_diag"][e], r["GR_up"][e], r["GR_low"][e]], "tip": [r["G_tip"][e][None]],
            "row": [r["G_row"][e]], "col": [r["G_col"][e]]}


def _ref_families(ref):
    return {"GR": [ref["GR_diag"], ref["GR_up"], ref["GR_low"]], "tip": [ref["G_tip"][None]],
            "row": [ref["G_row"]], "col": [ref["G_col"]]}


def _check(r, dev, gate, tol):
    for e in range(dev.ne):
        z = dev.energy[e] + 1j * dev.eta
        ref = O.arrowhead_dense(dev, z, r["sigma_L"][e], r["sigma_R"][e], gate[0], gate[1], sigR_scat=dev.sigR_scat)
        got, want = _families(r, e), _ref_families(ref)
        for k in want:
            num = max(np.linalg.norm(g - w) for gs, ws in zip(got[k], want[k]) for g, w in zip(gs, ws))
            den = max(np.linalg.norm(w) for ws in want[k] for w in ws)
            assert num <= tol * den, (dev.name, e, k, num / den)


@pytest.mark.parametrize("prec", ["FP64", "MIXED"])
@pytest.mark.parametrize("nb,b", [(2, 8), (3, 24), (5, 16), (3, 70)])
def test_arrowhead_matches_dense_bordered_inverse(P, ctx, prec, nb, b):
    dev = W.small_scattering_device(nb, b, 4, seed=130 + nb + b, overlap=True, strength=0.05)
    strong_leads(dev, seed=7)
    gate = W.arrowhead_gate(dev, seed=140 + nb, coupling=0.2)
    r = _run(P, ctx, [dev], [gate], getattr(P, prec))[0]
    assert np.all(r["status"] == 0)
    _check(r, dev, gate, TOL_FP64 if prec == "FP64" else TOL_MIXED)


def test_arrowhead_uneven_batch(P, ctx):
    devs = [strong_leads(W.small_scattering_device(3, 16, 3, seed=150, overlap=True), seed=1),
            strong_leads(W.small_scattering_device(4, 8, 2, seed=151, overlap=True), seed=2)]
    gates = [W.arrowhead_gate(d, seed=160 + k, coupling=0.2) for k, d in enumerate(devs)]
    rs = _run(P, ctx, devs, gates, P.FP64)
    for dev, gate, r in zip(devs, gates, rs):
        _check(r, dev, gate, TOL_FP64)
