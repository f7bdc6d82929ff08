"""Partitioned selected inversion of G^R (negf_rgf_partitioned, Fig. 3) through the
C ABI, against the CPU oracle: the dense inverse at small sizes, the block recursion at
the config-2 block shape with nb = 128, for P = 1 .. 4 partitions."""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import negf_oracle as O
from negf_testutil import GR_KEYS, TOL_FP64, TOL_MIXED, block_err, gf_err, strong_leads

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
    c = P.Context(0, 4 << 30)
    yield c
    c.close()


def _run(P, ctx, devs, prec, parts, scat=True):
    if not isinstance(devs, (list, tuple)):
        devs = [devs]
    sys_ = P.upload(devs)
    out = P.allocate_outputs(sys_, lesser=False)
    P.negf_obc(ctx, sys_, out["sigma_L"], out["sigma_R"], out["iters"], out["obc_status"], prec=P.FP64)
    sc = P.Scattering.from_devices(devs) if scat and devs[0].sigR_scat is not None else None
    P.negf_rgf_partitioned(ctx, sys_, prec, parts, out["sigma_L"], out["sigma_R"], sc, out["GR_diag"],
                           out["GR_up"], out["GR_low"], out["status"])
    assert ctx.sync() == 0
    L = sys_.layout()
    res = []
    for d, dev in enumerate(devs):
        o, nb, b, ne = L[d], dev.nb, dev.b, dev.ne
        bb = b * b
        r = {"sigma_L": out["sigma_L"][o[3]:o[3] + ne * bb].cpu().numpy().reshape(ne, b, b),
             "sigma_R": out["sigma_R"][o[3]:o[3] + ne * bb].cpu().numpy().reshape(ne, b, b),
             "status": out["status"][o[2]:o[2] + ne].cpu().numpy(),
             "GR_diag": out["GR_diag"][o[4]:o[4] + ne * nb * bb].cpu().numpy().reshape(ne, nb, b, b)}
        for k in ("GR_up", "GR_low"):
            r[k] = out[k][o[5]:o[5] + ne * (nb - 1) * bb].cpu().numpy().reshape(ne, nb - 1, b, b)
        res.append(r)
    return res


@pytest.mark.parametrize("prec", ["FP64", "MIXED"])
@pytest.mark.parametrize("nb,b,parts", [(4, 8, 2), (6, 24, 3), (8, 24, 4), (12, 16, 4), (8, 70, 2), (5, 8, 1)])
def test_partitioned_matches_dense_inverse(P, ctx, prec, nb, b, parts):
    dev = W.small_scattering_device(nb, b, 4, seed=90 + nb + b + parts, overlap=True, strength=0.05)
    strong_leads(dev, seed=4)
    r = _run(P, ctx, dev, getattr(P, prec), parts)[0]
    assert np.all(r["status"] == 0)
    for e in range(dev.ne):
        ref = O.solve_energy(dev, e, lesser=False, sigma=(r["sigma_L"][e], r["sigma_R"][e]))
        if prec == "FP64":
            for k in GR_KEYS:
                assert block_err(r[k][e], ref[k]) <= TOL_FP64, (k, e)
        else:
            assert gf_err(r, e, ref, GR_KEYS) <= TOL_MIXED, e


def test_partitioned_uneven_batch(P, ctx):
    devs = [strong_leads(W.banded_device(nb, b, ne, seed=110 + k, overlap=True), seed=k)
            for k, (nb, b, ne) in enumerate([(8, 16, 3), (4, 40, 2), (12, 8, 0), (6, 24, 4)])]
    rs = _run(P, ctx, devs, P.FP64, 2)
    for dev, r in zip(devs, rs):
        for e in range(dev.ne):
            ref = O.solve_energy(dev, e, lesser=False, sigma=(r["sigma_L"][e], r["sigma_R"][e]))
            for k in GR_KEYS:
                assert block_err(r[k][e], ref[k]) <= TOL_FP64, (dev.name, k, e)


def test_partitioned_rejects_partitions_that_do_not_divide_nb(P, ctx):
    dev = W.banded_device(6, 8, 2, seed=3, overlap=False)
    sys_ = P.upload(dev)
    out = P.allocate_outputs(sys_, lesser=False)
    for parts in (4, 6, 0):
        with pytest.raises(P.NegfError) as ei:
            P.negf_rgf_partitioned(ctx, sys_, P.FP64, parts, out["sigma_L"], out["sigma_R"], None,
                                   out["GR_diag"], out["GR_up"], out["GR_low"], out["status"])
        assert ei.value.code == P.negf.NEGF_ERR_ARG


@pytest.mark.parametrize("parts", [2, 4])
def test_partitioned_config2_shape_nb128_against_block_recursion(P, parts):
    """nb = 128 blocks of the config-2 shape (b = 128, global-band decay, S != I), a few
    energies in and out of the band; mixed precision against the oracle's block
    recursion (pinned to dense inversion), normwise over G^R."""
    dev = W.config2(nb=128, b=128, ne=1024)
    dev = dev.truncated(energies=[300, 470, 528])
    ctx = P.Context(0, 16 << 30)
    try:
        r = _run(P, ctx, dev, P.MIXED, parts)[0]
        assert np.all(r["status"] == 0)
        for e in range(dev.ne):
            ref = O.solve_energy(dev, e, lesser=False, use_rgf=True, sigma=(r["sigma_L"][e], r["sigma_R"][e]))
            assert gf_err(r, e, ref, GR_KEYS) <= TOL_MIXED, e
    finally:
        ctx.close()
