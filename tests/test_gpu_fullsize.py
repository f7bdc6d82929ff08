"""Parity at the workloads' full sizes, on outputs the oracle can compute one by one.

* config 2 (nb=64, b=128, 1024 energies) in the launch configuration bench.py times
  (one call over all energies, mixed precision, 24 GB workspace); sampled energies are
  compared with the oracle's block recursion (itself pinned to dense inversion).
* config 4 (nb=32, b=512) on sampled energies, FP64 and mixed.
* config 3's uneven batch: devices of every block size at their full nb in one call,
  on sampled energies.
"""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import negf_oracle as O
from negf_testutil import GL_KEYS, GR_KEYS, TOL_FP64, TOL_MIXED, gf_err, run_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2602_03438_gb300 as P
    P.negf.load_library()
    return P


def _blocks(out, key, e, nblk, b):
    return out[key].view(-1, nblk, b, b)[e].cpu().numpy()


def test_config2_full_launch_sampled_energies(P):
    dev = W.config2()
    ctx = P.Context(0, 24 << 30)
    try:
        sys_ = P.upload(dev)
        out = P.allocate_outputs(sys_)
        fL = torch.from_numpy(dev.f_L()).cuda()
        fR = torch.from_numpy(dev.f_R()).cuda()
        w = torch.from_numpy(dev.weights()).cuda()
        P.negf_obc(ctx, sys_, out["sigma_L"], out["sigma_R"], out["iters"], out["obc_status"])
        P.negf_rgf_lesser(ctx, sys_, P.MIXED, out["sigma_L"], out["sigma_R"], fL, fR, None, out["GR_diag"],
                          out["GR_up"], out["GR_low"], out["GL_diag"], out["GL_low"], out["status"])
        P.negf_observables(ctx, sys_, out["sigma_L"], w, out["GR_diag"], out["GR_up"], out["GR_low"],
                           out["GL_diag"], out["GL_low"], out["T"], out["dos"], out["current"], out["density"],
                           prec=P.MIXED)
        assert ctx.sync() == 0
        assert int((out["obc_status"] != 0).sum()) == 0
        assert int((out["status"] != 0).sum()) == 0
        nb, b = dev.nb, dev.b
        # in-band (|E| < 0.5, near-resonant blocks; 529 is the peak of the current, so that
        # the sample's largest |J| is the grid's) and out-of-band energies
        sample = [2, 430, 470, 511, 528, 529, 540, 600, 1021]
        J_got, J_ref, n_ref = [], [], np.zeros(nb * b)
        wh = dev.weights()
        for e in sample:
            sL = out["sigma_L"].view(-1, b, b)[e].cpu().numpy()
            sR = out["sigma_R"].view(-1, b, b)[e].cpu().numpy()
            sub = dev.truncated(energies=[e])
            ref_obc = O.solve_energy(sub, 0, lesser=False, use_rgf=True)
            for got, ref in ((sL, ref_obc["sigma_L"]), (sR, ref_obc["sigma_R"])):
                assert np.linalg.norm(got - ref) <= TOL_FP64 * max(np.linalg.norm(ref), 1e-300)
            ref = O.solve_energy(sub, 0, use_rgf=True, sigma=(sL, sR))
            r = {k: _blocks(out, k, e, nb if k.endswith("diag") else nb - 1, b)[None] for k in GR_KEYS + GL_KEYS}
            for keys in (GR_KEYS, GL_KEYS):
                assert gf_err(r, 0, ref, keys) <= TOL_MIXED, (e, keys)
            # first-order bounds from the blockwise error: T = Tr[Gamma X] terms, DOS = Tr over 3nb-2 blocks
            gmax = max(np.linalg.norm(ref[k][i]) for k in GR_KEYS for i in range(ref[k].shape[0]))
            gam = np.linalg.norm(1j * (sL - sL.conj().T))
            tscale = gam * gmax + (gam * gmax) ** 2
            assert abs(out["T"][e].item() - ref["T"]) <= 4 * TOL_MIXED * tscale
            smax = max(np.linalg.norm(dev.S_diag[0]) if dev.S_diag is not None else 1.0, 1.0)
            assert abs(out["dos"][e].item() - ref["dos"]) <= TOL_MIXED * gmax * smax * (3 * nb) / np.pi
            J_got.append(out["current"].view(-1, nb - 1)[e].cpu().numpy())
            J_ref.append(ref["J"])
            n_ref += wh[e] * ref["n_E"]
        # mixed current against the oracle, scalar reading: |dJ| / max(|J|, 1e-3 max |J|)
        J_got, J_ref = np.array(J_got), np.array(J_ref)
        floor = 1e-3 * np.abs(J_ref).max()
        assert floor > 0
        assert (np.abs(J_got - J_ref) / np.maximum(np.abs(J_ref), floor)).max() <= TOL_MIXED
        # mixed density of the sampled energies (the grid's weights), normwise: the sampled
        # blocks of the full launch go through negf_observables as a sub-batch
        sub = dev.truncated(energies=sample)
        s2 = P.upload(sub)
        o2 = P.allocate_outputs(s2)
        sel = torch.tensor(sample, device="cuda")
        for key in ("GL_diag", "GL_low"):
            o2[key].copy_(out[key].view(dev.ne, -1)[sel].reshape(-1))
        w2 = torch.from_numpy(wh[sample]).cuda()
        P.negf_observables(ctx, s2, None, w2, None, None, None, o2["GL_diag"], o2["GL_low"], None, None,
                           None, o2["density"], prec=P.MIXED)
        assert ctx.sync() == 0
        n_got = o2["density"].cpu().numpy()
        assert np.linalg.norm(n_got - n_ref) <= TOL_MIXED * np.linalg.norm(n_ref)
    finally:
        ctx.close()


@pytest.mark.parametrize("prec", ["FP64", "MIXED"])
def test_config4_full_blocks_sampled_energies(P, prec):
    full = W.config4()
    idx = [120, 255, 300]                    # out of band, in band, in band
    dev = full.truncated(energies=idx)
    ctx = P.Context(0, 16 << 30)
    try:
        r = run_gpu(P, ctx, dev, getattr(P, prec), obs=False)[0]
        assert np.all(r["obc_status"] == 0)
        tol = TOL_FP64 if prec == "FP64" else TOL_MIXED
        for e in range(dev.ne):
            ref = O.solve_energy(dev, e, use_rgf=True, sigma=(r["sigma_L"][e], r["sigma_R"][e]))
            for keys in (GR_KEYS, GL_KEYS):
                assert gf_err(r, e, ref, keys) <= tol, (prec, e, keys)
    finally:
        ctx.close()


def test_config3_uneven_batch_full_shapes_sampled_energies(P):
    shapes = W.config3_shapes()
    picked = []
    for bval in W.CONFIG3_BS:      # the first device of every block size, at its full nb
        k = next(i for i, s in enumerate(shapes) if s[1] == bval)
        picked.append(k)
    devs = []
    for k in picked:
        d = W.config3_device(k, shapes)
        sel = np.linspace(0, d.ne - 1, 3).round().astype(int)
        devs.append(d.truncated(energies=sel))
    ctx = P.Context(0, 16 << 30)
    try:
        rs = run_gpu(P, ctx, devs, P.MIXED, obs=False)
        for dev, r in zip(devs, rs):
            assert np.all(r["obc_status"] == 0)
            for e in range(dev.ne):
                ref = O.solve_energy(dev, e, use_rgf=True, sigma=(r["sigma_L"][e], r["sigma_R"][e]))
                for keys in (GR_KEYS, GL_KEYS):
                    assert gf_err(r, e, ref, keys) <= TOL_MIXED, (dev.name, e, keys)
    finally:
        ctx.close()
