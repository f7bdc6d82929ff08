"""Helpers shared by the GPU parity tests: run the CUDA path through the C ABI
and compare with the CPU oracle using the block-normwise error metric."""
import numpy as np
import torch

import workloads as W
from oracle import negf_oracle as O

# tolerances of the two precision modes (relative, block-normwise)
TOL_FP64 = 1e-10
TOL_MIXED = 1e-6


GR_KEYS = ("GR_diag", "GR_up", "GR_low")
GL_KEYS = ("GL_diag", "GL_low")


def gf_err(r, e, ref, keys):
    """Normwise error of one Green's function over its whole BT pattern for energy e:
    max over all its blocks of ||got - ref||_F / max over all its blocks of ||ref||_F."""
    num, den = 0.0, 0.0
    for k in keys:
        for i in range(ref[k].shape[0]):
            num = max(num, np.linalg.norm(r[k][e][i] - ref[k][i]))
            den = max(den, np.linalg.norm(ref[k][i]))
    return num / max(den, 1e-300)


def block_err(got, ref):
    """max_i ||got_i - ref_i||_F / max_i ||ref_i||_F over the blocks of one energy."""
    if ref.size == 0:
        return 0.0
    num = max(np.linalg.norm(got[i] - ref[i]) for i in range(ref.shape[0]))
    den = max(np.linalg.norm(ref[i]) for i in range(ref.shape[0]))
    return num / max(den, 1e-300)


def run_gpu(P, ctx, devs, prec, lesser=True, obc=True, sigma=None, scat=True, obs=True, obc_prec=None):
    """Run OBC (or use given sigma), RGF and observables on the GPU; return numpy outputs
    split per device."""
    if not isinstance(devs, (list, tuple)):
        devs = [devs]
    sys_ = P.upload(devs)
    out = P.allocate_outputs(sys_, lesser=lesser)
    sc = P.Scattering.from_devices(devs) if scat else None
    if obc:
        P.negf_obc(ctx, sys_, out["sigma_L"], out["sigma_R"], out["iters"], out["obc_status"],
                   prec=P.FP64 if obc_prec is None else obc_prec)
    else:
        sl, sr = sigma
        out["sigma_L"].copy_(torch.from_numpy(np.ascontiguousarray(sl).reshape(-1)))
        out["sigma_R"].copy_(torch.from_numpy(np.ascontiguousarray(sr).reshape(-1)))
    fL = torch.from_numpy(np.concatenate([d.f_L() for d in devs])).cuda()
    fR = torch.from_numpy(np.concatenate([d.f_R() for d in devs])).cuda()
    w = torch.from_numpy(np.concatenate([d.weights() for d in devs])).cuda()
    if lesser:
        P.negf_rgf_lesser(ctx, sys_, prec, out["sigma_L"], out["sigma_R"], fL, fR, sc, out["GR_diag"],
                          out["GR_up"], out["GR_low"], out["GL_diag"], out["GL_low"], out["status"])
    else:
        P.negf_rgf_retarded(ctx, sys_, prec, out["sigma_L"], out["sigma_R"], sc, out["GR_diag"], out["GR_up"],
                            out["GR_low"], out["status"])
    if obs:
        P.negf_observables(ctx, sys_, out["sigma_L"], w, out["GR_diag"], out["GR_up"], out["GR_low"],
                           out.get("GL_diag"), out.get("GL_low"), out["T"], out["dos"], out.get("current"),
                           out.get("density"), prec=prec)
    assert ctx.sync() == 0
    L = sys_.layout()
    res = []
    host = {k: (v.cpu().numpy() if isinstance(v, torch.Tensor) else None) for k, v in out.items()}
    for d, dev in enumerate(devs):
        o = L[d]
        nb, b, ne = dev.nb, dev.b, dev.ne
        bb = b * b
        r = {}
        r["sigma_L"] = host["sigma_L"][o[3]:o[3] + ne * bb].reshape(ne, b, b)
        r["sigma_R"] = host["sigma_R"][o[3]:o[3] + ne * bb].reshape(ne, b, b)
        r["iters"] = host["iters"][2 * o[2]:2 * (o[2] + ne)].reshape(ne, 2)
        r["obc_status"] = host["obc_status"][o[2]:o[2] + ne]
        r["status"] = host["status"][o[2]:o[2] + ne]
        r["GR_diag"] = host["GR_diag"][o[4]:o[4] + ne * nb * bb].reshape(ne, nb, b, b)
        r["GR_up"] = host["GR_up"][o[5]:o[5] + ne * (nb - 1) * bb].reshape(ne, nb - 1, b, b)
        r["GR_low"] = host["GR_low"][o[5]:o[5] + ne * (nb - 1) * bb].reshape(ne, nb - 1, b, b)
        r["T"] = host["T"][o[2]:o[2] + ne]
        r["dos"] = host["dos"][o[2]:o[2] + ne]
        if lesser:
            r["GL_diag"] = host["GL_diag"][o[4]:o[4] + ne * nb * bb].reshape(ne, nb, b, b)
            r["GL_low"] = host["GL_low"][o[5]:o[5] + ne * (nb - 1) * bb].reshape(ne, nb - 1, b, b)
            r["current"] = host["current"][o[6]:o[6] + ne * (nb - 1)].reshape(ne, nb - 1)
            r["density"] = host["density"][o[7]:o[7] + nb * b]
        res.append(r)
    return res


def oracle_energy(dev, e, sigma=None, lesser=True, rgf=False):
    return O.solve_energy(dev, e, lesser=lesser, use_rgf=rgf, sigma=sigma)


def oracle_density(dev, outs):
    """Energy-integrated density from per-energy oracle outputs (trapezoid weights)."""
    w = dev.weights()
    n = np.zeros(dev.nb * dev.b)
    for e, o in enumerate(outs):
        n += w[e] * o["n_E"]
    return n


def strong_leads(dev, seed=0, scale=0.3):
    """Add a dense random coupling so that the leads carry current (the
    banded generator couples blocks only near the corner)."""
    rng = np.random.default_rng(seed)
    if dev.nb > 1:
        dev.H_up = dev.H_up + scale * (rng.normal(size=dev.H_up.shape) + 1j * rng.normal(size=dev.H_up.shape)) / np.sqrt(dev.b)
    return dev
