"""CUDA path (through the C ABI) against the CPU oracle, element by element.

Sizes span several GEMM tiles and a ragged tail (b = 70 over 64-wide tiles),
plus the degenerate cases (b = 1, nb = 1, nb = 2, an empty device)."""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import negf_oracle as O
from negf_testutil import (GL_KEYS, GR_KEYS, TOL_FP64, TOL_MIXED, block_err, gf_err, oracle_density, run_gpu,
                           strong_leads)

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
    c = P.Context(0, 2 << 30)
    yield c
    c.close()


def _check_energy(r, e, ref, tol, lesser=True, keys=None):
    """FP64: every output family on its own (max block error / max block norm)."""
    keys = keys or (["GR_diag", "GR_up", "GR_low"] + (["GL_diag", "GL_low"] if lesser else []))
    for k in keys:
        err = block_err(r[k][e], ref[k])
        assert err <= tol, (k, e, err)


def _check_energy_mixed(r, e, ref, tol, lesser=True, keys=None):
    """Mixed precision: normwise over the BT pattern of G^R and of G^< (the products
    are accurate relative to row/column scales, not to blocks that are 1e-30 of
    their neighbours)."""
    gr = [k for k in GR_KEYS if keys is None or k in keys]
    gl = [k for k in GL_KEYS if keys is None or k in keys] if lesser else []
    for ks in (gr, gl):
        if ks:
            err = gf_err(r, e, ref, ks)
            assert err <= tol, (ks, e, err)


# --- config 1, in full -----------------------------------------------------------

def test_config1_fp64_full(P, ctx):
    dev = W.config1()
    r = run_gpu(P, ctx, dev, P.FP64, lesser=True)[0]
    assert np.all(r["obc_status"] == 0)
    assert np.all(r["status"] == 0)
    gold = np.loadtxt(__file__.replace("test_gpu_parity.py", "golden/config1_oracle.txt"))
    for e in range(dev.ne):
        ref = O.solve_energy(dev, e)
        for k in ("sigma_L", "sigma_R"):
            assert np.linalg.norm(r[k][e] - ref[k]) <= TOL_FP64 * max(np.linalg.norm(ref[k]), 1e-300)
        # OBC decimation steps agree with the oracle's (same stopping rule)
        assert np.abs(np.array(r["iters"][e]) - np.array(ref["obc"]["iters"])).max() <= 1
        # the sweeps are compared given the same Sigma: out of the band Gamma = i(Sigma - Sigma^H)
        # is O(eta), so G^< there amplifies last-bit differences of Sigma by ~1/eta
        ref = O.solve_energy(dev, e, sigma=(r["sigma_L"][e], r["sigma_R"][e]))
        _check_energy(r, e, ref, TOL_FP64)
        # T and DOS: |delta| / max(|ref|, 1e-3 max_E |ref|) (the tolerance reading for
        # the scalar observables; near-resonant energies at eta = 1e-6 amplify last-bit
        # differences of G by ~1/eta in a small DOS)
        tscale = max(1e-3 * np.abs(gold[:, 1]).max(), abs(gold[e, 1]))
        dscale = max(1e-3 * np.abs(gold[:, 3]).max(), abs(gold[e, 3]))
        assert abs(r["T"][e] - gold[e, 1]) <= 1e-8 * tscale
        assert abs(r["dos"][e] - gold[e, 3]) <= 1e-9 * dscale


def test_config1_mixed_full(P, ctx):
    dev = W.config1()
    r = run_gpu(P, ctx, dev, P.MIXED, lesser=True)[0]
    assert np.all(r["status"] == 0)
    for e in range(dev.ne):
        ref = O.solve_energy(dev, e, sigma=(r["sigma_L"][e], r["sigma_R"][e]))
        _check_energy_mixed(r, e, ref, TOL_MIXED)


# --- shape sweep: tiles, ragged tails, degenerate sizes --------------------------

SHAPES = [(2, 1), (3, 5), (5, 8), (3, 33), (4, 64), (3, 70), (2, 128)]


@pytest.mark.parametrize("nb,b", SHAPES)
@pytest.mark.parametrize("overlap", [False, True])
def test_shapes_fp64_lesser(P, ctx, nb, b, overlap):
    dev = strong_leads(W.banded_device(nb, b, 5, seed=100 + nb * b, overlap=overlap), seed=b)
    r = run_gpu(P, ctx, dev, P.FP64)[0]
    assert np.all(r["obc_status"] == 0)
    outs = []
    for e in range(dev.ne):
        ref = O.solve_energy(dev, e)
        for k in ("sigma_L", "sigma_R"):
            assert np.linalg.norm(r[k][e] - ref[k]) <= TOL_FP64 * max(np.linalg.norm(ref[k]), 1e-300)
        ref = O.solve_energy(dev, e, sigma=(r["sigma_L"][e], r["sigma_R"][e]))
        outs.append(ref)
        _check_energy(r, e, ref, TOL_FP64)
        assert abs(r["T"][e] - ref["T"]) <= 1e-9 * max(abs(ref["T"]), 1e-6)
        assert abs(r["dos"][e] - ref["dos"]) <= 1e-9 * abs(ref["dos"])
        jscale = max(np.linalg.norm(dev.H_up[i]) * np.linalg.norm(ref["GL_low"][i]) for i in range(nb - 1))
        assert np.abs(r["current"][e] - ref["J"]).max() <= 1e-10 * jscale + 1e-300
    n_ref = oracle_density(dev, outs)
    assert np.abs(r["density"] - n_ref).max() <= 1e-9 * np.abs(n_ref).max()


@pytest.mark.parametrize("nb,b", SHAPES)
def test_shapes_mixed_lesser(P, ctx, nb, b):
    dev = strong_leads(W.banded_device(nb, b, 5, seed=200 + nb * b, overlap=True), seed=b)
    r = run_gpu(P, ctx, dev, P.MIXED)[0]
    for e in range(dev.ne):
        ref = O.solve_energy(dev, e, sigma=(r["sigma_L"][e], r["sigma_R"][e]))
        _check_energy_mixed(r, e, ref, TOL_MIXED)


def test_uneven_batch_mixed_block_sizes(P, ctx):
    """Config-3 style: devices with different block sizes (incl. 192, 256) and block
    counts in one call, mixed precision, each against the oracle."""
    shapes = [(3, 32, 4), (2, 96, 3), (2, 192, 2), (2, 256, 2), (5, 64, 0)]
    devs = [strong_leads(W.banded_device(nb, b, ne, seed=300 + k, overlap=True), seed=k)
            for k, (nb, b, ne) in enumerate(shapes)]
    rs = run_gpu(P, ctx, devs, P.MIXED)
    for dev, r in zip(devs, rs):
        assert np.all(r["obc_status"] == 0)
        for e in range(dev.ne):
            ref = O.solve_energy(dev, e, sigma=(r["sigma_L"][e], r["sigma_R"][e]))
            _check_energy_mixed(r, e, ref, TOL_MIXED)


@pytest.mark.parametrize("nb", [4, 9])
def test_banded_weak_coupling_mixed(P, ctx, nb):
    """The config-2 generator itself (corner-coupled blocks, G^< spanning 30 decades)."""
    dev = W.banded_device(nb, 128, 8, seed=77, overlap=True)
    r = run_gpu(P, ctx, dev, P.MIXED)[0]
    for e in range(dev.ne):
        ref = O.solve_energy(dev, e, sigma=(r["sigma_L"][e], r["sigma_R"][e]))
        _check_energy_mixed(r, e, ref, TOL_MIXED)


@pytest.mark.parametrize("prec", ["FP64", "MIXED"])
def test_scattering_lesser(P, ctx, prec):
    dev = W.small_scattering_device(4, 24, 6, seed=31, overlap=True, strength=0.05)
    strong_leads(dev, seed=3)
    p = getattr(P, prec)
    tol = TOL_FP64 if prec == "FP64" else TOL_MIXED
    r = run_gpu(P, ctx, dev, p)[0]
    for e in range(dev.ne):
        ref = O.solve_energy(dev, e, sigma=(r["sigma_L"][e], r["sigma_R"][e]))
        (_check_energy if prec == "FP64" else _check_energy_mixed)(r, e, ref, tol)
        # J is a small difference of large terms: scale by the size of its summands
        jscale = max(np.linalg.norm(dev.H_up[i]) * np.linalg.norm(ref["GL_low"][i]) for i in range(dev.nb - 1))
        assert np.abs(r["current"][e] - ref["J"]).max() <= tol * jscale


def test_nb1_with_given_sigma(P, ctx):
    """nb = 1: one block, both self-energies on it (no lead hop: Sigma given)."""
    b = 6
    dev = W.banded_device(1, b, 4, seed=5, overlap=False)
    rng = np.random.default_rng(1)
    q = rng.normal(size=(2, dev.ne, b, b)) + 1j * rng.normal(size=(2, dev.ne, b, b))
    qh = np.conj(np.swapaxes(q, -1, -2))
    sig = 0.1 * (q + qh) - 0.2j * (q @ qh)
    for prec, tol in ((P.FP64, TOL_FP64), (P.MIXED, TOL_MIXED)):
        r = run_gpu(P, ctx, dev, prec, obc=False, sigma=(sig[0], sig[1]), obs=False)[0]
        for e in range(dev.ne):
            ref = O.solve_energy(dev, e, sigma=(sig[0][e], sig[1][e]))
            chk = _check_energy if prec == P.FP64 else _check_energy_mixed
            chk(r, e, ref, tol, keys=["GR_diag", "GL_diag"])


def test_uneven_batch_matches_single_devices(P, ctx):
    devs = [strong_leads(W.banded_device(nb, b, ne, seed=40 + k, overlap=True), seed=k)
            for k, (nb, b, ne) in enumerate([(3, 16, 4), (5, 8, 0), (2, 40, 3), (4, 24, 5)])]
    rs = run_gpu(P, ctx, devs, P.FP64)
    for dev, r in zip(devs, rs):
        if dev.ne == 0:
            continue
        single = run_gpu(P, ctx, dev, P.FP64)[0]
        for k in ("GR_diag", "GR_up", "GL_diag", "GL_low", "sigma_L"):
            assert np.array_equal(r[k], single[k]), k
        assert np.array_equal(r["density"], single["density"])
        for e in range(dev.ne):
            ref = O.solve_energy(dev, e, sigma=(r["sigma_L"][e], r["sigma_R"][e]))
            _check_energy(r, e, ref, TOL_FP64)



@pytest.mark.parametrize("b", [3, 8, 16])
def test_small_block_sweep_matches_batched_steps(P, ctx, b):
    """Blocks of b <= 16 (FP64) run the whole sweep as one launch, one CTA per energy; the
    same devices batched with another device of their block size run one launch per
    sweep step over a work list.  With scattering, the two agree to rounding and each
    matches the oracle."""
    devs = [strong_leads(W.small_scattering_device(nb, b, ne, seed=700 + 10 * b + k, overlap=True,
                                                   strength=0.05), seed=k)
            for k, (nb, ne) in enumerate([(4, 5), (7, 3)])]
    batched = run_gpu(P, ctx, devs, P.FP64)
    for dev, rb in zip(devs, batched):
        one = run_gpu(P, ctx, dev, P.FP64)[0]
        assert np.all(one["status"] == 0) and np.all(rb["status"] == 0)
        for k in GR_KEYS + GL_KEYS:
            scale = np.abs(rb[k]).max()
            assert np.abs(one[k] - rb[k]).max() <= 1e-11 * scale, k
        for e in range(dev.ne):
            ref = O.solve_energy(dev, e, sigma=(one["sigma_L"][e], one["sigma_R"][e]))
            _check_energy(one, e, ref, TOL_FP64)
        jscale = np.abs(rb["current"]).max()
        assert np.abs(one["current"] - rb["current"]).max() <= 1e-10 * jscale
        assert np.abs(one["density"] - rb["density"]).max() <= 1e-10 * np.abs(rb["density"]).max()


# --- numerical status codes ---------------------------------------------------------

def test_singular_block_flags_energy(P, ctx):
    """An exactly zero diagonal block with no coupling makes a zero pivot."""
    b, nb = 3, 3
    Hd = np.zeros((nb, b, b), complex)
    Hu = np.zeros((nb - 1, b, b), complex)
    dev = W.Device(Hd, Hu, None, None, np.array([0.0, 0.5]), 1e-6)
    sys_ = P.upload(dev)
    out = P.allocate_outputs(sys_)
    zero = torch.zeros_like(out["sigma_L"])
    # z = E + i eta with E = 0: A_ii = i eta I is invertible; force singularity with Sigma = z I on block 0
    sig = torch.from_numpy(np.stack([(e + 1j * dev.eta) * np.eye(b) for e in dev.energy]).reshape(-1)).cuda()
    P.negf_rgf_retarded(ctx, sys_, P.FP64, sig, zero, None, out["GR_diag"], None, None, out["status"])
    assert ctx.sync() == 0
    st = out["status"].cpu().numpy()
    assert np.all(st == P.negf.NEGF_ERR_SINGULAR)


def test_obc_max_iter_one_reports_noconv(P, ctx):
    dev = W.config1()
    sys_ = P.upload(dev)
    out = P.allocate_outputs(sys_)
    P.negf_obc(ctx, sys_, out["sigma_L"], out["sigma_R"], out["iters"], out["obc_status"], max_iter=1)
    assert ctx.sync() == 0
    st = out["obc_status"].cpu().numpy()
    assert (st == P.negf.NEGF_ERR_NOCONV).sum() > dev.ne // 2


def test_argument_errors(P, ctx):
    dev = W.config1()
    sys_ = P.upload(dev)
    out = P.allocate_outputs(sys_)
    with pytest.raises(P.NegfError) as ei:
        P.negf_rgf_lesser(ctx, sys_, P.FP64, out["sigma_L"], out["sigma_R"], None, None)
    assert ei.value.code == P.negf.NEGF_ERR_ARG
    bad = P.upload(dev)
    bad.eta = -1.0
    with pytest.raises(P.NegfError):
        P.negf_rgf_retarded(ctx, bad, P.FP64, out["sigma_L"], out["sigma_R"], None, out["GR_diag"])


# --- OBC with the FP64-class sliced products -------------------------------------------------

@pytest.mark.parametrize("nb,b", [(2, 16), (3, 33), (2, 64), (2, 128), (2, 192), (2, 256)])
def test_obc_mixed_products_match_oracle(P, ctx, nb, b):
    dev = strong_leads(W.banded_device(nb, b, 6, seed=500 + b, overlap=True), seed=b)
    r64 = run_gpu(P, ctx, dev, P.FP64, lesser=False, obs=False)[0]
    rmx = run_gpu(P, ctx, dev, P.FP64, lesser=False, obs=False, obc_prec=P.MIXED)[0]
    assert np.all(rmx["obc_status"] == 0)
    for e in range(dev.ne):
        ref = O.lead_self_energies(dev, dev.energy[e] + 1j * dev.eta)
        for k, sref in (("sigma_L", ref[0]), ("sigma_R", ref[1])):
            assert np.linalg.norm(rmx[k][e] - sref) <= TOL_FP64 * np.linalg.norm(sref), (e, k)
        # the same stopping rule: decimation steps agree with the FP64 run's
        assert np.abs(rmx["iters"][e] - r64["iters"][e]).max() <= 1


# --- observables with T's products on the sliced path --------------------------------------

@pytest.mark.parametrize("nb,b", [(3, 24), (2, 128), (2, 200)])
def test_observables_mixed_products_match_fp64(P, ctx, nb, b):
    """T's two block products (Gamma_L G_00, G_00 Gamma_L) on the sliced tensor-core path
    against FP64 products on the same G^R and Sigma: T within 1e-10 of max |T|; DOS,
    current and density use no products and are identical."""
    dev = strong_leads(W.banded_device(nb, b, 4, seed=300 + b, overlap=True), seed=b)
    sys_ = P.upload(dev)
    out = P.allocate_outputs(sys_)
    fL = torch.from_numpy(dev.f_L()).cuda()
    fR = torch.from_numpy(dev.f_R()).cuda()
    w = torch.from_numpy(dev.weights()).cuda()
    P.negf_obc(ctx, sys_, out["sigma_L"], out["sigma_R"], out["iters"], out["obc_status"])
    P.negf_rgf_lesser(ctx, sys_, P.FP64, out["sigma_L"], out["sigma_R"], fL, fR, None, out["GR_diag"],
                      out["GR_up"], out["GR_low"], out["GL_diag"], out["GL_low"], out["status"])
    res = {}
    for prec in (P.FP64, P.MIXED):
        got = {k: torch.zeros_like(out[k]) for k in ("T", "dos", "current", "density")}
        P.negf_observables(ctx, sys_, out["sigma_L"], w, out["GR_diag"], out["GR_up"], out["GR_low"],
                           out["GL_diag"], out["GL_low"], got["T"], got["dos"], got["current"], got["density"],
                           prec=prec)
        assert ctx.sync() == 0
        res[prec] = {k: v.cpu().numpy() for k, v in got.items()}
    t64, tm = res[P.FP64]["T"], res[P.MIXED]["T"]
    assert np.abs(tm - t64).max() <= 1e-10 * max(np.abs(t64).max(), 1e-6)
    for k in ("dos", "current", "density"):
        assert np.array_equal(res[P.FP64][k], res[P.MIXED][k]), k
