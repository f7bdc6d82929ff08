"""The warm-start network and the guess-driven OBC on the GPU, through the C ABI,
against the CPU oracle: feature packing (bit-exact), inference, gradients and Adam
(BF16 operands, FP32 accumulation vs the oracle's FP64 on the same BF16 values),
training progress, and the warm-start / fallback logic of negf_obc."""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import mlp_oracle as M
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
    c = P.Context(0, 512 << 20)
    yield c
    c.close()


def _bf16_bits(x):
    """BF16 bit patterns (int16) of values that are exactly BF16 numbers."""
    return (np.asarray(x, dtype=np.float32).view(np.uint32) >> 16).astype(np.uint16).view(np.int16)


def _leads(b, count, seed0=0):
    H00 = np.stack([W.config5_lead(seed0 + k, b)[0] for k in range(count)])
    H01 = np.stack([W.config5_lead(seed0 + k, b)[1] for k in range(count)])
    return H00, H01


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


# --- packing --------------------------------------------------------------------------

@pytest.mark.parametrize("b,n", [(8, 5), (64, 130)])
def test_pack_is_bit_exact(P, ctx, b, n):
    H00, H01 = _leads(b, 3)
    rng = np.random.default_rng(b)
    lead = rng.integers(0, 3, size=n).astype(np.int32)
    E = rng.uniform(-3, 3, size=n)
    X = P.negf.negf_mlp_pack(ctx, b, _dev(H00), _dev(H01), _dev(lead), _dev(E))
    assert ctx.sync() == 0
    got = X.cpu().view(torch.int16).numpy()
    k0, k0p, _, _ = M.mlp_dims(b)
    assert got.shape == (P.negf.mlp_rows(n), k0p)
    ref = np.stack([M.bf16_round(M.pack_features(H00[l], H01[l], e)) for l, e in zip(lead, E)])
    assert np.array_equal(got[:n], _bf16_bits(ref))
    assert np.all(got[n:] == 0)


def test_pack_flags_a_bad_lead_index(P, ctx):
    H00, H01 = _leads(8, 2)
    X = P.negf.negf_mlp_pack(ctx, 8, _dev(H00), _dev(H01), _dev(np.array([0, 5], np.int32)),
                             _dev(np.array([0.1, 0.2])))
    with pytest.raises(P.NegfError) as ei:
        ctx.check(ctx.sync())
    assert ei.value.code == P.negf.NEGF_ERR_ARG
    assert np.all(X[1].cpu().view(torch.int16).numpy() == 0)


# --- network ----------------------------------------------------------------------------

def _net(b, hidden, n, seed=0, scale=1.0):
    rng = np.random.default_rng(seed)
    theta = W.mlp_init(b, hidden, seed).astype(np.float64)
    H00, H01 = _leads(b, 4, seed0=10 * seed)
    lead = rng.integers(0, 4, size=n).astype(np.int32)
    E = rng.uniform(-3, 3, size=n)
    X = np.stack([M.pack_features(H00[l], H01[l], e) for l, e in zip(lead, E)])
    G = scale * (rng.normal(size=(n, b, b)) + 1j * rng.normal(size=(n, b, b)))
    T = np.stack([M.pack_target(g) for g in G])
    return theta, H00, H01, lead, E, X, G, T


def _gpu_inputs(P, ctx, b, hidden, theta, H00, H01, lead, E):
    dims = P.negf.negf_mlp_get_dims(b, hidden)
    params = _dev(theta.astype(np.float32))
    X = P.negf.negf_mlp_pack(ctx, b, _dev(H00), _dev(H01), _dev(lead), _dev(E))
    return dims, params, X


def _relerr(got, ref):
    return np.linalg.norm(got - ref) / max(np.linalg.norm(ref), 1e-300)


@pytest.mark.parametrize("b,hidden,n", [(8, 128, 200), (16, 256, 300)])
def test_forward_matches_oracle(P, ctx, b, hidden, n):
    theta, H00, H01, lead, E, X, G, T = _net(b, hidden, n, seed=1)
    dims, params, Xd = _gpu_inputs(P, ctx, b, hidden, theta, H00, H01, lead, E)
    g0 = P.negf.negf_mlp_forward(ctx, dims, params, n, Xd)
    assert ctx.sync() == 0
    Y, _ = M.forward(theta.astype(np.float32).astype(np.float64), X, b, hidden, quant=True)
    ref = np.stack([M.unpack_output(y, b) for y in Y])
    # same BF16 operands; FP32 accumulation and the rare BF16 rounding flip of a hidden
    # activation (relative change 2^-8) set the difference
    assert _relerr(g0.cpu().numpy(), ref) <= 1e-3


@pytest.mark.parametrize("b,hidden,n", [(8, 128, 200), (16, 256, 300)])
def test_gradients_match_oracle(P, ctx, b, hidden, n):
    theta, H00, H01, lead, E, X, G, T = _net(b, hidden, n, seed=2)
    dims, params, Xd = _gpu_inputs(P, ctx, b, hidden, theta, H00, H01, lead, E)
    grad = torch.zeros(dims.n_params, dtype=torch.float32, device="cuda")
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    P.negf.negf_mlp_train_step(ctx, dims, params, None, None, grad, 1, 1e-3, n, Xd, _dev(G), loss, update=False)
    assert ctx.sync() == 0
    th32 = theta.astype(np.float32).astype(np.float64)
    l_ref, g_ref, _ = M.loss_and_grads(th32, X, T, b, hidden, quant=True)
    assert abs(loss.item() - l_ref) <= 1e-5 * l_ref
    gg = M.split_params(grad.cpu().numpy().astype(np.float64), b, hidden)
    rr = M.split_params(g_ref, b, hidden)
    for k in ("W1", "c1", "W2", "c2", "W3", "c3"):
        assert _relerr(gg[k], rr[k]) <= 2e-3, k
    # the padding columns of W1 get exactly zero gradient
    assert np.all(gg["W1"][:, M.mlp_dims(b, hidden)[0]:] == 0.0)
    assert np.allclose(params.cpu().numpy(), theta.astype(np.float32))   # no update


def test_adam_steps_match_oracle(P, ctx):
    b, hidden, n = 8, 128, 128
    theta, H00, H01, lead, E, X, G, T = _net(b, hidden, n, seed=3)
    dims, params, Xd = _gpu_inputs(P, ctx, b, hidden, theta, H00, H01, lead, E)
    m = torch.zeros(dims.n_params, dtype=torch.float32, device="cuda")
    v = torch.zeros_like(m)
    grad = torch.zeros_like(m)
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    th, mm, vv = theta.astype(np.float32).astype(np.float64), np.zeros(dims.n_params), np.zeros(dims.n_params)
    for step in (1, 2, 3):
        P.negf.negf_mlp_train_step(ctx, dims, params, m, v, grad, step, 1e-3, n, Xd, _dev(G), loss)
        assert ctx.sync() == 0
        g = grad.cpu().numpy().astype(np.float64)      # the update is checked given the GPU's gradient
        th, mm, vv = M.adam_step(th, g, mm, vv, step, 1e-3)
        assert np.abs(params.cpu().numpy() - th).max() <= 1e-6
        assert np.abs(m.cpu().numpy() - mm).max() <= 1e-6 * max(np.abs(mm).max(), 1e-30)
        th = params.cpu().numpy().astype(np.float64)    # continue from the GPU state
        mm = m.cpu().numpy().astype(np.float64)
        vv = v.cpu().numpy().astype(np.float64)


def test_training_reduces_the_loss(P, ctx):
    # a target that is a smooth function of the inputs: G = 0.3 (H00 cos E + H01 sin E)
    b, hidden, n = 16, 256, 256
    theta, H00, H01, lead, E, X, _, _ = _net(b, hidden, n, seed=4)
    G = 0.3 * (H00[lead] * np.cos(E)[:, None, None] + H01[lead] * np.sin(E)[:, None, None])
    dims, params, Xd = _gpu_inputs(P, ctx, b, hidden, theta, H00, H01, lead, E)
    m = torch.zeros(dims.n_params, dtype=torch.float32, device="cuda")
    v, grad = torch.zeros_like(m), torch.zeros_like(m)
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    Gd = _dev(G)
    hist = []
    for step in range(1, 201):
        P.negf.negf_mlp_train_step(ctx, dims, params, m, v, grad, step, 1e-3, n, Xd, Gd, loss)
        if step in (1, 200):
            hist.append(loss.item())
    assert ctx.sync() == 0
    assert hist[1] < 0.2 * hist[0]


# --- warm-started OBC ------------------------------------------------------------------------

def _lead_device(H00, H01, energies, eta):
    """nb = 2 device whose two leads are the lead (H00, H01): the right lead faces
    +x with hop H01, the left lead -x (hop H01^H as seen from its surface)."""
    return W.Device(H_diag=np.stack([H00, H00]), H_up=H01[None].copy(), S_diag=None, S_up=None,
                    energy=np.asarray(energies, dtype=np.float64), eta=eta, mu_L=0.1, mu_R=-0.1, kT=0.025,
                    name="lead")


def _oracle_surfaces(H00, H01, E, eta):
    a00 = (E + 1j * eta) * np.eye(H00.shape[0]) - H00
    gR = O.surface_gf(a00, -H01, -H01.conj().T)[0]
    gL = O.surface_gf(a00, -H01.conj().T, -H01)[0]
    return a00, gL, gR


@pytest.mark.parametrize("eta,expect_warm", [(5e-2, True), (1e-6, False)])
def test_obc_warm_start_keeps_or_falls_back_like_the_oracle(P, ctx, eta, expect_warm):
    b = 16
    H00, H01 = W.config5_lead(11, b)
    E = np.array([-2.1, -0.4, 0.9, 2.6])
    dev = _lead_device(H00, H01, E, eta)
    rng = np.random.default_rng(5)
    g0L, g0R, refs = [], [], []
    for e in E:
        a00, gL, gR = _oracle_surfaces(H00, H01, e, eta)
        noise = lambda g: 1e-3 * np.linalg.norm(g) * (lambda N: N / np.linalg.norm(N))(
            rng.normal(size=(b, b)) + 1j * rng.normal(size=(b, b)))
        gl0, gr0 = gL + noise(gL), gR + noise(gR)
        g0L.append(gl0)
        g0R.append(gr0)
        rL = O.warm_surface_gf(a00, -H01.conj().T, -H01, gl0)
        rR = O.warm_surface_gf(a00, -H01, -H01.conj().T, gr0)
        refs.append((rL, rR))
    sys_ = P.upload(dev)
    ne = len(E)
    z = lambda: torch.zeros(ne * b * b, dtype=torch.complex128, device="cuda")
    sL, sR, gsL, gsR = z(), z(), z(), z()
    iters = torch.zeros(2 * ne, dtype=torch.int32, device="cuda")
    newton = torch.zeros_like(iters)
    status = torch.zeros(ne, dtype=torch.int32, device="cuda")
    P.negf_obc(ctx, sys_, sL, sR, iters, status, g0_L=_dev(np.stack(g0L)), g0_R=_dev(np.stack(g0R)), gs_L=gsL,
               gs_R=gsR, newton=newton)
    assert ctx.sync() == 0
    assert np.all(status.cpu().numpy() == 0)
    it = iters.cpu().numpy().reshape(ne, 2)
    nw = newton.cpu().numpy().reshape(ne, 2)
    GL = gsL.cpu().numpy().reshape(ne, b, b)
    GR = gsR.cpu().numpy().reshape(ne, b, b)
    for e in range(ne):
        for side, got in ((0, GL[e]), (1, GR[e])):
            X, oit, ons, ores, owarm = refs[e][side]
            # whichever path produced it, the result is the unique retarded root
            assert np.linalg.norm(got - X) <= 1e-9 * np.linalg.norm(X)
            if expect_warm:
                # well inside Newton's basin both sides keep the guess, in the same steps
                assert it[e, side] == 0 and owarm, (e, side)
                assert abs(int(nw[e, side]) - ons) <= 1
            elif it[e, side] != 0:
                # fell back: the decimation ran, as in the oracle's fallback
                assert not owarm or oit == 0
    if not expect_warm:
        # at eta = 1e-6 the Newton basin is ~eta wide: a 1e-3 guess falls back for most
        # leads (whether a borderline Smith series converges depends on rounding order)
        assert (it != 0).sum() >= it.size // 2
    # the self-energies follow from the kept surfaces
    a01 = -H01
    for e in range(ne):
        assert np.linalg.norm(sR.cpu().numpy().reshape(ne, b, b)[e] - a01 @ GR[e] @ a01.conj().T) <= \
            1e-12 * np.linalg.norm(a01) ** 2 * np.linalg.norm(GR[e])


def test_obc_rejects_a_wrong_root_and_falls_back(P, ctx):
    # the wrong root solves the surface equation to rounding but is not retarded: the
    # Stein-inertia test rejects it and the decimation gives the retarded one
    b, eta = 3, 1e-6
    H00, H01 = W.config5_lead(5, b)
    E = np.array([0.3, -1.1])
    a01, a10 = -H01, -H01.conj().T
    wrongR, good = [], []
    for e in E:
        a00 = (e + 1j * eta) * np.eye(b) - H00
        I, Z = np.eye(b), np.zeros((b, b))
        lam, V = np.linalg.eig(np.linalg.solve(np.block([[I, Z], [Z, a01]]), np.block([[Z, I], [-a10, -a00]])))
        order = np.argsort(np.abs(lam))
        pick = list(order[:b])
        pick[-1] = order[b]
        U = V[:b, pick]
        Fm = U @ np.diag(lam[pick]) @ np.linalg.inv(U)
        wrongR.append(np.linalg.inv(a00 + a01 @ Fm))
        good.append(O.surface_gf(a00, a01, a10)[0])
    dev = _lead_device(H00, H01, E, eta)
    sys_ = P.upload(dev)
    ne = len(E)
    z = lambda: torch.zeros(ne * b * b, dtype=torch.complex128, device="cuda")
    sL, sR, gsR = z(), z(), z()
    iters = torch.zeros(2 * ne, dtype=torch.int32, device="cuda")
    status = torch.zeros(ne, dtype=torch.int32, device="cuda")
    P.negf_obc(ctx, sys_, sL, sR, iters, status, g0_R=_dev(np.stack(wrongR)), gs_R=gsR)
    assert ctx.sync() == 0
    assert np.all(status.cpu().numpy() == 0)
    it = iters.cpu().numpy().reshape(ne, 2)
    assert np.all(it[:, 1] > 0)      # the guess was not kept
    GR = gsR.cpu().numpy().reshape(ne, b, b)
    for e in range(ne):
        assert np.linalg.norm(GR[e] - good[e]) <= 1e-9 * np.linalg.norm(good[e])


def test_minibatch_rows_match_the_packed_subset(P, ctx):
    b, hidden, n = 8, 128, 300
    theta, H00, H01, lead, E, X, G, T = _net(b, hidden, n, seed=6)
    dims, params, Xd = _gpu_inputs(P, ctx, b, hidden, theta, H00, H01, lead, E)
    rows = np.random.default_rng(0).permutation(n)[:130].astype(np.int32)
    grad = torch.zeros(dims.n_params, dtype=torch.float32, device="cuda")
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    P.negf.negf_mlp_train_step(ctx, dims, params, None, None, grad, 1, 1e-3, len(rows), Xd, _dev(G), loss,
                               update=False, rows=_dev(rows), n_set=n)
    assert ctx.sync() == 0
    th32 = theta.astype(np.float32).astype(np.float64)
    l_ref, g_ref, _ = M.loss_and_grads(th32, X[rows], T[rows], b, hidden, quant=True)
    assert abs(loss.item() - l_ref) <= 1e-5 * l_ref
    gg = M.split_params(grad.cpu().numpy().astype(np.float64), b, hidden)
    rr = M.split_params(g_ref, b, hidden)
    for k in ("W1", "W2", "W3", "c3"):
        assert _relerr(gg[k], rr[k]) <= 2e-3, k
