"""Pins of the warm-start oracle (network, rounding, optimiser, guess-driven OBC)
against closed forms, finite differences and an independent construction of the
lead's roots from its Bloch modes."""
import numpy as np
import pytest

import workloads as W
from oracle import mlp_oracle as M
from oracle import negf_oracle as O


# --- BF16 rounding ----------------------------------------------------------------

def test_bf16_round_closed_cases():
    u = 2.0 ** -7                      # BF16 spacing on [1, 2)
    cases = {1.0: 1.0, 1 + u / 2: 1.0, 1 + 1.5 * u: 1 + 2 * u, 1 + 0.49 * u: 1.0, 1 + 0.51 * u: 1 + u,
             -(1 + 1.5 * u): -(1 + 2 * u), 3.0: 3.0, 2.0 ** -130 * 1.5: 2.0 ** -130 * 1.5, 0.0: 0.0}
    for x, r in cases.items():
        assert M.bf16_round(x) == r, x


def test_bf16_round_matches_bit_formula_on_float32():
    # for values that are float32 numbers, RNE to BF16 is the classic integer formula
    rng = np.random.default_rng(0)
    x = (rng.normal(size=20000) * 10.0 ** rng.uniform(-20, 20, size=20000)).astype(np.float32)
    bits = x.view(np.uint32).astype(np.uint64)
    r = ((bits + 0x7FFF + ((bits >> 16) & 1)) >> 16) << 16
    ref = r.astype(np.uint32).view(np.float32).astype(np.float64)
    assert np.array_equal(M.bf16_round(x.astype(np.float64)), ref)


# --- feature packing -------------------------------------------------------------------

def test_pack_features_round_trip():
    H00, H01 = W.config5_lead(3, b=6)
    x = M.pack_features(H00, H01, -1.25)
    k0, k0p, _, _ = M.mlp_dims(6)
    assert k0 == 3 * 36 + 1 + 64 and k0p % 128 == 0 and x.shape == (k0p,)
    assert np.all(x[k0:] == 0.0)
    w = 2.0 ** (np.arange(32) / 4.0)
    assert np.allclose(M.freqs(), w, rtol=1e-15, atol=0)
    assert np.allclose(x[3 * 36 + 1:k0:2], np.sin(-1.25 * w)) and np.allclose(x[3 * 36 + 2:k0:2], np.cos(-1.25 * w))
    A, B, E = M.unpack_features(x, 6)
    assert np.allclose(A, H00, atol=1e-15) and np.allclose(B, H01, atol=1e-15) and abs(E + 1.25) < 1e-15
    assert np.allclose(M.unpack_output(M.pack_target(H01), 6), H01, atol=0)


# --- network and gradients -------------------------------------------------------------

def _tiny(seed=0, b=2, hidden=8, n=5):
    rng = np.random.default_rng(seed)
    _, total = M.param_layout(b, hidden)
    theta = rng.normal(size=total) * 0.3
    k0, k0p, _, nout = M.mlp_dims(b, hidden)
    X = np.zeros((n, k0p))
    X[:, :k0] = rng.normal(size=(n, k0))
    T = rng.normal(size=(n, nout))
    return theta, X, T, b, hidden


def test_gradients_match_central_differences():
    theta, X, T, b, h = _tiny()
    loss, grad, _ = M.loss_and_grads(theta, X, T, b, h, quant=False)
    lay, _ = M.param_layout(b, h)
    rng = np.random.default_rng(1)
    k0 = M.mlp_dims(b, h)[0]
    checked = 0
    for name, (o, n) in lay.items():
        idx = rng.choice(n, size=min(n, 12), replace=False)
        if name == "W1":   # include live columns (k < K0) of W1
            idx = np.array([r * (n // h) + c for r in range(h) for c in (0, 3 * b * b, k0 - 1)])
        for i in idx:
            eps = 1e-6
            tp, tm = theta.copy(), theta.copy()
            tp[o + i] += eps
            tm[o + i] -= eps
            lp = M.loss_and_grads(tp, X, T, b, h, quant=False)[0]
            lm = M.loss_and_grads(tm, X, T, b, h, quant=False)[0]
            fd = (lp - lm) / (2 * eps)
            assert abs(fd - grad[o + i]) <= 1e-6 * max(1.0, abs(fd)), (name, i, fd, grad[o + i])
            checked += 1
    assert checked > 50


def test_padding_columns_get_zero_gradient():
    theta, X, T, b, h = _tiny(seed=2)
    _, grad, _ = M.loss_and_grads(theta, X, T, b, h, quant=True)
    p = M.split_params(grad, b, h)
    k0 = M.mlp_dims(b, h)[0]
    assert np.all(p["W1"][:, k0:] == 0.0)


def test_forward_closed_form_constant_output():
    theta, X, T, b, h = _tiny(seed=3, n=1)
    p = M.split_params(theta, b, h)
    p["W3"][:] = 0.0
    p["c3"][:] = T[0]
    loss, grad, Y = M.loss_and_grads(theta, X, T, b, h, quant=True)
    assert np.array_equal(Y[0], T[0]) and loss == 0.0 and np.all(grad == 0.0)


def test_relu_network_by_hand():
    # b = 1, hidden 2: z1 = W1 x + c1 etc. written out for one sample (feature 3 is E/3;
    # the Fourier features of E get zero weights)
    b, h = 1, 2
    lay, total = M.param_layout(b, h)
    theta = np.zeros(total)
    p = M.split_params(theta, b, h)
    p["W1"][0, 0], p["W1"][1, 3], p["c1"][:] = 1.0, -2.0, (0.5, 0.25)
    p["W2"][:] = [[1.0, 0.0], [1.0, 1.0]]
    p["W3"][:] = [[1.0, 2.0], [-1.0, 0.0]]
    p["c3"][:] = (0.0, 3.0)
    x = M.pack_features(np.array([[0.75]]), np.array([[0.0]]), 1.5)
    # x = [0.75, 0, 0, 0.5, 0...]; z1 = [0.75 + 0.5, -1 + 0.25]; h1 = [1.25, 0]
    # z2 = [1.25, 1.25]; y = [1.25 + 2.5, -1.25 + 3]
    Y, _ = M.forward(theta, x[None], b, h, quant=True)
    assert np.allclose(Y[0], [3.75, 1.75], atol=0)


def test_adam_first_step_closed_form():
    rng = np.random.default_rng(4)
    th, g = rng.normal(size=50), rng.normal(size=50)
    g[0] = 0.0
    new, m, v = M.adam_step(th, g, np.zeros(50), np.zeros(50), 1, 1e-3)
    # bias-corrected m/sqrt(v) = g/|g| on the first step
    assert np.allclose(new[1:], th[1:] - 1e-3 * g[1:] / (np.abs(g[1:]) + 1e-8), rtol=0, atol=1e-15)
    assert new[0] == th[0]
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


# --- guess-driven OBC and the retarded-root test ----------------------------------------

def _chain_roots(E, t, eta):
    z = E + 1j * eta
    s = np.sqrt(z * z - 4 * t * t)
    r1, r2 = (z - s) / (2 * t * t), (z + s) / (2 * t * t)
    # retarded root: the one with |g t| < 1 (decaying mode)
    return (r1, r2) if abs(r1 * t) < abs(r2 * t) else (r2, r1)


@pytest.mark.parametrize("E", [-2.5, -1.3, 0.2, 1.7, 2.4])
def test_retarded_check_on_chain_roots(E):
    t, eta = 1.0, 1e-6
    good, bad = _chain_roots(E, t, eta)
    a00 = np.array([[E + 1j * eta]])
    al = be = np.array([[-t]])
    for r in (good, bad):   # both solve the quadratic equation
        assert O.surface_residual(a00, al, be, np.array([[r]])) < 1e-12
    assert O.retarded_check(np.array([[good]]))
    assert not O.retarded_check(np.array([[bad]]))


def _mode_root(a00, a01, a10, swap=0):
    """Surface function (a00 + a01 F)^{-1} with F = U L U^{-1} built from b Bloch modes of
    a10 + a00 lam + a01 lam^2 = 0: the b decaying modes, or with ``swap`` of them
    exchanged for growing ones (another root of the same quadratic equation)."""
    b = a00.shape[0]
    I, Z = np.eye(b), np.zeros((b, b))
    # companion pencil for psi_{n+1} = lam psi_n: [[0, I], [-a10, -a00]] v = lam [[I, 0], [0, a01]] v
    Amat = np.block([[Z, I], [-a10, -a00]])
    Bmat = np.block([[I, Z], [Z, a01]])
    lam, V = np.linalg.eig(np.linalg.solve(Bmat, Amat))
    order = np.argsort(np.abs(lam))
    pick = list(order[:b])
    for k in range(swap):
        pick[b - 1 - k] = order[b + k]
    U = V[:b, pick]
    F = U @ np.diag(lam[pick]) @ np.linalg.inv(U)
    return np.linalg.inv(a00 + a01 @ F)


@pytest.mark.parametrize("eta,E", [(1e-6, 0.3), (1e-6, -1.1), (1e-3, 0.8)])
def test_mode_roots_pin_decimation_and_retarded_check(eta, E):
    H00, H01 = W.config5_lead(5, b=3)
    a00 = (E + 1j * eta) * np.eye(3) - H00
    a01, a10 = -H01, -H01.conj().T
    g_sr, it, ns, res, ok = O.surface_gf(a00, a01, a10)
    g_modes = _mode_root(a00, a01, a10)
    assert ok and np.linalg.norm(g_sr - g_modes) <= 1e-8 * np.linalg.norm(g_modes)
    assert O.retarded_check(g_sr)
    wrong = _mode_root(a00, a01, a10, swap=1)
    assert O.surface_residual(a00, a01, a10, wrong) < 1e-9
    assert np.linalg.norm(wrong - g_sr) > 1e-3 * np.linalg.norm(g_sr)
    assert not O.retarded_check(wrong)


def test_newton_warm_from_exact_root_takes_no_step():
    H00, H01 = W.config5_lead(1, b=4)
    a00 = (0.4 + 1e-6j) * np.eye(4) - H00
    g, *_ = O.surface_gf(a00, -H01, -H01.conj().T)
    X, steps, res = O.surface_newton_warm(a00, -H01, -H01.conj().T, g, target=1e-11)
    assert steps == 0 and res <= 1e-11 and X is g


def test_newton_warm_converges_at_large_eta_and_falls_back_at_small_eta():
    H00, H01 = W.config5_lead(2, b=8)
    a01, a10 = -H01, -H01.conj().T
    rng = np.random.default_rng(7)
    for eta, expect_warm in ((5e-2, True), (1e-6, False)):
        a00 = (0.7 + 1j * eta) * np.eye(8) - H00
        g, *_ = O.surface_gf(a00, a01, a10)
        N = rng.normal(size=(8, 8)) + 1j * rng.normal(size=(8, 8))
        g0 = g + 1e-3 * np.linalg.norm(g) * N / np.linalg.norm(N)
        X, it, ns, res, warm = O.warm_surface_gf(a00, a01, a10, g0)
        assert res <= 1e-10 and np.linalg.norm(X - g) <= 1e-8 * np.linalg.norm(g)
        assert warm == expect_warm
        assert (it == 0) == warm
