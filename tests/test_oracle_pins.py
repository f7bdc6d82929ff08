"""Pins of the CPU oracle against closed forms, invariants and brute force.

Each test ties an oracle function to something other than itself: a closed
form (1D chain surface function, integer transmission of a perfect wire), an
independent library routine (generalized eigendecomposition), brute force (a
long finite chain inverted densely), or an exact identity of Eqs. (1)-(2)
(anti-Hermiticity of G^<, the spectral identity, current continuity).
"""
import numpy as np
import pytest
import scipy.linalg as sla

import workloads as W
from oracle import negf_oracle as O

H = lambda x: np.conj(np.swapaxes(x, -1, -2))


# --- OBC: closed form of the 1D chain ------------------------------------------

def chain_surface_closed_form(E, t, eta):
    """g = (z - sqrt(z^2 - 4t^2)) / (2 t^2), branch with |g t| <= 1 (retarded)."""
    z = E + 1j * eta
    r = np.sqrt(z * z - 4 * t * t + 0j)
    g1 = (z - r) / (2 * t * t)
    g2 = (z + r) / (2 * t * t)
    return g1 if abs(g1 * t) <= abs(g2 * t) else g2


@pytest.mark.parametrize("t", [1.0, 0.7])
@pytest.mark.parametrize("E", [-2.5, -1.9, -1.0, -0.3, 0.0, 0.45, 1.3, 1.99, 2.01, 3.0])
def test_chain_surface_closed_form(E, t):
    eta = 1e-6
    z = E + 1j * eta
    a00 = np.array([[z]])
    a01 = np.array([[-t + 0j]])
    g, it, ns, res, ok = O.surface_gf(a00, a01, a01, 1e-12, 100)
    ref = chain_surface_closed_form(E, t, eta)
    assert ok
    assert res <= 1e-10
    assert abs(g[0, 0] - ref) <= 1e-9 * max(1.0, abs(ref))
    if abs(E) < 2 * t:
        assert g[0, 0].imag < 0      # retarded branch in the band


# --- OBC + assembly: brute force by a long finite chain ------------------------

def _embedded_device(dev, L):
    """The device with L explicit lead cells on each side (dense H, S)."""
    nb, b = dev.nb, dev.b
    Sd = [np.eye(b)] * nb if dev.S_diag is None else list(dev.S_diag)
    Su = [np.zeros((b, b))] * (nb - 1) if dev.S_up is None else list(dev.S_up)
    diag = [dev.H_diag[0]] * L + list(dev.H_diag) + [dev.H_diag[-1]] * L
    up = [dev.H_up[0]] * L + list(dev.H_up) + [dev.H_up[-1]] * L
    sdiag = [Sd[0]] * L + Sd + [Sd[-1]] * L
    sup = [Su[0]] * L + Su + [Su[-1]] * L
    return (O.dense_matrix(np.array(diag), np.array(up)),
            O.dense_matrix(np.array(sdiag), np.array(sup)))


@pytest.mark.parametrize("overlap", [False, True])
def test_obc_against_long_finite_chain(overlap):
    """With eta = 0.05 a chain of 500 explicit lead cells is indistinguishable
    (e^{-eta L / v}) from the semi-infinite one: the device blocks of its dense
    inverse must equal the OBC + device solution."""
    b, nb, L = 3, 4, 500
    dev = W.banded_device(nb, b, 3, seed=11, overlap=overlap)
    # make leads strongly coupled (a narrow band lead would hide index mistakes)
    rng = np.random.default_rng(5)
    dev.H_up = dev.H_up + 0.4 * (rng.normal(size=dev.H_up.shape) + 1j * rng.normal(size=dev.H_up.shape))
    dev.eta = 0.05
    Hbig, Sbig = _embedded_device(dev, L)
    for E in [-0.7, 0.05, 0.6]:
        z = E + 1j * dev.eta
        Gbig = np.linalg.inv(z * Sbig - Hbig)
        sL, sR, info = O.lead_self_energies(dev, z)
        out = O.greens_dense(dev, z, sL, sR)
        off = L * b
        for i in range(nb):
            ref = Gbig[off + i * b: off + (i + 1) * b, off + i * b: off + (i + 1) * b]
            assert np.abs(out["GR_diag"][i] - ref).max() <= 1e-9 * np.abs(ref).max()
        for i in range(nb - 1):
            ref_u = Gbig[off + i * b: off + (i + 1) * b, off + (i + 1) * b: off + (i + 2) * b]
            ref_l = Gbig[off + (i + 1) * b: off + (i + 2) * b, off + i * b: off + (i + 1) * b]
            assert np.abs(out["GR_up"][i] - ref_u).max() <= 1e-9 * np.abs(ref_u).max()
            assert np.abs(out["GR_low"][i] - ref_l).max() <= 1e-9 * np.abs(ref_l).max()


def test_stein_doubling_against_kronecker():
    rng = np.random.default_rng(3)
    n = 5
    P = rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))
    Q = rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))
    # Smith's series converges for rho(P) rho(Q) < 1; make it slow (0.97)
    P *= 0.97 / np.abs(np.linalg.eigvals(P)).max()
    Q /= np.abs(np.linalg.eigvals(Q)).max()
    P *= 1e3      # badly balanced factors: only the products matter
    Q *= 1e-3
    C = rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))
    D = O.stein_smith(P, Q, C)
    # vec(P D Q) = (Q^T kron P) vec(D) (column-major vec)
    M = np.eye(n * n) - np.kron(Q.T, P)
    ref = np.linalg.solve(M, C.reshape(-1, order="F")).reshape(n, n, order="F")
    assert np.abs(D - ref).max() <= 1e-12 * np.abs(ref).max()


def test_obc_residual_config1_all_energies():
    dev = W.config1()
    for e in range(dev.ne):
        z = dev.energy[e] + 1j * dev.eta
        _, _, info = O.lead_self_energies(dev, z)
        assert all(info["converged"])
        assert max(info["residual"]) <= 1e-10
        # Gamma = i(Sigma - Sigma^H) is positive semidefinite for a retarded lead
    for e in [10, 30, 50]:
        z = dev.energy[e] + 1j * dev.eta
        sL, sR, _ = O.lead_self_energies(dev, z)
        for s in (sL, sR):
            assert np.linalg.eigvalsh(O.gamma(s)).min() >= -1e-10


# --- transmission: integer in the band of a perfect wire -----------------------

def test_ideal_chain_transmission():
    E = np.array([-2.5, -1.9, -1.2, -0.4, 0.0, 0.7, 1.5, 1.95, 2.05, 2.8])
    dev = W.ideal_chain(6, 1.0, E)
    for e in range(dev.ne):
        out = O.solve_energy(dev, e, lesser=False)
        expect = 1.0 if abs(E[e]) < 2.0 else 0.0
        # O(eta N / v) absorption inside the device at eta = 1e-6
        assert abs(out["T_caroli"] - expect) <= 1e-4
        assert abs(out["T"] - expect) <= 1e-4


def test_ideal_multiorbital_integer_transmission():
    """A perfect wire of identical cells transmits an integer number of
    channels; a transposed or mis-signed self-energy breaks this."""
    H00, H01 = W.config5_lead(0, b=4)
    E = np.linspace(-3.0, 3.0, 41)
    dev = W.ideal_multiorbital(5, H00, H01, E)
    vals = []
    for e in range(dev.ne):
        out = O.solve_energy(dev, e, lesser=False)
        vals.append(out["T_caroli"])
        # band edges excluded: the O(eta) rounding there is not integer
        assert abs(out["T_caroli"] - round(out["T_caroli"])) <= 2e-3
    assert max(vals) >= 2.0 - 1e-3    # several channels open somewhere


# --- Eq. (1): dense inverse vs a generalized eigendecomposition ---------------

def test_closed_system_against_eigendecomposition():
    dev = W.banded_device(3, 4, 5, seed=2)
    Hd, Sd = O.dense_H_S(dev)
    lam, V = sla.eigh(Hd, Sd)               # V^H S V = I
    zero = np.zeros((4, 4), complex)
    for e in range(dev.ne):
        z = dev.energy[e] + 0.03j
        out = O.greens_dense(dev, z, zero, zero, keep_dense=True)
        Gref = (V / (z - lam)) @ H(V)
        assert np.abs(out["G"] - Gref).max() <= 1e-11 * np.abs(Gref).max()
        d_ref = float(-np.imag(np.sum(1.0 / (z - lam))) / np.pi)
        d = O.dos(dev, out["GR_diag"], out["GR_up"], out["GR_low"])
        assert abs(d - d_ref) <= 1e-10 * abs(d_ref)


# --- RGF recursion vs the definition -------------------------------------------

@pytest.mark.parametrize("nb,b,overlap,scat", [(1, 3, False, False), (2, 3, True, False),
                                               (5, 4, True, True), (7, 2, False, True)])
def test_rgf_blocks_equal_dense(nb, b, overlap, scat):
    if scat:
        dev = W.small_scattering_device(nb, b, 6, seed=7, overlap=overlap, strength=0.05)
    else:
        dev = W.banded_device(nb, b, 6, seed=7, overlap=overlap)
        rng = np.random.default_rng(1)
        if nb > 1:
            dev.H_up = dev.H_up + 0.3 * (rng.normal(size=dev.H_up.shape) + 1j * rng.normal(size=dev.H_up.shape))
    rng = np.random.default_rng(nb)
    for e in range(dev.ne):
        sigma = None
        if nb == 1:   # no inter-block hop to build leads from: random retarded Sigmas
            q = rng.normal(size=(2, b, b)) + 1j * rng.normal(size=(2, b, b))
            sigma = tuple(0.1 * (x + H(x)) - 0.2j * (x @ H(x)) for x in q)
        a = O.solve_energy(dev, e, sigma=sigma)
        r = O.solve_energy(dev, e, use_rgf=True, sigma=(a["sigma_L"], a["sigma_R"]))
        for k in ["GR_diag", "GR_up", "GR_low", "GL_diag", "GL_low"]:
            if a[k].size == 0:
                continue
            scale = np.abs(a[k]).max()
            assert np.abs(a[k] - r[k]).max() <= 1e-10 * scale, k


# --- Eq. (2) invariants -----------------------------------------------------------

def _full_lesser_setup(seed=9):
    dev = W.small_scattering_device(5, 3, 4, seed=seed, overlap=True, strength=0.05)
    e = 2
    z = dev.energy[e] + 1j * dev.eta
    sL, sR, _ = O.lead_self_energies(dev, z)
    fL, fR = dev.f_L()[e], dev.f_R()[e]
    sLs = dev.sigL_scale[e][:, None, None] * dev.sigL_base
    out = O.greens_dense(dev, z, sL, sR, fL, fR, dev.sigR_scat, sLs, keep_dense=True)
    return dev, z, sL, sR, fL, fR, sLs, out


def test_lesser_is_antihermitian():
    dev, z, sL, sR, fL, fR, sLs, out = _full_lesser_setup()
    GL = out["GL"]
    assert np.abs(GL + H(GL)).max() <= 1e-13 * np.abs(GL).max()
    for i in range(dev.nb - 1):
        assert np.abs(out["GL_up"][i] + H(out["GL_low"][i])).max() <= 1e-13 * np.abs(GL).max()


def _sigma_greater_dense(dev, sL, sR, fL, fR, sLs):
    """Sigma^> = Sigma^< + Sigma^R - Sigma^A, block-diagonal."""
    b, nb = dev.b, dev.nb
    N = nb * b
    SR = np.zeros((N, N), complex)
    SR[:b, :b] += sL
    SR[-b:, -b:] += sR
    for i in range(nb):
        SR[i * b:(i + 1) * b, i * b:(i + 1) * b] += dev.sigR_scat[i]
    SLs = O.assemble_sigma_lesser(dev, sL, sR, fL, fR, sLs)
    return SLs + SR - H(SR), SLs


def test_spectral_identity_with_eta_term():
    """i(G^R - G^A) = i(G^> - G^<) + 2 eta G^R S G^A, with G^> = G^R Sigma^> G^A."""
    dev, z, sL, sR, fL, fR, sLs, out = _full_lesser_setup()
    G = out["G"]
    _, S = O.dense_H_S(dev)
    Sg, SLs = _sigma_greater_dense(dev, sL, sR, fL, fR, sLs)
    Gg = G @ Sg @ H(G)
    lhs = 1j * (G - H(G))
    rhs = 1j * (Gg - out["GL"]) + 2 * dev.eta * G @ S @ H(G)
    assert np.abs(lhs - rhs).max() <= 1e-10 * np.abs(lhs).max()
    # without the eta term the identity is off by O(eta ||G||^2) only
    assert np.abs(lhs - 1j * (Gg - out["GL"])).max() <= 1e3 * dev.eta * np.abs(G).max() ** 2


def _continuity_source(dev, i, Sg, SLs, GLd, Ggd, G, S):
    """Right-hand side of the exact block-i continuity equation of Eq. (2):
    J_{i-1} - J_i = Tr[Sigma^> G^< - Sigma^< G^>]_ii
                    + 2i eta Tr[Sigma^<_ii (G S G^A)_ii] - 2i eta Tr[S_ii G^<_ii]
                    + 4 eta Im Tr[S_{i-1,i} G^<_{i,i-1}]."""
    b = dev.b
    s = slice(i * b, (i + 1) * b)
    sm = slice((i - 1) * b, i * b)
    GSGA = G @ S @ H(G)
    src = np.trace(Sg[s, s] @ GLd[s, s] - SLs[s, s] @ Ggd[s, s])
    src += 2j * dev.eta * np.trace(SLs[s, s] @ GSGA[s, s])
    src -= 2j * dev.eta * np.trace(S[s, s] @ GLd[s, s])
    src += 4 * dev.eta * np.imag(np.trace(S[sm, s] @ GLd[s, sm]))
    return src


def test_current_continuity_with_scattering():
    """Current is conserved block by block up to the scattering source and the
    eta sink (exact identity); with random scattering J_i varies along x."""
    dev, z, sL, sR, fL, fR, sLs, out = _full_lesser_setup()
    G = out["G"]
    _, S = O.dense_H_S(dev)
    Sg, SLs = _sigma_greater_dense(dev, sL, sR, fL, fR, sLs)
    Gg = G @ Sg @ H(G)
    J = O.interface_current(dev, z, out["GL_low"])
    scale = np.abs(J).max()
    for i in range(1, dev.nb - 1):
        src = _continuity_source(dev, i, Sg, SLs, out["GL"], Gg, G, S)
        assert abs(src.imag) <= 1e-9 * scale
        assert abs((J[i - 1] - J[i]) - src.real) <= 1e-9 * scale
    assert np.ptp(J) > 1e-4 * scale


def test_ballistic_current_conservation():
    """Ballistic: J_{i-1} - J_i is the eta sink alone (exact), and J_i equals
    T (f_L - f_R) up to O(eta ||G||^2) (the Sec. III conservation check)."""
    dev = W.config1()
    nb, b = dev.nb, dev.b
    _, S = O.dense_H_S(dev)
    for e in [21, 31, 33, 40, 44]:
        z = dev.energy[e] + 1j * dev.eta
        sL, sR, _ = O.lead_self_energies(dev, z)
        fL, fR = dev.f_L()[e], dev.f_R()[e]
        out = O.greens_dense(dev, z, sL, sR, fL, fR, keep_dense=True)
        G = out["G"]
        dev.sigR_scat = np.zeros((nb, b, b), complex)
        Sg, SLs = _sigma_greater_dense(dev, sL, sR, fL, fR, None)
        dev.sigR_scat = None
        Gg = G @ Sg @ H(G)
        J = O.interface_current(dev, z, out["GL_low"])
        scale = max(np.abs(J).max(), 1e-300)
        for i in range(1, nb - 1):
            src = _continuity_source(dev, i, Sg, SLs, out["GL"], Gg, G, S)
            assert abs((J[i - 1] - J[i]) - src.real) <= 1e-9 * scale
        if fL - fR > 0.1:
            Tc = O.transmission_caroli(sL, sR, out["GR_corner"])
            assert np.abs(J - Tc * (fL - fR)).max() <= 1e-3 * Tc * (fL - fR) + 1e-8


def test_transmission_g00_identity():
    """T_g00 - T_caroli = 2 eta Tr[Gamma_L (G S G^H)_00] exactly (ballistic)."""
    dev = W.config1()
    for e in [20, 31, 40, 55]:
        z = dev.energy[e] + 1j * dev.eta
        sL, sR, _ = O.lead_self_energies(dev, z)
        out = O.greens_dense(dev, z, sL, sR, keep_dense=True)
        G = out["G"]
        b = dev.b
        Tc = O.transmission_caroli(sL, sR, out["GR_corner"])
        Tg = O.transmission_g00(sL, out["GR_diag"][0])
        corr = 2 * dev.eta * np.real(np.trace(O.gamma(sL) @ (G @ H(G))[:b, :b]))
        assert abs(Tg - Tc - corr) <= 1e-9 * max(1.0, abs(Tc))


def test_equilibrium_density_is_occupied_spectral_function():
    """f_L = f_R = f:  -i G^< = f [ i(G - G^A) - 2 eta G S G^A ]  (Eq. (2) with
    Sigma^< = i f Gamma), so the density is the occupied spectral weight."""
    dev = W.banded_device(4, 3, 7, seed=4, overlap=True)
    dev.mu_L = dev.mu_R = 0.0
    rng = np.random.default_rng(2)
    dev.H_up = dev.H_up + 0.3 * (rng.normal(size=dev.H_up.shape) + 1j * rng.normal(size=dev.H_up.shape))
    _, S = O.dense_H_S(dev)
    for e in range(dev.ne):
        z = dev.energy[e] + 1j * dev.eta
        sL, sR, _ = O.lead_self_energies(dev, z)
        f = dev.f_L()[e]
        out = O.greens_dense(dev, z, sL, sR, f, f, keep_dense=True)
        G = out["G"]
        ref = f * (1j * (G - H(G)) - 2 * dev.eta * G @ S @ H(G))
        assert np.abs(-1j * out["GL"] - ref).max() <= 1e-10 * max(np.abs(ref).max(), 1e-300) + 1e-14
        # per-orbital density from blocks equals the dense diag(-i G^< S)/2pi
        nE = O.density_energy(dev, out["GL_diag"], out["GL_low"])
        dref = np.real(np.diag(-1j * out["GL"] @ S)) / (2 * np.pi)
        assert np.abs(nE - dref).max() <= 1e-12 * max(np.abs(dref).max(), 1e-300) + 1e-15


# --- input generators -----------------------------------------------------------

def test_generators_hermitian_and_positive_overlap():
    dev = W.config2(nb=4, b=16, ne=4)
    Hd, Sd = O.dense_H_S(dev)
    assert np.abs(Hd - H(Hd)).max() == 0.0
    assert np.linalg.eigvalsh(Sd).min() > 0.5
    c1 = W.config1()
    assert c1.H_diag.shape == (16, 8, 8) and c1.ne == 64
    assert c1.energy[0] == -3.0 and c1.energy[-1] == 3.0
    a, b2 = W.config1(), W.config1()
    assert np.array_equal(a.H_up, b2.H_up)


def test_config4_scattering_signs():
    dev = W.small_scattering_device(3, 6, 5, seed=1)
    for i in range(dev.nb):
        # Im Sigma^R <= 0  <=>  i(Sigma^R - Sigma^A) >= 0
        assert np.linalg.eigvalsh(1j * (dev.sigR_scat[i] - H(dev.sigR_scat[i]))).min() >= -1e-14
        sl = dev.sigL_base[i]
        assert np.abs(sl + H(sl)).max() <= 1e-15     # Sigma^< anti-Hermitian


# ---------------------------------------------------------------------------
# G^> (the greater Green's function of the G^> output)
# ---------------------------------------------------------------------------

def test_greater_fluctuation_dissipation_in_equilibrium():
    """Ballistic device, both leads at the same chemical potential: G^< = i f G (Gamma_L +
    Gamma_R) G^A and G^> = -i (1 - f) G (Gamma_L + Gamma_R) G^A, so that
    G^> = -((1 - f) / f) G^< exactly, block by block.  A wrong sign or a dropped (1 - f)
    in Sigma^> fails it."""
    dev = W.config1()
    dev.mu_R = dev.mu_L
    f = dev.f_L()
    picked = [e for e in range(dev.ne) if 0.05 < f[e] < 0.95]
    if not picked:   # widen kT until some energies sit inside the Fermi window
        dev.kT = 0.5
        f = dev.f_L()
        picked = [e for e in range(dev.ne) if 0.05 < f[e] < 0.95]
    assert picked
    for e in picked[:4]:
        out = O.solve_energy(dev, e, greater=True)
        r = -(1.0 - f[e]) / f[e]
        for kg, kl in (("GG_diag", "GL_diag"), ("GG_low", "GL_low")):
            scale = np.abs(out[kg]).max()
            assert scale > 0
            assert np.abs(out[kg] - r * out[kl]).max() <= 1e-11 * scale, (e, kg)


def test_greater_is_antihermitian_and_matches_spectral_identity():
    """G^> = -(G^>)^H, and G^> - G^< = G^R (Sigma^R - Sigma^A) G^A = G^R - G^A + 2 i eta
    G^R S G^A on every selected block (G^R - G^A also carries the eta broadening)."""
    dev, z, sL, sR, fL, fR, sLs, out0 = _full_lesser_setup()
    out = O.greens_dense(dev, z, sL, sR, fL, fR, dev.sigR_scat, sLs, keep_dense=True, greater=True)
    GG, GL, G = out["GG"], out["GL"], out["G"]
    assert np.abs(GG + H(GG)).max() <= 1e-13 * np.abs(GG).max()
    _, S = O.dense_H_S(dev)
    rhs = G - H(G) + 2j * dev.eta * G @ S @ H(G)
    b, nb = dev.b, dev.nb
    for i in range(nb):
        s = slice(i * b, (i + 1) * b)
        d = out["GG_diag"][i] - out["GL_diag"][i] - rhs[s, s]
        assert np.abs(d).max() <= 1e-10 * np.abs(rhs).max()
    for i in range(nb - 1):
        s1, s0 = slice((i + 1) * b, (i + 2) * b), slice(i * b, (i + 1) * b)
        d = out["GG_low"][i] - out["GL_low"][i] - rhs[s1, s0]
        assert np.abs(d).max() <= 1e-10 * np.abs(rhs).max()


def test_greater_block_recursion_matches_dense():
    """The block recursion's G^> (the lesser sweeps run on Sigma^>) equals the dense
    G^R Sigma^> G^A, with scattering and S != I.  Errors are measured against the
    spectral function's scale max|G^R - G^A|, which bounds both G^< and G^> (far above
    the chemical potentials G^> is many decades smaller)."""
    dev = W.small_scattering_device(5, 6, 6, seed=31)
    for e in range(dev.ne):
        d = O.solve_energy(dev, e, greater=True)
        r = O.solve_energy(dev, e, greater=True, use_rgf=True, sigma=(d["sigma_L"], d["sigma_R"]))
        scale = np.abs(d["GR_diag"] - H(d["GR_diag"])).max()
        for k in ("GG_diag", "GG_low", "GL_diag", "GL_low"):
            assert np.abs(r[k] - d[k]).max() <= 1e-11 * scale, (e, k)


# ---------------------------------------------------------------------------
# partitioned selected inversion (Fig. 3)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("nb,P", [(4, 2), (6, 3), (8, 4), (8, 2), (9, 3), (6, 1)])
def test_partitioned_retarded_matches_dense_inverse(nb, P):
    """Partitioned elimination + reduced system + reconstruction gives the selected
    blocks of the dense inverse (with scattering, S != I, and leads)."""
    dev = W.small_scattering_device(nb, 5, 3, seed=60 + nb + P, overlap=True, strength=0.05)
    for e in range(dev.ne):
        z = dev.energy[e] + 1j * dev.eta
        sL, sR, _ = O.lead_self_energies(dev, z)
        d = O.greens_dense(dev, z, sL, sR, sigR_scat=dev.sigR_scat)
        r = O.partitioned_retarded(dev, z, sL, sR, P, sigR_scat=dev.sigR_scat)
        scale = np.abs(d["GR_diag"]).max()
        for k in ("GR_diag", "GR_up", "GR_low"):
            assert np.abs(r[k] - d[k]).max() <= 1e-11 * scale, (k, e)


def test_partitioned_retarded_one_partition_is_the_block_recursion():
    dev = W.small_scattering_device(5, 4, 2, seed=71)
    z = dev.energy[1] + 1j * dev.eta
    sL, sR, _ = O.lead_self_energies(dev, z)
    a = O.partitioned_retarded(dev, z, sL, sR, 1, sigR_scat=dev.sigR_scat)
    b = O.rgf_blocks(dev, z, sL, sR, sigR_scat=dev.sigR_scat)
    for k in ("GR_diag", "GR_up", "GR_low"):
        assert np.abs(a[k] - b[k]).max() <= 1e-12 * np.abs(b[k]).max()


def test_partitioned_retarded_rejects_uneven_partitions():
    dev = W.small_scattering_device(5, 4, 1, seed=72)
    z = dev.energy[0] + 1j * dev.eta
    with pytest.raises(ValueError):
        O.partitioned_retarded(dev, z, np.zeros((4, 4)), np.zeros((4, 4)), 2)
    with pytest.raises(ValueError):
        O.partitioned_retarded(dev.truncated(nb=4), z, np.zeros((4, 4)), np.zeros((4, 4)), 4)


# ---------------------------------------------------------------------------
# Eq. (3) energy convolution and the self-consistent scattering loop (Fig. 2)
# ---------------------------------------------------------------------------

def test_energy_convolution_is_a_shift_for_a_delta_kernel():
    rng = np.random.default_rng(5)
    X = rng.normal(size=(40, 3, 2)) + 1j * rng.normal(size=(40, 3, 2))
    for M, k in ((3, 2), (3, -3), (5, 0)):
        w = np.zeros(2 * M + 1)
        w[k + M] = 1.5
        Y = O.energy_convolution(X, w)
        for n in range(40):
            ref = 1.5 * X[n - k] if 0 <= n - k < 40 else 0.0
            assert np.all(Y[n] == ref), (M, k, n)


def test_energy_convolution_matches_numpy_convolve_on_scalars():
    rng = np.random.default_rng(6)
    x = rng.normal(size=57) + 1j * rng.normal(size=57)
    w = rng.uniform(0, 1, size=9)
    full = np.convolve(x, w)            # full[i] = sum_j w[j] x[i - j]
    y = O.energy_convolution(x[:, None], w)[:, 0]
    assert np.abs(y - full[4:4 + 57]).max() <= 1e-13 * np.abs(full).max()


def _scba_setup(eta=None, g2=0.05):
    dev = W.scba_device(6, 8, 128)
    if eta is not None:
        dev.eta = eta
    wl, wg = W.einstein_kernel(dev.energy, 4, g2, dev.kT)
    return dev, wl, wg


def test_scba_without_coupling_is_the_ballistic_solution():
    dev, wl, wg = _scba_setup(g2=0.0)
    dev = dev.truncated(energies=np.arange(0, 128, 16))
    r = O.scba_loop(dev, wl, wg)
    assert r["iters"] == 1 and np.all(r["sigL"] == 0)
    for e in range(dev.ne):
        ref = O.solve_energy(dev, e, use_rgf=True)
        assert np.abs(r["out"][e]["GL_diag"] - ref["GL_diag"]).max() <= 1e-13 * np.abs(ref["GL_diag"]).max()


def test_scba_converges_to_a_fixed_point_that_conserves_the_integrated_current():
    """At the fixed point the scattering only moves electrons between energies: the
    energy-resolved current J_i(E) changes along the device, the energy-integrated one
    does not (the scattering sources cancel over the grid because w^>_m = w^<_-m).  The
    broadening eta is an additional sink of 2 eta x (electrons per block), so the
    check runs at eta = 1e-10."""
    dev, wl, wg = _scba_setup(eta=1e-10)
    r = O.scba_loop(dev, wl, wg, mixing=0.5, tol=1e-9, max_iter=80)
    assert r["change"] < 1e-9
    # fixed point: the self-energies of the final Green's functions are the mixed ones
    GLd = np.stack([o["GL_diag"] for o in r["out"]])
    GGd = np.stack([o["GG_diag"] for o in r["out"]])
    SR, SL, SG = O.scba_self_energies(GLd, GGd, wl, wg)
    scale = np.abs(SG).max()
    assert np.abs(SL - r["sigL"]).max() <= 1e-8 * scale
    assert np.abs(SG - r["sigG"]).max() <= 1e-8 * scale
    assert np.abs(SR + H(SR)).max() <= 1e-10 * scale        # anti-Hermitian Sigma^R (to rounding)
    J = np.stack([O.interface_current(dev, dev.energy[e] + 1j * dev.eta, r["out"][e]["GL_low"])
                  for e in range(dev.ne)])
    Jint = J.sum(axis=0)
    assert np.ptp(Jint) <= 1e-6 * np.abs(Jint).max()
    assert np.abs(np.ptp(J, axis=1)).max() >= 1e-2 * np.abs(J).max()


# ---------------------------------------------------------------------------
# arrowhead BT (a gate block coupled to every block)
# ---------------------------------------------------------------------------

def test_arrowhead_without_coupling_is_the_bt_result_and_a_free_tip():
    dev = W.small_scattering_device(4, 6, 2, seed=80)
    H_tip, H_arrow = W.arrowhead_gate(dev)
    z = dev.energy[1] + 1j * dev.eta
    sL, sR, _ = O.lead_self_energies(dev, z)
    r = O.arrowhead_dense(dev, z, sL, sR, H_tip, 0.0 * H_arrow, sigR_scat=dev.sigR_scat)
    d = O.greens_dense(dev, z, sL, sR, sigR_scat=dev.sigR_scat)
    for k in ("GR_diag", "GR_up", "GR_low"):
        assert np.abs(r[k] - d[k]).max() <= 1e-12 * np.abs(d[k]).max()
    tip = np.linalg.inv(z * np.eye(dev.b) - H_tip)
    assert np.abs(r["G_tip"] - tip).max() <= 1e-12 * np.abs(tip).max()
    assert np.abs(r["G_row"]).max() == 0 and np.abs(r["G_col"]).max() == 0


def test_arrowhead_schur_complement_of_the_tip():
    """With the tip eliminated, the device block of the inverse is the inverse of the
    device matrix minus the tip's Schur-complement term A_(.,t) A_tt^{-1} A_(t,.), a dense
    correction to every block pair: checked on the diagonal blocks and the corner block."""
    dev = W.small_scattering_device(5, 4, 1, seed=81)
    H_tip, H_arrow = W.arrowhead_gate(dev, coupling=0.3)
    z = dev.energy[0] + 1j * dev.eta
    sL, sR, _ = O.lead_self_energies(dev, z)
    r = O.arrowhead_dense(dev, z, sL, sR, H_tip, H_arrow, sigR_scat=dev.sigR_scat)
    A = O.assemble_A(dev, z, sL, sR, dev.sigR_scat)
    b, nb = dev.b, dev.nb
    col = np.concatenate([-H(H_arrow[i]) for i in range(nb)], axis=0)      # A_(.,t)
    row = np.concatenate([-H_arrow[i] for i in range(nb)], axis=1)         # A_(t,.)
    Att = z * np.eye(b) - H_tip
    G = np.linalg.inv(A - col @ np.linalg.solve(Att, row))
    for i in range(nb):
        blk = G[i * b:(i + 1) * b, i * b:(i + 1) * b]
        assert np.abs(r["GR_diag"][i] - blk).max() <= 1e-11 * np.abs(blk).max()
    # and the tip block is the inverse of the tip's own Schur complement, the arrow row
    # G_(t,.) = -S_t^{-1} A_(t,.) A^{-1} and the column G_(.,t) = -A^{-1} A_(.,t) S_t^{-1}
    Gt = np.linalg.inv(Att - row @ np.linalg.solve(A, col))
    assert np.abs(r["G_tip"] - Gt).max() <= 1e-11 * np.abs(Gt).max()
    Grow = -Gt @ row @ np.linalg.inv(A)
    Gcol = -np.linalg.solve(A, col) @ Gt
    for i in range(nb):
        s_i = slice(i * b, (i + 1) * b)
        assert np.abs(r["G_row"][i] - Grow[:, s_i]).max() <= 1e-11 * np.abs(Grow).max()
        assert np.abs(r["G_col"][i] - Gcol[s_i, :]).max() <= 1e-11 * np.abs(Gcol).max()
