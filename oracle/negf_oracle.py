"""CPU oracle for the batched RGF selected inversion.  TEST INFRASTRUCTURE ONLY.

Only the tests, the smoke check and the CPU-baseline leg of the benchmark may
import this module; the library path never does.  It shares no code with the
CUDA path: everything here is plain numpy complex128, written from the
paper's statement of the problem:

  * Eq. (1):  C^R = (A - B^R)^{-1}.  For electrons
              G^R(E) = (z S - H - Sigma^R_OBC - Sigma^R_scat)^{-1}, z = E + i eta.
  * Eq. (2):  (C^R)^{-1} C^< (C^R)^{-H} = B^<,  i.e.  G^< = G^R Sigma^< G^A;
              the same relation with B^> gives G^> = G^R Sigma^> G^A.
  * Sec. II:  A and B are block-tridiagonal; only the entries of C on that
              pattern (diagonal and first off-diagonal blocks) are wanted, and
              every energy is independent.

The primary functions are the plain definitions (dense inversion of the full
N x N matrix, then the block extraction).  ``rgf_blocks`` is the textbook
recursive Green's function (the RGF the paper cites in Sec. II) as a plain
block loop; it exists to reach sizes the dense inverse cannot, and is pinned
to the dense definition by the tests.

The open-boundary term (Sec. II: "an open boundary condition term not shown
here") is not written out in the paper.  It is computed here by the
Lopez Sancho - Lopez Sancho - Rubio decimation (J. Phys. F 15, 851 (1985)),
written in A-form; pinned by the closed-form 1D-chain surface function and a
long finite chain.  Parity: all functions below are pinned (see the oracle
tests).
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "dense_matrix", "dense_H_S", "lead_A_blocks", "sancho_rubio", "surface_residual",
    "lead_self_energies", "lead_lesser", "lead_greater", "scattering_greater", "gamma", "assemble_A",
    "assemble_sigma_lesser", "assemble_sigma_greater",
    "greens_dense", "rgf_blocks", "transmission_caroli", "transmission_g00", "dos",
    "interface_current", "density", "solve_energy", "retarded_check", "surface_newton_warm",
    "warm_surface_gf", "stein_smith", "surface_newton", "surface_gf", "partitioned_retarded",
    "energy_convolution", "scba_self_energies", "scba_loop", "arrowhead_dense",
]


def _H(x):
    """Conjugate transpose of the last two axes."""
    return np.conj(np.swapaxes(x, -1, -2))


# ---------------------------------------------------------------------------
# block-tridiagonal bookkeeping (Sec. II: BT shape of A and B)
# ---------------------------------------------------------------------------

def dense_matrix(diag, up, low=None):
    """Dense N x N matrix from BT blocks; lower blocks default to up^H."""
    nb, b = diag.shape[0], diag.shape[1]
    M = np.zeros((nb * b, nb * b), dtype=np.complex128)
    for i in range(nb):
        M[i * b:(i + 1) * b, i * b:(i + 1) * b] = diag[i]
    for i in range(nb - 1):
        M[i * b:(i + 1) * b, (i + 1) * b:(i + 2) * b] = up[i]
        M[(i + 1) * b:(i + 2) * b, i * b:(i + 1) * b] = _H(up[i]) if low is None else low[i]
    return M


def dense_H_S(dev):
    """Dense Hamiltonian and overlap (S = I when the device has none)."""
    H = dense_matrix(dev.H_diag, dev.H_up)
    if dev.S_diag is None:
        S = np.eye(H.shape[0], dtype=np.complex128)
    else:
        S = dense_matrix(dev.S_diag, dev.S_up)
    return H, S


def _blk(M, i, j, b):
    return M[i * b:(i + 1) * b, j * b:(j + 1) * b]


# ---------------------------------------------------------------------------
# open boundary conditions (Sec. II "LSE+OBC"; decimation of Lopez Sancho et al.)
# ---------------------------------------------------------------------------

def lead_A_blocks(dev, side, z):
    """A-form blocks of a semi-infinite lead, A = z S - H.

    The left lead repeats block 0 with cell-to-cell hop H_{0,1}; the right lead
    repeats block nb-1 with hop H_{nb-2,nb-1}.  Returns (a00, a01, a10) with
    a01 the coupling from a cell to the next cell on its right and a10 the
    coupling back: a01 = z S01 - H01, a10 = z S01^H - H01^H."""
    b = dev.b
    if side == "L":
        H00, H01 = dev.H_diag[0], dev.H_up[0]
        S00 = np.eye(b) if dev.S_diag is None else dev.S_diag[0]
        S01 = np.zeros((b, b)) if dev.S_up is None else dev.S_up[0]
    else:
        H00, H01 = dev.H_diag[-1], dev.H_up[-1]
        S00 = np.eye(b) if dev.S_diag is None else dev.S_diag[-1]
        S01 = np.zeros((b, b)) if dev.S_up is None else dev.S_up[-1]
    a00 = z * S00 - H00
    a01 = z * S01 - H01
    a10 = z * _H(S01) - _H(H01)
    return a00, a01, a10


def sancho_rubio(a00, alpha, beta, tol=1e-12, max_iter=100):
    """Surface Green's function of a semi-infinite chain by decimation.

    The chain has onsite A-block ``a00`` on every cell, coupling ``alpha`` from
    a cell to the next one away from the surface and ``beta`` back.  Each step
    eliminates every other cell (a Schur complement), doubling the reach of the
    effective couplings:
        g = eps^{-1};  eps_s -= alpha g beta;  eps -= alpha g beta + beta g alpha;
        alpha <- -alpha g alpha;  beta <- -beta g beta,
    until max|alpha|, max|beta| fall below ``tol`` times their initial size.
    Returns (g_surface = eps_s^{-1}, iterations, converged)."""
    eps = a00.copy()
    eps_s = a00.copy()
    al = alpha.copy()
    be = beta.copy()
    ref = max(np.abs(alpha).max(), np.abs(beta).max(), 1e-300)
    it = 0
    converged = False
    while it < max_iter:
        if max(np.abs(al).max(), np.abs(be).max()) < tol * ref:
            converged = True
            break
        g = np.linalg.inv(eps)
        agb = al @ g @ be
        bga = be @ g @ al
        eps_s = eps_s - agb
        eps = eps - agb - bga
        al = -(al @ g @ al)
        be = -(be @ g @ be)
        it += 1
    if not converged and max(np.abs(al).max(), np.abs(be).max()) < tol * ref:
        converged = True
    return np.linalg.inv(eps_s), it, converged


def surface_residual(a00, alpha, beta, g):
    """|| (a00 - alpha g beta) g - I ||_F / sqrt(b): how far g is from the
    fixed point g = (a00 - alpha g beta)^{-1} of the semi-infinite chain."""
    b = a00.shape[0]
    R = (a00 - alpha @ g @ beta) @ g - np.eye(b)
    return np.linalg.norm(R) / np.sqrt(b)


def stein_smith(P, Q, C, tol=1e-15, max_iter=200):
    """Solve D = C + P D Q by Smith's doubling: D = sum_k P^k C Q^k, summed
    as S <- S + P_j S Q_j, P_{j+1} = P_j^2, Q_{j+1} = Q_j^2."""
    S = C.copy()
    Pj = P.copy()
    Qj = Q.copy()
    for _ in range(max_iter):
        inc = Pj @ S @ Qj
        S = S + inc
        if np.abs(inc).max() <= tol * max(np.abs(S).max(), 1e-300):
            break
        Pj = Pj @ Pj
        Qj = Qj @ Qj
        # only the products P_j (.) Q_j matter: keep the two factors balanced so
        # that neither overflows while the other underflows (rho(P) rho(Q) ~ 1)
        p, q = np.abs(Pj).max(), np.abs(Qj).max()
        if p > 0 and q > 0:
            s = np.sqrt(q / p)
            Pj *= s
            Qj /= s
    return S


def surface_newton(a00, alpha, beta, g, target=1e-13, max_steps=3):
    """Newton steps on F(X) = (a00 - alpha X beta) X - I = 0 starting at ``g``.

    With K = a00 - alpha X beta the step D solves K D - alpha D beta X = -F,
    i.e. the Stein equation D = -K^{-1} F + (K^{-1} alpha) D (beta X).
    Returns (X, steps taken, final residual)."""
    X = g
    res = surface_residual(a00, alpha, beta, X)
    steps = 0
    b = a00.shape[0]
    while res > target and steps < max_steps:
        K = a00 - alpha @ X @ beta
        F = K @ X - np.eye(b)
        Kinv = np.linalg.inv(K)
        D = stein_smith(Kinv @ alpha, beta @ X, -(Kinv @ F))
        Xn = X + D
        rn = surface_residual(a00, alpha, beta, Xn)
        steps += 1
        if not rn < res:
            break
        X, res = Xn, rn
    return X, steps, res


def surface_gf(a00, alpha, beta, tol=1e-12, max_iter=100, target=1e-13, newton_steps=3):
    """Surface Green's function: decimation, then Newton polishing of the
    fixed-point equation when rounding in the decimation (ill-conditioned
    intermediate eps near band edges at small eta) left a residual above
    ``target``.  Returns (g, decimation iterations, newton steps, residual, converged)."""
    g, it, ok = sancho_rubio(a00, alpha, beta, tol, max_iter)
    g, ns, res = surface_newton(a00, alpha, beta, g, target, newton_steps)
    return g, it, ns, res, ok


def retarded_check(g, tol=1e-12):
    """Is ``g`` the retarded (decaying) root of the surface equation?

    For a lead with S = I, every root of g = (a00 - alpha g beta)^{-1} satisfies the
    Stein equation  A = 2 eta g g^H + (g H01) A (g H01)^H  for A = i (g - g^H), whose
    constant term is positive definite for eta > 0.  By the inertia theorem for Stein
    equations, A is then positive definite exactly when rho(g H01) < 1, i.e. when g is
    built from the decaying (retarded) modes; the other roots solve the same quadratic
    equation to the same residual but leave A indefinite.  The test is the LDL^H
    factorisation of A without pivoting (Sylvester's criterion): every pivot must
    exceed -tol * max_k A_kk; a pivot within +-tol of zero is taken as a semidefinite
    direction and its column skipped."""
    A = 1j * (g - g.conj().T)
    A = 0.5 * (A + A.conj().T)
    n = A.shape[0]
    scale = max(float(np.max(A.real.diagonal())), 1e-300)
    W = A.copy()
    for k in range(n):
        d = W[k, k].real
        if d < -tol * scale or not np.isfinite(d):
            return False
        if d <= tol * scale:
            continue
        l = W[k + 1:, k] / d
        W[k + 1:, k + 1:] -= np.outer(l, W[k, k + 1:])
    return True


def surface_newton_warm(a00, alpha, beta, g0, target=1e-13, max_steps=8, smith_levels=96):
    """Guess-driven surface solver: plain Newton steps on F(X) = (a00 - alpha X beta) X - I
    from the initial guess ``g0`` (every finite step is taken; the Stein equation of each
    step is summed by Smith doubling with at most ``smith_levels`` levels).
    Returns (X, steps, residual); the residual is inf when a step did not stay finite."""
    b = a00.shape[0]
    X = g0
    res = surface_residual(a00, alpha, beta, X)
    steps = 0
    while res > target and steps < max_steps:
        K = a00 - alpha @ X @ beta
        F = K @ X - np.eye(b)
        Kinv = np.linalg.inv(K)
        with np.errstate(all="ignore"):
            D = stein_smith(Kinv @ alpha, beta @ X, -(Kinv @ F), max_iter=smith_levels)
            X = X + D
            res = surface_residual(a00, alpha, beta, X)
        steps += 1
        if not np.isfinite(res):
            return X, steps, np.inf
    return X, steps, res


def warm_surface_gf(a00, alpha, beta, g0, accept=1e-10, tol=1e-12, max_iter=100, target=1e-13,
                    warm_steps=8):
    """Surface function from a warm start, with the decimation as fallback and arbiter:
    Newton from ``g0``; the result is taken when its residual is <= ``accept`` and it
    passes ``retarded_check``; otherwise the plain decimation + polishing runs.
    Returns (g, decimation iterations, newton steps, residual, warm_taken)."""
    X, steps, res = surface_newton_warm(a00, alpha, beta, g0, target, warm_steps)
    if res <= accept and retarded_check(X):
        return X, 0, steps, res, True
    g, it, ns, r, ok = surface_gf(a00, alpha, beta, tol, max_iter, target)
    return g, it, ns, r, False


def lead_self_energies(dev, z, tol=1e-12, max_iter=100, newton_steps=3):
    """Retarded lead self-energies on blocks 0 and nb-1.

    Right lead (cells nb, nb+1, ...): surface g_R from (a00, a01, a10) and
    Sigma_R = a01 g_R a10.  Left lead (cells -1, -2, ...): couplings swapped,
    Sigma_L = a10 g_L a01.  Returns (Sigma_L, Sigma_R, info)."""
    a00, a01, a10 = lead_A_blocks(dev, "L", z)
    gL, itL, nL, resL, okL = surface_gf(a00, a10, a01, tol, max_iter, newton_steps=newton_steps)
    sL = a10 @ gL @ a01
    a00, a01, a10 = lead_A_blocks(dev, "R", z)
    gR, itR, nR, resR, okR = surface_gf(a00, a01, a10, tol, max_iter, newton_steps=newton_steps)
    sR = a01 @ gR @ a10
    info = dict(iters=(itL, itR), newton=(nL, nR), converged=(okL, okR),
                residual=(resL, resR), g=(gL, gR))
    return sL, sR, info


def gamma(sigma):
    """Broadening Gamma = i (Sigma^R - Sigma^A)."""
    return 1j * (sigma - _H(sigma))


def lead_lesser(sigma, f):
    """Lead lesser self-energy Sigma^< = i f Gamma."""
    return 1j * f * gamma(sigma)


def lead_greater(sigma, f):
    """Lead greater self-energy Sigma^> = -i (1 - f) Gamma (holes injected by the lead)."""
    return -1j * (1.0 - f) * gamma(sigma)


def scattering_greater(sigR_scat_i, sigL_scat_i):
    """Sigma^>_scat = Sigma^<_scat + Sigma^R_scat - Sigma^A_scat: the retarded
    self-energy's anti-Hermitian part is Sigma^> - Sigma^< for any self-energy
    of the Keldysh form."""
    out = np.zeros_like(sigR_scat_i if sigR_scat_i is not None else sigL_scat_i, dtype=np.complex128)
    if sigL_scat_i is not None:
        out = out + sigL_scat_i
    if sigR_scat_i is not None:
        out = out + sigR_scat_i - _H(sigR_scat_i)
    return out


# ---------------------------------------------------------------------------
# Eq. (1) and Eq. (2) by dense inversion
# ---------------------------------------------------------------------------

def assemble_A(dev, z, sigma_L, sigma_R, sigR_scat=None):
    """Dense A(z) = z S - H - Sigma^R_OBC - Sigma^R_scat (Eq. (1) operand)."""
    H, S = dense_H_S(dev)
    b, nb = dev.b, dev.nb
    A = z * S - H
    _blk(A, 0, 0, b)[...] -= sigma_L
    _blk(A, nb - 1, nb - 1, b)[...] -= sigma_R
    if sigR_scat is not None:
        for i in range(nb):
            _blk(A, i, i, b)[...] -= sigR_scat[i]
    return A


def assemble_sigma_lesser(dev, sigma_L, sigma_R, fL, fR, sigL_scat=None):
    """Dense block-diagonal Sigma^< = Sigma^<_scat + i f_L Gamma_L (block 0)
    + i f_R Gamma_R (block nb-1)  (the B^< of Eq. (2))."""
    b, nb = dev.b, dev.nb
    N = nb * b
    SL = np.zeros((N, N), dtype=np.complex128)
    _blk(SL, 0, 0, b)[...] += lead_lesser(sigma_L, fL)
    _blk(SL, nb - 1, nb - 1, b)[...] += lead_lesser(sigma_R, fR)
    if sigL_scat is not None:
        for i in range(nb):
            _blk(SL, i, i, b)[...] += sigL_scat[i]
    return SL


def assemble_sigma_greater(dev, sigma_L, sigma_R, fL, fR, sigR_scat=None, sigL_scat=None):
    """Dense block-diagonal Sigma^> = Sigma^>_scat - i (1 - f_L) Gamma_L (block 0)
    - i (1 - f_R) Gamma_R (block nb-1), the B^> that gives C^> = C^R B^> C^A in the
    same way as Eq. (2) gives C^<."""
    b, nb = dev.b, dev.nb
    N = nb * b
    SG = np.zeros((N, N), dtype=np.complex128)
    _blk(SG, 0, 0, b)[...] += lead_greater(sigma_L, fL)
    _blk(SG, nb - 1, nb - 1, b)[...] += lead_greater(sigma_R, fR)
    if sigR_scat is not None or sigL_scat is not None:
        for i in range(nb):
            _blk(SG, i, i, b)[...] += scattering_greater(None if sigR_scat is None else sigR_scat[i],
                                                         None if sigL_scat is None else sigL_scat[i])
    return SG


def greens_dense(dev, z, sigma_L, sigma_R, fL=None, fR=None, sigR_scat=None, sigL_scat=None,
                 keep_dense=False, greater=False):
    """Selected blocks of G^R (Eq. (1)) and, when occupations are given, of
    G^< = G^R Sigma^< G^A (Eq. (2)), by inverting the full matrix; with
    `greater`, also G^> = G^R Sigma^> G^A.

    Returns a dict with GR_diag [nb], GR_up [nb-1] (block (i,i+1)),
    GR_low [nb-1] (block (i+1,i)), GL_diag, GL_low likewise, and GG_diag, GG_low."""
    b, nb = dev.b, dev.nb
    A = assemble_A(dev, z, sigma_L, sigma_R, sigR_scat)
    G = np.linalg.inv(A)
    out = dict(
        GR_diag=np.stack([_blk(G, i, i, b) for i in range(nb)]),
        GR_up=np.stack([_blk(G, i, i + 1, b) for i in range(nb - 1)]) if nb > 1 else np.zeros((0, b, b), complex),
        GR_low=np.stack([_blk(G, i + 1, i, b) for i in range(nb - 1)]) if nb > 1 else np.zeros((0, b, b), complex),
        GR_corner=_blk(G, 0, nb - 1, b).copy(),
    )
    if fL is not None:
        SL = assemble_sigma_lesser(dev, sigma_L, sigma_R, fL, fR, sigL_scat)
        GL = G @ SL @ _H(G)
        out["GL_diag"] = np.stack([_blk(GL, i, i, b) for i in range(nb)])
        out["GL_low"] = (np.stack([_blk(GL, i + 1, i, b) for i in range(nb - 1)])
                         if nb > 1 else np.zeros((0, b, b), complex))
        out["GL_up"] = (np.stack([_blk(GL, i, i + 1, b) for i in range(nb - 1)])
                        if nb > 1 else np.zeros((0, b, b), complex))
        if keep_dense:
            out["GL"] = GL
            out["SigmaL"] = SL
        if greater:
            SG = assemble_sigma_greater(dev, sigma_L, sigma_R, fL, fR, sigR_scat, sigL_scat)
            GG = G @ SG @ _H(G)
            out["GG_diag"] = np.stack([_blk(GG, i, i, b) for i in range(nb)])
            out["GG_low"] = (np.stack([_blk(GG, i + 1, i, b) for i in range(nb - 1)])
                             if nb > 1 else np.zeros((0, b, b), complex))
            if keep_dense:
                out["GG"] = GG
                out["SigmaG"] = SG
    if keep_dense:
        out["G"] = G
        out["A"] = A
    return out


# ---------------------------------------------------------------------------
# textbook RGF (the recursion the paper cites in Sec. II), plain block loop
# ---------------------------------------------------------------------------

def _A_blocks(dev, z, sigma_L, sigma_R, sigR_scat=None):
    nb, b = dev.nb, dev.b
    S_d = [np.eye(b)] * nb if dev.S_diag is None else list(dev.S_diag)
    S_u = [np.zeros((b, b))] * (nb - 1) if dev.S_up is None else list(dev.S_up)
    Ad = [z * S_d[i] - dev.H_diag[i] for i in range(nb)]
    Ad[0] = Ad[0] - sigma_L
    Ad[nb - 1] = Ad[nb - 1] - sigma_R
    if sigR_scat is not None:
        Ad = [Ad[i] - sigR_scat[i] for i in range(nb)]
    Au = [z * S_u[i] - dev.H_up[i] for i in range(nb - 1)]           # A_{i,i+1}
    Al = [z * _H(S_u[i]) - _H(dev.H_up[i]) for i in range(nb - 1)]   # A_{i+1,i}
    return Ad, Au, Al


def _keldysh_sweep(g, GR_d, GR_u, Au, Al, Sig):
    """Forward and backward sweeps of C^x = C^R Sigma^x C^A for one block-diagonal
    Sigma^x (x = <, or >: the recursion is linear in Sigma^x).  Returns the diagonal
    and lower blocks."""
    nb = len(g)
    gl = [None] * nb
    gl[0] = g[0] @ Sig[0] @ _H(g[0])
    for i in range(1, nb):
        gl[i] = g[i] @ (Sig[i] + Al[i - 1] @ gl[i - 1] @ _H(Al[i - 1])) @ _H(g[i])
    Gd = [None] * nb
    Gl = [None] * (nb - 1)
    Gd[nb - 1] = gl[nb - 1]
    for i in range(nb - 2, -1, -1):
        X = g[i] @ Au[i]
        Z = Al[i] @ gl[i]
        P = Gd[i + 1] @ _H(X)
        W = GR_u[i] @ Z
        Gd[i] = gl[i] + X @ P - W + _H(W)
        Gl[i] = -GR_d[i + 1] @ Z - P
    return Gd, Gl


def rgf_blocks(dev, z, sigma_L, sigma_R, fL=None, fR=None, sigR_scat=None, sigL_scat=None, greater=False):
    """Selected blocks of G^R and G^< (and, with `greater`, G^>) by the
    forward/backward block recursion.

    Forward:  g_0 = A_00^{-1},  g_i = (A_ii - A_{i,i-1} g_{i-1} A_{i-1,i})^{-1};
              g^<_i = g_i (Sigma^<_ii + A_{i,i-1} g^<_{i-1} A_{i,i-1}^H) g_i^H.
    Backward: G_{nb-1} = g_{nb-1};  with X = g_i A_{i,i+1}, Y = A_{i+1,i} g_i:
              G_{i,i+1} = -X G_{i+1,i+1},  G_{i+1,i} = -G_{i+1,i+1} Y,
              G_ii = g_i - G_{i,i+1} Y;
              with Z = A_{i+1,i} g^<_i, P = G^<_{i+1,i+1} X^H:
              G^<_ii = g^<_i + X P - G_{i,i+1} Z + (G_{i,i+1} Z)^H,
              G^<_{i+1,i} = -G_{i+1,i+1} Z - P.
    G^> runs the same lesser recursion with Sigma^> in place of Sigma^<."""
    nb = dev.nb
    Ad, Au, Al = _A_blocks(dev, z, sigma_L, sigma_R, sigR_scat)
    inv = np.linalg.inv
    g = [None] * nb
    g[0] = inv(Ad[0])
    for i in range(1, nb):
        g[i] = inv(Ad[i] - Al[i - 1] @ g[i - 1] @ Au[i - 1])
    GR_d = [None] * nb
    GR_u = [None] * (nb - 1)
    GR_l = [None] * (nb - 1)
    GR_d[nb - 1] = g[nb - 1]
    for i in range(nb - 2, -1, -1):
        X = g[i] @ Au[i]
        Y = Al[i] @ g[i]
        GR_u[i] = -X @ GR_d[i + 1]
        GR_l[i] = -GR_d[i + 1] @ Y
        GR_d[i] = g[i] - GR_u[i] @ Y
    out = dict(GR_diag=np.stack(GR_d))
    b = dev.b
    out["GR_up"] = np.stack(GR_u) if nb > 1 else np.zeros((0, b, b), complex)
    out["GR_low"] = np.stack(GR_l) if nb > 1 else np.zeros((0, b, b), complex)
    if fL is None:
        return out
    SigL = [np.zeros((b, b), complex) for _ in range(nb)]
    SigL[0] = SigL[0] + lead_lesser(sigma_L, fL)
    SigL[nb - 1] = SigL[nb - 1] + lead_lesser(sigma_R, fR)
    if sigL_scat is not None:
        SigL = [SigL[i] + sigL_scat[i] for i in range(nb)]
    GL_d, GL_l = _keldysh_sweep(g, GR_d, GR_u, Au, Al, SigL)
    out["GL_diag"] = np.stack(GL_d)
    out["GL_low"] = np.stack(GL_l) if nb > 1 else np.zeros((0, b, b), complex)
    if greater:
        SigG = [np.zeros((b, b), complex) for _ in range(nb)]
        SigG[0] = SigG[0] + lead_greater(sigma_L, fL)
        SigG[nb - 1] = SigG[nb - 1] + lead_greater(sigma_R, fR)
        if sigR_scat is not None or sigL_scat is not None:
            SigG = [SigG[i] + scattering_greater(None if sigR_scat is None else sigR_scat[i],
                                                 None if sigL_scat is None else sigL_scat[i]) for i in range(nb)]
        GG_d, GG_l = _keldysh_sweep(g, GR_d, GR_u, Au, Al, SigG)
        out["GG_diag"] = np.stack(GG_d)
        out["GG_low"] = np.stack(GG_l) if nb > 1 else np.zeros((0, b, b), complex)
    return out


# ---------------------------------------------------------------------------
# partitioned selected inversion (Sec. II and Fig. 3: Schur complements of P
# partitions, a reduced system solved sequentially, local reconstruction)
# ---------------------------------------------------------------------------

def _rgf_retarded_from_blocks(Ad, Au, Al):
    """G^R diagonal, upper and lower blocks of a BT matrix given by its blocks
    (the textbook recursion of ``rgf_blocks``, retarded part)."""
    nb = len(Ad)
    inv = np.linalg.inv
    g = [None] * nb
    g[0] = inv(Ad[0])
    for i in range(1, nb):
        g[i] = inv(Ad[i] - Al[i - 1] @ g[i - 1] @ Au[i - 1])
    Gd, Gu, Gl = [None] * nb, [None] * (nb - 1), [None] * (nb - 1)
    Gd[nb - 1] = g[nb - 1]
    for i in range(nb - 2, -1, -1):
        X = g[i] @ Au[i]
        Y = Al[i] @ g[i]
        Gu[i] = -X @ Gd[i + 1]
        Gl[i] = -Gd[i + 1] @ Y
        Gd[i] = g[i] - Gu[i] @ Y
    return Gd, Gu, Gl


def partitioned_retarded(dev, z, sigma_L, sigma_R, P, sigR_scat=None):
    """Selected blocks of G^R by partitioning the BT matrix (nb = P L blocks, L >= 2).

    Partition p holds blocks pL .. pL+L-1.  Its interior blocks pL .. pL+L-2 are
    eliminated downward (Schur complements), keeping its last block e_p = pL+L-1 and
    the previous partition's last block e_(p-1) (its top neighbour) as boundaries:
      D_0 = A_(pL,pL), F_(a,0) = A_(pL-1,pL), F_(0,a) = A_(pL,pL-1)  (F = 0 for p = 0);
      for k (block i, next block j = i+1):  g_k = D_k^{-1},
        Y_k = A_ji g_k,  X_k = g_k A_ij,  Xa_k = F_(a,k) g_k,  Wa_k = g_k F_(k,a),
        D_j = A_jj - Y_k A_ij,  F_(a,j) = -Xa_k A_ij,  F_(j,a) = -Y_k F_(k,a),
        dD_a -= Xa_k F_(k,a).
    The reduced system over the boundaries e_0 .. e_(P-1) is BT with diagonal
    D_(e_p) + dD_a of partition p+1 and couplings F_(a,b), F_(b,a) of partition p+1;
    its inverse (the textbook recursion) gives G on the boundaries.  Each partition
    then rebuilds its interior from j = e_p down to pL, with a = e_(p-1):
      G_jk = -(G_ja Xa_k + G_jj Y_k),  G_ak = -(G_aa Xa_k + G_aj Y_k),
      G_kj = -(Wa_k G_aj + X_k G_jj),  G_ka = -(Wa_k G_aa + X_k G_ja),
      G_kk = g_k - (Wa_k G_ak + X_k G_jk).
    With P = 1 this is the textbook recursion itself."""
    nb, b = dev.nb, dev.b
    if P < 1 or nb % P or nb // P < 2:
        raise ValueError("need nb = P L with L >= 2")
    L = nb // P
    Ad, Au, Al = _A_blocks(dev, z, sigma_L, sigma_R, sigR_scat)
    inv = np.linalg.inv
    Z = np.zeros((b, b), dtype=np.complex128)
    parts = []
    for p in range(P):
        s0 = p * L
        has_a = p > 0
        D = Ad[s0]
        Fak = Au[s0 - 1] if has_a else Z
        Fka = Al[s0 - 1] if has_a else Z
        dDa = Z
        st = dict(g=[], Y=[], X=[], Xa=[], Wa=[])
        for k in range(L - 1):
            i, j = s0 + k, s0 + k + 1
            gk = inv(D)
            Yk, Xk = Al[i] @ gk, gk @ Au[i]
            Xak, Wak = Fak @ gk, gk @ Fka
            for key, v in (("g", gk), ("Y", Yk), ("X", Xk), ("Xa", Xak), ("Wa", Wak)):
                st[key].append(v)
            D = Ad[j] - Yk @ Au[i]
            dDa = dDa - Xak @ Fka
            Fak, Fka = -Xak @ Au[i], -Yk @ Fka
        st.update(Db=D, dDa=dDa, Fab=Fak, Fba=Fka)
        parts.append(st)
    # reduced system over e_0 .. e_(P-1)
    Rd = [parts[r]["Db"] + (parts[r + 1]["dDa"] if r + 1 < P else Z) for r in range(P)]
    Ru = [parts[r + 1]["Fab"] for r in range(P - 1)]
    Rl = [parts[r + 1]["Fba"] for r in range(P - 1)]
    Gr_d, Gr_u, Gr_l = _rgf_retarded_from_blocks(Rd, Ru, Rl)
    GRd, GRu, GRl = [None] * nb, [None] * (nb - 1), [None] * (nb - 1)
    for p in range(P):
        s0, st = p * L, parts[p]
        has_a = p > 0
        Gjj = Gr_d[p]
        GRd[s0 + L - 1] = Gjj
        Gaa = Gr_d[p - 1] if has_a else Z
        Gaj = Gr_u[p - 1] if has_a else Z
        Gja = Gr_l[p - 1] if has_a else Z
        for k in range(L - 2, -1, -1):
            i = s0 + k
            Gjk = -(Gja @ st["Xa"][k] + Gjj @ st["Y"][k])
            Gak = -(Gaa @ st["Xa"][k] + Gaj @ st["Y"][k])
            Gkj = -(st["Wa"][k] @ Gaj + st["X"][k] @ Gjj)
            Gka = -(st["Wa"][k] @ Gaa + st["X"][k] @ Gja)
            Gkk = st["g"][k] - (st["Wa"][k] @ Gak + st["X"][k] @ Gjk)
            GRd[i], GRu[i], GRl[i] = Gkk, Gkj, Gjk
            Gjj, Gja, Gaj = Gkk, Gka, Gak
        if has_a:
            GRu[s0 - 1], GRl[s0 - 1] = Gaj, Gja
    return dict(GR_diag=np.stack(GRd),
                GR_up=np.stack(GRu) if nb > 1 else np.zeros((0, b, b), complex),
                GR_low=np.stack(GRl) if nb > 1 else np.zeros((0, b, b), complex))


# ---------------------------------------------------------------------------
# arrowhead BT matrices: a dense border block (a gate) coupled to every block
# ---------------------------------------------------------------------------

def arrowhead_dense(dev, z, sigma_L, sigma_R, H_tip, H_arrow, sigR_scat=None):
    """Eq. (1) for the block-tridiagonal-with-arrowhead (BTA) matrix: the device's A(z)
    bordered by one more block row and column, the tip t (size b, overlap I, Hamiltonian
    H_tip) coupled to block i by H_(t,i) = H_arrow[i] (overlap 0):
        A_tt = z I - H_tip,   A_(t,i) = -H_arrow[i],   A_(i,t) = -H_arrow[i]^H.
    Returns the selected blocks of G^R = A^{-1}: GR_diag, GR_up, GR_low of the device, the
    tip G_tt and the arrow blocks G_(t,i) (row) and G_(i,t) (column)."""
    b, nb = dev.b, dev.nb
    A = assemble_A(dev, z, sigma_L, sigma_R, sigR_scat)
    N = nb * b
    Ab = np.zeros((N + b, N + b), dtype=np.complex128)
    Ab[:N, :N] = A
    Ab[N:, N:] = z * np.eye(b) - H_tip
    for i in range(nb):
        Ab[N:, i * b:(i + 1) * b] = -H_arrow[i]
        Ab[i * b:(i + 1) * b, N:] = -_H(H_arrow[i])
    G = np.linalg.inv(Ab)
    return dict(
        GR_diag=np.stack([_blk(G, i, i, b) for i in range(nb)]),
        GR_up=np.stack([_blk(G, i, i + 1, b) for i in range(nb - 1)]) if nb > 1 else np.zeros((0, b, b), complex),
        GR_low=np.stack([_blk(G, i + 1, i, b) for i in range(nb - 1)]) if nb > 1 else np.zeros((0, b, b), complex),
        G_tip=G[N:, N:].copy(),
        G_row=np.stack([G[N:, i * b:(i + 1) * b] for i in range(nb)]),
        G_col=np.stack([G[i * b:(i + 1) * b, N:] for i in range(nb)]))


# ---------------------------------------------------------------------------
# Eq. (3): energy convolution and the self-consistent scattering loop (Fig. 2)
# ---------------------------------------------------------------------------

def energy_convolution(X, w):
    """Eq. (3) on a uniform energy grid with a scalar kernel: Y[n] = sum_m w[m] X[n - m]
    for m = -M..M (w has 2M+1 entries, w[0] is m = -M), X taken as zero outside the grid.
    X has the energy as its first axis; the sum runs element by element over the rest."""
    X = np.asarray(X)
    ne = X.shape[0]
    M = (len(w) - 1) // 2
    Y = np.zeros_like(X)
    for n in range(ne):
        for j, m in enumerate(range(-M, M + 1)):
            k = n - m
            if 0 <= k < ne and w[j] != 0.0:
                Y[n] = Y[n] + w[j] * X[k]
    return Y


def scba_self_energies(GL_diag, GG_diag, w_less, w_great):
    """Scattering self-energies of the self-consistent loop from the diagonal blocks of
    G^< and G^> over all energies ([ne][nb][b][b]): Sigma^<(E) = sum_m w^<_m G^<(E - w_m),
    Sigma^>(E) = sum_m w^>_m G^>(E - w_m) (Eq. (3), C1 = G, C2 = the scalar kernel), and
    Sigma^R = (Sigma^> - Sigma^<) / 2 (the anti-Hermitian part; the principal-value part
    is not kept)."""
    SL = energy_convolution(GL_diag, w_less)
    SG = energy_convolution(GG_diag, w_great)
    return 0.5 * (SG - SL), SL, SG


def scba_loop(dev, w_less, w_great, sigma=None, mixing=0.5, tol=1e-8, max_iter=100):
    """The self-consistent scattering loop of Fig. 2 for block-diagonal scattering:
    start from Sigma^{R,<,>} = 0; at every step solve Eq. (1)-(2) for G^R, G^<, G^> at all
    energies (block recursion), form the new self-energies by Eq. (3), and mix
    Sigma <- (1 - mixing) Sigma + mixing Sigma_new (for Sigma^< and Sigma^>, Sigma^R
    following from them); stop when max|Sigma^<_new - Sigma^<|, max|Sigma^>_new - Sigma^>|
    are both below tol times the largest entry of the new ones.  `sigma` = (Sigma_L,
    Sigma_R) per energy, else the decimation gives them.  Returns the self-energies, the
    last Green's functions, the step count and the last change."""
    ne, nb, b = dev.ne, dev.nb, dev.b
    if sigma is None:
        sig = [lead_self_energies(dev, dev.energy[e] + 1j * dev.eta)[:2] for e in range(ne)]
    else:
        sig = [(sigma[0][e], sigma[1][e]) for e in range(ne)]
    fL, fR = dev.f_L(), dev.f_R()
    SR = np.zeros((ne, nb, b, b), complex)
    SL = np.zeros_like(SR)
    SG = np.zeros_like(SR)
    change, it = np.inf, 0
    out = None
    while it < max_iter:
        it += 1
        out = [rgf_blocks(dev, dev.energy[e] + 1j * dev.eta, sig[e][0], sig[e][1], fL[e], fR[e],
                          sigR_scat=SR[e], sigL_scat=SL[e], greater=True) for e in range(ne)]
        GLd = np.stack([o["GL_diag"] for o in out])
        GGd = np.stack([o["GG_diag"] for o in out])
        _, SLn, SGn = scba_self_energies(GLd, GGd, w_less, w_great)
        scale = max(np.abs(SLn).max(), np.abs(SGn).max(), 1e-300)
        change = max(np.abs(SLn - SL).max(), np.abs(SGn - SG).max()) / scale
        SL = (1.0 - mixing) * SL + mixing * SLn
        SG = (1.0 - mixing) * SG + mixing * SGn
        SR = 0.5 * (SG - SL)
        if change < tol:
            break
    return dict(sigR=SR, sigL=SL, sigG=SG, out=out, iters=it, change=change)


# ---------------------------------------------------------------------------
# observables (Sec. III: DOS, spectral current and its conservation, density)
# ---------------------------------------------------------------------------

def transmission_caroli(sigma_L, sigma_R, G_corner):
    """Ballistic T(E) = Tr[Gamma_L G_{0,nb-1} Gamma_R G_{0,nb-1}^H]."""
    return float(np.real(np.trace(gamma(sigma_L) @ G_corner @ gamma(sigma_R) @ _H(G_corner))))


def transmission_g00(sigma_L, G00):
    """T from the first diagonal block only:
    Tr[Gamma_L i(G_00 - G_00^H)] - Tr[Gamma_L G_00 Gamma_L G_00^H]
    (equal to the Caroli form up to O(eta ||G||^2))."""
    GL = gamma(sigma_L)
    t = np.trace(GL @ (1j * (G00 - _H(G00)))) - np.trace(GL @ G00 @ GL @ _H(G00))
    return float(np.real(t))


def dos(dev, GR_diag, GR_up, GR_low):
    """DOS(E) = -(1/pi) Im Tr[G^R S], summed over the BT pattern of S."""
    nb = dev.nb
    if dev.S_diag is None:
        tr = sum(np.trace(GR_diag[i]) for i in range(nb))
    else:
        tr = sum(np.trace(GR_diag[i] @ dev.S_diag[i]) for i in range(nb))
        for i in range(nb - 1):
            tr += np.trace(GR_up[i] @ _H(dev.S_up[i]))   # G_{i,i+1} S_{i+1,i}
            tr += np.trace(GR_low[i] @ dev.S_up[i])      # G_{i+1,i} S_{i,i+1}
    return float(-np.imag(tr) / np.pi)


def interface_current(dev, z, GL_low):
    """Spectral current through each interface i | i+1:
    J_i(E) = 2 Re Tr[(H_{i,i+1} - z S_{i,i+1}) G^<_{i+1,i}]  (length nb-1)."""
    nb, b = dev.nb, dev.b
    J = np.zeros(max(nb - 1, 0))
    for i in range(nb - 1):
        Su = np.zeros((b, b)) if dev.S_up is None else dev.S_up[i]
        J[i] = 2.0 * np.real(np.trace((dev.H_up[i] - z * Su) @ GL_low[i]))
    return J


def density_energy(dev, GL_diag, GL_low):
    """Per-energy orbital occupation -i diag(G^< S) / (2 pi) over the BT pattern
    (real part), length N = nb * b."""
    nb, b = dev.nb, dev.b
    out = np.zeros(nb * b)
    for i in range(nb):
        if dev.S_diag is None:
            d = np.diag(GL_diag[i])
        else:
            M = GL_diag[i] @ dev.S_diag[i]
            if i + 1 < nb:   # G^<_{i,i+1} S_{i+1,i},  G^<_{i,i+1} = -(G^<_{i+1,i})^H
                M = M + (-_H(GL_low[i])) @ _H(dev.S_up[i])
            if i > 0:        # G^<_{i,i-1} S_{i-1,i}
                M = M + GL_low[i - 1] @ dev.S_up[i - 1]
            d = np.diag(M)
        out[i * b:(i + 1) * b] = np.real(-1j * d) / (2.0 * np.pi)
    return out


def density(dev, weights, GL_diag_E, GL_low_E):
    """Energy-integrated density n_k = sum_E w_E (-i)(G^< S)_kk(E) / (2 pi)."""
    n = np.zeros(dev.nb * dev.b)
    for e in range(len(weights)):
        n += weights[e] * density_energy(dev, GL_diag_E[e], GL_low_E[e])
    return n


# ---------------------------------------------------------------------------
# one energy, end to end
# ---------------------------------------------------------------------------

def solve_energy(dev, e, *, lesser=True, use_rgf=False, tol=1e-12, max_iter=100,
                 sigma=None, greater=False):
    """OBC + Eq. (1)/(2) + observables for energy index ``e`` of ``dev`` (and G^>
    with `greater`)."""
    z = dev.energy[e] + 1j * dev.eta
    if sigma is None:
        sL, sR, info = lead_self_energies(dev, z, tol, max_iter)
    else:
        sL, sR = sigma
        info = {}
    fL = dev.f_L()[e] if lesser else None
    fR = dev.f_R()[e] if lesser else None
    sR_scat = dev.sigR_scat
    sL_scat = None
    if lesser and dev.sigL_base is not None:
        sL_scat = dev.sigL_scale[e][:, None, None] * dev.sigL_base
    if use_rgf:
        out = rgf_blocks(dev, z, sL, sR, fL, fR, sR_scat, sL_scat, greater=greater and lesser)
    else:
        out = greens_dense(dev, z, sL, sR, fL, fR, sR_scat, sL_scat, greater=greater and lesser)
        out["T_caroli"] = transmission_caroli(sL, sR, out["GR_corner"])
    out["sigma_L"], out["sigma_R"], out["obc"] = sL, sR, info
    out["T"] = transmission_g00(sL, out["GR_diag"][0])
    out["dos"] = dos(dev, out["GR_diag"], out["GR_up"], out["GR_low"])
    if lesser:
        out["J"] = interface_current(dev, z, out["GL_low"])
        out["n_E"] = density_energy(dev, out["GL_diag"], out["GL_low"])
    return out
