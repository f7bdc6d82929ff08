"""Seeded synthetic inputs for the batched RGF workloads.

This module holds only random draws and the construction of the device
matrices (H, S), energy grids, occupations and quadrature weights.  It holds
none of the NEGF arithmetic (no inversion, no self-energies, no Green's
functions): both the CPU oracle and the CUDA path consume what it produces.

Conventions (shared by both sides):
  * complex matrices are numpy complex128, row-major, blocks stacked as
    ``[nb][b][b]`` (diagonal) and ``[nb-1][b][b]`` (upper, block (i, i+1)).
    The lower blocks are the conjugate transposes of the upper ones.
  * ``S_diag``/``S_up`` are ``None`` when S is the identity.
  * the left lead repeats block 0 (onsite H_00, hop H_01), the right lead
    repeats block nb-1 (onsite H_{nb-1,nb-1}, hop H_{nb-2,nb-1}).

Device model (block-tridiagonal shape of A and B, Sec. II of the paper):
a random Hermitian onsite block per slice, random inter-slice couplings, and
the flat / linear / flat electrostatic profile of the transistor of Sec. III
(0.2 V drop over the central half of the device).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

SEED_BASE = 20260000


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _cn(rng: np.random.Generator, shape, sigma: float = 1.0) -> np.ndarray:
    """Circular complex normal, E|x|^2 = sigma^2 (re and im each N(0, sigma^2/2))."""
    s = sigma / np.sqrt(2.0)
    return rng.normal(0.0, s, shape) + 1j * rng.normal(0.0, s, shape)


def _herm(x: np.ndarray) -> np.ndarray:
    return 0.5 * (x + np.conj(np.swapaxes(x, -1, -2)))


def potential_profile(nb: int, dv: float = 0.2) -> np.ndarray:
    """Onsite shift per block: +dv/2 on the first quarter, a linear drop over the
    central half, -dv/2 on the last quarter (the Sec. III transistor profile)."""
    v = np.empty(nb)
    q = nb / 4.0
    for i in range(nb):
        x = i + 0.5
        if x <= q:
            v[i] = 0.5 * dv
        elif x >= nb - q:
            v[i] = -0.5 * dv
        else:
            v[i] = 0.5 * dv - dv * (x - q) / (nb - 2.0 * q)
    return v


def fermi(energy: np.ndarray, mu: float, kT: float) -> np.ndarray:
    """Fermi-Dirac occupation 1 / (1 + exp((E - mu) / kT)) (an input of the method)."""
    x = (np.asarray(energy, dtype=np.float64) - mu) / kT
    return 0.5 * (1.0 - np.tanh(0.5 * x))


def trapezoid_weights(energy: np.ndarray) -> np.ndarray:
    """Trapezoid quadrature weights over a uniform energy grid."""
    e = np.asarray(energy, dtype=np.float64)
    if e.size < 2:
        return np.ones_like(e)
    de = (e[-1] - e[0]) / (e.size - 1)
    w = np.full(e.size, de)
    w[0] *= 0.5
    w[-1] *= 0.5
    return w


@dataclass
class Device:
    """One block-tridiagonal device and its energy grid."""
    H_diag: np.ndarray                 # [nb][b][b] complex128, Hermitian blocks
    H_up: np.ndarray                   # [nb-1][b][b] complex128, block (i, i+1)
    S_diag: Optional[np.ndarray]       # None => identity
    S_up: Optional[np.ndarray]         # None => zero
    energy: np.ndarray                 # [ne] float64 (real part of z)
    eta: float = 1e-6
    mu_L: float = 0.1
    mu_R: float = -0.1
    kT: float = 0.025
    # optional block-diagonal scattering self-energies
    sigR_scat: Optional[np.ndarray] = None   # [nb][b][b], energy independent
    sigL_base: Optional[np.ndarray] = None   # [nb][b][b]; Sigma^<_ii(E) = scale[E][i] * base_i
    sigL_scale: Optional[np.ndarray] = None  # [ne][nb] float64
    name: str = ""

    @property
    def nb(self) -> int:
        return self.H_diag.shape[0]

    @property
    def b(self) -> int:
        return self.H_diag.shape[1]

    @property
    def ne(self) -> int:
        return self.energy.shape[0]

    def f_L(self) -> np.ndarray:
        return fermi(self.energy, self.mu_L, self.kT)

    def f_R(self) -> np.ndarray:
        return fermi(self.energy, self.mu_R, self.kT)

    def weights(self) -> np.ndarray:
        return trapezoid_weights(self.energy)

    def sigL_scat_full(self) -> Optional[np.ndarray]:
        """[ne][nb][b][b] lesser scattering self-energy (scale x base)."""
        if self.sigL_base is None:
            return None
        return self.sigL_scale[:, :, None, None] * self.sigL_base[None]

    def truncated(self, nb: Optional[int] = None, energies=None) -> "Device":
        """A sub-problem: the first ``nb`` blocks and/or a subset of energies.
        Leads keep being repeats of the (new) first and last blocks."""
        nb = self.nb if nb is None else nb
        idx = np.arange(self.ne) if energies is None else np.asarray(energies)
        cut = lambda a, n: None if a is None else a[:n].copy()
        return Device(
            H_diag=self.H_diag[:nb].copy(), H_up=self.H_up[:nb - 1].copy(),
            S_diag=cut(self.S_diag, nb), S_up=cut(self.S_up, nb - 1),
            energy=self.energy[idx].copy(), eta=self.eta, mu_L=self.mu_L,
            mu_R=self.mu_R, kT=self.kT,
            sigR_scat=cut(self.sigR_scat, nb), sigL_base=cut(self.sigL_base, nb),
            sigL_scale=None if self.sigL_scale is None else self.sigL_scale[idx][:, :nb].copy(),
            name=self.name + f"[nb={nb},ne={idx.size}]")


# --------------------------------------------------------------------------
# generators
# --------------------------------------------------------------------------

def random_uniform_chain(nb: int, b: int, seed: int, *, offdiag_sigma: float = 0.3,
                         shift: bool = True) -> tuple:
    """Config-1 style blocks: H_ii = Herm(CN(0,1))/sqrt(b) + V_i I, H_{i,i+1} ~ CN(0, sigma^2)."""
    rng = _rng(seed)
    Hd = _herm(_cn(rng, (nb, b, b))) / np.sqrt(b)
    Hu = _cn(rng, (max(nb - 1, 0), b, b), offdiag_sigma)
    if shift:
        v = potential_profile(nb)
        Hd = Hd + v[:, None, None] * np.eye(b)[None]
    return Hd, Hu


def banded_blocks(nb: int, b: int, rng: np.random.Generator, decay: float = 4.0) -> tuple:
    """Hermitian matrix with entries CN(0,1)/sqrt(b) * exp(-|p-q|/decay) over the
    GLOBAL orbital index p, q, cut to its block-tridiagonal part."""
    r = np.arange(b)
    d_diag = np.exp(-np.abs(r[:, None] - r[None, :]) / decay)
    d_up = np.exp(-(b + r[None, :] - r[:, None]) / decay)      # |p-q| = b + c - r
    Hd = _herm(_cn(rng, (nb, b, b))) * d_diag[None] / np.sqrt(b)
    Hu = _cn(rng, (max(nb - 1, 0), b, b)) * d_up[None] / np.sqrt(b)
    return Hd, Hu


def config1(seed: int = SEED_BASE + 1) -> Device:
    """Ballistic, plain method: nb=16, b=8, S=I, 64 energies in [-3,3], eta=1e-6."""
    Hd, Hu = random_uniform_chain(16, 8, seed)
    return Device(Hd, Hu, None, None, np.linspace(-3.0, 3.0, 64), 1e-6, name="config1")


def banded_device(nb: int, b: int, ne: int, seed: int, *, overlap: bool = True,
                  e_min: float = -3.0, e_max: float = 3.0, name: str = "") -> Device:
    """Config-2/3/4 generator: global-band decay H, S = I + 0.05 R (same pattern)."""
    rng = _rng(seed)
    Hd, Hu = banded_blocks(nb, b, rng)
    Hd = Hd + potential_profile(nb)[:, None, None] * np.eye(b)[None]
    Sd = Su = None
    if overlap:
        Rd, Ru = banded_blocks(nb, b, rng)
        Sd = np.eye(b)[None] + 0.05 * Rd
        Su = 0.05 * Ru
    return Device(Hd, Hu, Sd, Su, np.linspace(e_min, e_max, ne), 1e-6, name=name)


def config2(nb: int = 64, b: int = 128, ne: int = 1024, seed: int = SEED_BASE + 2) -> Device:
    """Ballistic batched RGF: nb=64, b=128, 1024 energies, S = I + 0.05 R."""
    return banded_device(nb, b, ne, seed, name="config2")


CONFIG3_BS = (32, 64, 96, 128, 192, 256)


def config3_shapes(ndev: int = 256, seed: int = SEED_BASE + 3) -> List[tuple]:
    """(nb, b, ne) per device of the uneven batch."""
    rng = _rng(seed)
    bs = rng.choice(np.array(CONFIG3_BS), size=ndev)
    nbs = rng.integers(8, 129, size=ndev)
    nes = rng.integers(64, 513, size=ndev)
    return [(int(n), int(b), int(e)) for n, b, e in zip(nbs, bs, nes)]


def config3_device(k: int, shapes=None, seed: int = SEED_BASE + 3) -> Device:
    shapes = config3_shapes(seed=seed) if shapes is None else shapes
    nb, b, ne = shapes[k]
    return banded_device(nb, b, ne, seed + 1 + k, name=f"config3.dev{k}")


def config4(nb: int = 32, b: int = 512, ne: int = 512, seed: int = SEED_BASE + 4) -> Device:
    """Lesser G with block-diagonal scattering self-energies.

    Sigma^R_ii = 0.01 R_i - i P_i with P_i = 0.01 Q Q^H / b (Im Sigma^R <= 0),
    Sigma^<_ii(E) = 2 i f_i(E) P_i with f_i the Fermi function at the local
    chemical potential (linear from mu_L to mu_R along the device)."""
    dev = banded_device(nb, b, ne, seed, name="config4")
    rng = _rng(seed + 1000)
    R = _herm(_cn(rng, (nb, b, b))) / np.sqrt(b)
    Q = _cn(rng, (nb, b, b))
    P = 0.01 * (Q @ np.conj(np.swapaxes(Q, -1, -2))) / b
    dev.sigR_scat = 0.01 * R - 1j * P
    dev.sigL_base = 2j * P
    mu_i = dev.mu_L + (dev.mu_R - dev.mu_L) * (np.arange(nb) + 0.5) / nb
    dev.sigL_scale = np.stack([fermi(dev.energy, m, dev.kT) for m in mu_i], axis=1)
    return dev


def small_scattering_device(nb: int, b: int, ne: int, seed: int, *, overlap: bool = True,
                            strength: float = 0.01) -> Device:
    """A config-4 style device at oracle-friendly sizes."""
    dev = banded_device(nb, b, ne, seed, overlap=overlap, name="scatter-small")
    rng = _rng(seed + 1000)
    R = _herm(_cn(rng, (nb, b, b))) / np.sqrt(b)
    Q = _cn(rng, (nb, b, b))
    P = strength * (Q @ np.conj(np.swapaxes(Q, -1, -2))) / b
    dev.sigR_scat = strength * R - 1j * P
    dev.sigL_base = 2j * P
    mu_i = dev.mu_L + (dev.mu_R - dev.mu_L) * (np.arange(nb) + 0.5) / nb
    dev.sigL_scale = np.stack([fermi(dev.energy, m, dev.kT) for m in mu_i], axis=1)
    return dev


def config5_lead(k: int, b: int = 64, seed: int = SEED_BASE + 5) -> tuple:
    """Lead k of the warm-start set: H00 = Herm(CN(0,1))/sqrt(b), H01 ~ CN(0, 0.3^2)."""
    rng = _rng(seed + 17 * k)
    H00 = _herm(_cn(rng, (b, b))) / np.sqrt(b)
    H01 = _cn(rng, (b, b), 0.3)
    return H00, H01


def config5_sets(b: int = 64, n_leads: int = 16, n_train_e: int = 256, n_held_e: int = 64,
                 n_unseen: int = 4, seed: int = SEED_BASE + 5) -> dict:
    """The warm-start workload: 16 leads x 256 training energies (4096 pairs, uniform
    grid on [-3, 3]), 1024 held-out energies on the same leads (64 per lead, uniform
    random, off the grid), and 4 unseen leads with 64 random energies each."""
    rng = _rng(seed + 999)
    leads = [config5_lead(k, b, seed) for k in range(n_leads + n_unseen)]
    H00 = np.stack([h for h, _ in leads])
    H01 = np.stack([t for _, t in leads])
    grid = np.linspace(-3.0, 3.0, n_train_e)
    train = (np.repeat(np.arange(n_leads), n_train_e).astype(np.int32), np.tile(grid, n_leads))
    held = (np.repeat(np.arange(n_leads), n_held_e).astype(np.int32),
            rng.uniform(-3.0, 3.0, size=n_leads * n_held_e))
    unseen = (np.repeat(np.arange(n_leads, n_leads + n_unseen), n_held_e).astype(np.int32),
              rng.uniform(-3.0, 3.0, size=n_unseen * n_held_e))
    return dict(H00=H00, H01=H01, train=train, held=held, unseen=unseen)


def mlp_init(b: int, hidden: int = 512, seed: int = SEED_BASE + 50) -> np.ndarray:
    """Initial parameters of the warm-start network as one float32 vector in the
    layout W1 [hidden][K0P], c1, W2 [hidden][hidden], c2, W3 [2b^2][hidden], c3:
    weights uniform in +-sqrt(6 / fan_in) (He), biases zero, and the padding
    columns of W1 (k >= 3b^2+65) zero."""
    rng = _rng(seed)
    k0 = 3 * b * b + 1 + 64          # lead blocks, E, 32 sine/cosine pairs of E
    k0p = (k0 + 127) // 128 * 128
    nout = 2 * b * b
    W1 = np.zeros((hidden, k0p))
    W1[:, :k0] = rng.uniform(-1, 1, size=(hidden, k0)) * np.sqrt(6.0 / k0)
    W2 = rng.uniform(-1, 1, size=(hidden, hidden)) * np.sqrt(6.0 / hidden)
    W3 = rng.uniform(-1, 1, size=(nout, hidden)) * np.sqrt(6.0 / hidden) * 0.1
    parts = [W1.ravel(), np.zeros(hidden), W2.ravel(), np.zeros(hidden), W3.ravel(), np.zeros(nout)]
    return np.concatenate(parts).astype(np.float32)


def ideal_chain(nb: int, t: float, energy, eta: float = 1e-6, onsite: float = 0.0) -> Device:
    """b = 1 chain with every block equal to the lead (onsite, hop t)."""
    Hd = np.full((nb, 1, 1), onsite, dtype=np.complex128)
    Hu = np.full((max(nb - 1, 0), 1, 1), t, dtype=np.complex128)
    return Device(Hd, Hu, None, None, np.asarray(energy, dtype=np.float64), eta, name="ideal-chain")


def ideal_multiorbital(nb: int, H00: np.ndarray, H01: np.ndarray, energy, eta: float = 1e-6) -> Device:
    """Device made of nb identical copies of a lead cell (H00, H01)."""
    b = H00.shape[0]
    Hd = np.broadcast_to(H00, (nb, b, b)).astype(np.complex128).copy()
    Hu = np.broadcast_to(H01, (max(nb - 1, 0), b, b)).astype(np.complex128).copy()
    return Device(Hd, Hu, None, None, np.asarray(energy, dtype=np.float64), eta, name="ideal")


# --------------------------------------------------------------------------
# self-consistent scattering (Fig. 2 loop): a device that carries current, and the
# phonon-like scalar kernel of the energy convolution of Eq. (3)
# --------------------------------------------------------------------------

def scba_device(nb: int = 8, b: int = 16, ne: int = 256, seed: int = SEED_BASE + 6,
                e_min: float = -4.5, e_max: float = 4.5) -> Device:
    """Config-4 style device for the self-consistent loop, at loop-friendly sizes: the
    banded generator plus a dense random inter-slice coupling (sigma 0.3 / sqrt(b)) so
    that current flows, S = I + 0.05 R, mu_L - mu_R = 0.2, kT = 0.025, on a uniform
    grid wide enough that no spectral weight leaves it when shifted by the kernel."""
    dev = banded_device(nb, b, ne, seed, overlap=True, e_min=e_min, e_max=e_max, name="scba")
    rng = _rng(seed + 500)
    if nb > 1:
        dev.H_up = dev.H_up + 0.3 * _cn(rng, dev.H_up.shape) / np.sqrt(b)
    return dev


def einstein_kernel(energy: np.ndarray, steps: int, g2: float, kT: float):
    """Weights of an Einstein boson of energy hw0 = steps * dE (dE the grid step) for the
    convolution Sigma^x(E) = sum_m w^x_m G^x(E - m dE), m = -steps..steps: absorption
    (m = +steps) with N, emission (m = -steps) with N + 1 for Sigma^<; the reverse for
    Sigma^>; N the Bose occupation at kT, g2 the squared coupling.  Returns (w_less,
    w_great), each of length 2 steps + 1 (entry 0 is m = -steps)."""
    de = float(energy[1] - energy[0])
    w0 = steps * de
    nbose = 1.0 / np.expm1(w0 / kT)
    wl = np.zeros(2 * steps + 1)
    wg = np.zeros(2 * steps + 1)
    wl[2 * steps], wl[0] = g2 * nbose, g2 * (nbose + 1.0)
    wg[2 * steps], wg[0] = g2 * (nbose + 1.0), g2 * nbose
    return wl, wg


def arrowhead_gate(dev: Device, seed: int = SEED_BASE + 7, coupling: float = 0.1):
    """A gate block for the arrowhead BT matrix of a device: a random Hermitian tip
    Hamiltonian (CN(0,1)/sqrt(b), shifted by +1) and a random coupling of the tip to every
    block (CN(0, coupling^2)/sqrt(b)).  Returns (H_tip [b][b], H_arrow [nb][b][b])."""
    rng = _rng(seed)
    b, nb = dev.b, dev.nb
    H_tip = _herm(_cn(rng, (b, b))) / np.sqrt(b) + np.eye(b)
    H_arrow = coupling * _cn(rng, (nb, b, b)) / np.sqrt(b)
    return H_tip, H_arrow
