"""The seeded input recipe: shapes, value structure and determinism of the generated
workloads, checked against the stated recipe (configs 1-5 of the benchmark plan).
CPU only; the generators hold no NEGF arithmetic."""
import numpy as np

import workloads as W


def _herm_err(x):
    return np.abs(x - np.conj(np.swapaxes(x, -1, -2))).max()


def test_config1_recipe():
    dev = W.config1()
    assert dev.H_diag.shape == (16, 8, 8) and dev.H_up.shape == (15, 8, 8)
    assert dev.S_diag is None and dev.S_up is None
    assert dev.ne == 64 and dev.energy[0] == -3.0 and dev.energy[-1] == 3.0
    assert dev.eta == 1e-6
    assert _herm_err(dev.H_diag) == 0.0


def test_config2_recipe_at_reduced_size():
    # the full generator at nb = 4 (same construction as nb = 64): global-band decay,
    # S = I + 0.05 R with the same pattern, Hermitian diagonal blocks
    dev = W.config2(nb=4, b=128, ne=1024)
    assert dev.H_diag.shape == (4, 128, 128) and dev.H_up.shape == (3, 128, 128)
    assert dev.S_diag.shape == (4, 128, 128) and dev.S_up.shape == (3, 128, 128)
    assert dev.ne == 1024 and np.isclose(dev.energy[1] - dev.energy[0], 6.0 / 1023)
    assert _herm_err(dev.H_diag) < 1e-15 and _herm_err(dev.S_diag) < 1e-15
    # overlap: identity plus a small perturbation, positive definite
    off = dev.S_diag - np.eye(128)[None]
    assert 0 < np.abs(off).max() < 0.05
    assert np.linalg.eigvalsh(dev.S_diag).min() > 0.5
    # band decay over the global orbital index: H_up[r][c] couples orbitals b apart plus
    # c - r, so its corner (0, b-1) is at distance 2b - 1 (tiny), (b-1, 0) at distance 1
    assert np.abs(dev.H_up[:, 0, -1]).max() < 1e-20 * np.abs(dev.H_up[:, -1, 0]).max()


def test_config2_full_size_shapes():
    dev = W.config2()
    assert (dev.nb, dev.b, dev.ne) == (64, 128, 1024)


def test_config3_shapes_recipe():
    shapes = W.config3_shapes()
    assert len(shapes) == 256
    nbs, bs, nes = (np.array(v) for v in zip(*shapes))
    assert set(bs.tolist()) <= set(W.CONFIG3_BS) and len(set(bs.tolist())) == len(W.CONFIG3_BS)
    assert nbs.min() >= 8 and nbs.max() <= 128
    assert nes.min() >= 64 and nes.max() <= 512
    assert W.config3_shapes() == shapes   # seeded


def test_config4_scattering_recipe_at_reduced_size():
    dev = W.config4(nb=3, b=32, ne=8)
    assert dev.sigR_scat.shape == (3, 32, 32)
    # Im Sigma^R <= 0: -i P with P positive semidefinite
    P = -(dev.sigR_scat - np.conj(np.swapaxes(dev.sigR_scat, -1, -2))) / 2j
    assert np.linalg.eigvalsh(P).min() > -1e-15
    # Sigma^< = 2 i f_i P_i with f_i in [0, 1] per block and energy
    assert dev.sigL_scale.shape == (8, 3)
    assert dev.sigL_scale.min() >= 0.0 and dev.sigL_scale.max() <= 1.0
    assert np.allclose(dev.sigL_base, 2j * P)


def test_config5_sets_recipe():
    s = W.config5_sets()
    assert s["H00"].shape == (20, 64, 64) and s["H01"].shape == (20, 64, 64)
    lead, E = s["train"]
    assert lead.size == 16 * 256 and set(lead.tolist()) == set(range(16))
    assert np.array_equal(np.unique(E), np.linspace(-3.0, 3.0, 256))
    lead_h, E_h = s["held"]
    assert lead_h.size == 16 * 64 and E_h.min() >= -3.0 and E_h.max() <= 3.0
    lead_u, _ = s["unseen"]
    assert set(lead_u.tolist()) == set(range(16, 20))


def test_generators_are_deterministic():
    a, b = W.config2(nb=2, b=16, ne=4), W.config2(nb=2, b=16, ne=4)
    assert np.array_equal(a.H_diag, b.H_diag) and np.array_equal(a.S_up, b.S_up)
    assert np.array_equal(W.mlp_init(8), W.mlp_init(8))
