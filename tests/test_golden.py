"""The stored config-1 table still matches the oracle (guards the fixture)."""
import os

import numpy as np

import workloads as W
from oracle import negf_oracle as O

GOLD = os.path.join(os.path.dirname(__file__), "golden", "config1_oracle.txt")


def test_config1_golden_matches_oracle():
    tab = np.loadtxt(GOLD)
    dev = W.config1()
    assert tab.shape == (dev.ne, 6)
    assert np.array_equal(tab[:, 0], dev.energy)
    for e in [0, 17, 31, 40, 63]:
        out = O.solve_energy(dev, e, lesser=False)
        assert abs(out["T"] - tab[e, 1]) <= 1e-12 * max(1.0, abs(tab[e, 1]))
        assert abs(out["dos"] - tab[e, 3]) <= 1e-12 * max(1.0, abs(tab[e, 3]))
