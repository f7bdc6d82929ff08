"""Writes the stored expected values under tests/golden/ from the CPU oracle.

Run from the repository root:  python tests/golden/make_golden.py
It calls only ``oracle`` (and the seeded generators in ``workloads``).
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402
from oracle import negf_oracle as O  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


def config1_table():
    """Ballistic config (nb=16, b=8, 64 energies): T (G_00 form and Caroli), DOS,
    and the trace of G^R_00 per energy, by dense inversion."""
    dev = W.config1()
    rows = []
    for e in range(dev.ne):
        out = O.solve_energy(dev, e, lesser=False)
        tr = np.trace(out["GR_diag"][0])
        rows.append((dev.energy[e], out["T"], out["T_caroli"], out["dos"], tr.real, tr.imag))
    hdr = ("config 1 (nb=16, b=8, S=I, eta=1e-6, seed 20260001): oracle by dense inversion\n"
           "columns: E  T_g00  T_caroli  DOS  Re Tr G00  Im Tr G00")
    np.savetxt(os.path.join(HERE, "config1_oracle.txt"), np.array(rows), fmt="%.17e", header=hdr)


if __name__ == "__main__":
    config1_table()
