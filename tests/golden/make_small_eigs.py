"""Writes small_eigs.json: the lowest eigenvalues of the 48^3 test cell's Hamiltonian.

Calls only the oracle: the dense Hamiltonian (4 259 plane waves) of the
'small' workload (cubic L = 10 bohr, E_cut = 20 Ha, k = (0.1, 0.2, 0.3),
8 Gaussian atoms, 32 projectors) diagonalised by LAPACK.  E_ref = 2 x the
sum of the lowest 16 (f = 2 per band).

    python tests/golden/make_small_eigs.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import planewave as pw  # noqa: E402
from synth import WORKLOADS, atom_positions  # noqa: E402


def main():
    w = WORKLOADS["small"]
    atoms = atom_positions(w.R, w.natoms, w.seed_atoms)
    basis = pw.Basis.build(w.R, w.S, w.kfrac[0], w.ecut)
    V = pw.vloc_realspace(w.R, w.S, atoms)
    P = pw.projectors(w.R, basis.kfrac, basis.iG, atoms)
    H = pw.dense_H(basis, V, P, pw.dmatrix(w.natoms))
    eigs = np.linalg.eigvalsh(H / basis.Omega)[:w.nbands + 4]
    out = {"workload": "small: cubic L=10 bohr, Ecut=20 Ha, 48^3, k=(0.1,0.2,0.3), 8 atoms seed 1",
           "npw": int(basis.npw), "nbands": w.nbands, "eigs": [float(e) for e in eigs],
           "E_ref": float(2.0 * eigs[:w.nbands].sum()),
           "gap": float(eigs[w.nbands] - eigs[w.nbands - 1])}
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "small_eigs.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(out["E_ref"], out["gap"])


if __name__ == "__main__":
    main()
