"""Writes scf_small.json: the self-consistent LDA solution of the 48^3 test cell.

Calls only the oracle (oracle/scf.py): the 'small' workload (cubic L = 10 bohr,
E_cut = 20 Ha, box 48^3, k = (0.1, 0.2, 0.3), 8 Gaussian atoms with 32
projectors, 16 bands with f = 2) as the ionic potential and projectors, Hartree
and Perdew-Zunger LDA added self-consistently, Pulay mixing (8 pairs,
alpha = 0.5) from the density of the seeded starting block, every band solve
by dense diagonalisation of the 4 259-plane-wave Hamiltonian.  Stored: total
energy and its parts, the 16 eigenvalues, and the density at a few grid points.

    python tests/golden/make_scf_small.py
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import planewave as pw  # noqa: E402
from oracle import scf  # noqa: E402
from synth import WORKLOADS, atom_positions, random_coefficients  # noqa: E402

#: grid points whose density is stored (linear box indices)
SAMPLE = [0, 1, 4321, 55296, 77777, 110591]


def main():
    w = WORKLOADS["small"]
    atoms = atom_positions(w.R, w.natoms, w.seed_atoms)
    basis = pw.Basis.build(w.R, w.S, w.kfrac[0], w.ecut)
    Vion = pw.vloc_realspace(w.R, w.S, atoms)
    P = pw.projectors(w.R, basis.kfrac, basis.iG, atoms)
    C0 = random_coefficients(2 * basis.T, w.nbands, w.seed_coeffs).T
    cells = [scf.KCell(basis, P, pw.dmatrix(w.natoms), 1.0, C0)]
    t0 = time.time()
    res = scf.scf(cells, Vion, alpha=0.5, history=8, tol_energy=1e-10, tol_density=1e-8)
    out = {
        "workload": "small (L=10, Ecut=20, 48^3, k=(0.1,0.2,0.3), 8 atoms, 16 bands, f=2), LDA (PZ81), "
                    "Pulay 8 pairs alpha 0.5",
        "converged": bool(res.converged),
        "iterations": res.iterations,
        "energy": res.energy,
        "parts": res.parts,
        "eigs": [float(x) for x in res.eigs[0]],
        "density_samples": {str(j): float(res.n[j]) for j in SAMPLE},
        "electrons": float(basis.Omega / basis.N * np.sum(res.n)),
        "oracle_seconds": time.time() - t0,
    }
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "scf_small.json"), "w") as fh:
        json.dump(out, fh, indent=1)
    print(json.dumps(out, indent=1))


if __name__ == "__main__":
    main()
