"""Seeded synthetic inputs shared by the oracle-side tests and the GPU side.

This module draws random numbers and lays out workload presets; it holds none
of the method's arithmetic (no sphere enumeration, no transforms, no
potentials, no Hamiltonian).  Anything derived from the plane-wave basis, such
as the kinetic energies used to damp the random coefficients, is passed in by
the caller, who computes it on its own side.

Workloads (all cells cubic unless stated; lengths in bohr, energies in Ha):
  small   L = 10, E_cut = 20, box 48^3, k_frac = (0.1, 0.2, 0.3), 16 bands,
          8 atoms at uniform-random positions, 4 Gaussian projectors per atom.
  large   L = 20, E_cut = 30, box 128^3, k_frac = (0.1, 0.2, 0.3), 256 bands,
          64 atoms, 256 projectors.
  slab    orthorhombic 40 x 20 x 20, E_cut = 30, box 256 x 128 x 128,
          256 atoms in a perturbed fcc slab filling x < 20 (vacuum above),
          1024 projectors, 1024 bands, 4 k-points uniform in the zone, w = 1/4.
  tiny_*  small boxes for exhaustive element-by-element checks.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

#: FFT box edge lengths the library accepts for generated cells, smallest first.
BOX_CHOICES = (40, 48, 54, 60, 64, 72, 80)


@dataclass(frozen=True)
class Workload:
    name: str
    L: tuple            # cell edge lengths (orthorhombic), bohr
    ecut: float         # Ha
    S: tuple            # FFT box
    kfrac: tuple        # tuple of k-points, fractional reciprocal coordinates
    natoms: int
    nbands: int
    seed_atoms: int
    seed_coeffs: int
    kweights: tuple = field(default=())
    layout: str = "uniform"   # atom placement: "uniform" in the cell, or "fcc_slab"

    @property
    def R(self) -> np.ndarray:
        """Lattice vectors as the columns of a 3x3 matrix."""
        return np.diag(np.asarray(self.L, dtype=np.float64))

    @property
    def nk(self) -> int:
        return len(self.kfrac)

    def weights(self) -> np.ndarray:
        if self.kweights:
            return np.asarray(self.kweights, dtype=np.float64)
        return np.full(self.nk, 1.0 / self.nk)


def _kpoints(nk: int, seed: int) -> tuple:
    rng = np.random.default_rng(seed)
    return tuple(tuple(float(x) for x in row) for row in rng.uniform(-0.5, 0.5, size=(nk, 3)))


WORKLOADS = {
    "small": Workload("small", (10.0, 10.0, 10.0), 20.0, (48, 48, 48),
                      ((0.1, 0.2, 0.3),), 8, 16, 1, 2),
    "large": Workload("large", (20.0, 20.0, 20.0), 30.0, (128, 128, 128),
                      ((0.1, 0.2, 0.3),), 64, 256, 11, 12),
    "tiny_cubic": Workload("tiny_cubic", (6.0, 6.0, 6.0), 4.0, (12, 12, 12),
                           ((0.1, 0.2, 0.3),), 2, 6, 101, 102),
    "tiny_ortho": Workload("tiny_ortho", (7.0, 5.0, 6.0), 5.0, (16, 12, 15),
                           ((0.25, -0.1, 0.4),), 3, 5, 103, 104),
    "mid": Workload("mid", (10.0, 10.0, 10.0), 12.0, (40, 40, 40),
                    ((0.1, 0.2, 0.3),), 8, 24, 105, 106),
    "slab": Workload("slab", (40.0, 20.0, 20.0), 30.0, (256, 128, 128), _kpoints(4, 51), 256, 1024, 51, 52,
                     (0.25, 0.25, 0.25, 0.25), "fcc_slab"),
}


def atom_positions(R: np.ndarray, natoms: int, seed: int) -> np.ndarray:
    """Cartesian positions (natoms x 3) uniform in the cell spanned by R's columns."""
    rng = np.random.default_rng(seed)
    frac = rng.uniform(0.0, 1.0, size=(natoms, 3))
    return frac @ np.asarray(R, dtype=np.float64).T


def fcc_slab_positions(seed: int, a: float = 5.0, cells=(4, 4, 4), sigma: float = 0.2) -> np.ndarray:
    """Cartesian positions of an fcc crystal of conventional edge a (4 atoms per
    cell, cells[0] x cells[1] x cells[2] cells from the origin), each atom
    displaced by independent N(0, sigma^2) per axis."""
    basis = np.array([[0.0, 0.0, 0.0], [0.5, 0.5, 0.0], [0.5, 0.0, 0.5], [0.0, 0.5, 0.5]])
    grid = np.array([(i, j, k) for i in range(cells[0]) for j in range(cells[1]) for k in range(cells[2])],
                    dtype=np.float64)
    pos = (grid[:, None, :] + basis[None, :, :]).reshape(-1, 3) * a
    rng = np.random.default_rng(seed)
    return pos + rng.normal(0.0, sigma, size=pos.shape)


def workload_atoms(w: Workload) -> np.ndarray:
    """The workload's atom positions (Cartesian, natoms x 3)."""
    if w.layout == "fcc_slab":
        pos = fcc_slab_positions(w.seed_atoms)
        assert pos.shape[0] == w.natoms
        return pos
    return atom_positions(w.R, w.natoms, w.seed_atoms)


def random_coefficients(kinetic2: np.ndarray, nbands: int, seed: int) -> np.ndarray:
    """Band-major random block Y (nbands x npw, complex128).

    Y[b, G] = (x + i y) / (1 + |k+G|^2) with x, y independent standard normals;
    ``kinetic2`` is |k+G|^2 per plane wave, supplied by the caller.
    """
    rng = np.random.default_rng(seed)
    z = rng.standard_normal(size=(nbands, kinetic2.size, 2))
    # (re, im) pairs are adjacent: the same draws viewed as complex, damped in place
    y = z.reshape(nbands, -1).view(np.complex128)
    y /= (1.0 + np.asarray(kinetic2, dtype=np.float64))[None, :]
    return y


def random_kpoints(nk: int, seed: int) -> np.ndarray:
    """nk k-points uniform in [-1/2, 1/2)^3 (fractional reciprocal coordinates)."""
    rng = np.random.default_rng(seed)
    return rng.uniform(-0.5, 0.5, size=(nk, 3))


def box_for(L: float, ecut: float) -> int:
    """Smallest box edge in BOX_CHOICES that holds twice the sphere radius.

    The sphere reaches |G| <= sqrt(2 E_cut); along one axis of a cubic cell
    that is sqrt(2 E_cut) L / (2 pi) grid steps, and the box must hold 4x that
    plus one (products of two sphere functions alias-free).  40 is the floor.
    """
    need = 4.0 * np.sqrt(2.0 * ecut) * L / (2.0 * np.pi) + 1.0
    for s in BOX_CHOICES:
        if s >= need:
            return s
    return BOX_CHOICES[-1]


def random_cells(n: int, seed: int, L_range=(8.0, 16.0), ecut: float = 20.0):
    """Independent cubic cells for the mixed-cell batch workload."""
    rng = np.random.default_rng(seed)
    cells = []
    for c in range(n):
        L = float(rng.uniform(*L_range))
        natoms = int(rng.integers(4, 33))
        nb = int(rng.integers(16, 129))
        cells.append(Workload(f"cell{c}", (L, L, L), ecut, (box_for(L, ecut),) * 3,
                              (tuple(rng.uniform(-0.5, 0.5, size=3)),), natoms, nb,
                              seed * 100 + 2 * c, seed * 100 + 2 * c + 1))
    return cells


def mlp_init(seed: int, hidden: int = 64) -> np.ndarray:
    """Seeded starting parameters of the preconditioner network (4481 floats for
    hidden = 64): weights N(0, 1/fan_in), zero biases, in the order
    W1 (hidden x 3), b1, W2 (hidden x hidden), b2, W3 (hidden), b3."""
    rng = np.random.default_rng(seed)
    W1 = rng.standard_normal((hidden, 3)) / np.sqrt(3.0)
    W2 = rng.standard_normal((hidden, hidden)) / np.sqrt(hidden)
    W3 = rng.standard_normal(hidden) / np.sqrt(hidden)
    return np.concatenate([W1.ravel(), np.zeros(hidden), W2.ravel(), np.zeros(hidden), W3, [0.0]])


def training_cells(n: int, seed0: int = 1000, L_range=(16.0, 24.0), ecut: float = 20.0):
    """Seeded cells for the preconditioner's training data: cubic L ~ U(L_range),
    n_atoms = round(8 (L/10)^3) uniform in the cell, n_bands = 2 n_atoms, k = 0."""
    cells = []
    for c in range(n):
        rng = np.random.default_rng(seed0 + c)
        L = float(rng.uniform(*L_range))
        natoms = int(round(8 * (L / 10.0) ** 3))
        cells.append(Workload(f"train{seed0 + c}", (L, L, L), ecut, (box_for(L, ecut),) * 3, ((0.0, 0.0, 0.0),),
                              natoms, 2 * natoms, seed0 + c, 10 ** 6 + seed0 + c))
    return cells
