"""FP64 CPU oracle of the plane-wave Hamiltonian hot path.

TEST INFRASTRUCTURE ONLY.  This module is the slow, plain statement of what
the GPU library computes.  Only ``tests/``, the smoke check and the
benchmark's CPU-baseline leg may import it; the product path never does, and
it shares no code with the CUDA library.

The JDFTx paper (Sec. 2.1, "Software Architecture") names the algebraic
operators of the DFT++ formulation -- I and J (reciprocal <-> real space by
FFT), O (overlap, diagonal in the plane-wave basis), pointwise multiplication
by a real-space field, projectors of the pseudopotentials (Sec. 2.2) -- but
prints no formula for them.  The formulas below are the standard plane-wave
readings:

* Lattice vectors are the columns a_d of R, Omega = |det R|, reciprocal
  vectors the columns of B = 2 pi R^{-T} (so a_i . b_j = 2 pi delta_ij).
* FFT box S = (S0, S1, S2), N = S0 S1 S2, grid points r_j = R (j0/S0, j1/S1,
  j2/S2), linear index j2 + S2 (j1 + S1 j0).
* Basis at k (fractional, k_cart = B k): integer triples iG with
  (1/2) |B (iG + k)|^2 <= E_cut, ordered lexicographically by (i0, i1, i2).
* (I X)_j = sum_G X_G exp(+2 pi i iG.j/S);  (J x)_G = (1/N) sum_j x_j exp(-...).
  Idag = N J and Jdag = I / N (adjoints on the full box).  O = Omega * 1.
* H C = Omega [ (1/2)|k+G|^2 C + J(V . I C) ] + P D P^dag C.
* n(r_j) = sum_k w_k sum_b f_b |(I C_b)_j|^2.

Coefficient blocks are handled here as (npw, nbands) arrays (one column per
band); the binding's band-major device layout is its transpose.  "Parity
unpinned" applies to nothing in this module: every function is pinned by a
test against a closed form, a brute-force sum or a library routine.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import cfft

# --------------------------------------------------------------------------
# Lattice and basis
# --------------------------------------------------------------------------


def reciprocal(R: np.ndarray) -> np.ndarray:
    """B = 2 pi R^{-T}: columns are the reciprocal lattice vectors."""
    return 2.0 * np.pi * np.linalg.inv(np.asarray(R, dtype=np.float64)).T


def cell_volume(R: np.ndarray) -> float:
    return float(abs(np.linalg.det(np.asarray(R, dtype=np.float64))))


def sphere(R: np.ndarray, kfrac, ecut: float) -> np.ndarray:
    """Integer triples iG with (1/2)|B(iG+k)|^2 <= ecut, lexicographic (i0,i1,i2).

    Brute force over the bounding box: along axis d, (iG + k)_d = a_d . q / 2pi,
    so |iG_d + k_d| <= |a_d| |q| / 2pi <= |a_d| sqrt(2 ecut) / 2pi.
    """
    R = np.asarray(R, dtype=np.float64)
    k = np.asarray(kfrac, dtype=np.float64)
    B = reciprocal(R)
    qmax = np.sqrt(2.0 * ecut)
    lo, hi = [], []
    for d in range(3):
        reach = np.linalg.norm(R[:, d]) * qmax / (2.0 * np.pi)
        lo.append(int(np.floor(-reach - k[d])) - 1)
        hi.append(int(np.ceil(reach - k[d])) + 1)
    axes = [np.arange(lo[d], hi[d] + 1) for d in range(3)]
    g = np.stack(np.meshgrid(*axes, indexing="ij"), axis=-1).reshape(-1, 3)
    q = (g + k) @ B.T
    keep = 0.5 * np.einsum("ij,ij->i", q, q) <= ecut
    return g[keep].astype(np.int64)  # meshgrid 'ij' order is already lexicographic


def kvectors(R, kfrac, iG) -> np.ndarray:
    """Cartesian k+G (npw x 3)."""
    return (np.asarray(iG, dtype=np.float64) + np.asarray(kfrac, dtype=np.float64)) @ reciprocal(R).T


def kinetic(R, kfrac, iG) -> np.ndarray:
    """(1/2)|k+G|^2 per plane wave."""
    q = kvectors(R, kfrac, iG)
    return 0.5 * np.einsum("ij,ij->i", q, q)


def box_slots(iG, S) -> np.ndarray:
    """Linear box index of each sphere point: iG mod S, j2 fastest."""
    m = np.mod(np.asarray(iG), np.asarray(S))
    return (m[:, 0] * S[1] + m[:, 1]) * S[2] + m[:, 2]


def grid_points(R, S) -> np.ndarray:
    """Cartesian grid points r_j (N x 3) in linear-index order."""
    axes = [np.arange(S[d]) / S[d] for d in range(3)]
    f = np.stack(np.meshgrid(*axes, indexing="ij"), axis=-1).reshape(-1, 3)
    return f @ np.asarray(R, dtype=np.float64).T


def signed_box_frequencies(S) -> np.ndarray:
    """Integer frequency triple of every box slot, mapped into [-S/2, S/2)."""
    axes = [np.fft.fftfreq(S[d], 1.0 / S[d]).round().astype(np.int64) for d in range(3)]
    return np.stack(np.meshgrid(*axes, indexing="ij"), axis=-1).reshape(-1, 3)


# --------------------------------------------------------------------------
# Local potential: a sum of Gaussians per atom
# --------------------------------------------------------------------------


def vloc_realspace(R, S, atoms, depth: float = 4.0, width: float = 1.0,
                   image_cut: float = 10.0, method: str = "auto") -> np.ndarray:
    """V(r_j) = -depth sum_a sum_T exp(-|r_j - R_a - T|^2 / (2 width^2)).

    Atoms and grid points lie in the cell (fractional coordinates in [0, 1)),
    so an image T = R n can come within ``image_cut`` of a grid point only if
    |n_d| <= 1 + image_cut / h_d, h_d = 2 pi / |b_d| being the spacing of the
    lattice planes normal to b_d.  All those images are summed; terms farther
    than ``image_cut`` are dropped (below 1e-21 at the default width).
    For an orthorhombic cell the Gaussian factorises over the axes and the
    sum is taken axis by axis over the same block of images, keeping also its
    corner terms beyond ``image_cut`` (each below 1e-21); ``method="direct"``
    forces the point-by-point sum.  Returns a flat array in linear-index order.
    """
    R = np.asarray(R, dtype=np.float64)
    atoms = np.asarray(atoms, dtype=np.float64)
    B = reciprocal(R)
    nmax = [1 + int(np.ceil(image_cut * np.linalg.norm(B[:, d]) / (2 * np.pi))) for d in range(3)]
    inv2w2 = 1.0 / (2.0 * width * width)
    if method == "auto" and np.count_nonzero(R - np.diag(np.diag(R))) == 0:
        Ld = np.diag(R)
        V = np.zeros(tuple(S))
        for a in atoms:
            g = []
            for d in range(3):
                x = Ld[d] * np.arange(S[d]) / S[d]
                n = np.arange(-nmax[d], nmax[d] + 1)
                dx = x[:, None] - a[d] - n[None, :] * Ld[d]
                g.append(np.exp(-dx * dx * inv2w2).sum(axis=1))
            V -= depth * np.einsum("i,j,k->ijk", g[0], g[1], g[2])
        return V.reshape(-1)
    r = grid_points(R, S)
    V = np.zeros(r.shape[0])
    for a in atoms:
        for n0 in range(-nmax[0], nmax[0] + 1):
            for n1 in range(-nmax[1], nmax[1] + 1):
                for n2 in range(-nmax[2], nmax[2] + 1):
                    d = r - (a + R @ np.array([n0, n1, n2], dtype=np.float64))
                    d2 = np.einsum("ij,ij->i", d, d)
                    near = d2 < image_cut * image_cut
                    if near.any():
                        V[near] -= depth * np.exp(-d2[near] * inv2w2)
    return V


def vloc_fourier(R, S, atoms, depth: float = 4.0, width: float = 1.0) -> np.ndarray:
    """The same potential from its Fourier series, inverse-transformed on the box.

    V(r) = sum_G Vt(G) exp(i G.r) with
    Vt(G) = -(depth / Omega) (2 pi width^2)^{3/2} exp(-width^2 |G|^2 / 2) sum_a exp(-i G.R_a),
    summed over the box's signed frequencies (aliasing is below
    exp(-width^2 G_nyquist^2 / 2)).
    """
    R = np.asarray(R, dtype=np.float64)
    Omega = cell_volume(R)
    g = signed_box_frequencies(S)
    G = g.astype(np.float64) @ reciprocal(R).T
    G2 = np.einsum("ij,ij->i", G, G)
    struct = np.exp(-1j * (G @ np.asarray(atoms, dtype=np.float64).T)).sum(axis=1)
    Vt = -(depth / Omega) * (2 * np.pi * width * width) ** 1.5 * np.exp(-0.5 * width * width * G2) * struct
    box = Vt.reshape(S)
    return cfft.fft3d(box, +1).reshape(-1).real.copy()


# --------------------------------------------------------------------------
# Nonlocal projectors: Gaussian s and p channels per atom
# --------------------------------------------------------------------------

PROJ_PER_ATOM = 4          # s, p_x, p_y, p_z
D_PER_ATOM = (0.5, -0.3, -0.3, -0.3)


def projector_ft(q: np.ndarray, sigma: float = 1.0) -> np.ndarray:
    """F_l(q) = integral beta_l(r) exp(-i q.r) d^3r for l = s, p_x, p_y, p_z.

    beta_s = N_s exp(-r^2 / 2 sigma^2),  beta_p_x = N_p x exp(-r^2 / 2 sigma^2),
    each normalised to integral beta^2 = 1:  N_s = (pi sigma^2)^{-3/4},
    N_p = N_s sqrt(2) / sigma.  Closed forms:
      F_s(q)   = N_s (2 pi sigma^2)^{3/2} exp(-sigma^2 q^2 / 2)
      F_p_x(q) = -i sigma^2 q_x (N_p / N_s) F_s(q).
    Returns (npw x 4) complex.
    """
    Ns = (np.pi * sigma * sigma) ** -0.75
    Np = Ns * np.sqrt(2.0) / sigma
    q2 = np.einsum("ij,ij->i", q, q)
    Fs = Ns * (2 * np.pi * sigma * sigma) ** 1.5 * np.exp(-0.5 * sigma * sigma * q2)
    out = np.empty((q.shape[0], 4), dtype=np.complex128)
    out[:, 0] = Fs
    for d in range(3):
        out[:, 1 + d] = -1j * sigma * sigma * q[:, d] * (Np / Ns) * Fs
    return out


def projectors(R, kfrac, iG, atoms, sigma: float = 1.0) -> np.ndarray:
    """P (npw x 4 natoms): column (a, l) = F_l(k+G) exp(-i (k+G).R_a).

    With this P, (P^dag C)_{(a,l), b} = integral beta_l(r - R_a) psi_b(r) d^3r
    over all space, psi_b(r) = sum_G C_Gb exp(i (k+G).r).  Columns are
    atom-major: 4a + {0: s, 1: p_x, 2: p_y, 3: p_z}.
    """
    q = kvectors(R, kfrac, iG)
    F = projector_ft(q, sigma)
    atoms = np.asarray(atoms, dtype=np.float64)
    P = np.empty((q.shape[0], PROJ_PER_ATOM * atoms.shape[0]), dtype=np.complex128)
    for a in range(atoms.shape[0]):
        phase = np.exp(-1j * (q @ atoms[a]))
        P[:, 4 * a:4 * a + 4] = F * phase[:, None]
    return P


def dmatrix(natoms: int) -> np.ndarray:
    """Block-diagonal D: diag(0.5, -0.3, -0.3, -0.3) Ha per atom."""
    return np.diag(np.tile(np.asarray(D_PER_ATOM, dtype=np.float64), natoms))


# --------------------------------------------------------------------------
# The algebraic operators
# --------------------------------------------------------------------------


def _scatter(iG, S, C):
    """Box of shape (nb, S0, S1, S2) holding C[G, b] at slot iG mod S, zero elsewhere."""
    C = np.asarray(C)
    nb = C.shape[1]
    box = np.zeros((nb, int(np.prod(S))), dtype=np.complex128)
    box[:, box_slots(iG, S)] = C.T
    return box.reshape((nb,) + tuple(S))


def _gather(iG, S, boxes):
    """(npw, nb) values of boxes (nb, S0, S1, S2) at the sphere's slots."""
    nb = boxes.shape[0]
    return boxes.reshape(nb, -1)[:, box_slots(iG, S)].T.copy()


def op_I(iG, S, C) -> np.ndarray:
    """psi = I C: (nb, S0, S1, S2), sum_G C_G exp(+2 pi i iG.j / S)."""
    return cfft.fft3d(_scatter(iG, S, C), +1)


def op_Jdag(iG, S, C) -> np.ndarray:
    """Jdag C = I C / N."""
    return op_I(iG, S, C) / float(np.prod(S))


def op_J(iG, S, psi) -> np.ndarray:
    """(J psi)_G = (1/N) sum_j psi_j exp(-2 pi i iG.j / S), restricted to the sphere."""
    psi = np.asarray(psi, dtype=np.complex128).reshape((-1,) + tuple(S))
    return _gather(iG, S, cfft.fft3d(psi, -1)) / float(np.prod(S))


def op_Idag(iG, S, psi) -> np.ndarray:
    """Idag psi = N J psi (the unnormalised forward sum)."""
    return op_J(iG, S, psi) * float(np.prod(S))


def op_O(Omega: float, C) -> np.ndarray:
    """O C = Omega C (norm-conserving overlap, diagonal in the basis)."""
    return Omega * np.asarray(C)


@dataclass
class Basis:
    """One cell at one k-point: everything the operators need."""
    R: np.ndarray
    S: tuple
    kfrac: np.ndarray
    iG: np.ndarray
    Omega: float
    T: np.ndarray          # (1/2)|k+G|^2

    @classmethod
    def build(cls, R, S, kfrac, ecut) -> "Basis":
        R = np.asarray(R, dtype=np.float64)
        k = np.asarray(kfrac, dtype=np.float64)
        iG = sphere(R, k, ecut)
        return cls(R, tuple(int(s) for s in S), k, iG, cell_volume(R), kinetic(R, k, iG))

    @property
    def npw(self) -> int:
        return self.iG.shape[0]

    @property
    def N(self) -> int:
        return int(np.prod(self.S))


def apply_H(basis: Basis, V, C, P=None, D=None) -> np.ndarray:
    """H C = Omega [T C + J(V . I C)] + P D P^dag C   (C: npw x nb)."""
    C = np.asarray(C, dtype=np.complex128)
    psi = op_I(basis.iG, basis.S, C)
    phi = psi * np.asarray(V, dtype=np.float64).reshape(basis.S)[None]
    HC = basis.Omega * (basis.T[:, None] * C + op_J(basis.iG, basis.S, phi))
    if P is not None:
        HC = HC + P @ (np.asarray(D) @ (P.conj().T @ C))
    return HC


def density(basis: Basis, C, f, weight: float = 1.0) -> np.ndarray:
    """n(r_j) = weight sum_b f_b |(I C_b)_j|^2, flat in linear-index order."""
    psi = op_I(basis.iG, basis.S, C)
    f = np.asarray(f, dtype=np.float64)
    return weight * np.einsum("b,bj->j", f, (psi.real ** 2 + psi.imag ** 2).reshape(len(f), -1))


def subspace(basis: Basis, C, HC):
    """(C^dag H C, C^dag O C) as full Hermitian nb x nb matrices."""
    C = np.asarray(C, dtype=np.complex128)
    return C.conj().T @ HC, basis.Omega * (C.conj().T @ C)


def potential_ft(S, V) -> np.ndarray:
    """Vt = J V on the full box (S0, S1, S2), by the direct per-axis transform."""
    return cfft.fft3d(np.asarray(V, dtype=np.complex128).reshape(S), -1) / float(np.prod(S))


def dense_H(basis: Basis, V, P=None, D=None, Vt=None) -> np.ndarray:
    """Dense H (npw x npw): Omega [T delta_GG' + Vt((G - G') mod S)] + P D P^dag.

    With it, apply_H(C) = dense_H @ C exactly (up to rounding) for any box
    large enough that the sphere's slots are distinct, and the band energies
    are the eigenvalues of the pencil (H, Omega 1).
    """
    if Vt is None:
        Vt = potential_ft(basis.S, V)
    S = basis.S
    m = [np.mod(basis.iG[:, None, d] - basis.iG[None, :, d], S[d]) for d in range(3)]
    H = basis.Omega * Vt.reshape(-1)[(m[0] * S[1] + m[1]) * S[2] + m[2]]
    H[np.diag_indices_from(H)] += basis.Omega * basis.T
    if P is not None:
        H = H + P @ np.asarray(D) @ P.conj().T
    return H


def lowdin(C, Omega: float) -> np.ndarray:
    """C (C^dag O C)^{-1/2}: the symmetric (Loewdin) orthonormalisation."""
    U = Omega * (C.conj().T @ C)
    w, Q = np.linalg.eigh(U)
    return C @ (Q @ np.diag(w ** -0.5) @ Q.conj().T)


def column_structure(iG):
    """Disk columns of a lexicographic sphere.

    Returns (pairs, start, count, i2lo): the distinct (i0, i1) pairs in order,
    each column's first index into the sphere, its length, and its lowest i2.
    Each column's i2 values are consecutive because the sphere meets a line in
    an interval.
    """
    iG = np.asarray(iG)
    key = iG[:, :2]
    change = np.ones(iG.shape[0], dtype=bool)
    change[1:] = np.any(key[1:] != key[:-1], axis=1)
    start = np.flatnonzero(change)
    count = np.diff(np.append(start, iG.shape[0]))
    return key[start].copy(), start, count, iG[start, 2].copy()
