"""Pins of the spinor oracle (oracle/spinor.py): reduction to the scalar
operator, the Zeeman splitting of a uniform field, Hermiticity, covariance
under spin rotations (with the rotation built from traces of Pauli matrices),
and the density and magnetisation of rotated spin states."""
from __future__ import annotations

import numpy as np

from oracle import planewave as pw
from oracle import spinor
from synth import atom_positions, random_coefficients

R = np.diag([6.0, 6.5, 5.5])
S = (12, 15, 10)
K = (0.1, 0.2, 0.3)
ECUT = 3.0
PAULI = [np.array([[0, 1], [1, 0]], dtype=complex), np.array([[0, -1j], [1j, 0]]),
         np.array([[1, 0], [0, -1]], dtype=complex)]


def _system(seed=3):
    b = pw.Basis.build(R, S, K, ECUT)
    atoms = atom_positions(R, 2, seed)
    V = pw.vloc_realspace(R, S, atoms)
    P = pw.projectors(R, b.kfrac, b.iG, atoms)
    return b, V, P, pw.dmatrix(2)


def _field(seed):
    rng = np.random.default_rng(seed)
    r = pw.grid_points(R, S)
    B = pw.reciprocal(R)
    M = np.empty((3, r.shape[0]))
    for c in range(3):
        G = B @ rng.integers(-2, 3, size=3)
        M[c] = 0.3 * rng.normal() + 0.2 * np.cos(r @ G + rng.normal())
    return M


def _block(b, nb, seed):
    return random_coefficients(2 * b.T, 2 * nb, seed).T      # (npw, 2 nb), columns up, down, up, ...


def _su2(theta, axis):
    n = np.asarray(axis, float) / np.linalg.norm(axis)
    return np.cos(theta / 2) * np.eye(2) - 1j * np.sin(theta / 2) * sum(n[i] * PAULI[i] for i in range(3))


def _so3(U):
    """R_jk = (1/2) tr(sigma_j U sigma_k U^dag)."""
    return np.array([[0.5 * np.trace(PAULI[j] @ U @ PAULI[k] @ U.conj().T).real for k in range(3)]
                     for j in range(3)])


def _rotate_block(U, C):
    out = np.empty_like(C)
    out[:, 0::2] = U[0, 0] * C[:, 0::2] + U[0, 1] * C[:, 1::2]
    out[:, 1::2] = U[1, 0] * C[:, 0::2] + U[1, 1] * C[:, 1::2]
    return out


def test_zero_field_is_the_scalar_operator_on_each_component():
    b, V, P, D = _system()
    C = _block(b, 3, 5)
    got = spinor.apply_H_spinor(b, V, np.zeros((3, b.N)), C, P, D)
    assert np.max(np.abs(got - pw.apply_H(b, V, C, P, D))) < 1e-13 * np.max(np.abs(got))


def test_uniform_field_splits_every_level_by_plus_minus_its_magnitude():
    """M uniform: H = H0 x 1 + Omega (m.sigma), so the pencil's eigenvalues are eps_n -+ |m|."""
    b, V, P, D = _system()
    m0 = np.array([0.05, -0.12, 0.08])
    M = np.repeat(m0[:, None], b.N, axis=1)
    n2 = 2 * b.npw
    # dense spinor matrix, index 2g + s for plane wave g and component s
    Hs = np.zeros((n2, n2), dtype=complex)
    for g in range(b.npw):
        for s in range(2):
            C = np.zeros((b.npw, 2), dtype=complex)
            C[g, s] = 1.0
            out = spinor.apply_H_spinor(b, V, M, C, P, D)    # one spinor band: (up, down) columns
            Hs[0::2, 2 * g + s] = out[:, 0]
            Hs[1::2, 2 * g + s] = out[:, 1]
    w = np.linalg.eigvalsh(0.5 * (Hs + Hs.conj().T)) / b.Omega
    e0 = np.linalg.eigvalsh(pw.dense_H(b, V, P, D)) / b.Omega
    want = np.sort(np.concatenate([e0 - np.linalg.norm(m0), e0 + np.linalg.norm(m0)]))
    assert np.max(np.abs(w - want)) < 1e-11


def test_spinor_operator_is_hermitian():
    b, V, P, D = _system()
    M = _field(7)
    X, Y = _block(b, 2, 8), _block(b, 2, 9)
    HX = spinor.apply_H_spinor(b, V, M, X, P, D)
    HY = spinor.apply_H_spinor(b, V, M, Y, P, D)
    lhs = np.sum(np.conj(Y) * HX)
    rhs = np.sum(np.conj(HY) * X)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_operator_is_covariant_under_spin_rotations():
    """H[R M](U C) = U (H[M] C) for U in SU(2) and R its rotation (from Pauli traces)."""
    b, V, P, D = _system()
    M = _field(11)
    C = _block(b, 2, 12)
    U = _su2(0.9, (0.3, -0.5, 0.8))
    Rm = _so3(U)
    lhs = spinor.apply_H_spinor(b, V, Rm @ M, _rotate_block(U, C), P, D)
    rhs = _rotate_block(U, spinor.apply_H_spinor(b, V, M, C, P, D))
    assert np.max(np.abs(lhs - rhs)) < 1e-12 * np.max(np.abs(rhs))


def test_density_and_magnetisation_of_rotated_spin_states():
    """Spin-up bands: m = (0, 0, n).  Rotated by U: m = n R e_z, and the total
    density is the scalar density of both components."""
    b, V, P, D = _system()
    C = _block(b, 3, 13)
    C[:, 1::2] = 0.0
    f = np.array([2.0, 1.0, 0.5])
    n, m = spinor.density_spinor(b, C, f)
    assert np.max(np.abs(m[2] - n)) < 1e-14 * np.max(n) and np.max(np.abs(m[:2])) < 1e-14 * np.max(n)
    U = _su2(1.3, (1.0, 2.0, -0.5))
    n2, m2 = spinor.density_spinor(b, _rotate_block(U, C), f)
    want = _so3(U)[:, 2][:, None] * n[None, :]
    assert np.max(np.abs(n2 - n)) < 1e-13 * np.max(n)
    assert np.max(np.abs(m2 - want)) < 1e-13 * np.max(n)
    Cr = _rotate_block(U, C)
    scalar = pw.density(b, Cr, np.repeat(f, 2))
    assert np.max(np.abs(n2 - scalar)) < 1e-13 * np.max(n)
