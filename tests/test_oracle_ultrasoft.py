"""Pins of the augmented-overlap oracle (oracle/ultrasoft.py): the
norm-conserving limit, the generalised secular equation of one augmented
projector in a free-electron basis, exact generalised Rayleigh-Ritz on an
invariant subspace, invariance under a change of basis, and S-orthonormality."""
from __future__ import annotations

import numpy as np
import scipy.linalg
import scipy.optimize

from oracle import planewave as pw
from oracle import ultrasoft as us
from synth import atom_positions, random_coefficients

R = np.diag([6.0, 6.5, 5.5])
S = (12, 15, 10)
K = (0.1, 0.2, 0.3)


def _system(ecut=3.0):
    b = pw.Basis.build(R, S, K, ecut)
    atoms = atom_positions(R, 2, 3)
    V = pw.vloc_realspace(R, S, atoms)
    P = pw.projectors(R, b.kfrac, b.iG, atoms)
    D = pw.dmatrix(2)
    Q = np.diag(np.tile([0.4, 0.1, 0.1, 0.1], 2))
    Q[0, 4] = Q[4, 0] = 0.05
    return b, V, P, D, Q


def test_zero_augmentation_is_the_plain_overlap():
    b, V, P, D, Q = _system()
    C = random_coefficients(2 * b.T, 4, 5).T
    assert np.max(np.abs(us.op_S(b, C, P, 0 * Q) - b.Omega * C)) < 1e-15 * np.max(np.abs(b.Omega * C))


def test_one_augmented_projector_obeys_the_generalised_secular_equation():
    """H = Omega T (free electrons), S = Omega + q p p^dag: every eigenvalue l of the
    pencil that is not a free level solves 1 = l q sum_G |p_G|^2 / (Omega (T_G - l))."""
    b, V, P, D, Q = _system(ecut=2.0)
    p = P[:, 0]
    q = 0.7
    Hd = np.diag(b.Omega * b.T).astype(complex)
    Sd = us.dense_S(b, P[:, :1], np.array([[q]]))
    lam = scipy.linalg.eigh(Hd, Sd, eigvals_only=True)
    w = np.abs(p) ** 2 / b.Omega
    T = b.T
    levels = np.unique(np.round(T, 12))

    def f(x):
        return 1.0 - x * q * np.sum(w / (T - x))

    roots = []
    for lo, hi in zip(levels[:-1], levels[1:]):
        a, c = lo + 1e-9, hi - 1e-9
        if f(a) * f(c) < 0:
            roots.append(scipy.optimize.brentq(f, a, c, xtol=1e-14, rtol=1e-15))
    # below the lowest level (the augmentation pulls one state down)
    a, c = -50.0, levels[0] - 1e-9
    if f(a) * f(c) < 0:
        roots.append(scipy.optimize.brentq(f, a, c, xtol=1e-14, rtol=1e-15))
    roots = np.sort(roots)
    assert len(roots) >= 5
    for x in roots:
        assert np.min(np.abs(lam - x)) < 1e-9


def test_rayleigh_ritz_on_an_invariant_subspace_is_exact():
    b, V, P, D, Q = _system()
    H = pw.dense_H(b, V, P, D)
    Sd = us.dense_S(b, P, Q)
    lam, X = scipy.linalg.eigh(H, Sd)
    C = X[:, :6] @ (np.eye(6) + 0.3 * np.random.default_rng(1).normal(size=(6, 6)))   # any basis of the span
    A, B, eigs = us.subspace_generalized(b, C, H @ C, P, Q)
    assert np.max(np.abs(eigs - lam[:6])) < 1e-10
    # and op_S agrees with the dense overlap
    assert np.max(np.abs(us.op_S(b, C, P, Q) - Sd @ C)) < 1e-12 * np.max(np.abs(Sd @ C))


def test_subspace_eigenvalues_do_not_depend_on_the_basis_of_the_block():
    b, V, P, D, Q = _system()
    C = random_coefficients(2 * b.T, 5, 6).T
    HC = pw.apply_H(b, V, C, P, D)
    Xm = np.random.default_rng(2).normal(size=(5, 5)) + 1j * np.random.default_rng(3).normal(size=(5, 5))
    e1 = us.subspace_generalized(b, C, HC, P, Q)[2]
    e2 = us.subspace_generalized(b, C @ Xm, HC @ Xm, P, Q)[2]
    assert np.max(np.abs(e1 - e2)) < 1e-10 * np.max(np.abs(e1))


def test_orthonormalised_block_is_S_orthonormal_with_the_same_span():
    b, V, P, D, Q = _system()
    C = random_coefficients(2 * b.T, 5, 7).T
    Co = us.orthonormalize_generalized(b, C, P, Q)
    assert np.max(np.abs(Co.conj().T @ us.op_S(b, Co, P, Q) - np.eye(5))) < 1e-12
    # same span: the projector onto span(C) is unchanged
    Pc = C @ np.linalg.pinv(C)
    assert np.max(np.abs(Pc @ Co - Co)) < 1e-10 * np.max(np.abs(Co))


def test_generalised_minimiser_finds_the_lowest_pencil_eigenvalues():
    """Converged bands span the lowest nb eigenvectors of the dense pencil (H, S):
    their Rayleigh-Ritz values are LAPACK's lowest generalised eigenvalues."""
    b, V, P, D, Q = _system()
    Sd = us.dense_S(b, P, Q)
    H = pw.dense_H(b, V, P, D)
    lam = scipy.linalg.eigh(H, Sd, eigvals_only=True)
    C0 = random_coefficients(2 * b.T, 5, 9).T
    C, eigs, it, res = us.minimize_bands_generalized(b, lambda X: pw.apply_H(b, V, X, P, D), P, Q, C0, tol=1e-9)
    assert res < 1e-9
    assert np.max(np.abs(eigs - lam[:5])) < 1e-12 * max(1.0, np.max(np.abs(lam[:5]))) + 1e-13
    assert np.max(np.abs(C.conj().T @ us.op_S(b, C, P, Q) - np.eye(5))) < 1e-10


def test_generalised_minimiser_without_augmentation_is_the_plain_one():
    from oracle import minimize as mz
    b, V, P, D, Q = _system()
    C0 = random_coefficients(2 * b.T, 5, 10).T
    Hap = lambda X: pw.apply_H(b, V, X, P, D)  # noqa: E731
    _, e1, _, _ = us.minimize_bands_generalized(b, Hap, P, 0 * Q, C0, tol=1e-9)
    e2 = mz.minimize_bands(b, Hap, C0, tol=1e-9).eigs
    assert np.max(np.abs(e1 - e2)) < 1e-12
