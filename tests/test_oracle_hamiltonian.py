"""Pins of the oracle's operators, Hamiltonian, density and subspace (CPU).

The operators I, J, O and the pointwise multiply are those of the JDFTx
paper's algebraic formulation (Sec. 2.1); the Hamiltonian they build is the
Kohn-Sham one of the plane-wave method (Sec. 2), with the nonlocal projector
term of the pseudopotentials (Sec. 2.2).  Pins: plane-wave closed forms, the
adjoint relations, the free-electron spectrum, the analytic matrix elements of
a single-cosine potential and its spectrum as a union of tridiagonal chains
(LAPACK), a rank-one secular equation for a single
projector, Hermiticity, the k -> -k and grid-translation symmetries of the
spectrum, a brute-force dense Hamiltonian built from a direct O(N^2) DFT,
direct real-space sums for the density, and the Loewdin orthonormalisation's
closed forms and minimal-distance property.
"""
import numpy as np
import pytest

from oracle import cfft
from oracle import planewave as pw
from synth import atom_positions, random_coefficients

rng = np.random.default_rng(5)


def tiny_system(R=None, S=(12, 12, 12), k=(0.1, 0.2, 0.3), ecut=4.0, natoms=2, seed=1):
    R = np.eye(3) * 6.0 if R is None else np.asarray(R, float)
    basis = pw.Basis.build(R, S, k, ecut)
    atoms = atom_positions(R, natoms, seed)
    V = pw.vloc_realspace(R, S, atoms)
    P = pw.projectors(R, basis.kfrac, basis.iG, atoms)
    D = pw.dmatrix(natoms)
    return basis, atoms, V, P, D


def rand_block(basis, nb, seed=3):
    return random_coefficients(2 * basis.T, nb, seed).T.copy()


def test_I_of_single_coefficient_is_plane_wave():
    basis, *_ = tiny_system()
    g = 17
    C = np.zeros((basis.npw, 1), complex)
    C[g, 0] = 1.0
    psi = pw.op_I(basis.iG, basis.S, C)[0]
    j = np.stack(np.meshgrid(*[np.arange(s) for s in basis.S], indexing="ij"), -1)
    phase = sum(basis.iG[g, d] * j[..., d] / basis.S[d] for d in range(3))
    assert np.max(np.abs(psi - np.exp(2j * np.pi * phase))) < 1e-13


def test_J_inverts_I_and_adjoints():
    basis, *_ = tiny_system(S=(12, 10, 14), R=np.diag([6.0, 5.0, 7.0]))
    C = rand_block(basis, 3)
    psi = pw.op_I(basis.iG, basis.S, C)
    assert np.max(np.abs(pw.op_J(basis.iG, basis.S, psi) - C)) < 1e-14
    x = rng.standard_normal((3,) + basis.S) + 1j * rng.standard_normal((3,) + basis.S)
    # <x, I C> = <Idag x, C> and <x, Jdag C> = <J x, C>
    lhs = np.vdot(x.reshape(3, -1), psi.reshape(3, -1))
    rhs = np.vdot(pw.op_Idag(basis.iG, basis.S, x), C)
    assert abs(lhs - rhs) < 1e-10 * abs(lhs)
    lhs2 = np.vdot(x, pw.op_Jdag(basis.iG, basis.S, C))
    rhs2 = np.vdot(pw.op_J(basis.iG, basis.S, x), C)
    assert abs(lhs2 - rhs2) < 1e-10 * abs(lhs2)


def test_parseval_normalisation():
    basis, *_ = tiny_system()
    C = pw.lowdin(rand_block(basis, 4), basis.Omega)
    psi = pw.op_I(basis.iG, basis.S, C)
    norms = basis.Omega / basis.N * np.sum(np.abs(psi.reshape(4, -1)) ** 2, axis=1)
    assert np.allclose(norms, 1.0, atol=1e-13)
    assert np.allclose(pw.subspace(basis, C, C)[1], np.eye(4), atol=1e-13)


def test_apply_H_equals_bruteforce_dense_matrix():
    """Dense H from a direct O(N^2) DFT of V (no factorised transform involved)."""
    basis, atoms, V, P, D = tiny_system(S=(10, 12, 11), R=np.diag([5.5, 6.0, 5.8]))
    Vt = cfft.dft3d_direct(V.reshape(basis.S).astype(complex), -1) / basis.N
    H = pw.dense_H(basis, V, P, D, Vt=Vt)
    C = rand_block(basis, 5)
    HC = pw.apply_H(basis, V, C, P, D)
    assert np.max(np.abs(HC - H @ C)) < 1e-12 * np.max(np.abs(HC))
    assert np.max(np.abs(H - H.conj().T)) < 1e-13 * np.max(np.abs(H))


def test_free_electron_spectrum():
    basis, *_ = tiny_system(R=np.diag([6.0, 7.0, 5.0]), S=(12, 14, 10))
    V0 = np.zeros(basis.N)
    H = pw.dense_H(basis, V0)
    eps = np.linalg.eigvalsh(H / basis.Omega)
    # closed form: 1/2 |k+G|^2 with k+G = 2 pi (iG + k) / L on this orthorhombic cell
    L = np.array([6.0, 7.0, 5.0])
    exact = np.sort(0.5 * np.sum((2 * np.pi * (basis.iG + basis.kfrac) / L) ** 2, 1))
    assert np.max(np.abs(eps - exact)) < 1e-12
    C = rand_block(basis, 2)
    assert np.allclose(pw.apply_H(basis, V0, C), basis.Omega * exact_T(basis, L)[:, None] * C, atol=1e-12)


def exact_T(basis, L):
    return 0.5 * np.sum((2 * np.pi * (basis.iG + basis.kfrac) / L) ** 2, 1)


def test_single_cosine_matrix_elements():
    """V = 2 V0 cos(b_1 . r): <G|V|G'> = V0 iff G - G' = +-b_1, else 0."""
    R = np.diag([6.0, 6.5, 5.5])
    S = (12, 13, 11)
    basis = pw.Basis.build(R, S, (0.1, 0.2, 0.3), 4.0)
    r = pw.grid_points(R, S)
    b1 = pw.reciprocal(R)[:, 1]
    V0 = 0.37
    V = 2 * V0 * np.cos(r @ b1)
    H = pw.dense_H(basis, V)
    diffG = basis.iG[:, None, :] - basis.iG[None, :, :]
    plus = np.all(diffG == np.array([0, 1, 0]), -1) | np.all(diffG == np.array([0, -1, 0]), -1)
    off = H / basis.Omega - np.diag(basis.T)
    assert np.max(np.abs(off[plus] - V0)) < 1e-13
    assert np.max(np.abs(off[~plus])) < 1e-13
    C = rand_block(basis, 2)
    assert np.max(np.abs(pw.apply_H(basis, V, C) - H @ C)) < 1e-12 * np.max(np.abs(H @ C))


def test_single_projector_secular_equation():
    """V = 0, one s projector with weight d: eigenvalues solve 1 + (d/Omega) sum |p|^2/(T - e) = 0."""
    R = np.diag([6.0, 6.0, 6.0])
    basis = pw.Basis.build(R, (12, 12, 12), (0.1, 0.2, 0.3), 4.0)
    atom = np.array([[1.0, 2.0, 3.0]])
    p = pw.projectors(R, basis.kfrac, basis.iG, atom)[:, :1]
    d = -0.7
    H = pw.dense_H(basis, np.zeros(basis.N), p, np.array([[d]]))
    eps = np.linalg.eigvalsh(H / basis.Omega)
    w = np.abs(p[:, 0]) ** 2
    T = basis.T
    # the lowest eigenvalue lies below min T and is a root of the secular function
    e0 = eps[0]
    assert e0 < T.min()
    f = 1 + (d / basis.Omega) * np.sum(w / (T - e0))
    df = (d / basis.Omega) * np.sum(w / (T - e0) ** 2)
    assert abs(f / df) < 1e-10


def test_hermiticity_of_apply_H():
    basis, atoms, V, P, D = tiny_system(S=(12, 12, 12))
    X = rand_block(basis, 3, 8)
    Y = rand_block(basis, 3, 9)
    a = np.vdot(X, pw.apply_H(basis, V, Y, P, D))
    b = np.vdot(pw.apply_H(basis, V, X, P, D), Y)
    assert abs(a - b) < 1e-13 * abs(a)


def test_time_reversal_spectrum():
    R = np.diag([6.0, 5.5, 6.5])
    S = (12, 11, 13)
    atoms = atom_positions(R, 2, 4)
    V = pw.vloc_realspace(R, S, atoms)
    spectra = []
    for k in ((0.1, 0.2, 0.3), (-0.1, -0.2, -0.3)):
        b = pw.Basis.build(R, S, k, 4.0)
        P = pw.projectors(R, b.kfrac, b.iG, atoms)
        spectra.append(np.linalg.eigvalsh(pw.dense_H(b, V, P, pw.dmatrix(2)) / b.Omega))
    assert np.max(np.abs(spectra[0] - spectra[1])) < 1e-12


def test_grid_translation_leaves_spectrum():
    R = np.diag([6.0, 6.0, 6.0])
    S = (12, 12, 12)
    basis = pw.Basis.build(R, S, (0.1, 0.2, 0.3), 4.0)
    atoms = atom_positions(R, 2, 6)
    shift = R @ (np.array([3, 5, 2]) / np.array(S))
    out = []
    for a in (atoms, atoms + shift):
        V = pw.vloc_realspace(R, S, a)
        P = pw.projectors(R, basis.kfrac, basis.iG, a)
        out.append(np.linalg.eigvalsh(pw.dense_H(basis, V, P, pw.dmatrix(2)) / basis.Omega))
    assert np.max(np.abs(out[0] - out[1])) < 1e-12


def test_density_direct_sum_and_invariances():
    basis, atoms, V, P, D = tiny_system(S=(12, 12, 12))
    C = pw.lowdin(rand_block(basis, 4), basis.Omega)
    f = np.array([2.0, 2.0, 1.0, 0.5])
    n = pw.density(basis, C, f)
    # integral of n = sum f for orthonormal bands
    assert np.isclose(basis.Omega / basis.N * n.sum(), f.sum(), rtol=1e-13)
    # direct evaluation of |u_b(r_j)|^2 at a few grid points
    for j in (0, 77, 1000):
        jj = np.array(np.unravel_index(j, basis.S))
        u = np.exp(2j * np.pi * (basis.iG @ (jj / np.array(basis.S)))) @ C
        assert np.isclose(n[j], np.sum(f * np.abs(u) ** 2), rtol=1e-12)
    # invariance under a unitary rotation of equally occupied bands
    fe = np.full(4, 2.0)
    Q, _ = np.linalg.qr(rng.standard_normal((4, 4)) + 1j * rng.standard_normal((4, 4)))
    assert np.max(np.abs(pw.density(basis, C, fe) - pw.density(basis, C @ Q, fe))) < 1e-13 * np.max(n)


def test_subspace_trace_invariance_and_hermitian():
    basis, atoms, V, P, D = tiny_system()
    C = pw.lowdin(rand_block(basis, 5), basis.Omega)
    CHC, COC = pw.subspace(basis, C, pw.apply_H(basis, V, C, P, D))
    assert np.max(np.abs(CHC - CHC.conj().T)) < 1e-13 * np.max(np.abs(CHC))
    Q, _ = np.linalg.qr(rng.standard_normal((5, 5)) + 1j * rng.standard_normal((5, 5)))
    C2 = C @ Q
    CHC2, _ = pw.subspace(basis, C2, pw.apply_H(basis, V, C2, P, D))
    assert np.isclose(np.trace(CHC).real, np.trace(CHC2).real, rtol=1e-13)
    assert np.allclose(COC, np.eye(5), atol=1e-13)


def test_rayleigh_ritz_bounds_exact_eigenvalues():
    """Subspace eigenvalues of the pencil (C^dag H C, C^dag O C) are upper bounds
    of the lowest exact ones (Courant-Fischer), and equal them on the exact
    eigenvectors."""
    basis, atoms, V, P, D = tiny_system()
    H = pw.dense_H(basis, V, P, D)
    ex, X = np.linalg.eigh(H / basis.Omega)
    C = pw.lowdin(rand_block(basis, 3), basis.Omega)
    CHC, COC = pw.subspace(basis, C, pw.apply_H(basis, V, C, P, D))
    ritz = np.sort(np.linalg.eigvals(np.linalg.solve(COC, CHC)).real)
    assert np.all(ritz >= ex[:3] - 1e-12)
    Cx = X[:, :3] / np.sqrt(basis.Omega)
    CHCx, COCx = pw.subspace(basis, Cx, pw.apply_H(basis, V, Cx, P, D))
    assert np.allclose(np.sort(np.linalg.eigvalsh(CHCx)), ex[:3], atol=1e-12)


def test_single_cosine_spectrum_is_union_of_tridiagonal_chains():
    """V = 2 V0 cos(b_1 . r) couples only plane waves that differ by b_1, so H
    splits into one chain per line of the sphere along b_1: a tridiagonal
    (Mathieu-type) matrix with diagonal 1/2 |k+G|^2 and off-diagonal V0.
    LAPACK's tridiagonal eigensolver on those chains, with the kinetic
    energies written out for this orthorhombic cell, fixes the whole spectrum;
    the oracle's dense H and its band minimiser (through the FFT apply_H) must
    reproduce it."""
    from scipy.linalg import eigh_tridiagonal

    from oracle import minimize as mn

    L = np.array([6.0, 6.5, 5.5])
    S = (12, 13, 11)
    kfrac = np.array([0.1, 0.2, 0.3])
    basis = pw.Basis.build(np.diag(L), S, kfrac, 4.0)
    b1 = 2 * np.pi / L[1] * np.array([0.0, 1.0, 0.0])
    V0 = 0.37
    V = 2 * V0 * np.cos(pw.grid_points(np.diag(L), S) @ b1)
    T = 0.5 * np.sum((2 * np.pi * (basis.iG + kfrac) / L) ** 2, 1)
    chains = {}
    for g, (i0, i1, i2) in enumerate(basis.iG):
        chains.setdefault((i0, i2), []).append((i1, g))
    eigs = []
    for members in chains.values():
        members.sort()
        i1 = [m[0] for m in members]
        assert i1 == list(range(i1[0], i1[0] + len(i1)))  # a line through a ball is one run
        d = T[[m[1] for m in members]]
        eigs.extend(eigh_tridiagonal(d, np.full(len(d) - 1, V0), eigvals_only=True) if len(d) > 1 else d)
    eigs = np.sort(eigs)
    assert len(eigs) == basis.npw
    dense = np.linalg.eigvalsh(pw.dense_H(basis, V) / basis.Omega)
    assert np.max(np.abs(dense - eigs)) < 1e-12
    nb = 6
    assert eigs[nb] - eigs[nb - 1] > 1e-2
    res = mn.minimize_bands(basis, lambda X: pw.apply_H(basis, V, X), rand_block(basis, nb, 11),
                            precond=mn.precond_teter, tol=1e-10, max_iter=1000)
    assert res.converged
    assert np.max(np.abs(np.sort(res.eigs) - eigs[:nb])) < 1e-12


def test_lowdin_closed_forms_and_minimal_distance():
    """Loewdin orthonormalisation C (C^dag O C)^{-1/2}, O = Omega: one column is
    just normalised; mutually orthogonal columns are each normalised; in
    general the result is O-orthonormal, C^dag O C_L is Hermitian positive
    definite (C_L = C times a positive matrix), and no other O-orthonormal basis
    of the same span (C_L W, W unitary) is closer to C."""
    Om = 3.7
    x = rng.standard_normal((40, 1)) + 1j * rng.standard_normal((40, 1))
    assert np.allclose(pw.lowdin(x, Om), x / np.sqrt(Om * np.vdot(x, x).real), atol=1e-14)
    Q, _ = np.linalg.qr(rng.standard_normal((40, 3)) + 1j * rng.standard_normal((40, 3)))
    D = Q * np.array([0.3, 2.0, 5.0])
    assert np.allclose(pw.lowdin(D, Om), Q / np.sqrt(Om), atol=1e-13)
    C = rng.standard_normal((40, 4)) + 1j * rng.standard_normal((40, 4))
    L = pw.lowdin(C, Om)
    assert np.allclose(Om * L.conj().T @ L, np.eye(4), atol=1e-13)
    G = Om * C.conj().T @ L
    assert np.allclose(G, G.conj().T, atol=1e-12) and np.all(np.linalg.eigvalsh(G) > 0)
    d0 = np.linalg.norm(L - C)
    for _ in range(20):
        W, _ = np.linalg.qr(rng.standard_normal((4, 4)) + 1j * rng.standard_normal((4, 4)))
        assert np.linalg.norm(L @ W - C) >= d0 - 1e-12
