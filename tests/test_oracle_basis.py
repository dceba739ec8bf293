"""Pins of the oracle's lattice, basis, local potential and projectors (CPU).

The plane-wave basis follows from the `elec-cutoff` setting of the paper's
input file (Sec. 3, Listing 2) and the plane-wave formulation (Sec. 2); the
local potential and the Gaussian projectors are the synthetic stand-ins for
the pseudopotentials of Sec. 2.2.  Each construction is pinned to an
independent one: definitions of the reciprocal lattice, symmetry and shift
properties of the sphere, a Fourier-series construction of the potential and
its closed-form mean, and direct real-space quadrature of the projector
overlaps.
"""
import numpy as np
import pytest

from oracle import planewave as pw
from synth import atom_positions, random_coefficients

rng = np.random.default_rng(11)


def skew_cell():
    return np.array([[6.0, 0.7, -0.4], [0.3, 5.5, 0.6], [-0.2, 0.5, 7.0]])


def test_reciprocal_definition():
    R = skew_cell()
    B = pw.reciprocal(R)
    assert np.allclose(R.T @ B, 2 * np.pi * np.eye(3), atol=1e-13)


def test_cell_volume_triple_product():
    # Omega = |a0 . (a1 x a2)| (columns of R), and the reciprocal cell holds (2 pi)^3 / Omega
    R = skew_cell()
    a0, a1, a2 = R[:, 0], R[:, 1], R[:, 2]
    om = abs(a0 @ np.cross(a1, a2))
    assert np.isclose(pw.cell_volume(R), om, rtol=1e-14)
    B = pw.reciprocal(R)
    assert np.isclose(abs(B[:, 0] @ np.cross(B[:, 1], B[:, 2])), (2 * np.pi) ** 3 / om, rtol=1e-13)
    assert np.isclose(pw.cell_volume(np.diag([6.0, 6.5, 5.5])), 6.0 * 6.5 * 5.5, rtol=1e-15)


def test_sphere_bounding_box_misses_nothing():
    R = skew_cell()
    k = np.array([0.3, -0.2, 0.45])
    ecut = 6.0
    iG = pw.sphere(R, k, ecut)
    # every lattice point of a much larger box that lies in the sphere is listed
    ax = np.arange(-20, 21)
    g = np.stack(np.meshgrid(ax, ax, ax, indexing="ij"), -1).reshape(-1, 3)
    q = (g + k) @ pw.reciprocal(R).T
    inside = g[0.5 * np.sum(q * q, 1) <= ecut]
    assert {tuple(x) for x in inside} == {tuple(x) for x in iG}
    # lexicographic (i0, i1, i2) order
    keys = iG[:, 0] * 10 ** 6 + iG[:, 1] * 10 ** 3 + iG[:, 2]
    assert np.all(np.diff(keys) > 0)


def test_sphere_shift_and_time_reversal():
    R = np.diag([9.0, 8.0, 10.0])
    k = np.array([0.1, 0.2, 0.3])
    ecut = 8.0
    a = pw.sphere(R, k, ecut)
    # k -> k + e0 relabels the sphere: iG -> iG - e0
    b = pw.sphere(R, k + np.array([1.0, 0, 0]), ecut)
    assert {tuple(x) for x in b} == {tuple(x - np.array([1, 0, 0])) for x in a}
    # k -> -k: iG -> -iG
    c = pw.sphere(R, -k, ecut)
    assert {tuple(x) for x in c} == {tuple(-x) for x in a}


def test_sphere_cubic_symmetry_at_gamma():
    iG = pw.sphere(np.eye(3) * 8.0, [0, 0, 0], 10.0)
    s = {tuple(x) for x in iG}
    for perm in [(1, 0, 2), (2, 1, 0), (0, 2, 1)]:
        assert s == {tuple(x[list(perm)]) for x in iG}
    assert s == {tuple(x * np.array([-1, 1, -1])) for x in iG}


def test_sphere_count_near_continuum_volume():
    # N_pw ~ Omega (4/3 pi qmax^3) / (2 pi)^3 with a surface correction ~ N^(2/3)
    L, ecut = 20.0, 30.0
    n = pw.sphere(np.eye(3) * L, [0.1, 0.2, 0.3], ecut).shape[0]
    est = L ** 3 * (4 / 3) * np.pi * (2 * ecut) ** 1.5 / (2 * np.pi) ** 3
    assert abs(n - est) < 3 * est ** (2 / 3)


def test_column_structure_reconstructs_sphere():
    iG = pw.sphere(np.eye(3) * 10.0, [0.1, 0.2, 0.3], 20.0)
    pairs, start, count, lo = pw.column_structure(iG)
    rebuilt = np.concatenate([
        np.column_stack([np.full(c, p[0]), np.full(c, p[1]), l + np.arange(c)])
        for p, c, l in zip(pairs, count, lo)])
    assert np.array_equal(rebuilt, iG)
    assert np.array_equal(start, np.concatenate([[0], np.cumsum(count)[:-1]]))


def test_kinetic_is_laplacian_of_bloch_wave():
    """-(1/2) lap psi at random points, by finite differences of the direct sum."""
    R = skew_cell()
    k = np.array([0.2, -0.1, 0.35])
    iG = pw.sphere(R, k, 3.0)
    T = pw.kinetic(R, k, iG)
    C = rng.standard_normal(len(iG)) + 1j * rng.standard_normal(len(iG))
    # independent route: k+G from a . q = 2 pi (iG + k) solved directly
    q = np.linalg.solve(R.T, 2 * np.pi * (iG + k).T).T

    def psi(r):
        return np.sum(C * np.exp(1j * (q @ r)))

    h = 1e-3
    for _ in range(3):
        r = rng.uniform(0, 5, 3)
        lap = sum(psi(r + h * e) - 2 * psi(r) + psi(r - h * e) for e in np.eye(3)) / h ** 2
        direct = np.sum(C * T * np.exp(1j * (q @ r)))
        assert abs(-0.5 * lap - direct) < 1e-5 * np.sum(np.abs(C * T))


def test_vloc_two_constructions_agree():
    R = np.eye(3) * 10.0
    S = (48, 48, 48)
    atoms = atom_positions(R, 8, 1)
    a = pw.vloc_realspace(R, S, atoms)
    b = pw.vloc_fourier(R, S, atoms)
    assert np.max(np.abs(a - b)) < 1e-12


def test_vloc_skew_cell_direct_vs_fourier():
    R = skew_cell()
    S = (30, 30, 32)
    atoms = atom_positions(R, 3, 5)
    a = pw.vloc_realspace(R, S, atoms)
    b = pw.vloc_fourier(R, S, atoms)
    assert np.max(np.abs(a - b)) < 1e-10


def test_vloc_separable_equals_direct_loop():
    R = np.diag([7.0, 6.0, 8.0])
    S = (14, 12, 16)
    atoms = atom_positions(R, 3, 9)
    a = pw.vloc_realspace(R, S, atoms)
    b = pw.vloc_realspace(R, S, atoms, method="direct")
    assert np.max(np.abs(a - b)) < 1e-14


def test_vloc_mean_closed_form():
    # cell average = (1/Omega) integral over all space = -depth natoms (2 pi w^2)^{3/2} / Omega
    R = np.eye(3) * 10.0
    S = (40, 40, 40)
    atoms = atom_positions(R, 5, 3)
    V = pw.vloc_realspace(R, S, atoms)
    assert np.isclose(V.mean(), -4.0 * 5 * (2 * np.pi) ** 1.5 / 1000.0, rtol=1e-12)


def test_vloc_single_isolated_gaussian():
    R = np.eye(3) * 30.0
    S = (30, 30, 30)
    atom = np.array([[15.0, 15.0, 15.0]])
    V = pw.vloc_realspace(R, S, atom).reshape(S)
    for j in [(15, 15, 15), (16, 15, 14), (18, 12, 15)]:
        d = np.array(j) - 15.0
        assert np.isclose(V[j], -4 * np.exp(-0.5 * d @ d), rtol=1e-14, atol=1e-300)


def test_projector_ft_by_quadrature():
    # direct 3-D quadrature of beta_l(r) exp(-i q.r) on a fine grid (Gaussian decays by r=8)
    h = 0.2
    ax = np.arange(-8, 8 + h / 2, h)
    X, Y, Z = np.meshgrid(ax, ax, ax, indexing="ij")
    Ns = np.pi ** -0.75
    Np = Ns * np.sqrt(2)
    g = np.exp(-(X * X + Y * Y + Z * Z) / 2)
    betas = [Ns * g, Np * X * g, Np * Y * g, Np * Z * g]
    for b in betas:  # normalisation
        assert np.isclose(np.sum(b * b) * h ** 3, 1.0, rtol=1e-10)
    for q in [np.array([0.3, -0.7, 1.1]), np.array([1.5, 0.2, 0.0])]:
        F = pw.projector_ft(q[None, :])[0]
        ph = np.exp(-1j * (q[0] * X + q[1] * Y + q[2] * Z))
        for l, b in enumerate(betas):
            assert abs(np.sum(b * ph) * h ** 3 - F[l]) < 1e-10


def test_projector_overlap_by_realspace_quadrature():
    """P^dag C = integral beta(r - R_a) psi(r) over all space (Bloch images)."""
    R = np.diag([6.0, 7.0, 6.5])
    k = np.array([0.15, -0.25, 0.3])
    iG = pw.sphere(R, k, 4.0)
    atoms = atom_positions(R, 2, 21)
    P = pw.projectors(R, k, iG, atoms)
    C = random_coefficients(2 * pw.kinetic(R, k, iG), 2, 22).T
    PdC = P.conj().T @ C
    # psi on a fine grid of the cell, with its Bloch phase
    S = (36, 42, 39)
    r = pw.grid_points(R, S)
    q = pw.kvectors(R, k, iG)
    psi = np.exp(1j * (r @ q.T)) @ C                       # (N, nb), direct sum
    Omega = pw.cell_volume(R)
    Ns = np.pi ** -0.75
    Np = Ns * np.sqrt(2)
    for a in range(2):
        acc = np.zeros((4, 2), complex)
        for n in np.ndindex(5, 5, 5):
            T = R @ (np.array(n) - 2.0)
            # integral over cell of beta(r + T - R_a) psi(r + T) = e^{ik.T} ...
            d = r + T - atoms[a]
            g = np.exp(-0.5 * np.sum(d * d, 1))
            bl = np.stack([Ns * g, Np * d[:, 0] * g, Np * d[:, 1] * g, Np * d[:, 2] * g])
            kT = np.exp(1j * (pw.reciprocal(R) @ k) @ T)
            acc += kT * (bl @ psi) * Omega / r.shape[0]
        assert np.max(np.abs(acc - PdC[4 * a:4 * a + 4])) < 1e-9 * np.max(np.abs(PdC))
