"""Pins of the SCF oracle (oracle/scf.py): Hartree, LDA, Pulay, the loop.

Each check fixes a value by something other than the oracle's own formula:
closed forms of Poisson's equation, an isolated Gaussian charge, the textbook
exchange constant and high-density correlation limit, finite differences of
the energy density, the finite termination of Pulay mixing on a linear map,
constrained least squares written another way, the uniform electron gas, and
the stationarity of the Kohn-Sham energy at self-consistency.
"""
from __future__ import annotations

from math import erf, log, pi

import numpy as np
import pytest

from oracle import planewave as pw
from oracle import scf
from synth import atom_positions, random_coefficients

TRICLINIC = np.array([[7.0, 1.2, 0.4], [0.0, 6.5, -0.9], [0.3, 0.0, 8.0]])


def _cos_density(R, S, waves):
    r = pw.grid_points(R, S)
    B = pw.reciprocal(R)
    n = np.zeros(r.shape[0])
    for A, m, ph in waves:
        G = B @ np.asarray(m, dtype=np.float64)
        n += A * np.cos(r @ G + ph)
    return n


def test_hartree_of_cosines_is_the_poisson_closed_form():
    """-lap V = 4 pi n for n = sum A cos(G.r + ph): V = sum 4 pi A / |G|^2 cos(...),
    E_H = sum pi A^2 Omega / |G|^2 (distinct waves do not interact)."""
    S = (18, 16, 20)
    waves = [(0.7, (1, 0, 0), 0.3), (-0.4, (1, -2, 1), 1.1), (0.25, (0, 3, -2), -0.5)]
    n = _cos_density(TRICLINIC, S, waves)
    V, EH = scf.hartree(TRICLINIC, S, n)
    B = pw.reciprocal(TRICLINIC)
    Omega = pw.cell_volume(TRICLINIC)
    want = np.zeros_like(n)
    E = 0.0
    for A, m, ph in waves:
        G2 = float(np.sum((B @ np.asarray(m, float)) ** 2))
        want += _cos_density(TRICLINIC, S, [(4 * pi * A / G2, m, ph)])
        E += pi * A * A * Omega / G2
    assert np.max(np.abs(V - want)) < 1e-12 * np.max(np.abs(want))
    assert abs(EH - E) < 1e-12 * E
    # the same energy from the real-space integral (1/2) int n V
    assert abs(0.5 * Omega / n.size * np.dot(n, V) - E) < 1e-12 * E


def test_hartree_of_a_uniform_density_is_zero():
    S = (12, 10, 9)
    V, EH = scf.hartree(TRICLINIC, S, np.full(int(np.prod(S)), 0.37))
    assert np.max(np.abs(V)) < 1e-14 and abs(EH) < 1e-14


def test_hartree_of_a_gaussian_charge_matches_the_isolated_potential():
    """A Gaussian charge Q in a large cube with its neutralising background:
    near the charge V(r) - V(0) = Q [erf(r / sqrt2 s) / r - sqrt(2/pi)/s]
    + (2 pi Q / 3 Omega) r^2, up to image terms of order (r/L)^4 Q/L."""
    L, S, s, Q = 16.0, (64, 64, 64), 0.8, 1.0
    R = np.eye(3) * L
    d = pw.grid_points(R, S) - L / 2
    d2 = np.sum(d * d, axis=1)
    n = Q * (2 * pi * s * s) ** -1.5 * np.exp(-d2 / (2 * s * s))
    V, _ = scf.hartree(R, S, n)
    r = np.sqrt(d2)
    sel = (r > 0) & (r < 2.5)
    ana = np.array([Q * erf(x / (np.sqrt(2.0) * s)) / x for x in r[sel]])
    ana += -Q * np.sqrt(2.0 / pi) / s + 2 * pi * Q / (3 * L ** 3) * r[sel] ** 2
    got = V[sel] - V[np.argmin(d2)]
    assert np.max(np.abs(got - ana)) < 1e-4


def test_slater_exchange_is_the_textbook_constant():
    """e_x(r_s) = -(3/4)(9/(4 pi^2))^{1/3} / r_s = -0.458165... / r_s Ha."""
    rs = np.array([0.5, 1.0, 2.0, 5.0])
    n = 3.0 / (4.0 * pi * rs ** 3)
    e, v = scf.lda_pz(n)
    # isolate exchange: the correlation part is bounded and computed separately below
    ec_free = e - (-0.4581652932831429 / rs)
    e_c, _ = _pz_correlation_only(rs)
    assert np.max(np.abs(ec_free - e_c)) < 1e-14


def _pz_correlation_only(rs):
    n = 3.0 / (4.0 * pi * np.asarray(rs) ** 3)
    e, v = scf.lda_pz(n)
    ex = -0.75 * (3.0 * n / pi) ** (1.0 / 3.0)
    return e - ex, v - 4.0 / 3.0 * ex


def test_xc_potential_is_the_derivative_of_the_energy_density():
    """v_xc = d(n e_xc)/dn by central differences, both correlation branches."""
    n = np.geomspace(1e-4, 50.0, 60)
    _, v = scf.lda_pz(n)
    h = 1e-6 * n
    ep, _ = scf.lda_pz(n + h)
    em, _ = scf.lda_pz(n - h)
    fd = ((n + h) * ep - (n - h) * em) / (2 * h)
    # skip the two points straddling r_s = 1, where the fit switches branch
    rs = np.cbrt(3.0 / (4.0 * pi * n))
    ok = np.abs(rs - 1.0) > 1e-3
    assert np.max(np.abs(fd - v)[ok] / np.abs(v[ok])) < 1e-8


def test_pz_branches_meet_at_rs_one():
    """The two halves of the fit join at r_s = 1 to within the fit's rounding."""
    lo, vlo = _pz_correlation_only(np.array([1.0 - 1e-12]))
    hi, vhi = _pz_correlation_only(np.array([1.0 + 1e-12]))
    assert abs(lo[0] - hi[0]) < 1e-4
    assert abs(vlo[0] - vhi[0]) < 1e-3


def test_correlation_has_the_high_density_log_coefficient():
    """Gell-Mann-Brueckner: e_c -> ((1 - ln 2)/pi^2) ln r_s + const as r_s -> 0."""
    e, _ = _pz_correlation_only(np.array([1e-4, 2e-4]))
    slope = (e[1] - e[0]) / log(2.0)
    assert abs(slope - (1.0 - log(2.0)) / pi ** 2) < 2e-4


def test_xc_of_nonpositive_density_is_zero():
    e, v = scf.lda_pz(np.array([0.0, -1e-12, -3.0]))
    assert np.all(e == 0) and np.all(v == 0)


def test_pulay_terminates_on_a_linear_map():
    """Pulay mixing on x -> M x + b (dim d, full history) is a Krylov method:
    it reaches the fixed point to rounding within d + 1 steps."""
    rng = np.random.default_rng(3)
    d = 6
    M = rng.normal(size=(d, d))
    M = 0.5 * M / np.linalg.norm(M, 2)
    b = rng.normal(size=d)
    xs = np.linalg.solve(np.eye(d) - M, b)
    x = np.zeros(d)
    mix = scf.Pulay(10, 0.7)
    for _ in range(d + 1):
        x = mix.step(x, M @ x + b)
    assert np.linalg.norm(x - xs) < 1e-12 * np.linalg.norm(xs)


def test_pulay_coefficients_are_the_constrained_least_squares_minimiser():
    """c minimises |sum c_i R_i| with sum c_i = 1: eliminate c_m = 1 - sum_{i<m} c_i
    and solve the unconstrained problem with numpy's least squares."""
    rng = np.random.default_rng(5)
    N, m, alpha = 40, 4, 0.3
    xs = [rng.normal(size=N) for _ in range(m)]
    fs = [rng.normal(size=N) for _ in range(m)]
    mix = scf.Pulay(8, alpha)
    for x, fx in zip(xs, fs):
        out = mix.step(x, fx)
    Rs = [f - x for x, f in zip(xs, fs)]
    Dm = np.stack([Rs[i] - Rs[-1] for i in range(m - 1)], axis=1)
    a, *_ = np.linalg.lstsq(Dm, -Rs[-1], rcond=None)
    c = np.append(a, 1.0 - a.sum())
    want = sum(ci * (x + alpha * r) for ci, x, r in zip(c, xs, Rs))
    assert np.max(np.abs(out - want)) < 1e-12 * np.max(np.abs(want))


def test_pulay_first_step_is_linear_mixing_and_fixed_points_stay():
    rng = np.random.default_rng(6)
    x, fx = rng.normal(size=30), rng.normal(size=30)
    assert np.allclose(scf.Pulay(5, 0.4).step(x, fx), x + 0.4 * (fx - x), rtol=0, atol=1e-15)
    mix = scf.Pulay(5, 0.4)
    mix.step(rng.normal(size=30), rng.normal(size=30))
    y = rng.normal(size=30)
    assert np.allclose(mix.step(y, y), y, rtol=0, atol=1e-12)


def test_pulay_history_is_bounded_and_drops_dependent_pairs():
    rng = np.random.default_rng(8)
    mix = scf.Pulay(3, 0.5)
    base = rng.normal(size=20)
    for _ in range(5):
        mix.step(base, base + rng.normal(size=20))
    assert len(mix.n_in) == 3 and mix.used == 3
    mix2 = scf.Pulay(4, 0.5)
    r = rng.normal(size=20)
    mix2.step(base, base + r)
    out = mix2.step(base, base + r)      # identical residual: singular system, oldest dropped
    assert mix2.used == 1
    assert np.allclose(out, base + 0.5 * r)


def _uniform_gas(nb=7):
    L = 8.0
    R = np.eye(3) * L
    S = (20, 20, 20)
    b = pw.Basis.build(R, S, (0.0, 0.0, 0.0), 3.0)
    C0 = random_coefficients(2 * b.T, nb, 4).T
    return R, S, b, [scf.KCell(b, None, None, 1.0, C0)]


def test_scf_uniform_electron_gas_closed_form():
    """V_ion = 0, k = 0, 7 bands filling the G = 0 and |G| = 2 pi/L shells: the
    self-consistent density is uniform n0 = 14/Omega, V_H = 0, the bands are
    (1/2)|G|^2 + v_xc(n0), and E = 2 sum (1/2)|G_b|^2 + Omega n0 e_xc(n0)."""
    R, S, b, cells = _uniform_gas()
    res = scf.scf(cells, np.zeros(b.N), alpha=0.5, tol_energy=1e-11, tol_density=1e-9)
    assert res.converged
    Omega = b.Omega
    n0 = 14.0 / Omega
    e0, v0 = scf.lda_pz(np.array([n0]))
    g2 = 0.5 * (2 * pi / 8.0) ** 2
    eig_want = np.array([0.0] + [g2] * 6) + v0[0]
    assert np.max(np.abs(res.eigs[0] - eig_want)) < 1e-9
    E_want = 2.0 * 6 * g2 + Omega * n0 * e0[0]
    assert abs(res.energy - E_want) < 1e-9
    assert np.max(np.abs(res.n - n0)) < 1e-8


def _small_cell():
    R = np.diag([8.0, 8.5, 7.5])
    S = (24, 25, 20)
    atoms = atom_positions(R, 4, 5)
    cells = []
    for i, k in enumerate([(0.1, 0.2, 0.3), (-0.25, 0.0, 0.4)]):
        b = pw.Basis.build(R, S, k, 6.0)
        P = pw.projectors(R, b.kfrac, b.iG, atoms)
        C0 = random_coefficients(2 * b.T, 6, 7 + i).T
        cells.append(scf.KCell(b, P, pw.dmatrix(4), 0.5, C0))
    return R, S, pw.vloc_realspace(R, S, atoms), cells


@pytest.fixture(scope="module")
def small_scf():
    R, S, Vion, cells = _small_cell()
    return R, S, Vion, cells, scf.scf(cells, Vion, alpha=0.5, tol_energy=1e-11, tol_density=1e-9)


def test_scf_energy_equals_the_direct_kohn_sham_functional(small_scf):
    """At self-consistency the band-sum form of E equals the functional
    evaluated from the orbitals directly (no eigenvalues)."""
    R, S, Vion, cells, res = small_scf
    assert res.converged
    Ed, n = scf.direct_energy(cells, res.C, Vion, 2.0)
    assert abs(Ed - res.energy) < 1e-9
    assert np.max(np.abs(n - res.n)) < 1e-12


def test_scf_solution_is_stationary(small_scf):
    """The Kohn-Sham energy is stationary at the SCF orbitals: a perturbation
    t X (re-orthonormalised) changes it by O(t^2), and the change is positive."""
    R, S, Vion, cells, res = small_scf
    rng = np.random.default_rng(9)
    X = [rng.normal(size=C.shape) + 1j * rng.normal(size=C.shape) for C in res.C]
    X = [x * np.linalg.norm(C) / np.linalg.norm(x) for x, C in zip(X, res.C)]
    E0, _ = scf.direct_energy(cells, res.C, Vion, 2.0)
    dE = []
    for t in (1e-3, 5e-4):
        Ct = [pw.lowdin(C + t * x, kc.basis.Omega) for C, x, kc in zip(res.C, X, cells)]
        dE.append(scf.direct_energy(cells, Ct, Vion, 2.0)[0] - E0)
    assert dE[0] > 0 and dE[1] > 0
    assert 3.5 < dE[0] / dE[1] < 4.5      # quadratic, not linear (ratio 2)


def test_scf_result_does_not_depend_on_the_mixing(small_scf):
    R, S, Vion, cells, res = small_scf
    other = scf.scf(cells, Vion, alpha=0.2, history=4, tol_energy=1e-11, tol_density=1e-9)
    assert other.converged
    assert abs(other.energy - res.energy) < 1e-9
    assert np.max(np.abs(other.n - res.n)) < 1e-7
