"""Pins of the LinearPCM oracle (oracle/pcm.py): the hessian of the paper's
Listing 1 against a hand-derived divergence, the uniform-dielectric closed
form, the vacuum case, and the CG solve against a dense linear solve."""
from __future__ import annotations

import numpy as np
import pytest

from oracle import pcm
from oracle import planewave as pw
from oracle import scf

TRICLINIC = np.array([[7.0, 1.2, 0.4], [0.0, 6.5, -0.9], [0.3, 0.0, 8.0]])
S = (18, 16, 20)


def _charge(R, S):
    """A neutral-background charge: two Gaussians (the solve ignores G = 0)."""
    return -pw.vloc_realspace(R, S, np.array([[1.0, 2.0, 3.0], [4.0, 1.0, 2.0]]), depth=0.3)


def test_hessian_of_a_cosine_in_a_cosine_dielectric_is_the_hand_divergence():
    """phi = cos(G.r), eps = 1 + a cos(Q.r):  div(eps grad phi) = -G^2 cos(G.r)
    - (a/2)[G.(G+Q) cos((G+Q).r) + G.(G-Q) cos((G-Q).r)]; the hessian is -1/(4 pi) of it."""
    r = pw.grid_points(TRICLINIC, S)
    B = pw.reciprocal(TRICLINIC)
    Q, G, a = B @ np.array([1.0, 0.0, -1.0]), B @ np.array([0.0, 1.0, 1.0]), 0.3
    eps = 1 + a * np.cos(r @ Q)
    H = pcm.hessian(TRICLINIC, S, eps, pcm.op_J(S, np.cos(r @ G)))
    div = -(G @ G) * np.cos(r @ G) - a / 2 * (G @ (G + Q) * np.cos(r @ (G + Q)) + G @ (G - Q) * np.cos(r @ (G - Q)))
    assert np.max(np.abs(pcm.op_I(S, H) + div / (4 * np.pi))) < 1e-13


def test_hessian_is_hermitian_and_positive():
    rng = np.random.default_rng(2)
    eps = 1.0 + rng.random(int(np.prod(S)))
    X = rng.normal(size=eps.size) + 1j * rng.normal(size=eps.size)
    Y = rng.normal(size=eps.size) + 1j * rng.normal(size=eps.size)
    HX, HY = pcm.hessian(TRICLINIC, S, eps, X), pcm.hessian(TRICLINIC, S, eps, Y)
    assert abs(np.vdot(Y, HX) - np.vdot(HY, X)) < 1e-12 * abs(np.vdot(Y, HX))
    assert np.vdot(X, HX).real > 0


@pytest.mark.parametrize("e", [1.0, 2.5, 78.4])
def test_uniform_dielectric_closed_form(e):
    """eps uniform: phi~ = 4 pi rho~ / (eps G^2) and A_diel = (1/eps - 1) E_H[rho]."""
    n = _charge(TRICLINIC, S)
    rt = pcm.op_J(S, n)
    res = pcm.solve(TRICLINIC, S, np.full(n.size, e), rt, tol=1e-12)
    assert res.converged
    want = pcm.coulomb(TRICLINIC, S, rt) / e
    assert np.max(np.abs(res.phi - want)) < 1e-12 * np.max(np.abs(want))
    _, EH = scf.hartree(TRICLINIC, S, n)
    assert abs(res.A_diel - (1.0 / e - 1.0) * EH) < 1e-12 * EH


def test_cg_solution_equals_a_dense_solve():
    """Tiny box, smooth varying dielectric: the CG result equals numpy's dense
    solve of the hessian matrix restricted to G != 0."""
    R, Sm = np.diag([5.0, 4.5, 4.0]), (6, 5, 4)
    r = pw.grid_points(R, Sm)
    eps = 1.0 + 0.5 * (1.0 + np.tanh(3.0 * np.cos(r @ pw.reciprocal(R)[:, 0])))
    N = int(np.prod(Sm))
    Hm = np.stack([pcm.hessian(R, Sm, eps, np.eye(N)[:, j]) for j in range(N)], axis=1)
    rng = np.random.default_rng(4)
    rt = rng.normal(size=N) + 1j * rng.normal(size=N)
    G = pcm.box_G(R, Sm)
    nz = np.einsum("ij,ij->i", G, G) > 0
    rt[~nz] = 0
    want = np.zeros(N, dtype=complex)
    want[nz] = np.linalg.solve(Hm[np.ix_(nz, nz)], rt[nz])
    res = pcm.solve(R, Sm, eps, rt, tol=1e-13, max_iter=200)
    assert res.converged
    assert np.max(np.abs(res.phi - want)) < 1e-10 * np.max(np.abs(want))


def test_screening_lowers_the_energy():
    """A_diel < 0 for eps >= 1 varying in space, and it lies between the
    uniform-eps bounds set by min and max eps."""
    n = _charge(TRICLINIC, S)
    rt = pcm.op_J(S, n)
    r = pw.grid_points(TRICLINIC, S)
    eps = 1.0 + 0.5 * (1.0 + np.tanh(3.0 * np.cos(r @ pw.reciprocal(TRICLINIC)[:, 0])))
    res = pcm.solve(TRICLINIC, S, eps, rt, tol=1e-12)
    _, EH = scf.hartree(TRICLINIC, S, n)
    assert res.converged
    assert (1 / eps.min() - 1) * EH >= res.A_diel >= (1 / eps.max() - 1) * EH
