"""Pins of the oracle's band minimiser (CPU).

Variational band minimisation (JDFTx paper, Sec. 2.1 Minimize, Sec. 2.2)
reaches the lowest eigenpairs of H: checked against LAPACK's dense
eigensolver, across preconditioners (the fixed point cannot depend on K), for
a variational (monotone) energy history, and the Teter polynomial against its
published closed form.
"""
import json
import os

import numpy as np
import pytest

from oracle import minimize as mn
from oracle import planewave as pw
from tests.systems import OracleSystem, workload

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "small_eigs.json")


def test_teter_closed_form_values():
    # K(0) = 1; K(1) = 65/81; large x: K ~ 8x^3 / 16x^4 = 1/(2x); strictly decreasing on x > 0
    assert mn.teter(0.0) == 1.0
    assert np.isclose(mn.teter(1.0), 65.0 / 81.0, rtol=1e-15)
    assert np.isclose(mn.teter(1e6) * 2e6, 1.0, rtol=1e-5)
    x = np.linspace(0, 20, 2001)
    assert np.all(np.diff(mn.teter(x)) < 0)


def test_band_kinetic_of_single_plane_wave():
    o = OracleSystem(workload("tiny_cubic"))
    C = np.zeros((o.basis.npw, 1), complex)
    C[7, 0] = 1.0 / np.sqrt(o.basis.Omega)
    assert np.isclose(mn.band_kinetic(o.basis, C)[0], o.basis.T[7], rtol=1e-15)


@pytest.mark.parametrize("name,nb", [("tiny_cubic", 6), ("tiny_ortho", 5)])
def test_minimiser_reaches_dense_eigenvalues(name, nb):
    o = OracleSystem(workload(name))
    H = lambda X: pw.apply_H(o.basis, o.V, X, o.P, o.D)
    exact = np.linalg.eigvalsh(pw.dense_H(o.basis, o.V, o.P, o.D) / o.basis.Omega)[:nb]
    energies = []
    for pc in (mn.precond_teter, mn.precond_identity):
        res = mn.minimize_bands(o.basis, H, o.coeffs(nb).T, precond=pc, tol=1e-9, max_iter=800)
        assert res.converged
        assert np.max(np.abs(np.sort(res.eigs) - exact)) < 1e-12
        r, *_ = mn.residual_norms(o.basis, res.C, res.HC)
        assert r.max() <= res.residual + 1e-15          # Frobenius bounds every band
        E = [h[0] for h in res.history]
        assert np.all(np.diff(E) <= 1e-12)               # variational
        assert np.allclose(pw.subspace(o.basis, res.C, res.C)[1], np.eye(nb), atol=1e-12)
        energies.append(res.energy)
    assert abs(energies[0] - energies[1]) < 1e-11


def test_golden_small_cell_eigenvalues_consistent():
    g = json.load(open(GOLDEN))
    assert g["npw"] == 4259 and g["nbands"] == 16
    e = np.array(g["eigs"])
    assert np.all(np.diff(e) >= 0)
    assert np.isclose(g["E_ref"], 2 * e[:16].sum(), rtol=1e-15)
    assert g["gap"] > 1e-3


def test_teter_beats_identity_in_iterations():
    o = OracleSystem(workload("tiny_ortho"))
    H = lambda X: pw.apply_H(o.basis, o.V, X, o.P, o.D)
    its = [mn.minimize_bands(o.basis, H, o.coeffs(5).T, precond=pc, tol=1e-8, max_iter=800).iterations
           for pc in (mn.precond_teter, mn.precond_identity)]
    assert its[0] < its[1]
