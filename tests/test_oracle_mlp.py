"""Pins of the oracle's preconditioner network (CPU): analytic gradients against
central finite differences, closed forms of the activations, the zero-weight
network, and the network as a preconditioner (it reaches the same minimum)."""
import numpy as np
import pytest

from oracle import minimize as mn
from oracle import mlp
from oracle import planewave as pw
from synth import mlp_init
from tests.systems import OracleSystem, workload

rng = np.random.default_rng(9)


def random_rows(n):
    X = np.column_stack([rng.uniform(0, 20, n), rng.uniform(0, 2, n), rng.uniform(0, 3, n)])
    a = rng.uniform(0.1, 2.0, n)
    q = rng.normal(0, 1, n)
    return np.column_stack([X, a, q])


def test_activation_closed_forms():
    assert mlp.softplus(0.0) == np.log(2.0)
    assert mlp.silu(0.0) == 0.0
    assert np.isclose(mlp.sigmoid(0.0), 0.5)
    z = np.linspace(-30, 30, 61)
    assert np.allclose(mlp.softplus(z), np.log1p(np.exp(z)), rtol=1e-12)
    assert np.allclose(mlp.silu(z), z / (1 + np.exp(-z)), rtol=1e-12, atol=1e-300)
    # silu' by central differences
    h = 1e-6
    assert np.allclose(mlp.dsilu(z), (mlp.silu(z + h) - mlp.silu(z - h)) / (2 * h), rtol=1e-7, atol=1e-9)


def test_gradient_matches_finite_differences():
    theta = mlp_init(3)
    theta[mlp.NPARAM - 1] = 0.3
    rows = random_rows(40)
    g = mlp.grad(theta, rows)
    idx = rng.choice(mlp.NPARAM, 60, replace=False)
    idx = np.append(idx, [0, 1, 200, mlp.NPARAM - 1, mlp.NPARAM - 2])
    h = 1e-5
    for i in idx:
        tp = theta.copy(); tp[i] += h
        tm = theta.copy(); tm[i] -= h
        fd = (mlp.loss(tp, rows) - mlp.loss(tm, rows)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-7 * max(1.0, abs(g[i])) + 1e-9, (i, fd, g[i])


def test_zero_weight_network_is_constant():
    theta = np.zeros(mlp.NPARAM)
    theta[-1] = 0.7
    rows = random_rows(25)
    K, _ = mlp.forward(theta, rows[:, :3])
    assert np.allclose(K, np.log1p(np.exp(0.7)))
    g = mlp.grad(theta, rows)
    k = np.log1p(np.exp(0.7))
    s = 1 / (1 + np.exp(-0.7))
    expect_b3 = np.sum((2 * k * rows[:, 3] - 2 * rows[:, 4]) * s) / np.sum(rows[:, 3])
    assert np.isclose(g[-1], expect_b3, rtol=1e-12)
    assert np.allclose(g[:-1 - mlp.H], 0.0)   # no gradient reaches W1, b1, W2, b2 through zero W3


def test_optimal_constant_minimises_loss():
    """With only b3 free the loss is a quadratic in K with minimum K* = sum q / sum a."""
    rows = random_rows(50)
    rows[:, 4] = np.abs(rows[:, 4])
    Kstar = rows[:, 4].sum() / rows[:, 3].sum()
    theta = np.zeros(mlp.NPARAM)
    theta[-1] = np.log(np.expm1(Kstar))
    assert abs(mlp.grad(theta, rows)[-1]) < 1e-12


def test_network_preconditioner_reaches_same_minimum():
    o = OracleSystem(workload("tiny_cubic"))
    Hf = lambda X: pw.apply_H(o.basis, o.V, X, o.P, o.D)
    exact = np.linalg.eigvalsh(pw.dense_H(o.basis, o.V, o.P, o.D) / o.basis.Omega)[:6]
    res = mn.minimize_bands(o.basis, Hf, o.coeffs(6).T, precond=mlp.make_precond(mlp_init(5)), tol=1e-9,
                            max_iter=1500)
    assert res.converged
    assert np.max(np.abs(np.sort(res.eigs) - exact)) < 1e-11
