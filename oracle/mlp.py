"""FP64 oracle of the learned per-coefficient preconditioner network.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Network (a reading: the JDFTx paper has no learned preconditioner; this is the
replacement for the Teter preconditioner in the band minimiser of Sec. 2.1):
  features of coefficient G of band b:
      f1 = (1/2)|k+G|^2 / T_b,  f2 = log(1 + T_b),  f3 = (h_b - min_b' h_b') / T_b
  with T_b the band kinetic energy and h_b = (C^dag H C)_bb;
  a1 = W1 f + b1, h1 = silu(a1)            (64)
  a2 = W2 h1 + b2, h2 = silu(a2)           (64)
  z  = W3 . h2 + b3,  K = softplus(z)       (K > 0 keeps -K G a descent direction)
Parameter vector (4481): W1 (64x3, row-major), b1, W2 (64x64), b2, W3 (64), b3.

Training rows: (f1, f2, f3, a, q) with a = |R|^2 and q = Re(conj(R) t) for the
residual R of a coefficient and its target correction t; the loss over rows is
    L = sum (K^2 a - 2 K q) / sum a
(= sum |K R - t|^2 / sum |R|^2 up to a constant).
"""
from __future__ import annotations

import numpy as np

H = 64
NPARAM = 3 * H + H + H * H + H + H + 1


def unpack(theta):
    theta = np.asarray(theta, dtype=np.float64)
    assert theta.size == NPARAM
    o = 0
    W1 = theta[o:o + 3 * H].reshape(H, 3); o += 3 * H
    b1 = theta[o:o + H]; o += H
    W2 = theta[o:o + H * H].reshape(H, H); o += H * H
    b2 = theta[o:o + H]; o += H
    W3 = theta[o:o + H]; o += H
    b3 = theta[o]
    return W1, b1, W2, b2, W3, b3


def pack(W1, b1, W2, b2, W3, b3):
    return np.concatenate([np.ravel(W1), b1, np.ravel(W2), b2, W3, [b3]]).astype(np.float64)


def sigmoid(z):
    """1 / (1 + e^-z), evaluated without cancellation on both sides of zero."""
    z = np.asarray(z, dtype=np.float64)
    e = np.exp(-np.abs(z))
    return np.where(z >= 0, 1.0 / (1.0 + e), e / (1.0 + e))


def silu(z):
    return z * sigmoid(z)


def dsilu(z):
    s = sigmoid(z)
    return s * (1.0 + z * (1.0 - s))


def softplus(z):
    return np.logaddexp(0.0, z)


def forward(theta, X):
    """K for feature rows X (n x 3), and the intermediates for backprop."""
    W1, b1, W2, b2, W3, b3 = unpack(theta)
    a1 = X @ W1.T + b1
    h1 = silu(a1)
    a2 = h1 @ W2.T + b2
    h2 = silu(a2)
    z = h2 @ W3 + b3
    return softplus(z), (X, a1, h1, a2, h2, z)


def loss(theta, rows) -> float:
    rows = np.asarray(rows, dtype=np.float64)
    K, _ = forward(theta, rows[:, :3])
    a, q = rows[:, 3], rows[:, 4]
    return float(np.sum(K * K * a - 2.0 * K * q) / np.sum(a))


def grad(theta, rows):
    """Analytic dL/dtheta (chain rule through softplus, SiLU and the affine layers)."""
    rows = np.asarray(rows, dtype=np.float64)
    W1, b1, W2, b2, W3, b3 = unpack(theta)
    K, (X, a1, h1, a2, h2, z) = forward(theta, rows[:, :3])
    a, q = rows[:, 3], rows[:, 4]
    dK = (2.0 * K * a - 2.0 * q) / np.sum(a)
    dz = dK * sigmoid(z)
    gW3 = h2.T @ dz
    gb3 = dz.sum()
    da2 = np.outer(dz, W3) * dsilu(a2)
    gW2 = da2.T @ h1
    gb2 = da2.sum(axis=0)
    da1 = (da2 @ W2) * dsilu(a1)
    gW1 = da1.T @ X
    gb1 = da1.sum(axis=0)
    return pack(gW1, gb1, gW2, gb2, gW3, gb3)


def features(kin, Tb, h):
    """Feature rows for every (G, b): returns (npw, nb, 3)."""
    kin = np.asarray(kin)[:, None]
    Tb = np.asarray(Tb)[None, :]
    f1 = kin / Tb
    f2 = np.broadcast_to(np.log1p(Tb), f1.shape)
    f3 = np.broadcast_to((np.asarray(h) - np.min(h))[None, :] / Tb, f1.shape)
    return np.stack([f1, f2, f3], axis=-1)


def make_precond(theta):
    """A preconditioner for oracle.minimize: K from the network, per coefficient."""
    from .minimize import band_kinetic

    def precond(basis, C, G, h):
        F = features(basis.T, band_kinetic(basis, C), h)
        K, _ = forward(theta, F.reshape(-1, 3))
        return K.reshape(G.shape) * G
    return precond
