"""FP64 oracle of the linear dielectric (LinearPCM) Poisson solve.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  Nothing here is shared
with the CUDA library.

The JDFTx paper's worked example (Sec. 2.1, Eq. (Poisson) and Eq. (Adiel),
Listing 1): the electrostatic potential phi of a charge density rho in an
inhomogeneous dielectric eps(r) solves  -4 pi rho = div(eps grad phi), and the
solvation energy is A_diel = (1/2) int (phi - K rho) rho, K the unscreened
Coulomb operator.  The listing solves it by conjugate gradients on fields in
reciprocal space with hessian(phi~) = -(1/4 pi) div J(eps * I(grad phi~)).

Readings (the paper prints the operator composition, not the discretisation):
  * Fields in reciprocal space are full FFT boxes X(G), G = B iG with the
    frequencies folded to [-S/2, S/2) per axis (the Nyquist slot takes -S/2).
    I X (r_j) = sum_G X(G) exp(i G.r_j);  J x (G) = (1/N) sum_j x_j exp(-i G.r_j).
  * gradient: (grad X)_d = i G_d X;  divergence: div Y = sum_d i G_d Y_d.
    With these, hessian = (1/4 pi N) sum_d (I iG_d)^dag eps (I iG_d): Hermitian
    and positive semi-definite for eps > 0, zero on G = 0.
  * coulomb(X) = 4 pi X / |G|^2 (0 at G = 0);  O = Omega;  dot(a, b) = sum_G conj(a) b.
  * The solve works on G != 0: rho~(0) is ignored (a neutral charge), phi~(0) = 0.
    A_diel = (1/2) Re dot(phi~ - coulomb(rho~), O rho~).
  * CG: preconditioned conjugate gradients (Hestenes-Stiefel) from phi~ = 0 with
    the preconditioner coulomb() (the exact inverse for eps = 1); converged when
    |r| <= tol |rho~| (plain sums over the box, G != 0).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import cfft
from . import planewave as pw


def box_G(R, S) -> np.ndarray:
    """Cartesian G of every box slot (N x 3), folded frequencies."""
    return pw.signed_box_frequencies(S).astype(np.float64) @ pw.reciprocal(R).T


def op_I(S, X) -> np.ndarray:
    """Full-box inverse transform of a reciprocal-space field (flat in, flat out)."""
    return cfft.fft3d(np.asarray(X, dtype=np.complex128).reshape(S), +1).reshape(-1)


def op_J(S, x) -> np.ndarray:
    """Full-box forward transform, normalised by 1/N (flat in, flat out)."""
    return cfft.fft3d(np.asarray(x, dtype=np.complex128).reshape(S), -1).reshape(-1) / float(np.prod(S))


def coulomb(R, S, X) -> np.ndarray:
    G = box_G(R, S)
    G2 = np.einsum("ij,ij->i", G, G)
    K = np.zeros_like(G2)
    K[G2 > 0] = 4.0 * np.pi / G2[G2 > 0]
    return K * np.asarray(X)


def hessian(R, S, eps, X) -> np.ndarray:
    """-(1/4 pi) div J(eps * I(grad X)) for a reciprocal-space field X (flat)."""
    G = box_G(R, S)
    X = np.asarray(X, dtype=np.complex128)
    out = np.zeros_like(X)
    for d in range(3):
        Ed = np.asarray(eps) * op_I(S, 1j * G[:, d] * X)
        out += 1j * G[:, d] * op_J(S, Ed)
    return -out / (4.0 * np.pi)


@dataclass
class SolveResult:
    phi: np.ndarray
    iterations: int
    converged: bool
    residual: float           # |r| / |rho~| at exit
    A_diel: float


def solve(R, S, eps, rho_t, tol: float = 1e-10, max_iter: int = 500) -> SolveResult:
    """Preconditioned CG for hessian(phi~) = rho~ on G != 0; A_diel of the result."""
    rho_t = np.asarray(rho_t, dtype=np.complex128).copy()
    G = box_G(R, S)
    g0 = np.einsum("ij,ij->i", G, G) == 0
    rho_t[g0] = 0.0
    x = np.zeros_like(rho_t)
    r = rho_t.copy()
    bnorm = np.linalg.norm(rho_t)
    z = coulomb(R, S, r)
    d = z.copy()
    rz = np.vdot(r, z).real
    it = 0
    res = np.linalg.norm(r) / bnorm if bnorm > 0 else 0.0
    while res > tol and it < max_iter:
        Hd = hessian(R, S, eps, d)
        alpha = rz / np.vdot(d, Hd).real
        x = x + alpha * d
        r = r - alpha * Hd
        it += 1
        res = np.linalg.norm(r) / bnorm
        if res <= tol:
            break
        z = coulomb(R, S, r)
        rz_new = np.vdot(r, z).real
        d = z + (rz_new / rz) * d
        rz = rz_new
    Omega = pw.cell_volume(R)
    A = 0.5 * np.vdot(x - coulomb(R, S, rho_t), Omega * rho_t).real
    return SolveResult(x, it, res <= tol, float(res), float(A))
