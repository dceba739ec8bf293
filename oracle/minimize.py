"""FP64 oracle of the preconditioned band conjugate-gradient minimiser.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The JDFTx paper names variational minimisation by nonlinear conjugate
gradients (Sec. 2.1, class Minimize) and the stable variational total-energy
minimiser (Sec. 2.2) but prints no algorithm.  Reading used here, for a fixed
local potential (non-self-consistent), all bands at once:

  state      C (npw x nb) with C^dag O C = 1, O = Omega
  energy     E = f tr(C^dag H C)            (f = 2 for every band)
  gradient   G = H C - O C (C^dag H C)      (the residual block; zero at a
             stationary point, where C spans an invariant subspace)
  residual   ||G||_F / sqrt(Omega), the Frobenius norm of the residual
             block of the normalised eigenproblem.  It is invariant under
             rotations within the subspace and bounds every band's residual
             after rotation to the subspace eigenbasis Q, ||(G Q)_b|| /
             sqrt(Omega); converged when it is below tol
  precond.   K G per coefficient, then projected: K G - C (C^dag O K G)
             Teter (Teter, Payne & Allan, PRB 40, 12255 (1989)):
             K(x) = (27 + 18x + 12x^2 + 8x^3) / (27 + 18x + 12x^2 + 8x^3 + 16x^4),
             x = (1/2)|k+G|^2 / T_b, T_b the band's kinetic energy
  direction  Polak-Ribiere: d = -K G + beta d_prev, beta = <G, KG - KG_prev> / <G_prev, KG_prev>,
             reset to 0 when negative; d projected to be O-orthogonal to C
  line step  E(lambda) along Y = C + lambda d is expanded to second order
             with the small matrices C^dag H d, d^dag H d, d^dag O d (one
             application of H to d per iteration):
               E(l)/f = tr A0 + l a1 + l^2 a2,   a1 = 2 Re tr(C^dag H d),
               a2 = tr(d^dag H d) - Re tr(A0 d^dag O d)
             lambda = -a1 / (2 a2) (when a2 > 0), halved while the exact
             E(lambda) = f tr[(Y^dag H Y)(Y^dag O Y)^{-1}] exceeds E(0) by
             more than rounding (64 ulp of |E|: near convergence the energy
             change, ~ residual^2, is below FP64 resolution)
  update     Y = C + lambda d, HY = HC + lambda Hd; U = Y^dag O Y = L L^dag
             (Cholesky); C = Y L^{-dag}, HC = HY L^{-dag}.

Preconditioners are plain functions (basis, C, G, h) -> K G, h being the
bands' Rayleigh quotients diag(C^dag H C), so the learned one plugs in beside
Teter and the identity.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import planewave as pw


def teter(x):
    """Teter-Payne-Allan preconditioner polynomial ratio."""
    x = np.asarray(x, dtype=np.float64)
    num = 27.0 + x * (18.0 + x * (12.0 + 8.0 * x))
    return num / (num + 16.0 * x ** 4)


def band_kinetic(basis: pw.Basis, C) -> np.ndarray:
    """T_b = Omega sum_G (1/2)|k+G|^2 |C_Gb|^2 for O-normalised bands."""
    return basis.Omega * np.einsum("g,gb->b", basis.T, np.abs(C) ** 2)


def precond_identity(basis, C, G, h=None):
    return G.copy()


def precond_teter(basis, C, G, h=None):
    Tb = band_kinetic(basis, C)
    return teter(basis.T[:, None] / Tb[None, :]) * G


@dataclass
class MinResult:
    C: np.ndarray
    HC: np.ndarray
    eigs: np.ndarray
    energy: float
    iterations: int
    converged: bool
    residual: float
    history: list = field(default_factory=list)


def residual_norms(basis, C, HC):
    """Per-band residuals of the normalised eigenproblem (after rotation to the
    subspace eigenbasis), the subspace eigenvalues, C^dag H C and the gradient."""
    Hs = C.conj().T @ HC
    Hs = 0.5 * (Hs + Hs.conj().T)
    eps, Q = np.linalg.eigh(Hs)
    G = HC - basis.Omega * C @ Hs
    r = np.linalg.norm(G @ Q, axis=0) / np.sqrt(basis.Omega)
    return r, eps, Hs, G


def residual_frobenius(basis, G) -> float:
    return float(np.linalg.norm(G) / np.sqrt(basis.Omega))


def minimize_bands(basis: pw.Basis, Happly, C0, precond=precond_teter, tol=1e-8, max_iter=1000, f=2.0,
                   record=None) -> MinResult:
    """Minimise E = f tr(C^dag H C) over O-orthonormal C, starting from C0.

    Happly(X) returns H X for an (npw, m) block.  `record`, if given, is
    called as record(it, C, G, KG, h) every iteration, h = diag(C^dag H C).
    """
    Om = basis.Omega
    C = pw.lowdin(np.asarray(C0, dtype=np.complex128), Om)
    HC = Happly(C)
    d_prev = None
    KG_prev = G_prev = None
    hist = []
    for it in range(max_iter + 1):
        r, eps, Hs, G = residual_norms(basis, C, HC)
        E = f * float(np.trace(Hs).real)
        res = residual_frobenius(basis, G)
        hist.append((E, res))
        if res < tol:
            return MinResult(C, HC, eps, E, it, True, res, hist)
        if it == max_iter:
            break
        KG = precond(basis, C, G, np.real(np.diag(Hs)))
        KG = KG - C @ (Om * (C.conj().T @ KG))
        if record is not None:
            record(it, C, G, KG, np.real(np.diag(Hs)))
        beta = 0.0
        if d_prev is not None:
            beta = np.vdot(G, KG - KG_prev).real / np.vdot(G_prev, KG_prev).real
            beta = max(beta, 0.0)
        d = -KG + beta * d_prev if d_prev is not None else -KG
        d = d - C @ (Om * (C.conj().T @ d))
        Hd = Happly(d)
        a1 = 2.0 * np.vdot(HC, d).real
        dHd = d.conj().T @ Hd
        dOd = Om * (d.conj().T @ d)
        a2 = float(np.trace(dHd).real - np.trace(Hs @ dOd).real)
        if a1 >= 0:               # not a descent direction: restart along -KG
            d = -KG
            Hd = Happly(d)
            a1 = 2.0 * np.vdot(HC, d).real
            dHd = d.conj().T @ Hd
            dOd = Om * (d.conj().T @ d)
            a2 = float(np.trace(dHd).real - np.trace(Hs @ dOd).real)
        lam = -a1 / (2.0 * a2) if a2 > 0 else 1.0
        E0 = E
        noise = 64.0 * np.finfo(np.float64).eps * abs(E0)
        for _ in range(30):
            Y = C + lam * d
            HY = HC + lam * Hd
            U = Om * (Y.conj().T @ Y)
            E1 = f * float(np.trace(np.linalg.solve(U, Y.conj().T @ HY)).real)
            if E1 <= E0 + noise:
                break
            lam *= 0.5
        L = np.linalg.cholesky(U)
        Linv_h = np.linalg.inv(L).conj().T
        C = Y @ Linv_h
        HC = HY @ Linv_h
        d_prev, KG_prev, G_prev = d, KG, G
    r, eps, Hs, G = residual_norms(basis, C, HC)
    return MinResult(C, HC, eps, f * float(np.trace(Hs).real), max_iter, False, residual_frobenius(basis, G), hist)
