"""FP64 oracle of the augmented (ultrasoft-type) overlap and the generalised
eigenproblem it makes.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  Nothing here is shared
with the CUDA library.

The JDFTx paper lists ultrasoft pseudopotentials among its features
(Sec. 2.2) and names the overlap operator O (Sec. 2.1); it prints no
formula.  Readings:

  * With augmentation charges Q (nproj x nproj, real symmetric) on the same
    projectors P as the nonlocal term, the overlap of coefficient blocks is
        S C = Omega C + P Q P^dag C,
    the norm-conserving O = Omega plus the projectors' augmentation (no Omega
    on the second term: P^dag C is already the integral <beta|psi>, as in the
    nonlocal term P D P^dag C).
  * Band energies are the eigenvalues of the pencil (C^dag H C, C^dag S C)
    (generalised Rayleigh-Ritz); orthonormal blocks satisfy C^dag S C = 1,
    reached by C <- C L^{-dag} with C^dag S C = L L^dag.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg

from . import planewave as pw


def op_S(basis: pw.Basis, C, P, Q) -> np.ndarray:
    """S C = Omega C + P Q P^dag C (C: npw x nb)."""
    C = np.asarray(C, dtype=np.complex128)
    return basis.Omega * C + P @ (np.asarray(Q) @ (P.conj().T @ C))


def dense_S(basis: pw.Basis, P, Q) -> np.ndarray:
    return basis.Omega * np.eye(basis.npw) + P @ np.asarray(Q) @ P.conj().T


def subspace_generalized(basis: pw.Basis, C, HC, P, Q):
    """(C^dag H C, C^dag S C, eigenvalues of the pencil) for a block C and H C."""
    C = np.asarray(C, dtype=np.complex128)
    A = C.conj().T @ HC
    B = C.conj().T @ op_S(basis, C, P, Q)
    A = 0.5 * (A + A.conj().T)
    B = 0.5 * (B + B.conj().T)
    return A, B, scipy.linalg.eigh(A, B, eigvals_only=True)


def orthonormalize_generalized(basis: pw.Basis, C, P, Q) -> np.ndarray:
    """C L^{-dag} with C^dag S C = L L^dag."""
    C = np.asarray(C, dtype=np.complex128)
    U = C.conj().T @ op_S(basis, C, P, Q)
    L = np.linalg.cholesky(0.5 * (U + U.conj().T))
    return C @ np.linalg.inv(L).conj().T


def minimize_bands_generalized(basis: pw.Basis, Happly, P, Q, C0, tol: float = 1e-8, max_iter: int = 2000,
                               f: float = 2.0, teter: bool = True):
    """All-band preconditioned CG for the lowest nb states of H c = e S c.

    The norm-conserving minimiser (oracle/minimize.py) with O replaced by S:
      state      C with C^dag S C = 1;  Hs = C^dag H C;  E = f tr Hs
      gradient   G = H C - S C Hs;  converged when ||G||_F / sqrt(Omega) < tol
      direction  K G (Teter, x = (1/2)|k+G|^2 / T_b with T_b = Omega sum kin |C|^2,
                 or K = 1), Polak-Ribiere with reset at beta < 0, projected
                 S-orthogonal to C: d - C (C^dag S d)
      line step  lambda = -a1 / (2 a2), a1 = 2 Re <H C, d>,
                 a2 = Re tr(d^dag H d) - Re tr(Hs d^dag S d); halved while
                 E(Y) = f tr[(Y^dag H Y)(Y^dag S Y)^{-1}] exceeds E by more than
                 64 FP64 ulp of |E|
      update     Y = C + lambda d, C = Y L^{-dag} with Y^dag S Y = L L^dag.
    Returns (C, eigenvalues of the final Hs, iterations, residual)."""
    Om = basis.Omega
    C = orthonormalize_generalized(basis, np.asarray(C0, dtype=np.complex128), P, Q)
    d_prev = KG_prev = G_prev = None
    res = np.inf
    it = 0
    for it in range(max_iter + 1):
        HC = Happly(C)
        SC = op_S(basis, C, P, Q)
        Hs = C.conj().T @ HC
        Hs = 0.5 * (Hs + Hs.conj().T)
        G = HC - SC @ Hs
        res = float(np.linalg.norm(G) / np.sqrt(Om))
        if res < tol or it == max_iter:
            break
        if teter:
            Tb = Om * np.einsum("g,gb->b", basis.T, np.abs(C) ** 2)
            x = basis.T[:, None] / Tb[None, :]
            num = 27.0 + x * (18.0 + x * (12.0 + 8.0 * x))
            KG = (num / (num + 16.0 * x ** 4)) * G
        else:
            KG = G.copy()
        beta = 0.0
        if d_prev is not None:
            beta = max(np.vdot(G, KG - KG_prev).real / np.vdot(G_prev, KG_prev).real, 0.0)
        d = -KG + beta * d_prev if d_prev is not None else -KG
        d = d - C @ (C.conj().T @ op_S(basis, d, P, Q))
        Hd = Happly(d)
        Sd = op_S(basis, d, P, Q)
        a1 = 2.0 * np.vdot(HC, d).real
        if a1 >= 0:
            d = -KG - C @ (C.conj().T @ op_S(basis, -KG, P, Q))
            Hd = Happly(d)
            Sd = op_S(basis, d, P, Q)
            a1 = 2.0 * np.vdot(HC, d).real
        dSd = d.conj().T @ Sd
        a2 = float(np.trace(d.conj().T @ Hd).real - np.trace(Hs @ dSd).real)
        lam = -a1 / (2.0 * a2) if a2 > 0 else 1.0
        E0 = f * float(np.trace(Hs).real)
        noise = 64.0 * np.finfo(np.float64).eps * abs(E0)
        for _ in range(30):
            Y = C + lam * d
            U = Y.conj().T @ (SC + lam * Sd)
            E1 = f * float(np.trace(np.linalg.solve(U, Y.conj().T @ (HC + lam * Hd))).real)
            if E1 <= E0 + noise:
                break
            lam *= 0.5
        L = np.linalg.cholesky(0.5 * (U + U.conj().T))
        C = Y @ np.linalg.inv(L).conj().T
        d_prev, KG_prev, G_prev = d, KG, G
    Hs = C.conj().T @ Happly(C)
    return C, np.linalg.eigvalsh(0.5 * (Hs + Hs.conj().T)), it, res
