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
