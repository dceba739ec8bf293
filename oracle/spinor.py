"""FP64 oracle of two-component (spinor) bands in a noncollinear potential.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  Nothing here is shared
with the CUDA library.

The JDFTx paper lists noncollinear magnetism and spin-orbit coupling among
its electronic features (Sec. 2.2, "spin-polarized, noncollinear") and holds
wavefunctions in ColumnBundles (Sec. 2.1); it prints no formula.  Readings:

  * A spinor band is two plane-wave blocks on the same sphere, (C_up, C_dn).
    Blocks here are (npw, 2 nb) arrays whose columns alternate up, down:
    column 2b is band b's up component, column 2b + 1 its down component.
  * The local potential is a 2 x 2 Hermitian field V(r) 1 + M(r) . sigma, with
    the Pauli matrices sigma_x = [[0, 1], [1, 0]], sigma_y = [[0, -i], [i, 0]],
    sigma_z = [[1, 0], [0, -1]]:
        phi_up = (V + M_z) psi_up + (M_x - i M_y) psi_dn
        phi_dn = (M_x + i M_y) psi_up + (V - M_z) psi_dn
  * H C = Omega [T C + J phi] + P D P^dag C per component (kinetic and
    projectors act on each component alike: no spin-orbit term).
  * Density and magnetisation of occupations f_b:
        n   = sum_b f_b (|psi_up|^2 + |psi_dn|^2)
        m_x = sum_b f_b 2 Re(conj(psi_up) psi_dn)
        m_y = sum_b f_b 2 Im(conj(psi_up) psi_dn)
        m_z = sum_b f_b (|psi_up|^2 - |psi_dn|^2)
"""
from __future__ import annotations

import numpy as np

from . import planewave as pw


def apply_H_spinor(basis: pw.Basis, V, M, C, P=None, D=None) -> np.ndarray:
    """H C for an interleaved spinor block C (npw, 2 nb); M: (3, N) real."""
    C = np.asarray(C, dtype=np.complex128)
    psi = pw.op_I(basis.iG, basis.S, C).reshape(C.shape[1], -1)
    up, dn = psi[0::2], psi[1::2]
    V = np.asarray(V, dtype=np.float64).reshape(-1)
    Mx, My, Mz = (np.asarray(M, dtype=np.float64).reshape(3, -1)[i] for i in range(3))
    phi = np.empty_like(psi)
    phi[0::2] = (V + Mz) * up + (Mx - 1j * My) * dn
    phi[1::2] = (Mx + 1j * My) * up + (V - Mz) * dn
    HC = basis.Omega * (basis.T[:, None] * C + pw.op_J(basis.iG, basis.S, phi.reshape((-1,) + basis.S)))
    if P is not None:
        HC = HC + P @ (np.asarray(D) @ (P.conj().T @ C))
    return HC


def density_spinor(basis: pw.Basis, C, f, weight: float = 1.0):
    """(n, m) with m of shape (3, N), for an interleaved spinor block."""
    C = np.asarray(C, dtype=np.complex128)
    psi = pw.op_I(basis.iG, basis.S, C).reshape(C.shape[1], -1)
    up, dn = psi[0::2], psi[1::2]
    f = np.asarray(f, dtype=np.float64)[:, None]
    au, ad = np.abs(up) ** 2, np.abs(dn) ** 2
    x = np.conj(up) * dn
    n = weight * np.sum(f * (au + ad), axis=0)
    m = weight * np.stack([np.sum(f * 2 * x.real, axis=0), np.sum(f * 2 * x.imag, axis=0),
                           np.sum(f * (au - ad), axis=0)])
    return n, m
