"""FP64 oracle of the self-consistent field (SCF) loop around the band solve.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  Nothing here is shared
with the CUDA library.

The JDFTx paper names the pieces but prints no formula for them: the Coulomb
kernel (class Coulomb) and the exchange-correlation functionals (class ExCorr,
local-density approximation among the "semilocal" ones), Sec. 2.1 and 2.2;
"self-consistency by Pulay mixing" (class Pulay, Sec. 2.1) as the alternative
to total-energy minimisation (Sec. 2.2).  The readings used here:

Hartree (3-D periodic Coulomb kernel, uniform neutralising background)
  nt = J n on the full box, frequencies folded to [-S/2, S/2) per axis,
  G = B iG.  V_H(G) = 4 pi nt(G) / |G|^2 for G != 0, V_H(0) = 0;
  V_H(r) = I V_H (real part).  E_H = (Omega/2) sum_{G != 0} 4 pi |nt(G)|^2 / |G|^2.

LDA (spin-unpolarised)
  r_s = (3 / (4 pi n))^{1/3}.
  Exchange (Dirac/Slater): e_x = -(3/4) (3/pi)^{1/3} n^{1/3}, v_x = (4/3) e_x.
  Correlation: the Perdew-Zunger 1981 fit (Phys. Rev. B 23, 5048) to the
  Ceperley-Alder electron gas,
    r_s >= 1:  e_c = g / (1 + b1 sqrt(r_s) + b2 r_s),  g = -0.1423, b1 = 1.0529, b2 = 0.3334
    r_s <  1:  e_c = A ln r_s + B + C r_s ln r_s + D r_s,
               A = 0.0311, B = -0.048, C = 0.0020, D = -0.0116
    v_c = e_c - (r_s / 3) de_c/dr_s.
  n <= 0 (possible after mixing) gives e_xc = v_xc = 0.
  E_xc = (Omega/N) sum_j n_j e_xc(n_j).

Kohn-Sham potential  V_KS[n] = V_ion + V_H[n] + V_xc[n].

Total energy of the orbitals C found in V_KS[n_in], with output density n_out:
  E = sum_k w_k sum_b f eps_kb - (Omega/N) sum_j n_out,j (V_H[n_in] + V_xc[n_in])_j
      + E_H[n_out] + E_xc[n_out]
  i.e. the Kohn-Sham functional of C (kinetic + nonlocal + int V_ion n_out +
  E_H + E_xc at n_out), written with the band-energy sum.

Pulay mixing (P. Pulay, Chem. Phys. Lett. 73, 393 (1980)), on the density
  Keep the last m pairs (n_in^i, R^i = n_out^i - n_in^i).  Coefficients c
  minimise |sum_i c_i R^i|^2 subject to sum_i c_i = 1: the bordered system
    [A 1; 1^T 0] [c; lam] = [0; 1],  A_ij = <R^i, R^j> (plain sum over the box).
  It is solved by Gaussian elimination with partial pivoting; when a pivot
  falls below 1e-13 times the largest |A_ii| the oldest pair is dropped and
  the system solved again.  Next input: n_in = sum_i c_i (n_in^i + alpha R^i).

SCF loop: n_in = density of the starting orbitals; repeat { V_KS[n_in];
lowest nb eigenpairs of H at every k; n_out; E; converged when
|E - E_prev| < tol_energy and sqrt((Omega/N) sum R^2) < tol_density;
else n_in = Pulay(n_in, n_out) }.  The band solve here is dense
diagonalisation of the plane-wave Hamiltonian (exact for the small cells it
is used on).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import cfft
from . import planewave as pw

FOUR_PI = 4.0 * np.pi

# --------------------------------------------------------------------------
# Hartree
# --------------------------------------------------------------------------


def coulomb_kernel(R, S) -> np.ndarray:
    """4 pi / |G|^2 on the box's folded frequencies (0 at G = 0), flat."""
    g = pw.signed_box_frequencies(S).astype(np.float64)
    G = g @ pw.reciprocal(R).T
    G2 = np.einsum("ij,ij->i", G, G)
    K = np.zeros_like(G2)
    nz = G2 > 0
    K[nz] = FOUR_PI / G2[nz]
    return K


def hartree(R, S, n):
    """(V_H flat real, E_H) of the real density n (flat, linear-index order)."""
    S = tuple(int(s) for s in S)
    N = int(np.prod(S))
    Omega = pw.cell_volume(R)
    nt = cfft.fft3d(np.asarray(n, dtype=np.float64).reshape(S), -1).reshape(-1) / N
    K = coulomb_kernel(R, S)
    VH = cfft.fft3d((K * nt).reshape(S), +1).reshape(-1).real.copy()
    EH = 0.5 * Omega * float(np.sum(K * (nt.real ** 2 + nt.imag ** 2)))
    return VH, EH


# --------------------------------------------------------------------------
# LDA exchange-correlation
# --------------------------------------------------------------------------

PZ_GAMMA, PZ_BETA1, PZ_BETA2 = -0.1423, 1.0529, 0.3334
PZ_A, PZ_B, PZ_C, PZ_D = 0.0311, -0.048, 0.0020, -0.0116


def lda_pz(n):
    """(e_xc, v_xc) per point: Slater exchange + Perdew-Zunger 1981 correlation."""
    n = np.asarray(n, dtype=np.float64)
    e = np.zeros_like(n)
    v = np.zeros_like(n)
    pos = n > 0
    x = n[pos]
    ex = -0.75 * (3.0 / np.pi) ** (1.0 / 3.0) * np.cbrt(x)
    vx = (4.0 / 3.0) * ex
    rs = np.cbrt(3.0 / (4.0 * np.pi * x))
    ec = np.empty_like(x)
    vc = np.empty_like(x)
    hi = rs >= 1.0
    r = rs[hi]
    sq = np.sqrt(r)
    den = 1.0 + PZ_BETA1 * sq + PZ_BETA2 * r
    ec[hi] = PZ_GAMMA / den
    # de/drs = -g (b1 / (2 sqrt rs) + b2) / den^2
    dec = -PZ_GAMMA * (0.5 * PZ_BETA1 / sq + PZ_BETA2) / den ** 2
    vc[hi] = ec[hi] - r / 3.0 * dec
    lo = ~hi
    r = rs[lo]
    lr = np.log(r)
    ec[lo] = PZ_A * lr + PZ_B + PZ_C * r * lr + PZ_D * r
    dec = PZ_A / r + PZ_C * (lr + 1.0) + PZ_D
    vc[lo] = ec[lo] - r / 3.0 * dec
    e[pos] = ex + ec
    v[pos] = vx + vc
    return e, v


def xc_energy(Omega, n) -> float:
    """E_xc = (Omega/N) sum_j n_j e_xc(n_j)."""
    n = np.asarray(n, dtype=np.float64)
    e, _ = lda_pz(n)
    return Omega / n.size * float(np.sum(n * e))


def ks_potential(R, S, n, Vion):
    """(V_KS, V_H, V_xc, E_H, E_xc) of density n."""
    Omega = pw.cell_volume(R)
    VH, EH = hartree(R, S, n)
    e, vxc = lda_pz(n)
    Exc = Omega / np.asarray(n).size * float(np.sum(np.asarray(n) * e))
    return np.asarray(Vion, dtype=np.float64) + VH + vxc, VH, vxc, EH, Exc


# --------------------------------------------------------------------------
# Pulay mixing
# --------------------------------------------------------------------------


def _solve_bordered(A: np.ndarray):
    """Solve [A 1; 1^T 0][c; lam] = [0; 1] by Gaussian elimination with partial
    pivoting.  Returns c, or None when a pivot is below 1e-13 max|A_ii|."""
    m = A.shape[0]
    M = np.zeros((m + 1, m + 2))
    M[:m, :m] = A
    M[:m, m] = 1.0
    M[m, :m] = 1.0
    M[m, m + 1] = 1.0
    thresh = 1e-13 * float(np.max(np.abs(np.diag(A))))
    for col in range(m + 1):
        p = col + int(np.argmax(np.abs(M[col:, col])))
        if abs(M[p, col]) <= thresh:
            return None
        if p != col:
            M[[col, p]] = M[[p, col]]
        for r in range(col + 1, m + 1):
            M[r, col:] -= (M[r, col] / M[col, col]) * M[col, col:]
    x = np.zeros(m + 1)
    for r in range(m, -1, -1):
        x[r] = (M[r, m + 1] - M[r, r + 1:m + 1] @ x[r + 1:m + 1]) / M[r, r]
    return x[:m]


@dataclass
class Pulay:
    """Density mixer: keeps the last `history` (n_in, residual) pairs."""
    history: int = 8
    alpha: float = 0.5
    n_in: list = field(default_factory=list)
    res: list = field(default_factory=list)
    used: int = 0            # pairs used by the last step

    def step(self, n_in, n_out) -> np.ndarray:
        n_in = np.asarray(n_in, dtype=np.float64)
        self.n_in.append(n_in.copy())
        self.res.append(np.asarray(n_out, dtype=np.float64) - n_in)
        if len(self.n_in) > self.history:
            self.n_in.pop(0)
            self.res.pop(0)
        first = 0
        while True:
            Rs = self.res[first:]
            A = np.array([[float(np.dot(a, b)) for b in Rs] for a in Rs])
            c = _solve_bordered(A)
            if c is not None or len(Rs) == 1:
                break
            first += 1
        if c is None:          # a single zero residual: the input is a fixed point
            c = np.ones(1)
        self.used = len(Rs)
        out = np.zeros_like(n_in)
        for ci, ni, ri in zip(c, self.n_in[first:], Rs):
            out += ci * (ni + self.alpha * ri)
        return out


# --------------------------------------------------------------------------
# The SCF loop
# --------------------------------------------------------------------------


@dataclass
class KCell:
    """One k-point of the cell: basis, projectors (or None), D, weight, start orbitals."""
    basis: pw.Basis
    P: object
    D: object
    weight: float
    C0: np.ndarray           # (npw, nb)


@dataclass
class ScfResult:
    energy: float
    n: np.ndarray
    eigs: list
    C: list
    iterations: int
    converged: bool
    residual: float
    parts: dict
    history: list


def lowest_bands(basis: pw.Basis, V, P, D, nb: int):
    """Lowest nb eigenpairs of the pencil (H, Omega 1) by dense diagonalisation.
    Returns (eigs, C) with C^dag O C = 1."""
    H = pw.dense_H(basis, V, P, D)
    w, Q = np.linalg.eigh(0.5 * (H + H.conj().T))
    return w[:nb] / basis.Omega, Q[:, :nb] / np.sqrt(basis.Omega)


def direct_energy(cells, C, Vion, f: float):
    """Kohn-Sham functional of the orbitals, without eigenvalues:
    sum_k w_k f sum_b <C_b| Omega T + P D P^dag |C_b> + int V_ion n + E_H[n] + E_xc[n]."""
    b0 = cells[0].basis
    n = np.zeros(b0.N)
    Ekin_nl = 0.0
    for kc, Ck in zip(cells, C):
        n += pw.density(kc.basis, Ck, np.full(Ck.shape[1], f), kc.weight)
        TC = kc.basis.Omega * kc.basis.T[:, None] * Ck
        if kc.P is not None:
            TC = TC + kc.P @ (np.asarray(kc.D) @ (kc.P.conj().T @ Ck))
        Ekin_nl += kc.weight * f * float(np.real(np.sum(Ck.conj() * TC)))
    Omega = b0.Omega
    _, EH = hartree(b0.R, b0.S, n)
    return Ekin_nl + Omega / b0.N * float(np.dot(Vion, n)) + EH + xc_energy(Omega, n), n


def scf(cells, Vion, f: float = 2.0, alpha: float = 0.5, history: int = 8, tol_energy: float = 1e-9,
        tol_density: float = 1e-7, max_iter: int = 100) -> ScfResult:
    """Pulay-mixed SCF for fixed occupations f on every band of every k-point."""
    b0 = cells[0].basis
    R, S, N, Omega = b0.R, b0.S, b0.N, b0.Omega
    n_in = np.zeros(N)
    for kc in cells:
        C = pw.lowdin(kc.C0, kc.basis.Omega)
        n_in += pw.density(kc.basis, C, np.full(C.shape[1], f), kc.weight)
    mixer = Pulay(history, alpha)
    E_prev = None
    hist = []
    for it in range(1, max_iter + 1):
        Vks, VH, vxc, _, _ = ks_potential(R, S, n_in, Vion)
        eigs, Cs = [], []
        n_out = np.zeros(N)
        Eband = 0.0
        for kc in cells:
            nb = kc.C0.shape[1]
            w, C = lowest_bands(kc.basis, Vks, kc.P, kc.D, nb)
            eigs.append(w)
            Cs.append(C)
            Eband += kc.weight * f * float(np.sum(w))
            n_out += pw.density(kc.basis, C, np.full(nb, f), kc.weight)
        Edc = -Omega / N * float(np.dot(n_out, VH + vxc))
        _, EH = hartree(R, S, n_out)
        Exc = xc_energy(Omega, n_out)
        E = Eband + Edc + EH + Exc
        res = float(np.sqrt(Omega / N * np.sum((n_out - n_in) ** 2)))
        hist.append((E, res))
        parts = {"band": Eband, "double_counting": Edc, "hartree": EH, "xc": Exc}
        if E_prev is not None and abs(E - E_prev) < tol_energy and res < tol_density:
            return ScfResult(E, n_out, eigs, Cs, it, True, res, parts, hist)
        E_prev = E
        n_in = mixer.step(n_in, n_out)
    return ScfResult(E, n_out, eigs, Cs, max_iter, False, res, parts, hist)
