"""Test systems built twice: once by the oracle (CPU, FP64) and once by the
GPU library through its C ABI, from the same seeded inputs (synth)."""
from __future__ import annotations

import numpy as np

from oracle import planewave as pw
from synth import WORKLOADS, Workload, atom_positions, random_coefficients, workload_atoms


class OracleSystem:
    def __init__(self, w: Workload, ik: int = 0, with_projectors: bool = True):
        self.w = w
        self.R = w.R
        self.atoms = workload_atoms(w)
        self.basis = pw.Basis.build(w.R, w.S, w.kfrac[ik], w.ecut)
        self.V = pw.vloc_realspace(w.R, w.S, self.atoms)
        if with_projectors:
            self.P = pw.projectors(w.R, self.basis.kfrac, self.basis.iG, self.atoms)
            self.D = pw.dmatrix(w.natoms)
        else:
            self.P = self.D = None

    def coeffs(self, nb=None, seed=None) -> np.ndarray:
        """Band-major (nb, npw) random block, damped by 1 + |k+G|^2."""
        nb = self.w.nbands if nb is None else nb
        seed = self.w.seed_coeffs if seed is None else seed
        return random_coefficients(2 * self.basis.T, nb, seed)

    def apply_H(self, Cbm: np.ndarray) -> np.ndarray:
        return pw.apply_H(self.basis, self.V, Cbm.T, self.P, self.D).T


class GpuSystem:
    def __init__(self, w: Workload, atoms, with_projectors: bool = True, device="cuda:0"):
        import torch

        from paper_1708_03621_gb300 import jdft
        self.jdft = jdft
        self.dev = torch.device(device)
        self.basis = jdft.Basis(w.R, w.S, w.ecut, w.kfrac, w.weights())
        self.N = int(np.prod(w.S))
        self.V = torch.empty(self.N, dtype=torch.float64, device=self.dev)
        jdft.jdft_gaussian_potential(self.basis, atoms, self.V)
        jdft.jdft_set_potential(self.basis, self.V)
        self.P = []
        for ik in range(w.nk):
            if with_projectors:
                P = torch.empty((4 * len(atoms), self.basis.npw(ik)), dtype=torch.complex128, device=self.dev)
                jdft.jdft_gaussian_projectors(self.basis, ik, atoms, P)
                D = torch.tensor(pw_dmatrix(len(atoms)), device=self.dev)
                jdft.jdft_set_projectors(self.basis, ik, P, D)
                self.P.append(P)
        torch.cuda.synchronize()


def pw_dmatrix(natoms):
    # Same block-diagonal D the oracle uses, written out as data (not imported from the oracle's code path
    # to the library: the library receives it as an input).
    return np.diag(np.tile([0.5, -0.3, -0.3, -0.3], natoms))


def band_rel_err(got: np.ndarray, ref: np.ndarray) -> float:
    """max over bands of ||got_b - ref_b|| / ||ref_b|| (band-major arrays)."""
    num = np.linalg.norm(got - ref, axis=-1)
    den = np.linalg.norm(ref, axis=-1)
    return float(np.max(num / np.maximum(den, 1e-300)))


def workload(name: str) -> Workload:
    return WORKLOADS[name]
