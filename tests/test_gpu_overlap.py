"""GPU parity of the augmented overlap S = Omega + P Q P^dag and the
generalised Rayleigh-Ritz / orthonormalisation (ultrasoft pseudopotentials,
paper Sec. 2.2; the overlap operator O, Sec. 2.1) against the FP64 oracle
(oracle/ultrasoft.py), through the C ABI."""
from __future__ import annotations

import numpy as np
import pytest
import scipy.linalg

from oracle import planewave as pw
from oracle import ultrasoft as us
from synth import WORKLOADS, atom_positions, random_coefficients

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1708_03621_gb300 import jdft  # noqa: E402

DEV = torch.device("cuda:0")

CASES = {
    "tiny": (np.diag([6.0, 6.5, 5.5]), (12, 15, 10), (0.1, 0.2, 0.3), 3.0, 2, 5),
    "cell24": (np.diag([8.0, 8.5, 7.5]), (24, 25, 20), (0.1, 0.2, 0.3), 6.0, 4, 8),
    "small": (WORKLOADS["small"].R, WORKLOADS["small"].S, WORKLOADS["small"].kfrac[0], WORKLOADS["small"].ecut,
              WORKLOADS["small"].natoms, 16),
    # the bench's S C workload (128^3, 256 projectors), 32 sampled bands of its 256
    "large": (WORKLOADS["large"].R, WORKLOADS["large"].S, WORKLOADS["large"].kfrac[0], WORKLOADS["large"].ecut,
              WORKLOADS["large"].natoms, 32),
}


def _Q(natoms):
    Q = np.diag(np.tile([0.4, 0.1, 0.1, 0.1], natoms))
    for a in range(natoms - 1):          # couple neighbouring atoms' s channels too
        Q[4 * a, 4 * a + 4] = Q[4 * a + 4, 4 * a] = 0.05
    return Q


def _setup(case):
    R, S, k, ecut, natoms, nb = CASES[case]
    atoms = atom_positions(R, natoms, 31)
    ob = pw.Basis.build(R, S, k, ecut)
    V = pw.vloc_realspace(R, S, atoms)
    P = pw.projectors(R, ob.kfrac, ob.iG, atoms)
    D = pw.dmatrix(natoms)
    basis = jdft.Basis(R, S, ecut, [k])
    Vd = torch.empty(int(np.prod(S)), dtype=torch.float64, device=DEV)
    jdft.jdft_gaussian_potential(basis, atoms, Vd)
    jdft.jdft_set_potential(basis, Vd)
    Pd = torch.empty((4 * natoms, basis.npw(0)), dtype=torch.complex128, device=DEV)
    jdft.jdft_gaussian_projectors(basis, 0, atoms, Pd)
    jdft.jdft_set_projectors(basis, 0, Pd, torch.tensor(np.diag(np.tile([0.5, -0.3, -0.3, -0.3], natoms)),
                                                        device=DEV))
    Q = _Q(natoms)
    jdft.jdft_set_augmentation(basis, 0, torch.tensor(Q, device=DEV))
    C = random_coefficients(2 * ob.T, nb, 32)        # (nb, npw)
    return ob, V, P, D, Q, basis, C, nb


OPS_CASES = [(c, p, t) for c in ("tiny", "small") for p, t in (("fp64", 1e-12), ("fp32", 1e-6), ("bf16x3", 2e-6))]
OPS_CASES += [("large", "bf16x3", 2e-6)]


@pytest.mark.parametrize("case,prec,tol", OPS_CASES, ids=[f"{c}-{p}" for c, p, _ in OPS_CASES])
def test_op_S_matches_oracle(case, prec, tol):
    ob, V, P, D, Q, basis, C, nb = _setup(case)
    ct = torch.complex128 if prec == "fp64" else torch.complex64
    Cd = torch.tensor(C, device=DEV).to(ct)
    SC = torch.empty_like(Cd)
    jdft.jdft_op_S(basis, 0, Cd, SC, prec)
    torch.cuda.synchronize()
    ref = us.op_S(ob, C.T, P, Q).T
    err = np.max(np.linalg.norm(SC.cpu().numpy() - ref, axis=1) / np.linalg.norm(ref, axis=1))
    assert err < tol, err
    # cleared augmentation: the plain overlap
    jdft.jdft_set_augmentation(basis, 0, None)
    jdft.jdft_op_S(basis, 0, Cd, SC, prec)
    torch.cuda.synchronize()
    assert np.max(np.abs(SC.cpu().numpy() - ob.Omega * Cd.cpu().numpy())) < 1e-12 * ob.Omega * np.max(np.abs(C))
    basis.close()


@pytest.mark.parametrize("case", ["tiny", "small"])
def test_generalised_subspace_matches_oracle(case):
    ob, V, P, D, Q, basis, C, nb = _setup(case)
    Cd = torch.tensor(C, device=DEV)
    HC = torch.empty_like(Cd)
    jdft.jdft_apply_H(basis, 0, Cd, HC, "fp64")
    CHC = torch.empty((nb, nb), dtype=torch.complex128, device=DEV)
    CSC = torch.empty_like(CHC)
    eigs = torch.empty(nb, dtype=torch.float64, device=DEV)
    jdft.jdft_subspace_generalized(basis, 0, Cd, HC, CHC, CSC, eigs)
    torch.cuda.synchronize()
    HCo = pw.apply_H(ob, V, C.T, P, D)
    A, B, e = us.subspace_generalized(ob, C.T, HCo, P, Q)
    assert np.max(np.abs(CHC.cpu().numpy() - A)) < 1e-12 * np.max(np.abs(A))
    assert np.max(np.abs(CSC.cpu().numpy() - B)) < 1e-12 * np.max(np.abs(B))
    assert np.max(np.abs(eigs.cpu().numpy() - e)) < 1e-10 * max(1.0, np.max(np.abs(e)))
    basis.close()


def test_generalised_orthonormalisation():
    ob, V, P, D, Q, basis, C, nb = _setup("small")
    Cd = torch.tensor(C, device=DEV)
    jdft.jdft_orthonormalize_generalized(basis, 0, Cd)
    HC = torch.empty_like(Cd)
    jdft.jdft_apply_H(basis, 0, Cd, HC, "fp64")
    CHC = torch.empty((nb, nb), dtype=torch.complex128, device=DEV)
    CSC = torch.empty_like(CHC)
    jdft.jdft_subspace_generalized(basis, 0, Cd, HC, CHC, CSC)
    torch.cuda.synchronize()
    assert np.max(np.abs(CSC.cpu().numpy() - np.eye(nb))) < 1e-12
    Co = us.orthonormalize_generalized(ob, C.T, P, Q)
    got = Cd.cpu().numpy().T
    # the same S-orthonormal block up to rounding (Cholesky fixes it uniquely)
    assert np.max(np.abs(got - Co)) < 1e-10 * np.max(np.abs(Co))
    basis.close()


@pytest.mark.parametrize("case,precond", [("tiny", "teter"), ("cell24", "teter"), ("cell24", "identity")])
def test_generalised_minimiser_finds_the_lowest_pencil_eigenvalues(case, precond):
    """GPU band CG for H c = e S c against LAPACK's dense pencil (the oracle's H and S)."""
    ob, V, P, D, Q, basis, C, nb = _setup(case)
    Cd = torch.tensor(C, device=DEV)
    eigs = torch.empty(nb, dtype=torch.float64, device=DEV)
    rep = jdft.jdft_minimize_bands_generalized(basis, 0, Cd, eigs, tol=1e-9, max_iter=3000, precond=precond)
    assert rep["converged"] == 1
    lam = scipy.linalg.eigh(pw.dense_H(ob, V, P, D), us.dense_S(ob, P, Q), eigvals_only=True)[:nb]
    assert np.max(np.abs(np.sort(eigs.cpu().numpy()) - lam)) < 1e-9 * max(1.0, np.max(np.abs(lam)))
    assert rep["energy"] == pytest.approx(2.0 * lam.sum(), abs=1e-8)
    got = Cd.cpu().numpy().T
    assert np.max(np.abs(got.conj().T @ us.op_S(ob, got, P, Q) - np.eye(nb))) < 1e-10
    basis.close()


def test_augmentation_needs_projectors_and_a_symmetric_Q():
    R, S, k = np.diag([6.0, 6.5, 5.5]), (12, 15, 10), (0.1, 0.2, 0.3)
    basis = jdft.Basis(R, S, 3.0, [k])
    with pytest.raises(jdft.JdftError):
        jdft.jdft_set_augmentation(basis, 0, torch.eye(8, dtype=torch.float64, device=DEV))
    atoms = atom_positions(R, 2, 31)
    Pd = torch.empty((8, basis.npw(0)), dtype=torch.complex128, device=DEV)
    jdft.jdft_gaussian_projectors(basis, 0, atoms, Pd)
    jdft.jdft_set_projectors(basis, 0, Pd, torch.eye(8, dtype=torch.float64, device=DEV))
    Q = torch.zeros((8, 8), dtype=torch.float64, device=DEV)
    Q[0, 1] = 0.1
    with pytest.raises(jdft.JdftError):
        jdft.jdft_set_augmentation(basis, 0, Q)
    basis.close()
