"""GPU parity of the spinor calls (noncollinear potential V + M.sigma; paper
Sec. 2.2 noncollinear magnetism, Sec. 2.1 ColumnBundles) against the FP64
oracle (oracle/spinor.py), through the C ABI."""
from __future__ import annotations

import numpy as np
import pytest

from oracle import planewave as pw
from oracle import spinor
from synth import WORKLOADS, atom_positions, random_coefficients

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1708_03621_gb300 import jdft  # noqa: E402

DEV = torch.device("cuda:0")
TOL = {"fp64": 1e-10, "fp32": 2e-5, "bf16x3": 2e-5}


def _field(R, S, seed):
    rng = np.random.default_rng(seed)
    r = pw.grid_points(R, S)
    B = pw.reciprocal(R)
    M = np.empty((3, r.shape[0]))
    for c in range(3):
        G = B @ rng.integers(-2, 3, size=3)
        M[c] = 0.3 * rng.normal() + 0.2 * np.cos(r @ G + rng.normal())
    return M


CASES = {
    "tiny": (np.diag([6.0, 6.5, 5.5]), (12, 15, 10), (0.1, 0.2, 0.3), 3.0, 2, 3),
    # 16 x 12 planes: the band-pair plane kernel serves them (the fused FP32 spinor pass)
    "pair16x12": (WORKLOADS["tiny_ortho"].R, WORKLOADS["tiny_ortho"].S, WORKLOADS["tiny_ortho"].kfrac[0],
                  WORKLOADS["tiny_ortho"].ecut, 3, 5),
    # the 128^3 workload with a few spinor bands (fused FP32 pass on 128 x 128 planes)
    "large": (WORKLOADS["large"].R, WORKLOADS["large"].S, WORKLOADS["large"].kfrac[0], WORKLOADS["large"].ecut,
              WORKLOADS["large"].natoms, 4),
    "small": (WORKLOADS["small"].R, WORKLOADS["small"].S, WORKLOADS["small"].kfrac[0], WORKLOADS["small"].ecut,
              WORKLOADS["small"].natoms, 16),
}


def _setup(case, prec):
    R, S, k, ecut, natoms, nb = CASES[case]
    atoms = atom_positions(R, natoms, 21)
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
    C = random_coefficients(2 * ob.T, 2 * nb, 22)            # (2 nb, npw): rows up, down, up, ...
    ct = torch.complex128 if prec == "fp64" else torch.complex64
    return ob, V, P, D, basis, C, torch.tensor(C, device=DEV).to(ct), nb


SPIN_CASES = [(c, p) for c in ("tiny", "pair16x12", "small") for p in ("fp64", "fp32")]
SPIN_CASES += [("small", "bf16x3"), ("large", "fp32"), ("large", "bf16x3")]


@pytest.mark.parametrize("case,prec", SPIN_CASES, ids=[f"{c}-{p}" for c, p in SPIN_CASES])
def test_apply_H_spinor_matches_oracle(case, prec):
    ob, V, P, D, basis, C, Cd, nb = _setup(case, prec)
    M = _field(ob.R, ob.S, 23)
    HC = torch.empty_like(Cd)
    jdft.jdft_apply_H_spinor(basis, 0, torch.tensor(M.reshape(-1), device=DEV), Cd, HC, prec)
    torch.cuda.synchronize()
    ref = spinor.apply_H_spinor(ob, V, M, C.T, P, D).T
    got = HC.cpu().numpy()
    err = np.max(np.linalg.norm(got - ref, axis=1) / np.linalg.norm(ref, axis=1))
    assert err < TOL[prec], err
    basis.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_density_spinor_matches_oracle(prec):
    ob, V, P, D, basis, C, Cd, nb = _setup("small", prec)
    f = np.linspace(2.0, 0.5, nb)
    N = ob.N
    n = torch.zeros(N, dtype=torch.float64, device=DEV)
    m = torch.zeros(3 * N, dtype=torch.float64, device=DEV)
    jdft.jdft_density_spinor(basis, 0, Cd, torch.tensor(f, device=DEV), n, m, prec)
    torch.cuda.synchronize()
    n_ref, m_ref = spinor.density_spinor(ob, C.T, f)
    tol = TOL[prec]
    assert np.max(np.abs(n.cpu().numpy() - n_ref)) < tol * np.max(n_ref)
    assert np.max(np.abs(m.cpu().numpy().reshape(3, N) - m_ref)) < tol * np.max(n_ref)
    basis.close()


def test_uniform_field_is_the_scalar_operator_plus_zeeman_term():
    """M uniform = m0: H_spinor C = H C (each row) + Omega (m0.sigma) C (no oracle involved)."""
    ob, V, P, D, basis, C, Cd, nb = _setup("small", "fp64")
    m0 = np.array([0.05, -0.12, 0.08])
    M = torch.tensor(np.repeat(m0[:, None], ob.N, axis=1).reshape(-1), device=DEV)
    HC = torch.empty_like(Cd)
    jdft.jdft_apply_H_spinor(basis, 0, M, Cd, HC, "fp64")
    H0 = torch.empty_like(Cd)
    jdft.jdft_apply_H(basis, 0, Cd, H0, "fp64")
    torch.cuda.synchronize()
    up, dn = C[0::2], C[1::2]
    Z = np.empty_like(C)
    Z[0::2] = m0[2] * up + (m0[0] - 1j * m0[1]) * dn
    Z[1::2] = (m0[0] + 1j * m0[1]) * up - m0[2] * dn
    want = H0.cpu().numpy() + ob.Omega * Z
    got = HC.cpu().numpy()
    assert np.max(np.abs(got - want)) < 1e-12 * np.max(np.abs(want))
    basis.close()


def test_single_spinor_band_on_the_fused_pass():
    """One spinor band (a single (up, down) pair) through the fused FP32 pass."""
    ob, V, P, D, basis, C, Cd, nb = _setup("pair16x12", "fp32")
    C1, Cd1 = C[:2], Cd[:2].contiguous()
    M = _field(ob.R, ob.S, 29)
    HC = torch.empty_like(Cd1)
    jdft.jdft_apply_H_spinor(basis, 0, torch.tensor(M.reshape(-1), device=DEV), Cd1, HC, "fp32")
    torch.cuda.synchronize()
    ref = spinor.apply_H_spinor(ob, V, M, C1.T, P, D).T
    err = np.max(np.linalg.norm(HC.cpu().numpy() - ref, axis=1) / np.linalg.norm(ref, axis=1))
    assert err < TOL["fp32"], err
    basis.close()
