"""GPU parity of the SCF pieces against the FP64 oracle (oracle/scf.py):
Hartree potential and energy, LDA exchange-correlation, the fused Kohn-Sham
potential, Pulay mixing and the whole SCF loop (paper Sec. 2.1: Coulomb,
ExCorr, Pulay; Sec. 2.2: SCF by Pulay mixing).  All through the C ABI."""
from __future__ import annotations

import json
import os

import numpy as np
import pytest

from oracle import planewave as pw
from oracle import scf
from synth import WORKLOADS, atom_positions, random_coefficients

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1708_03621_gb300 import jdft  # noqa: E402

DEV = torch.device("cuda:0")
TRICLINIC = np.array([[7.0, 1.2, 0.4], [0.0, 6.5, -0.9], [0.3, 0.0, 8.0]])
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "scf_small.json")


def _smooth_density(R, S, seed):
    """Positive smooth density: Gaussians at random points plus a modulation."""
    atoms = atom_positions(R, 5, seed)
    n = -pw.vloc_realspace(R, S, atoms, depth=0.05, width=1.3)
    r = pw.grid_points(R, S)
    B = pw.reciprocal(R)
    return n + 0.01 * (1.0 + np.cos(r @ B[:, 0] + 0.3))


def _dev(a):
    return torch.tensor(np.ascontiguousarray(a, dtype=np.float64), device=DEV)


def _rel(got, ref):
    return float(np.max(np.abs(got - ref)) / np.max(np.abs(ref)))


BOXES = [
    ("triclinic-18x16x20", TRICLINIC, (18, 16, 20)),
    ("orthorhombic-24x25x20", np.diag([8.0, 8.5, 7.5]), (24, 25, 20)),
    ("cubic-48", np.eye(3) * 10.0, (48, 48, 48)),
    ("cubic-60", np.eye(3) * 12.0, (60, 60, 60)),
    ("mixed-72x80x54", np.diag([14.0, 15.0, 11.0]), (72, 80, 54)),
    ("cubic-128", np.eye(3) * 20.0, (128, 128, 128)),
]


@pytest.mark.parametrize("name,R,S", BOXES, ids=[b[0] for b in BOXES])
def test_hartree_lda_ks_match_oracle(name, R, S):
    basis = jdft.Basis(R, S, 1.0, [(0.0, 0.0, 0.0)])
    n = _smooth_density(R, S, 31)
    n[:7] = [0.0, -1e-9, 1e-30, 3.0, 50.0, 1e-3, 0.2387]     # zero / negative / both r_s branches
    Vion = pw.vloc_realspace(R, S, atom_positions(R, 3, 32))
    VH_ref, EH_ref = scf.hartree(R, S, n)
    e_ref, vxc_ref = scf.lda_pz(n)
    Omega = pw.cell_volume(R)
    Exc_ref = Omega / n.size * float(np.sum(n * e_ref))
    nd, vion = _dev(n), _dev(Vion)
    vh = torch.empty_like(nd)
    vxc = torch.empty_like(nd)
    vks = torch.empty_like(nd)
    eh = torch.zeros(1, dtype=torch.float64, device=DEV)
    ex = torch.zeros(1, dtype=torch.float64, device=DEV)
    en = torch.zeros(2, dtype=torch.float64, device=DEV)
    jdft.jdft_hartree(basis, nd, vh, eh)
    jdft.jdft_xc_lda(basis, nd, vxc, ex)
    jdft.jdft_ks_potential(basis, nd, vion, vks, en)
    torch.cuda.synchronize()
    vh_h, vxc_h, vks_h = vh.cpu().numpy(), vxc.cpu().numpy(), vks.cpu().numpy()
    assert _rel(vh_h, VH_ref) < 1e-12
    assert abs(eh.item() - EH_ref) < 1e-12 * abs(EH_ref)
    assert np.max(np.abs(vxc_h - vxc_ref) / np.maximum(np.abs(vxc_ref), 1e-300)) < 1e-13
    assert np.all(vxc_h[:2] == 0.0)
    assert abs(ex.item() - Exc_ref) < 1e-13 * abs(Exc_ref)
    assert _rel(vks_h, Vion + VH_ref + vxc_ref) < 1e-12
    # the fused chain against the separate calls
    assert np.max(np.abs(vks_h - (Vion + vh_h + vxc_h))) < 1e-13 * np.max(np.abs(vks_h))
    assert en[0].item() == pytest.approx(eh.item(), rel=1e-14)
    assert en[1].item() == pytest.approx(ex.item(), rel=1e-14)
    basis.close()


def test_hartree_of_a_cosine_on_gpu_is_the_closed_form():
    """-lap V = 4 pi n for one cosine on the triclinic box (no oracle involved)."""
    S = (18, 16, 20)
    basis = jdft.Basis(TRICLINIC, S, 1.0, [(0.0, 0.0, 0.0)])
    B = pw.reciprocal(TRICLINIC)
    G = B @ np.array([1.0, -2.0, 1.0])
    r = pw.grid_points(TRICLINIC, S)
    n = 0.4 * np.cos(r @ G + 1.1)
    vh = torch.empty(n.size, dtype=torch.float64, device=DEV)
    eh = torch.zeros(1, dtype=torch.float64, device=DEV)
    jdft.jdft_hartree(basis, _dev(n), vh, eh)
    torch.cuda.synchronize()
    G2 = float(G @ G)
    assert _rel(vh.cpu().numpy(), 4 * np.pi / G2 * n) < 1e-12
    assert eh.item() == pytest.approx(np.pi * 0.16 * pw.cell_volume(TRICLINIC) / G2, rel=1e-12)
    basis.close()


def _pulay_inputs(N, steps, seed):
    """A contracting nonlinear map whose Pulay history stays well conditioned
    (full-rank coupling, slow convergence), so that rounding differences in the
    box sums cannot flip the mixer's drop decisions."""
    rng = np.random.default_rng(seed)
    M = 0.9 * rng.normal(size=(N, N)) / np.sqrt(N)
    b = rng.normal(size=N)
    F = lambda x: 0.6 * np.tanh(M @ x) + b  # noqa: E731
    return F


@pytest.mark.parametrize("history,alpha", [(4, 0.6), (8, 0.3)])
def test_pulay_matches_oracle(history, alpha):
    N, steps = 3000, 12
    F = _pulay_inputs(N, steps, 41)
    ref = scf.Pulay(history, alpha)
    mix = jdft.Pulay(N, history, alpha)
    x = np.zeros(N)
    nxt = torch.empty(N, dtype=torch.float64, device=DEV)
    for it in range(steps):
        fx = F(x)
        want = ref.step(x, fx)
        mix.step(_dev(x), _dev(fx), nxt)
        got = nxt.cpu().numpy()
        assert _rel(got, want) < 1e-10, it
        assert mix.used() == ref.used
        x = want
    mix.close()


def test_pulay_drops_a_dependent_pair_and_mixes_in_place():
    N = 500
    rng = np.random.default_rng(43)
    base, r = rng.normal(size=N), rng.normal(size=N)
    mix = jdft.Pulay(N, 4, 0.5)
    buf = _dev(base)
    mix.step(buf, _dev(base + r), buf)            # in place: n_next = n_in
    assert np.allclose(buf.cpu().numpy(), base + 0.5 * r, rtol=0, atol=1e-14)
    out = torch.empty(N, dtype=torch.float64, device=DEV)
    mix.step(_dev(base), _dev(base + r), out)     # the same residual again: singular, oldest dropped
    assert mix.used() == 1
    assert np.allclose(out.cpu().numpy(), base + 0.5 * r, rtol=0, atol=1e-14)
    mix.close()


def _gpu_cell(R, S, ecut, kpts, weights, atoms, nb, seeds, projectors=True):
    basis = jdft.Basis(R, S, ecut, kpts, weights)
    N = int(np.prod(S))
    vion = torch.zeros(N, dtype=torch.float64, device=DEV)
    if atoms is not None:
        jdft.jdft_gaussian_potential(basis, atoms, vion)
    blocks, Ps = [], []
    # one leading dimension for all k-points (the call takes a single ldc >= every npw)
    ld = max(basis.npw(ik) for ik in range(len(kpts)))
    for ik in range(len(kpts)):
        ob = pw.Basis.build(R, S, kpts[ik], ecut)
        if projectors:
            P = torch.empty((4 * len(atoms), basis.npw(ik)), dtype=torch.complex128, device=DEV)
            jdft.jdft_gaussian_projectors(basis, ik, atoms, P)
            D = torch.tensor(np.diag(np.tile([0.5, -0.3, -0.3, -0.3], len(atoms))), device=DEV)
            jdft.jdft_set_projectors(basis, ik, P, D)
            Ps.append(P)
        store = torch.zeros((nb, ld), dtype=torch.complex128, device=DEV)
        store[:, :ob.npw] = torch.tensor(random_coefficients(2 * ob.T, nb, seeds[ik]), device=DEV)
        blocks.append(store[:, :ob.npw])
    return basis, vion, blocks, Ps


def _small_cell_oracle():
    R = np.diag([8.0, 8.5, 7.5])
    S = (24, 25, 20)
    atoms = atom_positions(R, 4, 5)
    kpts = [(0.1, 0.2, 0.3), (-0.25, 0.0, 0.4)]
    cells = []
    for i, k in enumerate(kpts):
        b = pw.Basis.build(R, S, k, 6.0)
        P = pw.projectors(R, b.kfrac, b.iG, atoms)
        C0 = random_coefficients(2 * b.T, 6, 7 + i).T
        cells.append(scf.KCell(b, P, pw.dmatrix(4), 0.5, C0))
    return R, S, atoms, kpts, cells, pw.vloc_realspace(R, S, atoms)


def test_scf_two_kpoints_matches_oracle():
    R, S, atoms, kpts, cells, Vion = _small_cell_oracle()
    ref = scf.scf(cells, Vion, alpha=0.5, tol_energy=1e-11, tol_density=1e-9)
    assert ref.converged
    basis, vion, blocks, _ = _gpu_cell(R, S, 6.0, kpts, [0.5, 0.5], atoms, 6, [7, 8])
    n = torch.empty(int(np.prod(S)), dtype=torch.float64, device=DEV)
    eigs = torch.empty(2 * 6, dtype=torch.float64, device=DEV)
    rep = jdft.jdft_scf(basis, blocks, vion, n, eigs, tol_energy=1e-10, tol_density=1e-8, band_tol=1e-10)
    assert rep["converged"] == 1
    assert abs(rep["energy"] - ref.energy) < 1e-8
    for k in ("band_energy", "hartree", "xc"):
        want = {"band_energy": ref.parts["band"], "hartree": ref.parts["hartree"], "xc": ref.parts["xc"]}[k]
        assert abs(rep[k] - want) < 1e-6, k
    assert np.max(np.abs(eigs.cpu().numpy() - np.concatenate(ref.eigs))) < 1e-7
    assert _rel(n.cpu().numpy(), ref.n) < 1e-6
    basis.close()


def test_scf_uniform_electron_gas_on_gpu():
    """V_ion = 0, k = 0, 7 bands: uniform density 14/Omega, bands (1/2)|G|^2 + v_xc(n0),
    E = 2 sum (1/2)|G_b|^2 + Omega n0 e_xc(n0) (closed form)."""
    L = 8.0
    R = np.eye(3) * L
    S = (20, 20, 20)
    basis, vion, blocks, _ = _gpu_cell(R, S, 3.0, [(0.0, 0.0, 0.0)], [1.0], None, 7, [4], projectors=False)
    n = torch.empty(int(np.prod(S)), dtype=torch.float64, device=DEV)
    eigs = torch.empty(7, dtype=torch.float64, device=DEV)
    rep = jdft.jdft_scf(basis, blocks, vion, n, eigs, tol_energy=1e-11, tol_density=1e-9, band_tol=1e-10)
    assert rep["converged"] == 1
    Omega = L ** 3
    n0 = 14.0 / Omega
    e0, v0 = scf.lda_pz(np.array([n0]))
    g2 = 0.5 * (2 * np.pi / L) ** 2
    assert np.max(np.abs(eigs.cpu().numpy() - (np.array([0.0] + [g2] * 6) + v0[0]))) < 1e-9
    assert abs(rep["energy"] - (12.0 * g2 + Omega * n0 * e0[0])) < 1e-9
    assert np.max(np.abs(n.cpu().numpy() - n0)) < 1e-8
    assert abs(rep["hartree"]) < 1e-12
    basis.close()


def _small_workload_on_gpu(prec="fp64", band_tol=1e-9, band_tol_factor=0.0, precond="teter", mlp=None):
    w = WORKLOADS["small"]
    atoms = atom_positions(w.R, w.natoms, w.seed_atoms)
    ob = pw.Basis.build(w.R, w.S, w.kfrac[0], w.ecut)
    basis = jdft.Basis(w.R, w.S, w.ecut, w.kfrac, w.weights())
    N = int(np.prod(w.S))
    vion = torch.empty(N, dtype=torch.float64, device=DEV)
    jdft.jdft_gaussian_potential(basis, atoms, vion)
    P = torch.empty((4 * w.natoms, basis.npw(0)), dtype=torch.complex128, device=DEV)
    jdft.jdft_gaussian_projectors(basis, 0, atoms, P)
    D = torch.tensor(np.diag(np.tile([0.5, -0.3, -0.3, -0.3], w.natoms)), device=DEV)
    jdft.jdft_set_projectors(basis, 0, P, D)
    C = torch.tensor(random_coefficients(2 * ob.T, w.nbands, w.seed_coeffs), device=DEV)
    n = torch.empty(N, dtype=torch.float64, device=DEV)
    eigs = torch.empty(w.nbands, dtype=torch.float64, device=DEV)
    rep = jdft.jdft_scf(basis, [C], vion, n, eigs, tol_energy=1e-9, tol_density=1e-7, band_tol=band_tol,
                        prec=prec, band_tol_factor=band_tol_factor, precond=precond, mlp=mlp)
    out = (rep, n.cpu().numpy(), eigs.cpu().numpy())
    basis.close()
    return out


@pytest.mark.parametrize("prec,tol,factor", [("fp64", 1e-8, 0.0), ("fp64", 1e-8, -1.0), ("bf16x3", 1e-6, 0.0)],
                         ids=["fp64-adaptive-band-tol", "fp64-fixed-band-tol", "bf16x3-adaptive-band-tol"])
def test_scf_48cubed_matches_golden(prec, tol, factor):
    """The 'small' workload self-consistent (LDA, Pulay): energy, eigenvalues and
    density samples against the oracle's values (tests/golden/scf_small.json).
    BF16x3: the band solves run their bulk iterations with split-precision
    products and finish in FP64 (the minimiser's own schedule)."""
    g = json.load(open(GOLDEN))
    rep, n, eigs = _small_workload_on_gpu(prec, band_tol_factor=factor)
    assert rep["converged"] == 1
    assert abs(rep["energy"] - g["energy"]) < tol
    assert np.max(np.abs(eigs - np.array(g["eigs"]))) < 10 * tol
    for j, v in g["density_samples"].items():
        assert abs(n[int(j)] - v) < 1e-5 * max(abs(v), 1e-3)
    w = WORKLOADS["small"]
    Omega = float(np.prod(w.L))
    assert Omega / n.size * n.sum() == pytest.approx(2.0 * w.nbands, rel=1e-10)


def test_scf_with_the_learned_preconditioner_matches_golden():
    """Mixed-precision band solves with the committed network as preconditioner
    inside the SCF loop reach the oracle's self-consistent energy."""
    from paper_1708_03621_gb300 import learned
    wts = learned.load_weights()
    if wts is None:
        pytest.skip("no committed network weights")
    net = jdft.Mlp(wts)
    g = json.load(open(GOLDEN))
    rep, n, eigs = _small_workload_on_gpu("bf16x3", precond="mlp", mlp=net)
    assert rep["converged"] == 1
    assert abs(rep["energy"] - g["energy"]) < 1e-6
    assert np.max(np.abs(eigs - np.array(g["eigs"]))) < 1e-5


def test_pulay_with_one_pair_is_linear_mixing():
    N = 700
    rng = np.random.default_rng(44)
    mix = jdft.Pulay(N, 1, 0.35)
    out = torch.empty(N, dtype=torch.float64, device=DEV)
    for _ in range(3):
        x, fx = rng.normal(size=N), rng.normal(size=N)
        mix.step(_dev(x), _dev(fx), out)
        assert np.allclose(out.cpu().numpy(), x + 0.35 * (fx - x), rtol=0, atol=1e-14)
        assert mix.used() == 1
    mix.close()


def test_scf_iteration_limit_reports_not_converged():
    R, S, atoms, kpts, cells, Vion = _small_cell_oracle()
    basis, vion, blocks, _ = _gpu_cell(R, S, 6.0, kpts, [0.5, 0.5], atoms, 6, [7, 8])
    n = torch.empty(int(np.prod(S)), dtype=torch.float64, device=DEV)
    rep = jdft.jdft_scf(basis, blocks, vion, n, max_iter=2, check=False)
    assert rep["status"] == "ERR_NOT_CONVERGED" and rep["converged"] == 0 and rep["iterations"] == 2
    Omega = float(np.prod(np.diag(R)))
    # the output density still holds every electron
    assert Omega / n.numel() * n.sum().item() == pytest.approx(2.0 * 6, rel=1e-10)
    basis.close()
