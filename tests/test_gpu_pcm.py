"""GPU parity of the scalar-field transforms and the linear dielectric solve
(the paper's LinearPCM example: Sec. 2.1, Eq. Poisson, Eq. Adiel, Listing 1)
against the FP64 oracle (oracle/pcm.py), through the C ABI."""
from __future__ import annotations

import numpy as np
import pytest

from oracle import pcm
from oracle import planewave as pw
from oracle import scf
from synth import atom_positions

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1708_03621_gb300 import jdft  # noqa: E402

DEV = torch.device("cuda:0")
TRICLINIC = np.array([[7.0, 1.2, 0.4], [0.0, 6.5, -0.9], [0.3, 0.0, 8.0]])

BOXES = [
    ("triclinic-18x16x20", TRICLINIC, (18, 16, 20)),
    ("orthorhombic-24x25x20", np.diag([8.0, 8.5, 7.5]), (24, 25, 20)),
    ("cubic-48", np.eye(3) * 10.0, (48, 48, 48)),
    ("mixed-60x64x54", np.diag([12.0, 13.0, 11.0]), (60, 64, 54)),
]


def _c(a):
    return torch.tensor(np.ascontiguousarray(a, dtype=np.complex128), device=DEV)


def _d(a):
    return torch.tensor(np.ascontiguousarray(a, dtype=np.float64), device=DEV)


def _rel(got, ref):
    return float(np.max(np.abs(got - ref)) / np.max(np.abs(ref)))


def _cavity_eps(R, S, natoms, seed, eps_bulk=78.4, radius=2.0):
    """A solute-shaped dielectric: 1 inside spheres around seeded points, eps_bulk
    outside, joined by a smooth erfc-like switch (built from Gaussians)."""
    atoms = atom_positions(R, natoms, seed)
    shape = -pw.vloc_realspace(R, S, atoms, depth=1.0, width=radius)
    s = np.exp(-shape)            # ~0 near the atoms, 1 far away
    return 1.0 + (eps_bulk - 1.0) * s


@pytest.mark.parametrize("name,R,S", BOXES, ids=[b[0] for b in BOXES])
def test_field_I_J_match_oracle(name, R, S):
    basis = jdft.Basis(R, S, 1.0, [(0.0, 0.0, 0.0)])
    rng = np.random.default_rng(3)
    N = int(np.prod(S))
    X = rng.normal(size=N) + 1j * rng.normal(size=N)
    x = torch.empty(N, dtype=torch.complex128, device=DEV)
    Y = torch.empty_like(x)
    jdft.jdft_field_I(basis, _c(X), x)
    jdft.jdft_field_J(basis, x, Y)
    torch.cuda.synchronize()
    assert _rel(x.cpu().numpy(), pcm.op_I(S, X)) < 1e-13
    assert _rel(Y.cpu().numpy(), X) < 1e-13
    Z = _c(X)
    jdft.jdft_field_J(basis, Z, Z)         # in place
    torch.cuda.synchronize()
    assert _rel(Z.cpu().numpy(), pcm.op_J(S, X)) < 1e-13
    basis.close()


@pytest.mark.parametrize("name,R,S", BOXES, ids=[b[0] for b in BOXES])
def test_pcm_hessian_matches_oracle(name, R, S):
    basis = jdft.Basis(R, S, 1.0, [(0.0, 0.0, 0.0)])
    rng = np.random.default_rng(5)
    N = int(np.prod(S))
    eps = _cavity_eps(R, S, 3, 6, eps_bulk=20.0)
    X = rng.normal(size=N) + 1j * rng.normal(size=N)
    out = torch.empty(N, dtype=torch.complex128, device=DEV)
    jdft.jdft_pcm_hessian(basis, _d(eps), _c(X), out)
    torch.cuda.synchronize()
    assert _rel(out.cpu().numpy(), pcm.hessian(R, S, eps, X)) < 1e-12
    basis.close()


def test_pcm_hessian_of_a_cosine_is_the_hand_divergence():
    """phi = cos(G.r), eps = 1 + a cos(Q.r) on the triclinic box (no oracle involved)."""
    S = (18, 16, 20)
    basis = jdft.Basis(TRICLINIC, S, 1.0, [(0.0, 0.0, 0.0)])
    r = pw.grid_points(TRICLINIC, S)
    B = pw.reciprocal(TRICLINIC)
    Q, G, a = B @ np.array([1.0, 0.0, -1.0]), B @ np.array([0.0, 1.0, 1.0]), 0.3
    eps = 1 + a * np.cos(r @ Q)
    phi = torch.empty(r.shape[0], dtype=torch.complex128, device=DEV)
    jdft.jdft_field_J(basis, _c(np.cos(r @ G)), phi)
    H = torch.empty_like(phi)
    jdft.jdft_pcm_hessian(basis, _d(eps), phi, H)
    h = torch.empty_like(phi)
    jdft.jdft_field_I(basis, H, h)
    torch.cuda.synchronize()
    div = -(G @ G) * np.cos(r @ G) - a / 2 * (G @ (G + Q) * np.cos(r @ (G + Q)) + G @ (G - Q) * np.cos(r @ (G - Q)))
    assert np.max(np.abs(h.cpu().numpy() + div / (4 * np.pi))) < 1e-13
    basis.close()


SOLVE_CASES = [(b, p) for b in BOXES[:3] for p in ("fp64", "fp32")]


@pytest.mark.parametrize("box,prec", SOLVE_CASES, ids=[f"{b[0]}-{p}" for b, p in SOLVE_CASES])
def test_pcm_solve_matches_oracle(box, prec):
    """FP64 CG, and FP32 CG rounds refined with FP64 residuals, both to the
    oracle's FP64 CG solution at the same tolerance."""
    name, R, S = box
    basis = jdft.Basis(R, S, 1.0, [(0.0, 0.0, 0.0)])
    eps = _cavity_eps(R, S, 2, 7, eps_bulk=10.0, radius=1.5)
    rho = -pw.vloc_realspace(R, S, atom_positions(R, 2, 7), depth=0.5, width=0.9)
    rho_t = pcm.op_J(S, rho)
    ref = pcm.solve(R, S, eps, rho_t, tol=1e-11, max_iter=400)
    assert ref.converged
    phi = torch.empty(rho.size, dtype=torch.complex128, device=DEV)
    rep = jdft.jdft_pcm_solve(basis, _d(eps), _c(rho_t), phi, tol=1e-11, max_iter=400, prec=prec)
    assert rep["converged"] == 1
    if prec == "fp64":
        assert abs(rep["iterations"] - ref.iterations) <= 1
        assert rep["fp64_hessians"] == rep["iterations"]
    else:
        assert rep["fp64_hessians"] <= 6
    assert _rel(phi.cpu().numpy(), ref.phi) < 1e-9
    assert abs(rep["A_diel"] - ref.A_diel) < 1e-9 * abs(ref.A_diel)
    basis.close()


def test_pcm_uniform_dielectric_closed_form_128cubed():
    """eps uniform on the 128^3 box: one CG step, phi~ = 4 pi rho~ / (eps G^2),
    A_diel = (1/eps - 1) E_H with E_H from the library's Hartree call."""
    R, S = np.eye(3) * 20.0, (128, 128, 128)
    basis = jdft.Basis(R, S, 1.0, [(0.0, 0.0, 0.0)])
    N = int(np.prod(S))
    rho = torch.empty(N, dtype=torch.float64, device=DEV)
    jdft.jdft_gaussian_potential(basis, atom_positions(R, 8, 9), rho, depth=0.2, width=1.1)
    rho.neg_()
    rho_t = torch.empty(N, dtype=torch.complex128, device=DEV)
    jdft.jdft_field_J(basis, rho.to(torch.complex128), rho_t)
    vh = torch.empty_like(rho)
    eh = torch.zeros(1, dtype=torch.float64, device=DEV)
    jdft.jdft_hartree(basis, rho, vh, eh)
    e = 4.0
    phi = torch.empty_like(rho_t)
    rep = jdft.jdft_pcm_solve(basis, torch.full((N,), e, dtype=torch.float64, device=DEV), rho_t, phi, tol=1e-12)
    assert rep["converged"] == 1 and rep["iterations"] == 1
    assert rep["A_diel"] == pytest.approx((1 / e - 1) * eh.item(), rel=1e-11)
    # V_H = I(4 pi rho~ / G^2) = e * I(phi~)
    p = torch.empty_like(phi)
    jdft.jdft_field_I(basis, phi, p)
    torch.cuda.synchronize()
    assert _rel(e * p.real.cpu().numpy(), vh.cpu().numpy()) < 1e-11
    basis.close()


def test_pcm_energy_between_uniform_bounds_64cubed():
    """A solute-shaped dielectric on a 64^3 box: the CG converges and A_diel lies
    between the uniform-eps values for min and max eps (E_H from the oracle)."""
    R, S = np.eye(3) * 16.0, (64, 64, 64)
    basis = jdft.Basis(R, S, 1.0, [(0.0, 0.0, 0.0)])
    eps = _cavity_eps(R, S, 4, 11)
    rho = -pw.vloc_realspace(R, S, atom_positions(R, 4, 11), depth=0.5, width=0.8)
    rho_t = pcm.op_J(S, rho)
    phi = torch.empty(rho.size, dtype=torch.complex128, device=DEV)
    rep = jdft.jdft_pcm_solve(basis, _d(eps), _c(rho_t), phi, tol=1e-10, max_iter=1000)
    _, EH = scf.hartree(R, S, rho)
    assert rep["converged"] == 1
    assert (1 / eps.min() - 1) * EH >= rep["A_diel"] >= (1 / eps.max() - 1) * EH
    basis.close()


def test_pcm_mixed_equals_fp64_on_a_128cubed_cavity():
    """The bench's dielectric (eps 1 inside ~2 bohr of 64 centres, 78.4 outside)
    on the 128^3 box: the FP32-refined solve reaches the FP64 tolerance and
    agrees with the FP64 CG."""
    R, S = np.eye(3) * 20.0, (128, 128, 128)
    basis = jdft.Basis(R, S, 1.0, [(0.0, 0.0, 0.0)])
    N = int(np.prod(S))
    centres = atom_positions(R, 64, 78)
    shape = torch.empty(N, dtype=torch.float64, device=DEV)
    jdft.jdft_gaussian_potential(basis, centres, shape, depth=6.0, width=2.0)
    eps = (1.0 + 77.4 * torch.exp(shape)).contiguous()
    rho = torch.empty(N, dtype=torch.float64, device=DEV)
    jdft.jdft_gaussian_potential(basis, centres, rho, depth=0.5, width=0.8)
    rho_t = torch.empty(N, dtype=torch.complex128, device=DEV)
    jdft.jdft_field_J(basis, (-rho).to(torch.complex128), rho_t)
    p64 = torch.empty_like(rho_t)
    p32 = torch.empty_like(rho_t)
    r64 = jdft.jdft_pcm_solve(basis, eps, rho_t, p64, tol=1e-10, max_iter=2000, prec="fp64")
    r32 = jdft.jdft_pcm_solve(basis, eps, rho_t, p32, tol=1e-10, max_iter=2000, prec="fp32")
    assert r64["converged"] == 1 and r32["converged"] == 1
    assert r32["residual"] <= 1e-10
    assert _rel(p32.cpu().numpy(), p64.cpu().numpy()) < 1e-8
    assert r32["A_diel"] == pytest.approx(r64["A_diel"], rel=1e-10)
    basis.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_pcm_zero_charge_gives_zero_potential(prec):
    """Degenerate input: rho~ = 0 converges at once to phi~ = 0 and A_diel = 0."""
    S = (18, 16, 20)
    basis = jdft.Basis(TRICLINIC, S, 1.0, [(0.0, 0.0, 0.0)])
    N = int(np.prod(S))
    phi = torch.full((N,), 7.0 + 1j, dtype=torch.complex128, device=DEV)
    rep = jdft.jdft_pcm_solve(basis, torch.full((N,), 2.0, dtype=torch.float64, device=DEV),
                              torch.zeros(N, dtype=torch.complex128, device=DEV), phi, tol=1e-10, prec=prec)
    torch.cuda.synchronize()
    assert rep["converged"] == 1 and rep["iterations"] == 0
    assert rep["A_diel"] == 0.0
    assert torch.count_nonzero(phi).item() == 0
    basis.close()


def test_pcm_iteration_limit_reports_not_converged():
    R, S = np.diag([8.0, 8.5, 7.5]), (24, 25, 20)
    basis = jdft.Basis(R, S, 1.0, [(0.0, 0.0, 0.0)])
    eps = _cavity_eps(R, S, 2, 7, eps_bulk=10.0, radius=1.5)
    rho_t = pcm.op_J(S, -pw.vloc_realspace(R, S, atom_positions(R, 2, 7), depth=0.5, width=0.9))
    phi = torch.empty(rho_t.size, dtype=torch.complex128, device=DEV)
    rep = jdft.jdft_pcm_solve(basis, _d(eps), _c(rho_t), phi, tol=1e-12, max_iter=3, check=False)
    assert rep["status"] == "ERR_NOT_CONVERGED" and rep["converged"] == 0 and rep["iterations"] == 3
    assert 0 < rep["residual"] < 1
    basis.close()
