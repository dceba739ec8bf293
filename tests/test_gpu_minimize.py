"""GPU band minimisation (orthonormalisation, subspace eigenvalues, preconditioned
band CG) against the oracle and LAPACK, through the C ABI.

The minimiser (JDFTx paper, Sec. 2.1 Minimize; Sec. 2.2) must reach the lowest
eigenpairs: the 48^3 cell's energy within 1e-6 Ha of the dense-diagonalisation
reference (tests/golden/small_eigs.json, written by a script that calls only
the oracle), in FP64 and in the mixed FP32 -> FP64 mode, with the Teter and
identity preconditioners converging to the same energy.
"""
import json
import os

import numpy as np
import pytest

from oracle import planewave as pw
from tests.systems import GpuSystem, OracleSystem, workload

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GOLDEN = json.load(open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "small_eigs.json")))
_cache = {}


def systems(name):
    if name not in _cache:
        w = workload(name)
        o = OracleSystem(w)
        _cache[name] = (w, o, GpuSystem(w, o.atoms))
    return _cache[name]


def test_subspace_eigs_match_lapack():
    from paper_1708_03621_gb300 import jdft
    rng = np.random.default_rng(4)
    for n in (1, 2, 16, 37, 128):
        X = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
        A = X + X.conj().T
        e = torch.empty(n, dtype=torch.float64, device="cuda")
        jdft.jdft_subspace_eigs(torch.tensor(A, device="cuda"), e)
        ref = np.linalg.eigvalsh(A)
        assert np.max(np.abs(e.cpu().numpy() - ref)) < 1e-11 * max(1.0, np.max(np.abs(ref)))


@pytest.mark.parametrize("nb", [13, 70, 150])
@pytest.mark.parametrize("prec", ["fp64", "fp32", "tf32x3", "bf16x3"])
def test_orthonormalize_spans_same_subspace(prec, nb):
    """13 bands: one-block factorisation; 70 and 150: the blocked multi-block
    one (padded to 3 and 5 tiles; FP32 factorisation for the FP32 blocks)."""
    from paper_1708_03621_gb300 import jdft
    w, o, g = systems("mid")
    C = o.coeffs(nb, seed=31)
    Cd = torch.tensor(C.astype(np.complex128 if prec == "fp64" else np.complex64), device="cuda")
    jdft.jdft_orthonormalize(g.basis, 0, Cd, prec)
    Q = Cd.cpu().numpy().astype(np.complex128).T               # (npw, nb)
    tol = 1e-12 if prec == "fp64" else 2e-5
    assert np.allclose(o.basis.Omega * Q.conj().T @ Q, np.eye(nb), atol=tol)
    L = pw.lowdin(C.T, o.basis.Omega)                          # oracle's orthonormal basis of the same span
    P1 = Q @ Q.conj().T
    P2 = L @ L.conj().T
    assert np.max(np.abs(P1 - P2)) < tol * np.max(np.abs(P2))


@pytest.mark.parametrize("fp32,cluster", [("0", "1"), ("1", "1"), ("1", "0")])
def test_orthonormalize_fp32_factorisations(fp32, cluster, monkeypatch):
    """FP32 blocks of 150 bands (5 tiles): the default FP64 factorisation, and on
    request the FP32 ones (one-launch cluster with distributed shared memory,
    and multi-block) give the same span."""
    from paper_1708_03621_gb300 import jdft
    monkeypatch.setenv("JDFT_CHOL_FP32", fp32)
    monkeypatch.setenv("JDFT_CHOL_CLUSTER", cluster)
    w, o, g = systems("mid")
    nb = 150
    C = o.coeffs(nb, seed=37)
    Cd = torch.tensor(C.astype(np.complex64), device="cuda")
    jdft.jdft_orthonormalize(g.basis, 0, Cd, "fp32")
    Q = Cd.cpu().numpy().astype(np.complex128).T
    assert np.allclose(o.basis.Omega * Q.conj().T @ Q, np.eye(nb), atol=2e-5)
    L = pw.lowdin(C.T, o.basis.Omega)
    assert np.max(np.abs(Q @ Q.conj().T - L @ L.conj().T)) < 2e-5 * np.max(np.abs(L @ L.conj().T))


@pytest.mark.parametrize("name,nb,prec", [("tiny_cubic", 3, "fp64"), ("mid", 40, "fp64"), ("mid", 40, "fp32"),
                                          ("mid", 100, "tf32x3")])
def test_orthonormalize_rejects_dependent_bands(name, nb, prec):
    from paper_1708_03621_gb300 import jdft
    w, o, g = systems(name)
    C = o.coeffs(nb)
    C[nb - 1] = C[0]
    Cd = torch.tensor(C.astype(np.complex128 if prec == "fp64" else np.complex64), device="cuda")
    with pytest.raises(jdft.JdftError, match="NOT_POSDEF"):
        jdft.jdft_orthonormalize(g.basis, 0, Cd, prec)


@pytest.mark.parametrize("cluster", ["1", "0"])
def test_orthonormalize_fp32_factorisation_rejects_dependent_bands(cluster, monkeypatch):
    """The FP32 factorisation's pivot floor (2e-4 of the original diagonal) on
    100 bands with a duplicate."""
    from paper_1708_03621_gb300 import jdft
    monkeypatch.setenv("JDFT_CHOL_FP32", "1")
    monkeypatch.setenv("JDFT_CHOL_CLUSTER", cluster)
    w, o, g = systems("mid")
    C = o.coeffs(100)
    C[99] = C[3]
    with pytest.raises(jdft.JdftError, match="NOT_POSDEF"):
        jdft.jdft_orthonormalize(g.basis, 0, torch.tensor(C.astype(np.complex64), device="cuda"), "fp32")


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
def test_orthonormalize_async_matches_and_status_is_sticky(prec):
    """The asynchronous form gives the synchronous one's block (up to the order
    of the FP64 atomic split-K sums of C^dag C) and merges failures into a
    device word that a later good call does not clear."""
    from paper_1708_03621_gb300 import jdft
    w, o, g = systems("mid")
    ct = np.complex128 if prec == "fp64" else np.complex64
    C = o.coeffs(70, seed=41)
    A = torch.tensor(C.astype(ct), device="cuda")
    B = A.clone()
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    jdft.jdft_orthonormalize(g.basis, 0, A, prec)
    jdft.jdft_orthonormalize_async(g.basis, 0, B, st, prec)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    a, b = A.cpu().numpy().astype(np.complex128), B.cpu().numpy().astype(np.complex128)
    assert np.max(np.abs(a - b)) < (1e-12 if prec == "fp64" else 1e-5) * np.max(np.abs(a))
    D = o.coeffs(40)
    D[39] = D[0]
    Dd = torch.tensor(D.astype(ct), device="cuda")
    jdft.jdft_orthonormalize_async(g.basis, 0, Dd, st, prec)
    jdft.jdft_orthonormalize_async(g.basis, 0, B, st, prec)   # a good call afterwards
    torch.cuda.synchronize()
    assert int(st.item()) == jdft.STATUS_CODES["ERR_NOT_POSDEF"]


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
def test_orthonormalize_with_given_overlap(prec):
    """U = the COC output of jdft_subspace for the same block gives the block
    that recomputing the overlap gives, and C^dag O C = 1 afterwards."""
    from paper_1708_03621_gb300 import jdft
    w, o, g = systems("mid")
    ct = np.complex128 if prec == "fp64" else np.complex64
    C = o.coeffs(70, seed=43)
    A = torch.tensor(C.astype(ct), device="cuda")
    B = A.clone()
    nb = A.shape[0]
    COC = torch.empty((nb, nb), dtype=torch.complex128, device="cuda")
    jdft.jdft_subspace(g.basis, 0, B, None, None, COC, prec)
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    jdft.jdft_orthonormalize(g.basis, 0, A, prec)
    jdft.jdft_orthonormalize_async(g.basis, 0, B, st, prec, U=COC)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    a, b = A.cpu().numpy().astype(np.complex128), B.cpu().numpy().astype(np.complex128)
    assert np.max(np.abs(a - b)) < (1e-12 if prec == "fp64" else 1e-5) * np.max(np.abs(a))
    Q = b.T
    assert np.allclose(o.basis.Omega * Q.conj().T @ Q, np.eye(nb), atol=1e-12 if prec == "fp64" else 2e-5)


@pytest.mark.parametrize("precond", ["teter", "identity"])
def test_minimize_tiny_reaches_dense_eigenvalues(precond):
    from paper_1708_03621_gb300 import jdft
    w, o, g = systems("tiny_cubic")
    nb = 6
    exact = np.linalg.eigvalsh(pw.dense_H(o.basis, o.V, o.P, o.D) / o.basis.Omega)[:nb]
    C = torch.tensor(o.coeffs(nb), device="cuda")
    eigs = torch.empty(nb, dtype=torch.float64, device="cuda")
    rep = jdft.jdft_minimize_bands(g.basis, 0, C, eigs, tol=1e-9, max_iter=800, precond=precond)
    assert rep["converged"]
    assert np.max(np.abs(eigs.cpu().numpy() - exact)) < 1e-11
    assert abs(rep["energy"] - 2 * exact.sum()) < 1e-10
    Q = C.cpu().numpy().T
    assert np.allclose(o.basis.Omega * Q.conj().T @ Q, np.eye(nb), atol=1e-12)


@pytest.mark.parametrize("prec", ["fp64", "fp32", "tf32x3", "bf16x3"])
def test_minimize_small_cell_energy_within_1e6(prec):
    """The 48^3, 16-band system: |E - E_ref| < 1e-6 Ha, eigenvalues to 1e-7."""
    from paper_1708_03621_gb300 import jdft
    w, o, g = systems("small")
    C = torch.tensor(o.coeffs(16), device="cuda")
    eigs = torch.empty(16, dtype=torch.float64, device="cuda")
    rep = jdft.jdft_minimize_bands(g.basis, 0, C, eigs, tol=1e-8, max_iter=2000, precond="teter", prec=prec)
    assert rep["converged"], rep
    assert abs(rep["energy"] - GOLDEN["E_ref"]) < 1e-6
    assert np.max(np.abs(eigs.cpu().numpy() - np.array(GOLDEN["eigs"][:16]))) < 1e-7
    if prec != "fp64":
        assert rep["mixed_iterations"] > 0


def test_minimize_reports_not_converged():
    from paper_1708_03621_gb300 import jdft
    w, o, g = systems("tiny_cubic")
    C = torch.tensor(o.coeffs(6), device="cuda")
    rep = jdft.jdft_minimize_bands(g.basis, 0, C, tol=1e-12, max_iter=3, check=False)
    assert rep["status"] == "ERR_NOT_CONVERGED" and rep["iterations"] == 3 and not rep["converged"]
