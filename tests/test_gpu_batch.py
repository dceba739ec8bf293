"""Batches of Hamiltonian applications in one CUDA graph (k-points of one
cell with uneven spheres, plus independent cells with their own boxes):
the graph replay equals the individual calls and the oracle."""
import numpy as np
import pytest

from oracle import planewave as pw
from synth import Workload, atom_positions, random_cells, random_coefficients, random_kpoints

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _cell(w):
    from paper_1708_03621_gb300 import learned
    return learned.build_cell(w, "cuda")


def _block(b, w, ik, nb, seed, prec):
    from paper_1708_03621_gb300 import learned
    C = learned.start_block(b, w, ik=ik, nb=nb, seed=seed)
    return torch.tensor(C.astype(np.complex128 if prec == "fp64" else np.complex64), device="cuda")


@pytest.mark.parametrize("prec", ["fp64", "tf32x3"])
def test_batch_graph_equals_individual_calls(prec):
    from paper_1708_03621_gb300 import jdft
    kpts = tuple(tuple(k) for k in random_kpoints(3, 21))
    wk = Workload("kbatch", (10.0, 10.0, 10.0), 12.0, (40, 40, 40), kpts, 8, 12, 21, 22)
    cells = random_cells(2, 23, L_range=(7.0, 9.0), ecut=10.0)
    bases, items, refs = [], [], []
    bk = _cell(wk)
    bases.append(bk)
    for ik in range(3):
        C = _block(bk, wk, ik, 12, 100 + ik, prec)
        items.append((bk, ik, C, torch.empty_like(C), prec))
    for c, w in enumerate(cells):
        b = _cell(w)
        bases.append(b)
        C = _block(b, w, 0, 9, 200 + c, prec)
        items.append((b, 0, C, torch.empty_like(C), prec))
    for (b, ik, C, HC, pr) in items:
        R = torch.empty_like(C)
        jdft.jdft_apply_H(b, ik, C, R, pr)
        refs.append(R)
    torch.cuda.synchronize()
    batch = jdft.Batch(items)
    for rep in range(2):
        if rep == 1:
            for it in items:
                it[2].mul_(0.5)
            refs = [r * 0.5 for r in refs]
        for it in items:
            it[3].fill_(float("nan"))
        batch.launch()
        torch.cuda.synchronize()
        tol = 1e-12 if prec == "fp64" else 1e-5
        for it, R in zip(items, refs):
            got, ref = it[3].cpu().numpy(), R.cpu().numpy()
            assert np.all(np.isfinite(got))
            rel = np.linalg.norm(got - ref, axis=1) / np.linalg.norm(ref, axis=1)
            assert rel.max() < tol
    # one k-point of the batch against the oracle
    ob = pw.Basis.build(wk.R, wk.S, wk.kfrac[1], wk.ecut)
    atoms = atom_positions(wk.R, wk.natoms, wk.seed_atoms)
    V = pw.vloc_realspace(wk.R, wk.S, atoms)
    P = pw.projectors(wk.R, ob.kfrac, ob.iG, atoms)
    C1 = items[1][2].cpu().numpy().astype(np.complex128)
    ref = pw.apply_H(ob, V, C1.T, P, pw.dmatrix(wk.natoms)).T
    got = items[1][3].cpu().numpy().astype(np.complex128)
    rel = np.linalg.norm(got - ref, axis=1) / np.linalg.norm(ref, axis=1)
    assert rel.max() < (1e-10 if prec == "fp64" else 1e-5)
    batch.close()


def test_autotune_chunk_keeps_results():
    from paper_1708_03621_gb300 import jdft
    from synth import WORKLOADS
    w = WORKLOADS["mid"]
    b = _cell(w)
    C = _block(b, w, 0, 24, 5, "fp32")
    H0 = torch.empty_like(C)
    jdft.jdft_apply_H(b, 0, C, H0, "fp32")
    mb = jdft.jdft_autotune_chunk(b, 0, C, torch.empty_like(C), "fp32")
    assert mb in (32, 64, 128, 256, 512, 1024)
    H1 = torch.empty_like(C)
    jdft.jdft_apply_H(b, 0, C, H1, "fp32")
    torch.cuda.synchronize()
    assert torch.allclose(H0, H1, rtol=1e-5, atol=1e-6 * H0.abs().max().item())


@pytest.mark.parametrize("prec", ["bf16x3", "tf32x3"])
def test_autotune_schedules_keep_results(prec):
    """jdft_autotune on a 150-band block of the 40^3 cell: the chosen chunk
    budget and split-K schedules are valid, and H C and C^dag H C computed
    with them still match the oracle."""
    from oracle import planewave as pw
    from paper_1708_03621_gb300 import jdft
    from synth import WORKLOADS
    w = WORKLOADS["mid"]
    b = _cell(w)
    nb = 150
    C = _block(b, w, 0, nb, 7, prec)
    rep = jdft.jdft_autotune(b, 0, C, torch.empty_like(C), prec)
    assert rep["chunk_mb"] in (32, 64, 128, 256, 512, 1024)
    assert rep["splits_subspace"] >= 1 and rep["splits_projector"] >= 1
    assert rep["plane_bands"] == 0  # 40^3 planes have no band-pair kernel
    HC = torch.empty_like(C)
    jdft.jdft_apply_H(b, 0, C, HC, prec)
    CHC = torch.empty((nb, nb), dtype=torch.complex128, device="cuda")
    jdft.jdft_subspace(b, 0, C, HC, CHC, None, prec)
    ob = pw.Basis.build(w.R, w.S, w.kfrac[0], w.ecut)
    atoms = atom_positions(w.R, w.natoms, w.seed_atoms)
    V = pw.vloc_realspace(w.R, w.S, atoms)
    P = pw.projectors(w.R, ob.kfrac, ob.iG, atoms)
    Ch = C.cpu().numpy().astype(np.complex128)
    ref = pw.apply_H(ob, V, Ch.T, P, pw.dmatrix(w.natoms)).T
    got = HC.cpu().numpy().astype(np.complex128)
    assert (np.linalg.norm(got - ref, axis=1) / np.linalg.norm(ref, axis=1)).max() < 2e-5
    chc_ref = Ch.conj() @ ref.T
    assert np.max(np.abs(CHC.cpu().numpy() - chc_ref)) / np.max(np.abs(chc_ref)) < 2e-4
    jdft.jdft_device_status()


@pytest.mark.parametrize("prec", ["bf16x3", "fp32"])
def test_kbatched_kpoints_equal_individual_calls_and_oracle(prec):
    """k-points of the 128^3 cell with uneven spheres and odd band counts run
    as one k-batched chain (one launch per FFT stage over all of them, the
    paper's k-point parallelism, Sec. 3, folded into one GPU launch): equal to
    the individual jdft_apply_H calls, and to the oracle on sampled bands."""
    from paper_1708_03621_gb300 import jdft
    from tests.systems import OracleSystem
    kpts = tuple(tuple(k) for k in random_kpoints(3, 41))
    w = Workload("kbatch128", (20.0, 20.0, 20.0), 30.0, (128, 128, 128), kpts, 64, 9, 11, 12)
    b = _cell(w)
    nbs = [9, 6, 11]
    items, refs = [], []
    for ik, nb in enumerate(nbs):
        C = _block(b, w, ik, nb, 300 + ik, prec)
        items.append((b, ik, C, torch.empty_like(C), prec))
        R = torch.empty_like(C)
        jdft.jdft_apply_H(b, ik, C, R, prec)
        refs.append(R)
    torch.cuda.synchronize()
    batch = jdft.Batch(items)
    assert batch.kbatched
    for it in items:
        it[3].fill_(float("nan"))
    batch.launch()
    torch.cuda.synchronize()
    for it, R in zip(items, refs):
        got, ref = it[3].cpu().numpy(), R.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert np.max(np.abs(got - ref)) < 1e-6 * np.max(np.abs(ref))
    # the oracle on two bands of the second k-point
    o = OracleSystem(w, ik=1)
    C1 = items[1][2].cpu().numpy().astype(np.complex128)
    sample = [0, nbs[1] - 1]
    ref = o.apply_H(C1[sample])
    got = items[1][3].cpu().numpy().astype(np.complex128)[sample]
    err = np.max(np.linalg.norm(got - ref, axis=1) / np.linalg.norm(ref, axis=1))
    assert err < 2e-5
    batch.close()
    jdft.jdft_device_status()
