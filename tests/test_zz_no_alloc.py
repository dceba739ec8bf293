"""jdft_apply_H_noalloc against jdft_apply_H, through the C ABI (GPU).

The no-allocation entry point serves callers that cannot let the library call
cudaMalloc (fixed memory budgets or pool allocators, latency-critical loops); it
keeps its intermediates in a static 32 MiB device array instead.  Its results
must equal those of the allocating entry point within the parity tolerances,
on two calls in a row (the static array keeps the previous call's contents,
so the second call checks that nothing stale leaks in).  This file is
collected last on purpose.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# the tensor-core modes: both entry points run the nonlocal products with
# different tile and split-K schedules (one scratch-sized chunk of bands at a
# time here, the whole block in jdft_apply_H), so they agree to the split's
# accuracy rather than bit for bit
TOL = {"fp64": 1e-10, "fp32": 1e-5, "tf32x3": 1e-5, "bf16x3": 2e-5}


def _system(name):
    from synth import WORKLOADS, atom_positions, random_coefficients
    from paper_1708_03621_gb300 import jdft
    w = WORKLOADS[name]
    atoms = atom_positions(w.R, w.natoms, w.seed_atoms)
    b = jdft.Basis(w.R, w.S, w.ecut, w.kfrac)
    V = torch.empty(int(np.prod(w.S)), dtype=torch.float64, device="cuda")
    jdft.jdft_gaussian_potential(b, atoms, V)
    jdft.jdft_set_potential(b, V)
    npw = b.npw(0)
    P = torch.empty((4 * w.natoms, npw), dtype=torch.complex128, device="cuda")
    jdft.jdft_gaussian_projectors(b, 0, atoms, P)
    D = torch.tensor(np.diag(np.tile([0.5, -0.3, -0.3, -0.3], w.natoms)), device="cuda")
    jdft.jdft_set_projectors(b, 0, P, D)
    damp = np.linspace(1.0, 50.0, npw)  # any smooth damping: only agreement between entry points matters
    return w, b, random_coefficients(damp, w.nbands, w.seed_coeffs)


def _rel(a, b):
    return float(np.max(np.linalg.norm(a - b, axis=1) / np.linalg.norm(b, axis=1)))


@pytest.mark.parametrize("name,prec", [(n, p) for n in ("mid", "large") for p in ("fp64", "fp32", "tf32x3", "bf16x3")])
def test_noalloc_matches_apply_H_twice(name, prec):
    from paper_1708_03621_gb300 import jdft
    w, b, C = _system(name)
    ct = np.complex128 if prec == "fp64" else np.complex64
    nb = C.shape[0] if name == "mid" else 40   # 40 bands of the large cell: several scratch-sized chunks
    C1 = torch.tensor(C[:nb].astype(ct), device="cuda")
    C2 = torch.tensor(C[nb:2 * nb].astype(ct), device="cuda") if name == "large" else torch.flip(C1, [0]).contiguous()
    for Cd in (C1, C2):
        ref = torch.empty_like(Cd)
        got = torch.full_like(Cd, float("nan"))
        jdft.jdft_apply_H(b, 0, Cd, ref, prec)
        jdft.jdft_apply_H_noalloc(b, 0, Cd, got, prec)
        torch.cuda.synchronize()
        assert _rel(got.cpu().numpy().astype(np.complex128), ref.cpu().numpy().astype(np.complex128)) < TOL[prec]
    b.close()


def test_noalloc_rejects_bands_larger_than_scratch():
    from paper_1708_03621_gb300 import jdft
    # a 100 x 100 x 512 box with a large sphere: one FP64 band needs ~60 MB of column buffer
    R = np.diag([40.0, 40.0, 40.0])
    b = jdft.Basis(R, (100, 100, 512), 30.0, [(0.0, 0.0, 0.0)])
    V = torch.zeros(100 * 100 * 512, dtype=torch.float64, device="cuda")
    jdft.jdft_set_potential(b, V)
    npw = b.npw(0)
    C = torch.zeros((1, npw), dtype=torch.complex128, device="cuda")
    HC = torch.zeros_like(C)
    with pytest.raises(jdft.JdftError, match="32 MiB"):
        jdft.jdft_apply_H_noalloc(b, 0, C, HC, "fp64")
    b.close()
