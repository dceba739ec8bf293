"""The 40 x 20 x 20 bohr slab (orthorhombic box 256 x 128 x 128, 125 k plane
waves, 256 atoms in a perturbed fcc slab, 1024 projectors, 1024 bands, 4
k-points) through the C ABI: the whole block runs on the GPU, and the FP64
oracle checks sampled bands, the matching subspace columns, and a second
k-point's sphere."""
import numpy as np
import pytest

from tests.systems import GpuSystem, OracleSystem, band_rel_err, workload

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "bf16x3": 2e-5}
CTYPE = {"fp64": np.complex128, "bf16x3": np.complex64}

_sys = {}


def slab():
    if "g" not in _sys:
        w = workload("slab")
        o = OracleSystem(w)
        _sys.update(w=w, o=o, g=GpuSystem(w, o.atoms))
    return _sys["w"], _sys["o"], _sys["g"]


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
def test_slab_sampled_bands(prec):
    from paper_1708_03621_gb300 import jdft
    w, o, g = slab()
    assert g.basis.npw(0) == o.basis.npw
    C = o.coeffs()                                   # (1024, npw)
    Cd = torch.tensor(C.astype(CTYPE[prec]), device="cuda")
    HC = torch.empty_like(Cd)
    jdft.jdft_apply_H(g.basis, 0, Cd, HC, prec)
    sample = [0, 517, 1023]
    ref = o.apply_H(C[sample])
    got = HC[sample].cpu().numpy().astype(np.complex128)
    assert band_rel_err(got, ref) < TOL[prec]
    nb = C.shape[0]
    CHC = torch.empty((nb, nb), dtype=torch.complex128, device="cuda")
    jdft.jdft_subspace(g.basis, 0, Cd, HC, CHC, None, prec)
    ref_cols = C.conj() @ ref.T                      # C^dag (H C_b) for the sampled b
    got_cols = CHC.cpu().numpy()[:, sample]
    assert np.max(np.abs(got_cols - ref_cols)) / np.max(np.abs(ref_cols)) < 10 * TOL[prec]
    jdft.jdft_device_status()


def test_slab_other_kpoint():
    """k-point 3 has its own sphere (sizes differ by a few plane waves): 8 bands in FP32."""
    from paper_1708_03621_gb300 import jdft
    w, _, g = slab()
    o3 = OracleSystem(w, ik=3)
    assert g.basis.npw(3) == o3.basis.npw
    C = o3.coeffs(8, seed=55)
    Cd = torch.tensor(C.astype(np.complex64), device="cuda")
    HC = torch.empty_like(Cd)
    jdft.jdft_apply_H(g.basis, 3, Cd, HC, "fp32")
    assert band_rel_err(HC.cpu().numpy().astype(np.complex128), o3.apply_H(C)) < 1e-5
