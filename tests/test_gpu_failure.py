"""Failure detection on the device, without a GPU fault (GPU).

The tensor-core products wait on shared-memory barriers for their batches of
products.  Every such wait is bounded by a run-time limit
(jdft_set_wait_limit).  With the limit at 0 every wait gives up at once: the
product must stop issuing, wait for what it already committed, free its
tensor memory, return, and leave JDFT_ERR_TIMEOUT for jdft_device_status.  The
context must stay usable: the next call, with the default limit back, gives
the normal result and a clean status.
"""
import numpy as np
import pytest

from tests.systems import GpuSystem, OracleSystem, band_rel_err, workload

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", ["tf32x3", "bf16x3"])
def test_wait_limit_runs_out_and_context_survives(prec):
    from paper_1708_03621_gb300 import jdft
    w = workload("mid")
    o = OracleSystem(w)
    g = GpuSystem(w, o.atoms)
    C = o.coeffs()
    Cd = torch.tensor(C.astype(np.complex64), device="cuda")
    ref = torch.empty_like(Cd)
    jdft.jdft_apply_H(g.basis, 0, Cd, ref, prec)
    jdft.jdft_device_status()
    out = torch.zeros_like(Cd)
    jdft.jdft_set_wait_limit(0.0)
    try:
        # the projector products P^dag C and P (D P^dag C) both give up
        jdft.jdft_apply_H(g.basis, 0, Cd, out, prec)
        with pytest.raises(jdft.JdftError) as err:
            jdft.jdft_device_status()
        assert err.value.status == jdft.STATUS_CODES["ERR_TIMEOUT"]
    finally:
        jdft.jdft_set_wait_limit(2.0)
    # the status was cleared by the read; the same call now completes normally
    jdft.jdft_device_status()
    jdft.jdft_apply_H(g.basis, 0, Cd, out, prec)
    jdft.jdft_device_status()
    torch.cuda.synchronize()
    got = out.cpu().numpy().astype(np.complex128)
    assert band_rel_err(got, ref.cpu().numpy().astype(np.complex128)) < 1e-6
    assert band_rel_err(got, o.apply_H(C)) < 2e-5


def test_wait_limit_runs_out_in_split_operand_products():
    """The same for the BF16x3 subspace products that read split operands
    through the ring fed by bulk asynchronous copies (40 bands: both
    dimensions above 32)."""
    from paper_1708_03621_gb300 import jdft
    w = workload("mid")
    o = OracleSystem(w)
    g = GpuSystem(w, o.atoms)
    C = o.coeffs(40, seed=8)
    Cd = torch.tensor(C.astype(np.complex64), device="cuda")
    HC = torch.empty_like(Cd)
    jdft.jdft_apply_H(g.basis, 0, Cd, HC, "bf16x3")
    nb = C.shape[0]
    ref = torch.empty((nb, nb), dtype=torch.complex128, device="cuda")
    jdft.jdft_subspace(g.basis, 0, Cd, HC, ref, None, "bf16x3")
    jdft.jdft_device_status()
    got = torch.zeros_like(ref)
    jdft.jdft_set_wait_limit(0.0)
    try:
        jdft.jdft_subspace(g.basis, 0, Cd, HC, got, None, "bf16x3")
        with pytest.raises(jdft.JdftError) as err:
            jdft.jdft_device_status()
        assert err.value.status == jdft.STATUS_CODES["ERR_TIMEOUT"]
    finally:
        jdft.jdft_set_wait_limit(2.0)
    jdft.jdft_subspace(g.basis, 0, Cd, HC, got, None, "bf16x3")
    jdft.jdft_device_status()
    a, b = got.cpu().numpy(), ref.cpu().numpy()
    assert np.max(np.abs(a - b)) / np.max(np.abs(b)) < 1e-6
    HCo = o.apply_H(C)
    assert np.max(np.abs(a - C.conj() @ HCo.T)) / np.max(np.abs(b)) < 2e-5


def test_wait_limit_runs_out_in_persistent_products():
    """The same on the 128^3 block (62 759 plane waves, 256 bands), where
    P (D P^dag C) runs as the persistent product with separate copy, MMA and
    epilogue warps: every role gives up, the block drains and frees its
    tensor memory, and the next call is exact again."""
    from paper_1708_03621_gb300 import jdft
    w = workload("large")
    o = OracleSystem(w)
    g = GpuSystem(w, o.atoms)
    Cd = torch.tensor(o.coeffs().astype(np.complex64), device="cuda")
    ref = torch.empty_like(Cd)
    jdft.jdft_apply_H(g.basis, 0, Cd, ref, "bf16x3")
    jdft.jdft_device_status()
    out = torch.zeros_like(Cd)
    jdft.jdft_set_wait_limit(0.0)
    try:
        jdft.jdft_apply_H(g.basis, 0, Cd, out, "bf16x3")
        with pytest.raises(jdft.JdftError) as err:
            jdft.jdft_device_status()
        assert err.value.status == jdft.STATUS_CODES["ERR_TIMEOUT"]
    finally:
        jdft.jdft_set_wait_limit(2.0)
    jdft.jdft_device_status()
    jdft.jdft_apply_H(g.basis, 0, Cd, out, "bf16x3")
    jdft.jdft_device_status()
    torch.cuda.synchronize()
    assert torch.equal(out, ref)
