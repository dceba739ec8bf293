"""The C ABI library loads and exports every symbol include/jdft.h declares;
argument checks that need no GPU return the documented status (CPU only)."""
import ctypes
import os
import re

import pytest

from paper_1708_03621_gb300 import jdft

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    src = open(os.path.join(ROOT, "include", "jdft.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(jdft_\w+)\s*\(", src)))


def test_header_declarations_are_exported():
    L = jdft.lib()
    names = declared()
    assert len(names) >= 15
    for n in names:
        assert hasattr(L, n), n
    assert set(names) == set(jdft.EXPORTS)


def test_version_and_empty_error():
    assert "sm_103a" in jdft.jdft_version()
    assert jdft.lib().jdft_last_error() == b""


def test_null_arguments_rejected():
    L = jdft.lib()
    assert L.jdft_basis_create(None, None) == 1
    assert b"null" in L.jdft_last_error()
    assert L.jdft_apply_H(None, 0, None, 0, None, 0, 1, 0, None) == 1
    assert L.jdft_density(None, 0, None, 0, None, 1, None, 0, None) == 1
    assert L.jdft_apply_H_density(None, 0, None, 0, None, 0, 1, None, None, 0, None) == 1
    assert L.jdft_autotune(None, 0, None, 0, None, 0, 1, 3, None, None) == 1
    assert L.jdft_orthonormalize_async(None, 0, None, 1, 1, None, 0, None, None) == 1
    assert L.jdft_autotune_gemm(0, 1, 1, None, 1, None, 1, 3, None, None) == 1
    assert L.jdft_subspace(None, 0, None, 0, None, 0, 1, None, None, 0, None) == 1
    assert L.jdft_basis_npw(None, 0, None) == 1
    assert L.jdft_basis_destroy(None) == 0
    # the device-side wait limit is checked before any CUDA call
    assert L.jdft_set_wait_limit(ctypes.c_double(-1.0)) == 1
    assert L.jdft_set_wait_limit(ctypes.c_double(61.0)) == 1
    assert L.jdft_measure_fp32_peak(None, None, None, None) == 1


def test_bad_cell_descriptions_rejected():
    L = jdft.lib()
    desc = jdft._CellDesc()
    for i in range(3):
        desc.R[4 * i] = 6.0
        desc.S[i] = 12
    k = (ctypes.c_double * 3)(0.1, 0.2, 0.3)
    desc.kfrac = ctypes.cast(k, ctypes.POINTER(ctypes.c_double))
    h = ctypes.c_void_p()
    desc.nk = 0
    desc.ecut = 4.0
    assert L.jdft_basis_create(ctypes.byref(desc), ctypes.byref(h)) == 1
    desc.nk = 1
    desc.ecut = -1.0
    assert L.jdft_basis_create(ctypes.byref(desc), ctypes.byref(h)) == 1
    desc.ecut = 4.0
    desc.S[1] = 14  # 14 = 2 x 7: radix 7 unsupported
    assert L.jdft_basis_create(ctypes.byref(desc), ctypes.byref(h)) == 7
    desc.S[1] = 12
    desc.R[0] = 0.0
    desc.R[4] = 0.0
    assert L.jdft_basis_create(ctypes.byref(desc), ctypes.byref(h)) == 1
    assert not h.value


def test_more_null_and_size_arguments_rejected():
    """Every entry point checks its handle, pointers and sizes before any CUDA call."""
    L = jdft.lib()
    E = 1  # JDFT_ERR_ARG
    assert L.jdft_basis_gvectors(None, 0, None) == E
    assert L.jdft_basis_info(None, 0, None, None, None) == E
    assert L.jdft_set_potential(None, None, None) == E
    assert L.jdft_set_projectors(None, 0, None, 0, None, None) == E
    assert L.jdft_gaussian_potential(None, 1, None, 4.0, 1.0, None, None) == E
    assert L.jdft_gaussian_projectors(None, 0, 1, None, 1.0, None, None) == E
    for op in ("jdft_op_I", "jdft_op_Jdag"):
        assert getattr(L, op)(None, 0, None, 0, None, 1, 0, None) == E
    for op in ("jdft_op_J", "jdft_op_Idag"):
        assert getattr(L, op)(None, 0, None, None, 0, 1, 0, None) == E
    assert L.jdft_op_O(None, 0, None, 0, None, 0, 1, 0, None) == E
    assert L.jdft_apply_H_noalloc(None, 0, None, 0, None, 0, 1, 0, None) == E
    assert L.jdft_orthonormalize(None, 0, None, 1, 1, 0, None) == E
    assert L.jdft_subspace_eigs(0, None, None, None) == E
    assert L.jdft_minimize_bands(None, 0, None, 1, 1, None, None, None, None) == E
    assert L.jdft_autotune_chunk(None, 0, None, 0, None, 0, 1, 0, None, None) == E
    assert L.jdft_mlp_create(None, None) == E
    assert L.jdft_mlp_forward(None, 1, None, None, None) == E
    assert L.jdft_mlp_loss_grad(None, 1, None, None, None, None) == E
    assert L.jdft_mlp_adam_step(None, None, 1e-3, None) == E
    assert L.jdft_batch_create(0, None, None) == E
    assert L.jdft_batch_launch(None, None) == E
    buf = ctypes.create_string_buffer(1)
    assert L.jdft_profile_read(buf, 0) == E
    assert L.jdft_last_error() != b""


def test_scf_entry_points_check_arguments_first():
    """Hartree, LDA, Kohn-Sham potential, Pulay and SCF calls reject null
    handles, pointers and out-of-range options before any CUDA call."""
    L = jdft.lib()
    assert L.jdft_hartree(None, None, None, None, None) == 1
    assert L.jdft_xc_lda(None, None, None, None, None) == 1
    assert L.jdft_ks_potential(None, None, None, None, None, None) == 1
    h = ctypes.c_void_p()
    assert L.jdft_pulay_create(0, 4, ctypes.c_double(0.5), ctypes.byref(h)) == 1
    assert L.jdft_pulay_create(100, 0, ctypes.c_double(0.5), ctypes.byref(h)) == 1
    assert L.jdft_pulay_create(100, 17, ctypes.c_double(0.5), ctypes.byref(h)) == 1
    assert L.jdft_pulay_create(100, 4, ctypes.c_double(0.0), ctypes.byref(h)) == 1
    assert L.jdft_pulay_create(100, 4, ctypes.c_double(1.5), ctypes.byref(h)) == 1
    assert L.jdft_pulay_create(100, 4, ctypes.c_double(0.5), None) == 1
    assert not h.value
    assert L.jdft_pulay_step(None, None, None, None, None) == 1
    assert L.jdft_pulay_used(None, None, None) == 1
    assert L.jdft_pulay_reset(None) == 1
    assert L.jdft_pulay_destroy(None) == 0
    r = jdft.ScfReport()
    o = jdft.ScfOpts()
    assert L.jdft_scf(None, None, 0, 1, None, None, None, ctypes.byref(o), ctypes.byref(r), None) == 1


def test_field_and_dielectric_entry_points_check_arguments_first():
    L = jdft.lib()
    assert L.jdft_field_I(None, None, None, None) == 1
    assert L.jdft_field_J(None, None, None, None) == 1
    assert L.jdft_pcm_hessian(None, None, None, None, None) == 1
    r = jdft.PcmReport()
    assert L.jdft_pcm_solve(None, None, None, None, ctypes.c_double(1e-8), 10, 0, ctypes.byref(r), None) == 1


def test_spinor_entry_points_check_arguments_first():
    L = jdft.lib()
    assert L.jdft_apply_H_spinor(None, 0, None, None, 0, None, 0, 1, 0, None) == 1
    assert L.jdft_density_spinor(None, 0, None, 0, None, 1, None, None, 0, None) == 1


def test_overlap_entry_points_check_arguments_first():
    L = jdft.lib()
    assert L.jdft_set_augmentation(None, 0, None, None) == 1
    assert L.jdft_op_S(None, 0, None, 0, None, 0, 1, 0, None) == 1
    assert L.jdft_subspace_generalized(None, 0, None, 0, None, 0, 1, None, None, None, None) == 1
    assert L.jdft_orthonormalize_generalized(None, 0, None, 0, 1, None) == 1
    o, r = jdft.MinOpts(), jdft.MinReport()
    assert L.jdft_minimize_bands_generalized(None, 0, None, 0, 1, ctypes.byref(o), None, ctypes.byref(r), None) == 1
