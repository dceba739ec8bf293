"""Thin ctypes binding of libjdft.so (the C ABI declared in include/jdft.h).

Argument marshalling only: every step of the computation runs in the CUDA
library.  Tensors are PyTorch CUDA tensors; the binding passes their device
pointers, leading dimensions and the current CUDA stream.  Coefficient blocks
are (nb, ld) tensors, one band per row (band-major), complex128 for
``"fp64"`` and complex64 for the other precisions.

If libjdft.so has not been built, importing this module raises: there is no
CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libjdft.so")

PREC = {"fp64": 0, "fp32": 1, "tf32x3": 2, "bf16x3": 3}
STATUS = {0: "OK", 1: "ERR_ARG", 2: "ERR_CUDA", 3: "ERR_OOM", 4: "ERR_TIMEOUT",
          5: "ERR_NOT_POSDEF", 6: "ERR_NOT_CONVERGED", 7: "ERR_UNSUPPORTED"}
STATUS_CODES = {v: k for k, v in STATUS.items()}


class JdftError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: {STATUS.get(status, status)}: {msg}")
        self.status = status


class _CellDesc(ctypes.Structure):
    _fields_ = [("R", ctypes.c_double * 9), ("S", ctypes.c_int * 3), ("ecut", ctypes.c_double),
                ("nk", ctypes.c_int), ("kfrac", ctypes.POINTER(ctypes.c_double)),
                ("kweight", ctypes.POINTER(ctypes.c_double))]


class MinOpts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("max_iter", ctypes.c_int), ("precond", ctypes.c_int),
                ("prec", ctypes.c_int), ("switch_tol", ctypes.c_double), ("occupation", ctypes.c_double),
                ("mlp", ctypes.c_void_p)]


class MinReport(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("mixed_iterations", ctypes.c_int), ("converged", ctypes.c_int),
                ("energy", ctypes.c_double), ("residual", ctypes.c_double), ("seconds", ctypes.c_double),
                ("precond_fallback", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


PRECOND = {"identity": 0, "teter": 1, "mlp": 2}


class ScfOpts(ctypes.Structure):
    _fields_ = [("tol_energy", ctypes.c_double), ("tol_density", ctypes.c_double), ("max_iter", ctypes.c_int),
                ("history", ctypes.c_int), ("alpha", ctypes.c_double), ("band_tol", ctypes.c_double),
                ("band_max_iter", ctypes.c_int), ("precond", ctypes.c_int), ("prec", ctypes.c_int),
                ("occupation", ctypes.c_double), ("mlp", ctypes.c_void_p), ("band_tol_factor", ctypes.c_double)]


class ScfReport(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("converged", ctypes.c_int), ("band_iterations", ctypes.c_int),
                ("band_unconverged", ctypes.c_int), ("energy", ctypes.c_double), ("band_energy", ctypes.c_double),
                ("double_counting", ctypes.c_double), ("hartree", ctypes.c_double), ("xc", ctypes.c_double),
                ("residual", ctypes.c_double), ("seconds", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}

class ApplyItem(ctypes.Structure):
    _fields_ = [("basis", ctypes.c_void_p), ("ik", ctypes.c_int), ("C", ctypes.c_void_p), ("ldc", ctypes.c_int),
                ("HC", ctypes.c_void_p), ("ldhc", ctypes.c_int), ("nb", ctypes.c_int), ("prec", ctypes.c_int)]


_vp, _i, _d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
_SIGS = {
    "jdft_basis_create": [ctypes.POINTER(_CellDesc), ctypes.POINTER(_vp)],
    "jdft_basis_destroy": [_vp],
    "jdft_basis_npw": [_vp, _i, ctypes.POINTER(_i)],
    "jdft_basis_gvectors": [_vp, _i, _vp],
    "jdft_basis_info": [_vp, _i, ctypes.POINTER(_d), ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(_i)],
    "jdft_set_potential": [_vp, _vp, _vp],
    "jdft_set_projectors": [_vp, _i, _vp, _i, _vp, _vp],
    "jdft_gaussian_potential": [_vp, _i, _vp, _d, _d, _vp, _vp],
    "jdft_gaussian_projectors": [_vp, _i, _i, _vp, _d, _vp, _vp],
    "jdft_op_I": [_vp, _i, _vp, _i, _vp, _i, _i, _vp],
    "jdft_op_Jdag": [_vp, _i, _vp, _i, _vp, _i, _i, _vp],
    "jdft_op_J": [_vp, _i, _vp, _vp, _i, _i, _i, _vp],
    "jdft_op_Idag": [_vp, _i, _vp, _vp, _i, _i, _i, _vp],
    "jdft_op_O": [_vp, _i, _vp, _i, _vp, _i, _i, _i, _vp],
    "jdft_apply_H": [_vp, _i, _vp, _i, _vp, _i, _i, _i, _vp],
    "jdft_density": [_vp, _i, _vp, _i, _vp, _i, _vp, _i, _vp],
    "jdft_apply_H_density": [_vp, _i, _vp, _i, _vp, _i, _i, _vp, _vp, _i, _vp],
    "jdft_subspace": [_vp, _i, _vp, _i, _vp, _i, _i, _vp, _vp, _i, _vp],
    "jdft_apply_H_noalloc": [_vp, _i, _vp, _i, _vp, _i, _i, _i, _vp],
    "jdft_orthonormalize": [_vp, _i, _vp, _i, _i, _i, _vp],
    "jdft_subspace_eigs": [_i, _vp, _vp, _vp],
    "jdft_minimize_bands": [_vp, _i, _vp, _i, _i, ctypes.POINTER(MinOpts), _vp, ctypes.POINTER(MinReport), _vp],
    "jdft_mlp_create": [_vp, ctypes.POINTER(_vp)],
    "jdft_mlp_destroy": [_vp],
    "jdft_mlp_get_params": [_vp, _vp],
    "jdft_mlp_forward": [_vp, ctypes.c_int64, _vp, _vp, _vp],
    "jdft_mlp_loss_grad": [_vp, ctypes.c_int64, _vp, _vp, _vp, _vp],
    "jdft_mlp_adam_step": [_vp, _vp, ctypes.c_float, _vp],
    "jdft_mlp_rows": [_vp, _i, _vp, _vp, _i, ctypes.c_int64, ctypes.c_int64, _vp, ctypes.POINTER(ctypes.c_int64), _vp],
    "jdft_device_status": [_vp],
    "jdft_set_wait_limit": [_d],
    "jdft_hamiltonian_step": [_vp, _i, _vp, _i, _vp, _i, _i, _vp, _vp, _vp, _vp, _i, _vp, _i, _vp],
    "jdft_measure_fp32_peak": [ctypes.POINTER(_d), ctypes.POINTER(_d), ctypes.POINTER(_i), _vp],
    "jdft_batch_create": [_i, ctypes.POINTER(ApplyItem), ctypes.POINTER(_vp)],
    "jdft_batch_launch": [_vp, _vp],
    "jdft_batch_destroy": [_vp],
    "jdft_autotune_chunk": [_vp, _i, _vp, _i, _vp, _i, _i, _i, ctypes.POINTER(_i), _vp],
    "jdft_orthonormalize_async": [_vp, _i, _vp, _i, _i, _vp, _i, _vp, _vp],
    "jdft_autotune_gemm": [_i, _i, _i, _vp, _i, _vp, _i, _i, ctypes.POINTER(_i), _vp],
    "jdft_autotune": [_vp, _i, _vp, _i, _vp, _i, _i, _i, _vp, _vp],
    "jdft_hartree": [_vp, _vp, _vp, _vp, _vp],
    "jdft_xc_lda": [_vp, _vp, _vp, _vp, _vp],
    "jdft_ks_potential": [_vp, _vp, _vp, _vp, _vp, _vp],
    "jdft_pulay_create": [ctypes.c_int64, _i, _d, ctypes.POINTER(_vp)],
    "jdft_pulay_destroy": [_vp],
    "jdft_pulay_reset": [_vp],
    "jdft_pulay_step": [_vp, _vp, _vp, _vp, _vp],
    "jdft_pulay_used": [_vp, ctypes.POINTER(_i), _vp],
    "jdft_scf": [_vp, _vp, _i, _i, _vp, _vp, _vp, ctypes.POINTER(ScfOpts), ctypes.POINTER(ScfReport), _vp],
    "jdft_apply_H_spinor": [_vp, _i, _vp, _vp, _i, _vp, _i, _i, _i, _vp],
    "jdft_density_spinor": [_vp, _i, _vp, _i, _vp, _i, _vp, _vp, _i, _vp],
    "jdft_set_augmentation": [_vp, _i, _vp, _vp],
    "jdft_op_S": [_vp, _i, _vp, _i, _vp, _i, _i, _i, _vp],
    "jdft_subspace_generalized": [_vp, _i, _vp, _i, _vp, _i, _i, _vp, _vp, _vp, _vp],
    "jdft_orthonormalize_generalized": [_vp, _i, _vp, _i, _i, _vp],
    "jdft_minimize_bands_generalized": [_vp, _i, _vp, _i, _i, ctypes.POINTER(MinOpts), _vp,
                                        ctypes.POINTER(MinReport), _vp],
    "jdft_field_I": [_vp, _vp, _vp, _vp],
    "jdft_field_J": [_vp, _vp, _vp, _vp],
    "jdft_pcm_hessian": [_vp, _vp, _vp, _vp, _vp],
    "jdft_pcm_solve": [_vp, _vp, _vp, _vp, _d, _i, _i, _vp, _vp],
    "jdft_profile_enable": [_i],
    "jdft_profile_read": [ctypes.c_char_p, _i],
}
#: Every symbol include/jdft.h declares (the loader checks all are exported).
EXPORTS = sorted(list(_SIGS) + ["jdft_last_error", "jdft_version", "jdft_launch_count", "jdft_batch_is_kbatched"])

_lib = None


def lib() -> ctypes.CDLL:
    """The loaded library; raises if libjdft.so is missing (build it first)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libjdft.so not built at {LIB_PATH}: run "
                              "`python -m paper_1708_03621_gb300.build` (needs nvcc)")
        L = ctypes.CDLL(LIB_PATH)
        for name, args in _SIGS.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = ctypes.c_int
        L.jdft_last_error.restype = ctypes.c_char_p
        L.jdft_last_error.argtypes = []
        L.jdft_version.restype = ctypes.c_char_p
        L.jdft_version.argtypes = []
        L.jdft_launch_count.restype = ctypes.c_longlong
        L.jdft_launch_count.argtypes = []
        L.jdft_batch_is_kbatched.restype = ctypes.c_int
        L.jdft_batch_is_kbatched.argtypes = [ctypes.c_void_p]
        _lib = L
    return _lib


def _call(name: str, *args) -> None:
    L = lib()
    st = getattr(L, name)(*args)
    if st != 0:
        raise JdftError(st, name, L.jdft_last_error().decode())


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def _prec(p) -> int:
    return PREC[p] if isinstance(p, str) else int(p)


def _block(t, prec, name):
    """(pointer, ld, nb) of a band-major coefficient block."""
    import torch
    want = torch.complex128 if _prec(prec) == 0 else torch.complex64
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != want:
        raise ValueError(f"{name} must be {want} for precision {prec}")
    if t.dim() != 2 or t.stride(1) != 1:
        raise ValueError(f"{name} must be 2-D (nb, ld) with unit stride along the plane waves")
    return ctypes.c_void_p(t.data_ptr()), t.stride(0) if t.shape[0] > 1 else t.shape[1], t.shape[0]


def _ptr(t):
    return ctypes.c_void_p(0 if t is None else t.data_ptr())


class Basis:
    """Owner of a jdft_basis_t handle (see jdft_basis_create)."""

    def __init__(self, R, S, ecut, kfrac, kweight=None):
        R = np.asarray(R, dtype=np.float64)
        kf = np.ascontiguousarray(np.asarray(kfrac, dtype=np.float64).reshape(-1, 3))
        desc = _CellDesc()
        for i in range(3):
            for d in range(3):
                desc.R[3 * i + d] = R[i, d]
            desc.S[i] = int(S[i])
        desc.ecut = float(ecut)
        desc.nk = kf.shape[0]
        self._kf = kf
        desc.kfrac = kf.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        if kweight is not None:
            self._kw = np.ascontiguousarray(np.asarray(kweight, dtype=np.float64))
            desc.kweight = self._kw.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        h = ctypes.c_void_p()
        _call("jdft_basis_create", ctypes.byref(desc), ctypes.byref(h))
        self.handle = h
        self.S = tuple(int(s) for s in S)
        self.nk = kf.shape[0]

    def close(self):
        if getattr(self, "handle", None):
            lib().jdft_basis_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def npw(self, ik: int = 0) -> int:
        n = ctypes.c_int()
        _call("jdft_basis_npw", self.handle, ik, ctypes.byref(n))
        return n.value

    def gvectors(self, ik: int = 0) -> np.ndarray:
        out = np.empty((self.npw(ik), 3), dtype=np.int32)
        _call("jdft_basis_gvectors", self.handle, ik, ctypes.c_void_p(out.ctypes.data))
        return out

    def info(self, ik: int = 0):
        om, n, nc = ctypes.c_double(), ctypes.c_int64(), ctypes.c_int()
        _call("jdft_basis_info", self.handle, ik, ctypes.byref(om), ctypes.byref(n), ctypes.byref(nc))
        return {"omega": om.value, "N": n.value, "ncols": nc.value}


def jdft_basis_create(R, S, ecut, kfrac, kweight=None) -> Basis:
    return Basis(R, S, ecut, kfrac, kweight)


def jdft_set_potential(basis: Basis, V, stream=None) -> None:
    _call("jdft_set_potential", basis.handle, _ptr(V), _stream(stream))


def jdft_set_projectors(basis: Basis, ik: int, P, D, stream=None) -> None:
    """P: (nproj, npw) complex128 CUDA tensor (projector-major); D: (nproj, nproj) float64."""
    nproj = 0 if P is None else P.shape[0]
    _call("jdft_set_projectors", basis.handle, ik, _ptr(P), nproj, _ptr(D), _stream(stream))


def jdft_gaussian_potential(basis: Basis, atoms, V_out, depth=4.0, width=1.0, stream=None) -> None:
    a = np.ascontiguousarray(np.asarray(atoms, dtype=np.float64))
    _call("jdft_gaussian_potential", basis.handle, a.shape[0], ctypes.c_void_p(a.ctypes.data), depth, width,
          _ptr(V_out), _stream(stream))


def jdft_gaussian_projectors(basis: Basis, ik: int, atoms, P_out, sigma=1.0, stream=None) -> None:
    a = np.ascontiguousarray(np.asarray(atoms, dtype=np.float64))
    _call("jdft_gaussian_projectors", basis.handle, ik, a.shape[0], ctypes.c_void_p(a.ctypes.data), sigma,
          _ptr(P_out), _stream(stream))


def jdft_op_I(basis, ik, C, psi, prec="fp64", stream=None):
    p, ld, nb = _block(C, prec, "C")
    _call("jdft_op_I", basis.handle, ik, p, ld, _ptr(psi), nb, _prec(prec), _stream(stream))


def jdft_op_Jdag(basis, ik, C, psi, prec="fp64", stream=None):
    p, ld, nb = _block(C, prec, "C")
    _call("jdft_op_Jdag", basis.handle, ik, p, ld, _ptr(psi), nb, _prec(prec), _stream(stream))


def jdft_op_J(basis, ik, psi, C, prec="fp64", stream=None):
    p, ld, nb = _block(C, prec, "C")
    _call("jdft_op_J", basis.handle, ik, _ptr(psi), p, ld, nb, _prec(prec), _stream(stream))


def jdft_op_Idag(basis, ik, psi, C, prec="fp64", stream=None):
    p, ld, nb = _block(C, prec, "C")
    _call("jdft_op_Idag", basis.handle, ik, _ptr(psi), p, ld, nb, _prec(prec), _stream(stream))


def jdft_op_O(basis, ik, C, OC, prec="fp64", stream=None):
    p, ld, nb = _block(C, prec, "C")
    q, ldo, _ = _block(OC, prec, "OC")
    _call("jdft_op_O", basis.handle, ik, p, ld, q, ldo, nb, _prec(prec), _stream(stream))


def jdft_apply_H(basis, ik, C, HC, prec="fp64", stream=None):
    p, ld, nb = _block(C, prec, "C")
    q, ldh, nb2 = _block(HC, prec, "HC")
    if nb2 != nb:
        raise ValueError("C and HC must hold the same number of bands")
    _call("jdft_apply_H", basis.handle, ik, p, ld, q, ldh, nb, _prec(prec), _stream(stream))


def jdft_apply_H_noalloc(basis, ik, C, HC, prec="fp64", stream=None):
    """jdft_apply_H without device allocation (static 32 MiB scratch in the library)."""
    p, ld, nb = _block(C, prec, "C")
    q, ldh, nb2 = _block(HC, prec, "HC")
    if nb2 != nb:
        raise ValueError("C and HC must hold the same number of bands")
    _call("jdft_apply_H_noalloc", basis.handle, ik, p, ld, q, ldh, nb, _prec(prec), _stream(stream))


def jdft_apply_H_density(basis, ik, C, HC, f, n_r, prec="fp64", stream=None):
    """HC = H C and n_r += w_k sum_b f_b |I C_b|^2 in one pass over the box."""
    p, ld, nb = _block(C, prec, "C")
    q, ldh, nb2 = _block(HC, prec, "HC")
    if nb2 != nb:
        raise ValueError("C and HC must hold the same number of bands")
    _call("jdft_apply_H_density", basis.handle, ik, p, ld, q, ldh, nb, _ptr(f), _ptr(n_r), _prec(prec),
          _stream(stream))


def jdft_density(basis, ik, C, f, n_r, prec="fp64", stream=None):
    p, ld, nb = _block(C, prec, "C")
    _call("jdft_density", basis.handle, ik, p, ld, _ptr(f), nb, _ptr(n_r), _prec(prec), _stream(stream))


def jdft_subspace(basis, ik, C, HC, CHC, COC, prec="fp64", stream=None):
    p, ld, nb = _block(C, prec, "C")
    if HC is not None:
        q, ldh, _ = _block(HC, prec, "HC")
    else:
        q, ldh = ctypes.c_void_p(0), ld
    _call("jdft_subspace", basis.handle, ik, p, ld, q, ldh, nb, _ptr(CHC), _ptr(COC), _prec(prec),
          _stream(stream))


def jdft_orthonormalize(basis, ik, C, prec="fp64", stream=None):
    """C <- C L^{-dag}, Omega C^dag C = L L^dag (complex128 block for fp64, complex64 otherwise)."""
    p, ld, nb = _block(C, prec, "C")
    _call("jdft_orthonormalize", basis.handle, ik, p, ld, nb, _prec(prec), _stream(stream))


def jdft_orthonormalize_async(basis, ik, C, status, prec="fp64", stream=None, U=None):
    """jdft_orthonormalize without the wait; failures are merged into the device int32 tensor `status`.

    U: None, or the complex128 (nb, nb) CUDA tensor C^dag O C of this block
    (the COC output of jdft_subspace), read instead of recomputed."""
    import torch
    p, ld, nb = _block(C, prec, "C")
    if U is not None and not (U.is_cuda and U.dtype == torch.complex128 and tuple(U.shape) == (nb, nb)
                              and U.is_contiguous()):
        raise ValueError("U must be a contiguous complex128 (nb, nb) CUDA tensor")
    _call("jdft_orthonormalize_async", basis.handle, ik, p, ld, nb, _ptr(U) if U is not None else None,
          _prec(prec), _ptr(status), _stream(stream))


def jdft_hamiltonian_step(basis, ik, C, HC, f, n_r, CHC, COC, status=None, prec="bf16x3", stream=None):
    """One pass of the hot path: HC = H C, n_r += density, COC = C^dag O C, CHC = C^dag H C,
    and C <- C L^{-dag} (COC = L L^dag) when a device int32 status word is given."""
    p, ld, nb = _block(C, prec, "C")
    q, ldh, nbh = _block(HC, prec, "HC")
    if nbh != nb:
        raise ValueError("C and HC must have the same number of bands")
    _call("jdft_hamiltonian_step", basis.handle, ik, p, ld, q, ldh, nb, _ptr(f), _ptr(n_r), _ptr(CHC), _ptr(COC),
          1 if status is not None else 0, _ptr(status) if status is not None else None, _prec(prec),
          _stream(stream))


def jdft_subspace_eigs(A, eigs, stream=None):
    """Eigenvalues of the Hermitian complex128 (nb, nb) CUDA tensor A into eigs (float64, nb)."""
    _call("jdft_subspace_eigs", A.shape[0], _ptr(A), _ptr(eigs), _stream(stream))


def jdft_minimize_bands(basis, ik, C, eigs=None, tol=1e-8, max_iter=1000, precond="teter", prec="fp64",
                        switch_tol=0.0, occupation=2.0, mlp=None, stream=None, check=True) -> dict:
    """Preconditioned band CG in place on the complex128 block C; returns the report as a dict."""
    p, ld, nb = _block(C, "fp64", "C")
    o = MinOpts(tol, max_iter, PRECOND[precond] if isinstance(precond, str) else int(precond), _prec(prec),
                switch_tol, occupation, ctypes.c_void_p(0 if mlp is None else mlp.handle.value))
    r = MinReport()
    L = lib()
    st = L.jdft_minimize_bands(basis.handle, ik, p, ld, nb, ctypes.byref(o), _ptr(eigs), ctypes.byref(r),
                               _stream(stream))
    out = r.as_dict()
    out["status"] = STATUS.get(st, st)
    if check and st != 0:
        raise JdftError(st, "jdft_minimize_bands", L.jdft_last_error().decode())
    return out


def _field(t, name, N=None):
    """Pointer of a real FP64 box (a contiguous float64 CUDA tensor)."""
    import torch
    if not t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous float64 CUDA tensor")
    if N is not None and t.numel() != N:
        raise ValueError(f"{name} must hold {N} values")
    return ctypes.c_void_p(t.data_ptr())


def jdft_hartree(basis, n, vh, energy=None, stream=None):
    """vh = V_H[n]; energy (float64 CUDA tensor of 1, optional) = E_H."""
    N = int(np.prod(basis.S))
    _call("jdft_hartree", basis.handle, _field(n, "n", N), _field(vh, "vh", N),
          _ptr(energy), _stream(stream))


def jdft_xc_lda(basis, n, vxc=None, energy=None, stream=None):
    """vxc = v_xc[n] (optional); energy (float64 CUDA tensor of 1, optional) = E_xc."""
    N = int(np.prod(basis.S))
    _call("jdft_xc_lda", basis.handle, _field(n, "n", N), None if vxc is None else _field(vxc, "vxc", N),
          _ptr(energy), _stream(stream))


def jdft_ks_potential(basis, n, vion, vks, energies=None, stream=None):
    """vks = vion + V_H[n] + v_xc[n]; energies (float64 CUDA tensor of 2, optional) = (E_H, E_xc)."""
    N = int(np.prod(basis.S))
    _call("jdft_ks_potential", basis.handle, _field(n, "n", N), _field(vion, "vion", N), _field(vks, "vks", N),
          _ptr(energies), _stream(stream))


class Pulay:
    """Owner of a jdft_pulay_t density mixer (see jdft_pulay_create)."""

    def __init__(self, n: int, history: int = 8, alpha: float = 0.5):
        h = ctypes.c_void_p()
        _call("jdft_pulay_create", int(n), int(history), float(alpha), ctypes.byref(h))
        self.handle = h
        self.n = int(n)

    def step(self, n_in, n_out, n_next, stream=None):
        _call("jdft_pulay_step", self.handle, _field(n_in, "n_in", self.n), _field(n_out, "n_out", self.n),
              _field(n_next, "n_next", self.n), _stream(stream))

    def used(self, stream=None) -> int:
        u = ctypes.c_int()
        _call("jdft_pulay_used", self.handle, ctypes.byref(u), _stream(stream))
        return u.value

    def reset(self):
        _call("jdft_pulay_reset", self.handle)

    def close(self):
        if getattr(self, "handle", None):
            lib().jdft_pulay_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def jdft_scf(basis, C, vion, n_r, eigs=None, tol_energy=1e-8, tol_density=1e-6, max_iter=100, history=8,
             alpha=0.5, band_tol=1e-9, band_max_iter=1000, precond="teter", prec="fp64", occupation=2.0,
             mlp=None, band_tol_factor=0.0, stream=None, check=True) -> dict:
    """SCF loop; C: list of nk complex128 (nb, ld) CUDA blocks (updated in place).  Returns the report."""
    if len(C) != basis.nk:
        raise ValueError("one coefficient block per k-point is required")
    blocks = [_block(c, "fp64", f"C[{i}]") for i, c in enumerate(C)]
    ld, nb = blocks[0][1], blocks[0][2]
    if any(b[1] != ld or b[2] != nb for b in blocks):
        raise ValueError("all blocks need the same band count and row stride (views of (nb, ld) storage with "
                         "ld >= the largest npw)")
    ptrs = (ctypes.c_void_p * len(C))(*[b[0].value for b in blocks])
    N = int(np.prod(basis.S))
    o = ScfOpts(tol_energy, tol_density, max_iter, history, alpha, band_tol, band_max_iter,
                PRECOND[precond] if isinstance(precond, str) else int(precond), _prec(prec), occupation,
                ctypes.c_void_p(0 if mlp is None else mlp.handle.value), band_tol_factor)
    r = ScfReport()
    L = lib()
    st = L.jdft_scf(basis.handle, ctypes.cast(ptrs, ctypes.c_void_p), ld, nb, _field(vion, "vion", N),
                    _field(n_r, "n_r", N), _ptr(eigs), ctypes.byref(o), ctypes.byref(r), _stream(stream))
    out = r.as_dict()
    out["status"] = STATUS.get(st, st)
    if check and st != 0:
        raise JdftError(st, "jdft_scf", L.jdft_last_error().decode())
    return out


def jdft_apply_H_spinor(basis, ik, M, C, HC, prec="fp64", stream=None):
    """C, HC: (2 nb, ld) blocks, rows alternating up, down; M: float64 CUDA tensor of 3 N (M_x, M_y, M_z)."""
    p, ld, n2 = _block(C, prec, "C")
    q, ldh, n2h = _block(HC, prec, "HC")
    if n2 % 2 or n2h != n2:
        raise ValueError("spinor blocks need an even number of rows (up, down per band), equal for C and HC")
    N = int(np.prod(basis.S))
    _call("jdft_apply_H_spinor", basis.handle, ik, _field(M, "M", 3 * N), p, ld, q, ldh, n2 // 2, _prec(prec),
          _stream(stream))


def jdft_density_spinor(basis, ik, C, f, n_r, m_r, prec="fp64", stream=None):
    """n_r (N) and m_r (3 N) accumulate the density and magnetisation of the spinor block C (2 nb rows)."""
    p, ld, n2 = _block(C, prec, "C")
    if n2 % 2:
        raise ValueError("spinor blocks need an even number of rows")
    N = int(np.prod(basis.S))
    _call("jdft_density_spinor", basis.handle, ik, p, ld, _field(f, "f", n2 // 2), n2 // 2, _field(n_r, "n_r", N),
          _field(m_r, "m_r", 3 * N), _prec(prec), _stream(stream))


def jdft_set_augmentation(basis, ik, Q, stream=None):
    """Q: (nproj, nproj) float64 CUDA tensor (symmetric), or None to clear."""
    _call("jdft_set_augmentation", basis.handle, ik, _ptr(Q), _stream(stream))


def jdft_op_S(basis, ik, C, SC, prec="fp64", stream=None):
    p, ld, nb = _block(C, prec, "C")
    q, lds, nbs = _block(SC, prec, "SC")
    if nbs != nb:
        raise ValueError("C and SC must have the same number of bands")
    _call("jdft_op_S", basis.handle, ik, p, ld, q, lds, nb, _prec(prec), _stream(stream))


def jdft_subspace_generalized(basis, ik, C, HC, CHC, CSC, eigs=None, stream=None):
    p, ld, nb = _block(C, "fp64", "C")
    q, ldh, nbh = _block(HC, "fp64", "HC")
    if nbh != nb:
        raise ValueError("C and HC must have the same number of bands")
    _call("jdft_subspace_generalized", basis.handle, ik, p, ld, q, ldh, nb, _ptr(CHC), _ptr(CSC), _ptr(eigs),
          _stream(stream))


def jdft_orthonormalize_generalized(basis, ik, C, stream=None):
    p, ld, nb = _block(C, "fp64", "C")
    _call("jdft_orthonormalize_generalized", basis.handle, ik, p, ld, nb, _stream(stream))


def jdft_minimize_bands_generalized(basis, ik, C, eigs=None, tol=1e-8, max_iter=1000, precond="teter",
                                    occupation=2.0, stream=None, check=True) -> dict:
    """Generalised (S-orthonormal) band CG in place on the complex128 block C; returns the report."""
    p, ld, nb = _block(C, "fp64", "C")
    o = MinOpts(tol, max_iter, PRECOND[precond] if isinstance(precond, str) else int(precond), 0, 0.0, occupation,
                ctypes.c_void_p(0))
    r = MinReport()
    L = lib()
    st = L.jdft_minimize_bands_generalized(basis.handle, ik, p, ld, nb, ctypes.byref(o), _ptr(eigs), ctypes.byref(r),
                                           _stream(stream))
    out = r.as_dict()
    out["status"] = STATUS.get(st, st)
    if check and st != 0:
        raise JdftError(st, "jdft_minimize_bands_generalized", L.jdft_last_error().decode())
    return out


class PcmReport(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("converged", ctypes.c_int), ("residual", ctypes.c_double),
                ("A_diel", ctypes.c_double), ("seconds", ctypes.c_double), ("fp64_hessians", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


def _cfield(t, name, N):
    """Pointer of a complex128 box (a contiguous CUDA tensor of N values)."""
    import torch
    if not t.is_cuda or t.dtype != torch.complex128 or not t.is_contiguous() or t.numel() != N:
        raise ValueError(f"{name} must be a contiguous complex128 CUDA tensor of {N} values")
    return ctypes.c_void_p(t.data_ptr())


def jdft_field_I(basis, X, x, stream=None):
    N = int(np.prod(basis.S))
    _call("jdft_field_I", basis.handle, _cfield(X, "X", N), _cfield(x, "x", N), _stream(stream))


def jdft_field_J(basis, x, X, stream=None):
    N = int(np.prod(basis.S))
    _call("jdft_field_J", basis.handle, _cfield(x, "x", N), _cfield(X, "X", N), _stream(stream))


def jdft_pcm_hessian(basis, eps, phi_t, out_t, stream=None):
    N = int(np.prod(basis.S))
    _call("jdft_pcm_hessian", basis.handle, _field(eps, "eps", N), _cfield(phi_t, "phi_t", N),
          _cfield(out_t, "out_t", N), _stream(stream))


def jdft_pcm_solve(basis, eps, rho_t, phi_t, tol=1e-10, max_iter=500, prec="fp64", stream=None,
                   check=True) -> dict:
    """phi_t = hessian^{-1} rho_t (G != 0) by preconditioned CG ("fp64") or FP32 CG rounds with FP64
    residuals ("fp32"); returns the report (A_diel included)."""
    N = int(np.prod(basis.S))
    r = PcmReport()
    L = lib()
    st = L.jdft_pcm_solve(basis.handle, _field(eps, "eps", N), _cfield(rho_t, "rho_t", N), _cfield(phi_t, "phi_t", N),
                          float(tol), int(max_iter), _prec(prec), ctypes.byref(r), _stream(stream))
    out = r.as_dict()
    out["status"] = STATUS.get(st, st)
    if check and st != 0:
        raise JdftError(st, "jdft_pcm_solve", L.jdft_last_error().decode())
    return out


MLP_NPARAM = 4481


class Mlp:
    """Owner of a jdft_mlp_t (the learned preconditioner network)."""

    def __init__(self, params):
        p = np.ascontiguousarray(np.asarray(params, dtype=np.float32))
        if p.size != MLP_NPARAM:
            raise ValueError(f"need {MLP_NPARAM} parameters")
        h = ctypes.c_void_p()
        _call("jdft_mlp_create", ctypes.c_void_p(p.ctypes.data), ctypes.byref(h))
        self.handle = h

    def close(self):
        if getattr(self, "handle", None):
            lib().jdft_mlp_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def params(self) -> np.ndarray:
        out = np.empty(MLP_NPARAM, dtype=np.float32)
        _call("jdft_mlp_get_params", self.handle, ctypes.c_void_p(out.ctypes.data))
        return out


def jdft_mlp_forward(mlp, feats, K, stream=None):
    _call("jdft_mlp_forward", mlp.handle, feats.shape[0], _ptr(feats), _ptr(K), _stream(stream))


def jdft_mlp_loss_grad(mlp, rows, grad, loss, stream=None):
    """rows: (n, 5) float32 CUDA tensor; grad: float32 (4481,); loss: float64 (2,)."""
    _call("jdft_mlp_loss_grad", mlp.handle, rows.shape[0], _ptr(rows), _ptr(grad), _ptr(loss), _stream(stream))


def jdft_mlp_adam_step(mlp, grad, lr, stream=None):
    _call("jdft_mlp_adam_step", mlp.handle, _ptr(grad), float(lr), _stream(stream))


def jdft_mlp_rows(basis, ik, C, Cstar, stride=1, offset=0, stream=None):
    """Training rows (float32 CUDA tensor (n, 5)) from snapshot C and converged Cstar (complex128, ld = npw)."""
    import torch
    nb = C.shape[0]
    n = ctypes.c_int64()
    _call("jdft_mlp_rows", basis.handle, ik, _ptr(C), _ptr(Cstar), nb, stride, offset, ctypes.c_void_p(0),
          ctypes.byref(n), _stream(stream))
    out = torch.empty((n.value, 5), dtype=torch.float32, device=C.device)
    _call("jdft_mlp_rows", basis.handle, ik, _ptr(C), _ptr(Cstar), nb, stride, offset, _ptr(out), ctypes.byref(n),
          _stream(stream))
    return out


def jdft_version() -> str:
    return lib().jdft_version().decode()


def jdft_profile_enable(on: bool = True) -> None:
    _call("jdft_profile_enable", 1 if on else 0)


def jdft_profile_read() -> dict:
    """{kernel name: (launches, total ms)} since the last read (waits for the events)."""
    buf = ctypes.create_string_buffer(1 << 16)
    _call("jdft_profile_read", buf, len(buf))
    out = {}
    for line in buf.value.decode().splitlines():
        name, n, ms = line.split()
        out[name] = (int(n), float(ms))
    return out


def jdft_autotune_chunk(basis, ik, C, HC, prec="fp64", stream=None) -> int:
    """Pick and keep the fastest band-chunk budget (MB) for apply_H on these blocks."""
    p, ld, nb = _block(C, prec, "C")
    q, ldh, _ = _block(HC, prec, "HC")
    out = ctypes.c_int()
    _call("jdft_autotune_chunk", basis.handle, ik, p, ld, q, ldh, nb, _prec(prec), ctypes.byref(out),
          _stream(stream))
    return out.value


def jdft_autotune_gemm(A, B, prec="bf16x3", stream=None) -> int:
    """Tune and keep the split-K schedule of A^dag B (band-major complex64 blocks A: M x K, B: N x K)."""
    p, lda, M = _block(A, prec, "A")
    q, ldb, N = _block(B, prec, "B")
    K = A.shape[1]
    out = ctypes.c_int()
    _call("jdft_autotune_gemm", M, N, K, p, lda, q, ldb, _prec(prec), ctypes.byref(out), _stream(stream))
    return out.value


class TuneReport(ctypes.Structure):
    _fields_ = [("chunk_mb", ctypes.c_int), ("splits_subspace", ctypes.c_int), ("splits_projector", ctypes.c_int),
                ("plane_bands", ctypes.c_int)]


def jdft_autotune(basis, ik, C, HC, prec="bf16x3", stream=None) -> dict:
    """Tune the FFT-chain chunk budget and the GEMM schedules of this block (overwrites HC)."""
    p, ld, nb = _block(C, prec, "C")
    q, ldh, _ = _block(HC, prec, "HC")
    r = TuneReport()
    _call("jdft_autotune", basis.handle, ik, p, ld, q, ldh, nb, _prec(prec), ctypes.c_void_p(ctypes.addressof(r)),
          _stream(stream))
    return {"chunk_mb": r.chunk_mb, "splits_subspace": r.splits_subspace, "splits_projector": r.splits_projector,
            "plane_bands": r.plane_bands}


class Batch:
    """A CUDA graph of Hamiltonian applications (see jdft_batch_create).

    items: sequence of (basis, ik, C, HC, prec) with CUDA tensors C, HC."""

    def __init__(self, items):
        arr = (ApplyItem * len(items))()
        self._keep = []
        for i, (basis, ik, C, HC, prec) in enumerate(items):
            p, ld, nb = _block(C, prec, "C")
            q, ldh, _ = _block(HC, prec, "HC")
            arr[i] = ApplyItem(basis.handle.value, ik, p.value, ld, q.value, ldh, nb, _prec(prec))
            self._keep.append((basis, C, HC))
        h = ctypes.c_void_p()
        _call("jdft_batch_create", len(items), arr, ctypes.byref(h))
        self.handle = h

    @property
    def kbatched(self) -> bool:
        """Whether the chain runs one launch per stage over all items."""
        return bool(lib().jdft_batch_is_kbatched(self.handle))

    def launch(self, stream=None):
        _call("jdft_batch_launch", self.handle, _stream(stream))

    def close(self):
        if getattr(self, "handle", None):
            lib().jdft_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def jdft_device_status(stream=None) -> None:
    """Raise JdftError(ERR_TIMEOUT) if a bounded device-side wait gave up."""
    _call("jdft_device_status", _stream(stream))


def jdft_set_wait_limit(seconds: float) -> None:
    """Limit of the tensor-core products' device-side waits on the current device."""
    _call("jdft_set_wait_limit", ctypes.c_double(seconds))


def jdft_measure_fp32_peak(stream=None) -> dict:
    """Measured FP32 peak of the current device (scalar and packed FMA chains), TFLOP/s."""
    a, b, n = ctypes.c_double(), ctypes.c_double(), ctypes.c_int()
    _call("jdft_measure_fp32_peak", ctypes.byref(a), ctypes.byref(b), ctypes.byref(n), _stream(stream))
    return {"ffma_tflops": a.value, "ffma2_tflops": b.value, "sms": n.value}


def jdft_launch_count() -> int:
    """Kernels the library has launched in this process."""
    return int(lib().jdft_launch_count())
