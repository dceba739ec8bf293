"""GPU parity of the FFT chain, Hamiltonian, density and subspace against the
FP64 oracle, element by element, through the C ABI.

Tolerances: FP64 path 1e-10 relative (per band, and max-abs over max-abs);
FP32 path (FFT chain and products in FP32, accumulations in FP64) 1e-5
relative per band.  Workloads span several FFT lengths (12, 15, 16, 40, 48,
128 -> radices 2, 3, 4, 5, 8), ragged band counts and column groups, padded
leading dimensions and several band chunks.
"""
import os

import numpy as np
import pytest

from oracle import planewave as pw
from tests.systems import GpuSystem, OracleSystem, band_rel_err, workload

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# bf16x3: x = hi + lo in BF16 represents x to 2^-18 (3.8e-6) and the dropped lo*lo
# term is of the same size, so a product is good to ~1.1e-5 in the worst case.
TOL = {"fp64": 1e-10, "fp32": 1e-5, "tf32x3": 1e-5, "bf16x3": 2e-5}
# two runs of the same product: they differ only by the order of FP64 atomic
# additions (split-K) before the result is rounded to the block type
SAME = {"fp64": 1e-13, "fp32": 1e-6, "tf32x3": 1e-6, "bf16x3": 1e-6}
CTYPE = {"fp64": "complex128", "fp32": "complex64", "tf32x3": "complex64", "bf16x3": "complex64"}
CASES = ["tiny_cubic", "tiny_ortho", "mid", "small"]

_cache = {}


def systems(name):
    if name not in _cache:
        w = workload(name)
        o = OracleSystem(w)
        g = GpuSystem(w, o.atoms)
        _cache[name] = (w, o, g)
    return _cache[name]


def to_dev(a, prec, ld=None):
    t = torch.tensor(np.ascontiguousarray(a.astype(CTYPE[prec])), device="cuda")
    if ld is not None and ld > a.shape[1]:
        big = torch.zeros((a.shape[0], ld), dtype=t.dtype, device="cuda")
        big[:, :a.shape[1]] = t
        t = big[:, :a.shape[1]]
    return t


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy().astype(np.complex128)


def rel_max(got, ref):
    return float(np.max(np.abs(got - ref)) / np.max(np.abs(ref)))


@pytest.mark.parametrize("name", CASES + ["large"])
def test_gvectors_and_maps(name):
    w = workload(name)
    from paper_1708_03621_gb300 import jdft
    b = jdft.Basis(w.R, w.S, w.ecut, w.kfrac)
    ob = pw.Basis.build(w.R, w.S, w.kfrac[0], w.ecut)
    assert b.npw(0) == ob.npw
    assert np.array_equal(b.gvectors(0), ob.iG)
    info = b.info(0)
    assert info["N"] == ob.N
    assert np.isclose(info["omega"], ob.Omega, rtol=1e-14)
    assert info["ncols"] == len(pw.column_structure(ob.iG)[0])
    b.close()


@pytest.mark.parametrize("name", CASES)
def test_gaussian_potential_and_projectors(name):
    w, o, g = systems(name)
    V = g.V.cpu().numpy()
    assert np.max(np.abs(V - o.V)) < 1e-12
    P = g.P[0].cpu().numpy()
    assert rel_max(P, o.P.T) < 1e-13


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("name", CASES)
def test_operators_I_J_Idag_Jdag_O(name, prec):
    w, o, g = systems(name)
    from paper_1708_03621_gb300 import jdft
    nb = 3
    C = o.coeffs(nb, seed=77)
    Cd = to_dev(C, prec)
    psi = torch.empty((nb, g.N), dtype=Cd.dtype, device="cuda")
    jdft.jdft_op_I(g.basis, 0, Cd, psi, prec)
    ref_psi = pw.op_I(o.basis.iG, o.basis.S, C.T).reshape(nb, -1)
    assert band_rel_err(host(psi), ref_psi) < TOL[prec]
    jdft.jdft_op_Jdag(g.basis, 0, Cd, psi, prec)
    assert band_rel_err(host(psi), ref_psi / g.N) < TOL[prec]
    # forward operators on a random full box
    rng = np.random.default_rng(3)
    x = rng.standard_normal((nb, g.N)) + 1j * rng.standard_normal((nb, g.N))
    xd = torch.tensor(x.astype(CTYPE[prec]), device="cuda")
    out = torch.empty((nb, o.basis.npw), dtype=Cd.dtype, device="cuda")
    jdft.jdft_op_J(g.basis, 0, xd, out, prec)
    ref = pw.op_J(o.basis.iG, o.basis.S, x.reshape((nb,) + o.basis.S)).T
    assert band_rel_err(host(out), ref) < TOL[prec]
    jdft.jdft_op_Idag(g.basis, 0, xd, out, prec)
    assert band_rel_err(host(out), ref * g.N) < TOL[prec]
    jdft.jdft_op_O(g.basis, 0, Cd, out, prec)
    assert band_rel_err(host(out), o.basis.Omega * C) < TOL[prec]


@pytest.mark.parametrize("prec", ["fp64", "fp32", "tf32x3", "bf16x3"])
@pytest.mark.parametrize("name", CASES)
def test_apply_H(name, prec):
    w, o, g = systems(name)
    from paper_1708_03621_gb300 import jdft
    C = o.coeffs()
    ref = o.apply_H(C)
    Cd = to_dev(C, prec)
    HC = torch.empty_like(Cd)
    jdft.jdft_apply_H(g.basis, 0, Cd, HC, prec)
    got = host(HC)
    assert band_rel_err(got, ref) < TOL[prec]
    if prec == "fp64":
        assert rel_max(got, ref) < TOL[prec]
    jdft.jdft_device_status()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_apply_H_padded_ld_ragged_chunks(prec, monkeypatch):
    """ld > npw, an odd band count and a 1 MB chunk budget (several chunks)."""
    w, o, g = systems("mid")
    from paper_1708_03621_gb300 import jdft
    nb = 13
    C = o.coeffs(nb, seed=5)
    ref = o.apply_H(C)
    Cd = to_dev(C, prec, ld=o.basis.npw + 37)
    HC = to_dev(np.zeros_like(C), prec, ld=o.basis.npw + 5)
    monkeypatch.setenv("JDFT_CHUNK_MB", "1")
    jdft.jdft_apply_H(g.basis, 0, Cd, HC, prec)
    got = host(HC)
    assert band_rel_err(got, ref) < TOL[prec]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("name", CASES)
def test_density(name, prec):
    w, o, g = systems(name)
    from paper_1708_03621_gb300 import jdft
    C = o.coeffs()
    f = np.linspace(2.0, 0.5, C.shape[0])
    ref = pw.density(o.basis, C.T, f, weight=w.weights()[0])
    n = torch.full((g.N,), 0.25, dtype=torch.float64, device="cuda")  # accumulates onto existing values
    jdft.jdft_density(g.basis, 0, to_dev(C, prec), torch.tensor(f, device="cuda"), n, prec)
    got = n.cpu().numpy() - 0.25
    assert np.max(np.abs(got - ref)) / np.max(np.abs(ref)) < TOL[prec]


@pytest.mark.parametrize("prec", ["fp64", "fp32", "tf32x3", "bf16x3"])
@pytest.mark.parametrize("name", CASES)
def test_apply_H_density(name, prec):
    """The fused call: HC equal to jdft_apply_H's up to the order of the FP64
    atomic split-K sums of the nonlocal projections (same plane-pass
    arithmetic; the 16 x 12 planes of tiny_ortho take the fused kernel, the
    other boxes density-then-apply on one column buffer) and the density
    against the oracle's, accumulated onto existing values."""
    w, o, g = systems(name)
    from paper_1708_03621_gb300 import jdft
    C = o.coeffs()
    f = np.linspace(2.0, 0.5, C.shape[0])
    Cd = to_dev(C, prec)
    HC = torch.empty_like(Cd)
    HC1 = torch.empty_like(Cd)
    n = torch.full((g.N,), 0.25, dtype=torch.float64, device="cuda")
    jdft.jdft_apply_H_density(g.basis, 0, Cd, HC, torch.tensor(f, device="cuda"), n, prec)
    jdft.jdft_apply_H(g.basis, 0, Cd, HC1, prec)
    assert rel_max(host(HC), host(HC1)) < SAME[prec]
    assert band_rel_err(host(HC), o.apply_H(C)) < TOL[prec]
    ref = pw.density(o.basis, C.T, f, weight=w.weights()[0])
    got = n.cpu().numpy() - 0.25
    assert np.max(np.abs(got - ref)) / np.max(np.abs(ref)) < TOL[prec]
    jdft.jdft_device_status()


@pytest.mark.parametrize("prec", ["fp64", "fp32", "tf32x3", "bf16x3"])
@pytest.mark.parametrize("name", CASES)
def test_subspace(name, prec):
    w, o, g = systems(name)
    from paper_1708_03621_gb300 import jdft
    C = o.coeffs()
    HCo = o.apply_H(C)
    CHC_ref, COC_ref = pw.subspace(o.basis, C.T, HCo.T)
    nb = C.shape[0]
    CHC = torch.empty((nb, nb), dtype=torch.complex128, device="cuda")
    COC = torch.empty_like(CHC)
    jdft.jdft_subspace(g.basis, 0, to_dev(C, prec), to_dev(HCo, prec), CHC, COC, prec)
    assert rel_max(CHC.cpu().numpy(), CHC_ref) < TOL[prec]
    assert rel_max(COC.cpu().numpy(), COC_ref) < TOL[prec]
    jdft.jdft_device_status()


@pytest.mark.parametrize("prec", ["fp64", "fp32", "tf32x3", "bf16x3"])
def test_large_sampled_bands(prec):
    """128^3 box, 62 759 plane waves, 256 bands, 256 projectors: the whole block
    runs on the GPU; the oracle checks three sampled bands, the matching
    subspace columns and the density of those bands."""
    w = workload("large")
    o = OracleSystem(w)
    g = GpuSystem(w, o.atoms)
    from paper_1708_03621_gb300 import jdft
    C = o.coeffs()
    Cd = to_dev(C, prec)
    HC = torch.empty_like(Cd)
    jdft.jdft_apply_H(g.basis, 0, Cd, HC, prec)
    got = host(HC)
    sample = [0, 131, 255]
    ref = o.apply_H(C[sample])
    assert band_rel_err(got[sample], ref) < TOL[prec]
    nb = C.shape[0]
    CHC = torch.empty((nb, nb), dtype=torch.complex128, device="cuda")
    jdft.jdft_subspace(g.basis, 0, Cd, HC, CHC, None, prec)
    ref_cols = C.conj() @ ref.T            # (nb, 3): C^dag (H C_b) for sampled b
    assert rel_max(CHC.cpu().numpy()[:, sample], ref_cols) < 10 * TOL[prec]
    f = np.zeros(nb)
    f[sample] = 2.0
    n = torch.zeros(g.N, dtype=torch.float64, device="cuda")
    jdft.jdft_density(g.basis, 0, Cd, torch.tensor(f, device="cuda"), n, prec)
    nref = pw.density(o.basis, C[sample].T, f[sample])
    assert np.max(np.abs(n.cpu().numpy() - nref)) / np.max(nref) < TOL[prec]
    # the fused call in the launch configuration the benchmark times (128 x 128
    # planes: the fused kernel for the FP32 blocks; several band chunks)
    HC2 = torch.empty_like(Cd)
    n2 = torch.zeros(g.N, dtype=torch.float64, device="cuda")
    jdft.jdft_apply_H_density(g.basis, 0, Cd, HC2, torch.tensor(f, device="cuda"), n2, prec)
    assert rel_max(host(HC2), got) < SAME[prec]
    assert np.max(np.abs(n2.cpu().numpy() - nref)) / np.max(nref) < TOL[prec]
    jdft.jdft_device_status()


def test_split_operand_subspace_full_size_is_deterministic():
    """C^dag O C and C^dag B on split operands at the benchmark's shape (256
    bands, 62 759 plane waves, one wave of split-K blocks): the blocks' FP32
    partial tiles are summed in a fixed order, so two calls agree to
    the bit, and both agree with the complex128 product of the same FP32
    inputs within the BF16x3 bound."""
    from paper_1708_03621_gb300 import jdft
    w = workload("large")
    basis = jdft.Basis(w.R, w.S, w.ecut, w.kfrac, w.weights())
    npw, nb = basis.npw(0), 256
    rng = np.random.default_rng(1708)
    C = ((rng.standard_normal((nb, npw)) + 1j * rng.standard_normal((nb, npw))) / np.sqrt(npw)).astype(np.complex64)
    B = ((rng.standard_normal((nb, npw)) + 1j * rng.standard_normal((nb, npw))) / np.sqrt(npw)).astype(np.complex64)
    Cd, Bd = torch.tensor(C, device="cuda"), torch.tensor(B, device="cuda")
    out = [torch.empty((nb, nb), dtype=torch.complex128, device="cuda") for _ in range(4)]
    jdft.jdft_subspace(basis, 0, Cd, Bd, out[0], out[1], "bf16x3")
    jdft.jdft_subspace(basis, 0, Cd, Bd, out[2], out[3], "bf16x3")
    got = [host(t) for t in out]
    assert np.array_equal(got[0], got[2]) and np.array_equal(got[1], got[3])
    C64 = C.astype(np.complex128)
    ref_b = C64.conj() @ B.astype(np.complex128).T
    ref_o = abs(np.linalg.det(np.asarray(w.R, dtype=np.float64))) * (C64.conj() @ C64.T)  # O = cell volume
    assert rel_max(got[0], ref_b) < TOL["bf16x3"]
    assert rel_max(got[1], ref_o) < TOL["bf16x3"]
    jdft.jdft_device_status()


_large_ref = {}


@pytest.mark.parametrize("prec", ["bf16x3", "fp32"])
def test_large_autotuned_all_bands_occupied(prec):
    """The benchmark's launch configuration: jdft_autotune on the 256-band
    128^3 block (chunk budget: all bands in one chain launch; tuned split-K),
    then the fused jdft_apply_H_density with every band occupied (f_b from 2
    down to 0.5).  The whole density is compared with the oracle's
    n = sum_b f_b |I C_b|^2 over all 256 bands (about a minute of FP64 host
    work, in batches of 16 bands), and H C on eight sampled bands."""
    w = workload("large")
    if "o" not in _large_ref:
        _large_ref["o"] = OracleSystem(w)
    o = _large_ref["o"]
    g = GpuSystem(w, o.atoms)
    from paper_1708_03621_gb300 import jdft
    C = o.coeffs()
    nb = C.shape[0]
    f = np.linspace(2.0, 0.5, nb)
    if "n" not in _large_ref:
        n = np.zeros(g.N)
        for b0 in range(0, nb, 16):
            n += pw.density(o.basis, C[b0:b0 + 16].T, f[b0:b0 + 16])
        _large_ref["n"] = n
        sample = [0, 37, 74, 111, 148, 185, 222, 255]
        _large_ref["sample"] = sample
        _large_ref["HC"] = o.apply_H(C[sample])
    nref, sample, HCref = _large_ref["n"], _large_ref["sample"], _large_ref["HC"]
    Cd = to_dev(C, prec)
    HC = torch.empty_like(Cd)
    tune = jdft.jdft_autotune(g.basis, 0, Cd, HC, prec)
    assert tune["chunk_mb"] > 0
    # FP32 blocks on 128 x 128 planes: band pairs or single bands per plane-pass item, whichever ran faster
    assert tune["plane_bands"] in ((0,) if prec == "fp64" else (1, 2))
    n = torch.zeros(g.N, dtype=torch.float64, device="cuda")
    jdft.jdft_apply_H_density(g.basis, 0, Cd, HC, torch.tensor(f, device="cuda"), n, prec)
    got_n = n.cpu().numpy()
    assert np.max(np.abs(got_n - nref)) / np.max(np.abs(nref)) < TOL[prec]
    # the integral of n is sum_b f_b times each band's norm Omega sum |C_b|^2
    norms = o.basis.Omega * np.sum(np.abs(C) ** 2, axis=1)
    assert np.isclose(o.basis.Omega / g.N * got_n.sum(), np.sum(f * norms), rtol=TOL[prec])
    assert band_rel_err(host(HC)[sample], HCref) < TOL[prec]
    jdft.jdft_device_status()


def test_edge_cases():
    w, o, g = systems("tiny_cubic")
    from paper_1708_03621_gb300 import jdft
    L = jdft.lib()
    C = to_dev(o.coeffs(2), "fp64")
    HC = torch.empty_like(C)
    # nb = 0 is a no-op
    assert L.jdft_apply_H(g.basis.handle, 0, C.data_ptr(), C.shape[1], HC.data_ptr(), C.shape[1], 0, 0, None) == 0
    # out-of-range k-point, short leading dimension, misaligned pointer, bad precision
    assert L.jdft_apply_H(g.basis.handle, 1, C.data_ptr(), C.shape[1], HC.data_ptr(), C.shape[1], 2, 0, None) == 1
    assert L.jdft_apply_H(g.basis.handle, 0, C.data_ptr(), 3, HC.data_ptr(), C.shape[1], 2, 0, None) == 1
    assert L.jdft_apply_H(g.basis.handle, 0, C.data_ptr() + 8, C.shape[1], HC.data_ptr(), C.shape[1], 2, 0,
                          None) == 1
    assert L.jdft_apply_H(g.basis.handle, 0, C.data_ptr(), C.shape[1], HC.data_ptr(), C.shape[1], 2, 9, None) == 1
    # a box smaller than the sphere
    with pytest.raises(jdft.JdftError, match="smaller than the sphere"):
        jdft.Basis(w.R, (4, 12, 12), w.ecut, w.kfrac)
    # no potential set yet
    b2 = jdft.Basis(w.R, w.S, w.ecut, w.kfrac)
    with pytest.raises(jdft.JdftError, match="no potential"):
        jdft.jdft_apply_H(b2, 0, C, HC)
    b2.close()
    # single band, zero projectors
    g2 = GpuSystem(w, o.atoms, with_projectors=False)
    C1 = o.coeffs(1, seed=9)
    H1 = torch.empty((1, o.basis.npw), dtype=torch.complex128, device="cuda")
    jdft.jdft_apply_H(g2.basis, 0, to_dev(C1, "fp64"), H1)
    ref = pw.apply_H(o.basis, o.V, C1.T).T
    assert band_rel_err(host(H1), ref) < 1e-10


def test_free_electron_on_gpu():
    """V = 0, no projectors: H C = Omega (1/2)|k+G|^2 C exactly (closed form)."""
    w = workload("tiny_ortho")
    from paper_1708_03621_gb300 import jdft
    b = jdft.Basis(w.R, w.S, w.ecut, w.kfrac)
    V = torch.zeros(int(np.prod(w.S)), dtype=torch.float64, device="cuda")
    jdft.jdft_set_potential(b, V)
    ob = pw.Basis.build(w.R, w.S, w.kfrac[0], w.ecut)
    C = np.random.default_rng(1).standard_normal((4, ob.npw)) + 0j
    HC = torch.empty((4, ob.npw), dtype=torch.complex128, device="cuda")
    jdft.jdft_apply_H(b, 0, torch.tensor(C, device="cuda"), HC)
    assert band_rel_err(host(HC), ob.Omega * ob.T[None, :] * C) < 1e-13
    b.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("name", ["tiny_cubic", "small"])
def test_generic_plane_kernels_match_oracle(name, prec, monkeypatch):
    """The shared-memory Stockham plane kernels (used for box shapes without a
    register-FFT kernel) stay exact when the register path is switched off."""
    w, o, g = systems(name)
    from paper_1708_03621_gb300 import jdft
    monkeypatch.setenv("JDFT_FAST_PLANE", "0")
    C = o.coeffs()
    Cd = to_dev(C, prec)
    HC = torch.empty_like(Cd)
    jdft.jdft_apply_H(g.basis, 0, Cd, HC, prec)
    assert band_rel_err(host(HC), o.apply_H(C)) < TOL[prec]
    f = np.full(C.shape[0], 2.0)
    n = torch.zeros(g.N, dtype=torch.float64, device="cuda")
    jdft.jdft_density(g.basis, 0, Cd, torch.tensor(f, device="cuda"), n, prec)
    ref = pw.density(o.basis, C.T, f, weight=w.weights()[0])
    assert np.max(np.abs(n.cpu().numpy() - ref)) / np.max(ref) < TOL[prec]


@pytest.mark.parametrize("name", ["tiny_ortho", "large"])
def test_one_band_plane_kernels_match_band_pair_kernels(name, monkeypatch):
    """FP32 blocks with the band-pair plane kernels switched off run the
    one-band register-FFT kernels: same transforms, one band per lane, so the
    same H C and density up to FP32 rounding order, and both match the oracle
    (sampled bands on the 128^3 box)."""
    w, o, g = systems(name) if name != "large" else (workload("large"), None, None)
    from paper_1708_03621_gb300 import jdft
    if name == "large":
        o = _large_ref.setdefault("o", OracleSystem(w))
        g = GpuSystem(w, o.atoms)
    C = o.coeffs()
    nb = C.shape[0]
    f = torch.tensor(np.linspace(2.0, 0.5, nb), device="cuda")
    Cd = to_dev(C, "fp32")
    out = {}
    for mode in ("pair", "one"):
        if mode == "one":
            monkeypatch.setenv("JDFT_PAIR_PLANE", "0")
        HC = torch.empty_like(Cd)
        n = torch.zeros(g.N, dtype=torch.float64, device="cuda")
        jdft.jdft_apply_H_density(g.basis, 0, Cd, HC, f, n, "fp32")
        out[mode] = (host(HC), n.cpu().numpy())
    assert rel_max(out["one"][0], out["pair"][0]) < SAME["fp32"] * 10
    assert np.max(np.abs(out["one"][1] - out["pair"][1])) / np.max(np.abs(out["pair"][1])) < 1e-6
    sample = [0, nb // 2, nb - 1] if name == "large" else list(range(nb))
    ref = o.apply_H(C[sample])
    for mode in out:
        assert band_rel_err(out[mode][0][sample], ref) < TOL["fp32"]
    jdft.jdft_device_status()


@pytest.mark.parametrize("name,prec", [("mid", "fp64"), ("mid", "bf16x3"), ("large", "bf16x3"), ("large", "fp32")])
def test_hamiltonian_step_equals_separate_calls(name, prec):
    """jdft_hamiltonian_step (rows a1-a9 in one call, the overlap factored on a
    side stream while H is applied) against jdft_apply_H_density,
    jdft_subspace and jdft_orthonormalize_async on the same block, and its
    H C against the oracle on sampled bands."""
    w = workload(name)
    o = OracleSystem(w) if name != "large" else _large_ref.setdefault("o", OracleSystem(w))
    g = GpuSystem(w, o.atoms)
    from paper_1708_03621_gb300 import jdft
    C = o.coeffs(40, seed=31) if name == "mid" else o.coeffs()
    nb = C.shape[0]
    f = torch.tensor(np.linspace(2.0, 0.5, nb), device="cuda")
    # separate calls
    C1 = to_dev(C, prec)
    H1 = torch.empty_like(C1)
    n1 = torch.zeros(g.N, dtype=torch.float64, device="cuda")
    S1 = torch.empty((nb, nb), dtype=torch.complex128, device="cuda")
    O1 = torch.empty_like(S1)
    st1 = torch.zeros(1, dtype=torch.int32, device="cuda")
    jdft.jdft_apply_H_density(g.basis, 0, C1, H1, f, n1, prec)
    jdft.jdft_subspace(g.basis, 0, C1, H1, S1, O1, prec)
    jdft.jdft_orthonormalize_async(g.basis, 0, C1, st1, prec, U=O1)
    # one call
    C2 = to_dev(C, prec)
    H2 = torch.empty_like(C2)
    n2 = torch.zeros(g.N, dtype=torch.float64, device="cuda")
    S2 = torch.empty_like(S1)
    O2 = torch.empty_like(S1)
    st2 = torch.zeros(1, dtype=torch.int32, device="cuda")
    jdft.jdft_hamiltonian_step(g.basis, 0, C2, H2, f, n2, S2, O2, st2, prec)
    torch.cuda.synchronize()
    assert int(st1.item()) == 0 and int(st2.item()) == 0
    assert rel_max(host(H2), host(H1)) < SAME[prec]
    assert np.max(np.abs(n2.cpu().numpy() - n1.cpu().numpy())) < SAME[prec] * np.max(np.abs(n1.cpu().numpy()))
    S1h, S2h = S1.cpu().numpy(), S2.cpu().numpy()
    if prec == "bf16x3" and nb > 128:
        # the step forms its Hermitian C^dag H C from the upper-triangle 128 x 128
        # tiles (other split-K ranges) and mirrors the rest; jdft_subspace forms
        # every tile of C^dag (H C) for any H C.  They agree to the products'
        # accuracy (FP32 accumulation in tensor memory), and the mirror is exact.
        assert rel_max(S2h, S1h) < TOL[prec]
        assert np.array_equal(S2h[128:, :128], S2h[:128, 128:].conj().T)
    else:
        assert rel_max(S2h, S1h) < SAME[prec]
    assert rel_max(O2.cpu().numpy(), O1.cpu().numpy()) < SAME[prec]
    assert rel_max(host(C2), host(C1)) < (1e-12 if prec == "fp64" else 1e-5)
    sample = [0, nb // 2, nb - 1]
    assert band_rel_err(host(H2)[sample], o.apply_H(C[sample])) < TOL[prec]
    jdft.jdft_device_status()
