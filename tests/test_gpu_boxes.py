"""GPU parity against the FP64 oracle on every box shape the benchmark runs.

The 48^3 and 128^3 boxes are covered in test_gpu_chain.py.  Here:

* cubic cells whose boxes are 54^3, 60^3, 64^3, 72^3 and 80^3 (E_cut 20 Ha,
  L chosen so that the smallest admissible box is that size): the generic
  Stockham plane kernels with radix 3 (54, 60, 72) and 5 (60, 80), and the
  compiled 64- and 80-point register-FFT kernels;
* the eight independent cells of the benchmark's mixed-cell batch (seed 29:
  boxes 40, 40, 60, 40, 64, 72, 48, 72), each with its own atoms and band
  count.

Per cell, three sampled bands of the block are compared element by element
(per-band relative error) for jdft_apply_H, jdft_apply_H_density (H C and the
density of the sampled bands) and jdft_density, in FP64 (1e-10) and in the
mixed precisions (the tolerances of test_gpu_chain.py).  The I, J, multiply
chain follows the JDFTx paper, Sec. 2.1 (Listing 1's I, pointwise product, J
on temporaries); the nonlocal term is the projector form of Sec. 2.2.
"""
import numpy as np
import pytest

from oracle import planewave as pw
from synth import Workload, random_cells
from tests.systems import GpuSystem, OracleSystem, band_rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "fp32": 1e-5, "tf32x3": 1e-5, "bf16x3": 2e-5}
CTYPE = {"fp64": "complex128", "fp32": "complex64", "tf32x3": "complex64", "bf16x3": "complex64"}

# cubic cells at E_cut = 20 Ha whose smallest admissible box (synth.box_for) is the given edge
BOX_CELLS = {
    54: Workload("box54", (12.5, 12.5, 12.5), 20.0, (54, 54, 54), ((0.1, 0.2, 0.3),), 10, 12, 541, 542),
    60: Workload("box60", (14.0, 14.0, 14.0), 20.0, (60, 60, 60), ((-0.3, 0.05, 0.45),), 12, 12, 601, 602),
    64: Workload("box64", (15.2, 15.2, 15.2), 20.0, (64, 64, 64), ((0.1, 0.2, 0.3),), 16, 12, 641, 642),
    72: Workload("box72", (16.5, 16.5, 16.5), 20.0, (72, 72, 72), ((0.25, -0.4, 0.1),), 12, 12, 721, 722),
    80: Workload("box80", (18.5, 18.5, 18.5), 20.0, (80, 80, 80), ((0.1, 0.2, 0.3),), 20, 12, 801, 802),
}
BATCH_CELLS = random_cells(8, 29)

_cache = {}


def _systems(w):
    if w.name not in _cache:
        _cache.clear()  # one cell's device buffers at a time
        o = OracleSystem(w)
        g = GpuSystem(w, o.atoms)
        _cache[w.name] = (o, g)
    return _cache[w.name]


def _dev(a, prec):
    return torch.tensor(np.ascontiguousarray(a.astype(CTYPE[prec])), device="cuda")


def _host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy().astype(np.complex128)


def _check_cell(w, prec):
    from paper_1708_03621_gb300 import jdft
    o, g = _systems(w)
    C = o.coeffs()
    nb = C.shape[0]
    sample = sorted({0, nb // 2, nb - 1})
    ref_HC = o.apply_H(C[sample])
    f = np.zeros(nb)
    f[sample] = [2.0, 1.5, 0.5][:len(sample)]
    ref_n = pw.density(o.basis, C[sample].T, f[sample], weight=w.weights()[0])
    Cd = _dev(C, prec)
    # jdft_apply_H over the whole block
    HC = torch.empty_like(Cd)
    jdft.jdft_apply_H(g.basis, 0, Cd, HC, prec)
    got = _host(HC)[sample]
    assert band_rel_err(got, ref_HC) < TOL[prec], "apply_H"
    # the fused call: H C and the density of the block (only the sampled bands occupied)
    HC2 = torch.empty_like(Cd)
    n2 = torch.full((g.N,), 0.125, dtype=torch.float64, device="cuda")
    jdft.jdft_apply_H_density(g.basis, 0, Cd, HC2, torch.tensor(f, device="cuda"), n2, prec)
    assert band_rel_err(_host(HC2)[sample], ref_HC) < TOL[prec], "apply_H_density: H C"
    got_n = n2.cpu().numpy() - 0.125
    assert np.max(np.abs(got_n - ref_n)) / np.max(np.abs(ref_n)) < TOL[prec], "apply_H_density: n(r)"
    # the density call alone
    n1 = torch.zeros(g.N, dtype=torch.float64, device="cuda")
    jdft.jdft_density(g.basis, 0, Cd, torch.tensor(f, device="cuda"), n1, prec)
    assert np.max(np.abs(n1.cpu().numpy() - ref_n)) / np.max(np.abs(ref_n)) < TOL[prec], "density"
    jdft.jdft_device_status()


@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16x3"])
@pytest.mark.parametrize("edge", sorted(BOX_CELLS))
def test_box_shapes_match_oracle(edge, prec):
    w = BOX_CELLS[edge]
    from synth import box_for
    assert box_for(w.L[0], w.ecut) == edge   # the cell really is the one that needs this box
    _check_cell(w, prec)


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
@pytest.mark.parametrize("idx", range(len(BATCH_CELLS)))
def test_benchmark_batch_cells_match_oracle(idx, prec):
    """The eight cells of the benchmark's mixed-cell batch, one by one."""
    _check_cell(BATCH_CELLS[idx], prec)


def test_benchmark_batch_boxes_are_covered():
    """Every box edge of the benchmark's mixed-cell batch has a cell above."""
    edges = {w.S[0] for w in BATCH_CELLS}
    assert edges <= set(BOX_CELLS) | {40, 48}
