"""The bench's algorithmic work model (the numerators of `roofline.achieved`)
against the closed forms per unit: 5 n log2 n flops per complex length-n
transform, 8 M N K flops per complex product, and minimum DRAM bytes (inputs
read once, outputs written once).  Host logic only (CPU)."""
import importlib.util
import math
import os
import types

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


class _Elem:
    def __init__(self, size):
        self.size = size

    def element_size(self):
        return self.size


def _problem(nb=256, nproj=256, e=8):
    # the 128^3 workload: 62 759 plane waves, 1 908 (i0, i1) columns, 49 i0 rows
    return types.SimpleNamespace(w=types.SimpleNamespace(S=(128, 128, 128)), info={"ncols": 1908}, nrows=49,
                                 C=_Elem(e), N=128 ** 3, npw=62759, nproj=nproj, nb=nb)


def test_plane_pass_per_band(bench):
    p = _problem()
    fl, by = bench.kernel_work(p, "plane_apply_density_fast", 1, 1)
    # rows (49 lines) and columns (128 lines) of 128 points, each inverse and forward, on 128 planes
    per_plane = 2 * 49 * 5 * 128 * 7 + 2 * 128 * 5 * 128 * 7
    assert fl == pytest.approx(128 * per_plane)
    assert fl == pytest.approx(203.0e6, rel=1e-3)
    # column buffer read and written once (8-byte FP32 complex), V once (FP32), n(r) read + written (FP64)
    assert by == pytest.approx(2 * 128 * 1908 * 8 + 128 ** 3 * 4 + 128 ** 3 * 16)


def test_plane_pass_scales_with_bands_per_launch(bench):
    p = _problem()
    fl1, _ = bench.kernel_work(p, "plane_apply_density_fast", 1, 1)
    fl256, _ = bench.kernel_work(p, "plane_apply_density_fast", 1, 256)
    assert fl256 == pytest.approx(256 * fl1)


def test_z_passes(bench):
    p = _problem()
    fi, bi = bench.kernel_work(p, "zpass_inverse", 1, 1)
    ff, bf = bench.kernel_work(p, "zpass_forward", 1, 1)
    assert fi == ff == pytest.approx(5 * 1908 * 128 * math.log2(128))
    assert bi == pytest.approx((62759 + 128 * 1908) * 8)           # sphere in, column buffer out
    assert bf == pytest.approx((2 * 62759 + 128 * 1908) * 8)       # column buffer and C in, HC out


def test_tensor_products(bench):
    p = _problem(nb=256, nproj=256)
    fl, by = bench.kernel_work(p, "tc_zgemm_cn", 3, 256)
    assert fl == pytest.approx(8.0 * 256 * 256 * 62759)
    assert by == pytest.approx(2 * 256 * 62759 * 8)
    fl, _ = bench.kernel_work(p, "tc_zgemm_nn", 2, 256)
    assert fl == pytest.approx(8.0 * 62759 * 256 * 256)
    # unequal projector and band counts: P^dag C, C^dag HC and C^dag C averaged per launch
    q = _problem(nb=64, nproj=256)
    fl, _ = bench.kernel_work(q, "tc_zgemm_cn", 3, 64)
    assert fl == pytest.approx(8.0 * 62759 * (256 * 64 + 64 * 64 + 64 * 64) / 3)


def test_band_pair_kernels_use_the_same_work(bench):
    """The band-pair plane kernels do the transforms of the one-band ones."""
    p = _problem()
    assert bench.kernel_work(p, "plane_apply_density_pair", 1, 2) == bench.kernel_work(p, "plane_apply_density_fast",
                                                                                        1, 2)
    assert bench.kernel_work(p, "plane_apply_pair", 1, 2) == bench.kernel_work(p, "plane_apply_fast", 1, 2)


def test_traffic_figure_is_dropped_when_the_kernel_changes(bench, monkeypatch):
    name = "plane_apply_density_pair"
    sha = bench.sources_sha(name)
    monkeypatch.setitem(bench.TRAFFIC_PER_BAND, name, (3.7e6, sha))
    assert bench.traffic_per_band(name) == 3.7e6
    monkeypatch.setitem(bench.TRAFFIC_PER_BAND, name, (3.7e6, "0" * 16))
    assert bench.traffic_per_band(name) is None


def test_split_operand_products_and_split_pass(bench):
    p = _problem(nb=256, nproj=256)
    assert bench.kernel_work(p, "tcx_cn", 3, 256) == bench.kernel_work(p, "tc_zgemm_cn", 3, 256)
    # five splits per step: C, H C, C's transpose (256 x 62 759 values each), two 256 x 256
    fl, by = bench.kernel_work(p, "split_planes", 5, 256)
    assert fl == 0.0 and by == pytest.approx(16.0 * (3 * 256 * 62759 + 2 * 256 * 256) / 5)


def test_split_operand_nn_and_reduction(bench):
    p = _problem(nb=256, nproj=256)
    assert bench.kernel_work(p, "tcx_nn", 2, 256) == bench.kernel_work(p, "tc_zgemm_nn", 2, 256)
    # 76 splits x 2 tiles of 128 x 256 FP32 complex partials, the 256 x 256 FP64 output read and written
    p.tune = {"splits_subspace": 76}
    fl, by = bench.kernel_work(p, "tcx_reduce", 3, 256)
    assert fl == 0.0 and by == pytest.approx(76 * 2 * 128 * 256 * 8 + 2 * 256 * 256 * 16)
