"""The shared-memory layout constants of the register-FFT kernels
(csrc/plane_fast.cu) against the conflict count that chooses them
(paper_1708_03621_gb300/plane_layout.py): the table compiled into the kernels
must be the one the count prints, and the bench's 128 x 128 FP32 plane pass
must come out free of bank conflicts."""
import os
import re

from paper_1708_03621_gb300 import plane_layout as pl

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_1708_03621_gb300", "csrc",
                   "plane_fast.cu")


def _table(macro):
    text = open(SRC).read()
    return sorted(re.findall(rf"^{macro}\(([^)]*)\)$", text, flags=re.M))


def test_compiled_table_matches_the_conflict_count(capsys):
    pl.main()
    printed = capsys.readouterr().out.splitlines()
    for macro in ("JDFT_SCRATCH_SPACING", "JDFT_PLANE_STRIDE"):
        want = sorted(line[len(macro) + 1:-1] for line in printed if line.startswith(macro + "("))
        assert want and _table(macro) == want


def test_bench_plane_pass_is_conflict_free():
    n, es = 128, 8
    sp = pl.spacing(n, es)
    assert pl.conflicts(pl.Line(n).exchanges(sp), es) == 0
    nrows, i0min = pl.SHAPES[(n, n)]
    assert pl.conflicts(pl.plane_accesses(n, n, nrows, i0min, pl.stride(n, n, es)), es) == 0


def test_wavefront_rule():
    # 8-byte accesses: 16 lanes per group; two distinct addresses in one slot cost two wavefronts
    assert pl.wavefronts(list(range(32)), 8) == (2, 2)
    assert pl.wavefronts([16 * l for l in range(32)], 8) == (32, 2)
    assert pl.wavefronts([0] * 32, 8) == (2, 2)  # broadcast
    # 16-byte accesses: 8 lanes per group
    assert pl.wavefronts(list(range(32)), 16) == (4, 4)
    assert pl.wavefronts([None] * 32, 8) == (0, 0)
