"""Derives the shared-memory layout constants of the register-FFT kernels in
csrc/plane_fast.cu (the scratch-line spacing per line length and the plane
array stride per plane shape) by counting the bank conflicts of every shared
access those kernels make.

Rule used for the count: a warp's 8-byte shared access is served in two
halves of 16 lanes, a 16-byte access in four quarters of 8 lanes; within one
group, the number of wavefronts is the largest number of distinct addresses
that fall in the same bank slot (128 bytes hold 16 eight-byte or 8
sixteen-byte slots).  Under this rule the old layout (lanes of one line
adjacent, plane stride 132) has 8.25 M conflicts on one 34-band launch of
the 128^3 fused kernel, the number ncu reports for it; the layout printed
here has none.

Lanes: a line of N values is split over TL = N / E lanes and a warp serves
LPW = 32 / TL lines; lane l takes position t = l / LPW of line l % LPW.

    python -m paper_1708_03621_gb300.plane_layout

prints the C++ specialisations used in plane_fast.cu.  Nothing imports this
module; it is the record of how the constants were chosen.
"""
from __future__ import annotations

from collections import defaultdict

# (E values per lane, radix list) per compiled line length: FastCfg in plane_fast.cu
CFG = {12: (12, (4, 3)), 16: (16, (16,)), 40: (20, (2, 4, 5)), 48: (12, (4, 4, 3)), 64: (8, (8, 8)),
       80: (20, (4, 4, 5)), 128: (16, (16, 8)), 256: (16, (16, 16))}
# compiled plane shapes (S0, S1) with a typical sphere: rows touched and the first row's i0
SHAPES = {(12, 12): (5, -2), (16, 12): (7, -3), (40, 40): (17, -8), (48, 48): (21, -10), (64, 64): (25, -12),
          (80, 80): (31, -15), (128, 128): (49, -24), (256, 128): (49, -24)}
NWARPS = 8


def padx(i: int) -> int:
    return i + (i >> 4)


def padded_line(n: int) -> int:
    return n + (n >> 4)


class Line:
    """Index functions of LineFFT<N, E, Rad<...>> (fft_reg.cuh)."""

    def __init__(self, n: int):
        self.N = n
        self.E, self.R = CFG[n]
        self.TL = n // self.E
        self.LPW = 32 // self.TL
        self.stages = []
        ns = 1
        for r in self.R:
            self.stages.append((ns, r))
            ns *= r

    def lanes(self):
        return [(l % self.LPW, l // self.LPW) for l in range(32)]  # (line, position)

    def in_index(self, t, e):
        r0 = self.R[0]
        return t + self.TL * (e // r0) + (e % r0) * (self.N // r0)

    def stage_out(self, t, u, r, ns, rad):
        j = t + self.TL * u
        k = j % ns
        return (j - k) * rad + k + r * ns

    def out_index(self, t, e):
        ns, rad = self.stages[-1]
        return self.stage_out(t, e // rad, e % rad, ns, rad)

    def exchanges(self, sp):
        """Scratch accesses of one transform (the adjoint makes the same ones)."""
        out = []
        for i in range(len(self.stages) - 1):
            ns, rad = self.stages[i]
            r2 = self.stages[i + 1][1]
            for u in range(self.E // rad):
                for r in range(rad):
                    out.append([q * sp + padx(self.stage_out(t, u, r, ns, rad)) for q, t in self.lanes()])
            for u in range(self.E // r2):
                for r in range(r2):
                    out.append([q * sp + padx(t + self.TL * u + r * (self.N // r2)) for q, t in self.lanes()])
        return out


def wavefronts(addrs, es: int):
    """(wavefronts, ideal) of one warp access; addrs in elements of es bytes, None = inactive lane."""
    g = 128 // es
    tot = ideal = 0
    for h in range(0, 32, g):
        a = {addrs[l] for l in range(h, h + g) if addrs[l] is not None}
        if not a:
            continue
        slots = defaultdict(set)
        for x in a:
            slots[x % g].add(x)
        tot += max(len(v) for v in slots.values())
        ideal += 1
    return tot, ideal


def conflicts(accesses, es):
    t = i = 0
    for a in accesses:
        x, y = wavefronts(a, es)
        t += x
        i += y
    return t - i


def spacing(n: int, es: int) -> int:
    """Smallest scratch-line spacing >= padded_line(n) with the fewest exchange conflicts."""
    L = Line(n)
    cands = [padded_line(n) + d for d in range(128 // es)]
    return min(cands, key=lambda sp: (conflicts(L.exchanges(sp), es), sp))


def plane_accesses(n0, n1, nrows, i0min, ls):
    """Plane-array accesses of one (plane, band) item of the H plane pass (rows, columns, rows)."""
    L0, L1 = Line(n0), Line(n1)
    out = []
    for w in range(NWARPS):
        for base in range(w * L1.LPW, nrows, NWARPS * L1.LPW):
            for fn in (L1.out_index, L1.in_index):  # row inverse stores, row forward loads
                for e in range(L1.E):
                    out.append([(base + q) * ls + fn(t, e) if base + q < nrows else None for q, t in L1.lanes()])
        for base in range(w * L0.LPW, n1, NWARPS * L0.LPW):
            for _ in range(2):  # column loads and stores
                for e in range(L0.E):
                    acc = []
                    for q, t in L0.lanes():
                        r = (L0.in_index(t, e) - i0min) % n0
                        acc.append(r * ls + base + q if r < nrows and base + q < n1 else None)
                    out.append(acc)
    return out


def stride(n0: int, n1: int, es: int) -> int:
    nrows, i0min = SHAPES[(n0, n1)]
    cands = [n1 + p for p in range(1, 128 // es + 1)]
    return min(cands, key=lambda ls: (conflicts(plane_accesses(n0, n1, nrows, i0min, ls), es), ls))


def main():
    for t, es in (("float", 8), ("double", 16)):
        for n in CFG:
            print(f"JDFT_SCRATCH_SPACING({t}, {n}, {spacing(n, es)})")
    for t, es in (("float", 8), ("double", 16)):
        for n0, n1 in SHAPES:
            print(f"JDFT_PLANE_STRIDE({t}, {n0}, {n1}, {stride(n0, n1, es)})")


if __name__ == "__main__":
    main()
