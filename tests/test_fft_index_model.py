"""The index algebra of the register line FFTs (csrc/fft_reg.cuh), as written
out in paper_1708_03621_gb300/plane_layout.py, run as a transform on the CPU:
lane t of a line holds E values, a stage (span NS, radix R) twiddles and
transforms the butterflies j = t + TL u, the stages exchange values through a
scratch line, and the last stage leaves output out_index(t, e) in v[e].  The
adjoint runs the conjugate flow graph backwards from that layout.  Both must
equal the direct DFT for every compiled length, so the index functions that the
layout count uses are those of a correct transform."""
import numpy as np
import pytest

from paper_1708_03621_gb300 import plane_layout as pl


def _dft(x, sign):
    n = len(x)
    k = np.arange(n)
    return np.exp(sign * 2j * np.pi * np.outer(k, k) / n) @ x


def _twiddle(v, N, NS, R, t, u, TL, sign):
    j = t + TL * u
    k = j % NS
    if NS > 1 and k != 0:
        b = k * (N // (NS * R))
        for r in range(1, R):
            v[u * R + r] *= np.exp(sign * 2j * np.pi * r * b / N)


def _small_dft(v, u, R, sign):
    v[u * R:(u + 1) * R] = _dft(v[u * R:(u + 1) * R], sign)


def run(L, x, sign):
    """LineFFT::run: v[t][e] starts as x[in_index(t, e)]; returns v."""
    v = np.array([[x[L.in_index(t, e)] for e in range(L.E)] for t in range(L.TL)], complex)
    for i, (NS, R) in enumerate(L.stages):
        for t in range(L.TL):
            for u in range(L.E // R):
                _twiddle(v[t], L.N, NS, R, t, u, L.TL, sign)
                _small_dft(v[t], u, R, sign)
        if i + 1 < len(L.stages):
            scr = np.zeros(L.N, complex)
            for t in range(L.TL):
                for u in range(L.E // R):
                    for r in range(R):
                        scr[L.stage_out(t, u, r, NS, R)] = v[t][u * R + r]
            R2 = L.stages[i + 1][1]
            for t in range(L.TL):
                for u in range(L.E // R2):
                    for r in range(R2):
                        v[t][u * R2 + r] = scr[t + L.TL * u + r * (L.N // R2)]
    return v


def run_adjoint(L, v, sign2):
    """LineFFT::run_adjoint (transform of sign sign2 from the layout run() leaves)."""
    v = v.copy()
    for i in range(len(L.stages) - 1, -1, -1):
        NS, R = L.stages[i]
        if i + 1 < len(L.stages):
            Rn = L.stages[i + 1][1]
            scr = np.zeros(L.N, complex)
            for t in range(L.TL):
                for u in range(L.E // Rn):
                    for r in range(Rn):
                        scr[t + L.TL * u + r * (L.N // Rn)] = v[t][u * Rn + r]
            for t in range(L.TL):
                for u in range(L.E // R):
                    for r in range(R):
                        v[t][u * R + r] = scr[L.stage_out(t, u, r, NS, R)]
        for t in range(L.TL):
            for u in range(L.E // R):
                _small_dft(v[t], u, R, sign2)
                _twiddle(v[t], L.N, NS, R, t, u, L.TL, sign2)
    return v


@pytest.mark.parametrize("n", sorted(pl.CFG))
@pytest.mark.parametrize("sign", [+1, -1])
def test_line_fft_index_algebra(n, sign):
    L = pl.Line(n)
    rng = np.random.default_rng(n)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    v = run(L, x, sign)
    y = np.zeros(n, complex)
    seen = np.zeros(n, int)
    for t in range(L.TL):
        for e in range(L.E):
            y[L.out_index(t, e)] = v[t][e]
            seen[L.out_index(t, e)] += 1
    assert np.all(seen == 1)  # every output position exactly once
    assert np.allclose(y, _dft(x, sign), atol=1e-10 * n)
    # the adjoint flow graph from the output layout: the transform of the other sign
    w = np.array([[y[L.out_index(t, e)] for e in range(L.E)] for t in range(L.TL)], complex)
    back = run_adjoint(L, w, -sign)
    z = np.zeros(n, complex)
    for t in range(L.TL):
        for e in range(L.E):
            z[L.in_index(t, e)] = back[t][e]
    assert np.allclose(z, n * x, atol=1e-9 * n)
