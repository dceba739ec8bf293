// Batched 1-D FFTs over lines held in shared memory, for the I and J
// operators of the algebraic formulation (JDFTx paper, Sec. 2.1: Fourier
// transforms between reciprocal and real space "using Fast Fourier
// Transforms").
//
// Algorithm: Stockham autosort, mixed radix (2, 3, 4, 5, 8).  Pass t with
// radix R and span Ns (product of the earlier radices) reads R inputs spaced
// n/R apart, multiplies input r by W^{r (j mod Ns) n / (Ns R)}, takes the
// R-point DFT in registers and writes the outputs Ns apart from
// (j / Ns) Ns R + (j mod Ns).  Passes ping-pong between two buffers, so the
// output of an odd number of passes lands in the second buffer.  The sum is
// the unnormalised y_m = sum_t x_t exp(SIGN 2 pi i t m / n).
#pragma once

#include "common.cuh"

namespace jdft {

// R-point DFT in registers: out[m] = sum_r v[r] exp(SIGN 2 pi i r m / R).
template <typename T, int SIGN>
__device__ __forceinline__ void dft2(c_t<T>* v) {
    c_t<T> a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
}

template <typename T, int SIGN>
__device__ __forceinline__ void dft4(c_t<T>* v) {
    c_t<T> y0 = cadd(v[0], v[2]), y1 = csub(v[0], v[2]);
    c_t<T> y2 = cadd(v[1], v[3]), y3 = cmul_i<SIGN>(csub(v[1], v[3]));
    v[0] = cadd(y0, y2);
    v[2] = csub(y0, y2);
    v[1] = cadd(y1, y3);
    v[3] = csub(y1, y3);
}

template <typename T, int SIGN>
__device__ __forceinline__ void dft3(c_t<T>* v) {
    const T h = T(0.86602540378443864676372317075294);  // sqrt(3)/2
    c_t<T> t1 = cadd(v[1], v[2]);
    c_t<T> t2 = cscale(cmul_i<SIGN>(csub(v[1], v[2])), h);
    c_t<T> m = csub(v[0], cscale(t1, T(0.5)));
    v[0] = cadd(v[0], t1);
    v[1] = cadd(m, t2);
    v[2] = csub(m, t2);
}

template <typename T, int SIGN>
__device__ __forceinline__ void dft5(c_t<T>* v) {
    const T c1 = T(0.30901699437494742410229341718282);   // cos(2 pi / 5)
    const T c2 = T(-0.80901699437494742410229341718282);  // cos(4 pi / 5)
    const T s1 = T(0.95105651629515357211643933337938);   // sin(2 pi / 5)
    const T s2 = T(0.58778525229247312916870595463907);   // sin(4 pi / 5)
    c_t<T> a1 = cadd(v[1], v[4]), b1 = csub(v[1], v[4]);
    c_t<T> a2 = cadd(v[2], v[3]), b2 = csub(v[2], v[3]);
    c_t<T> x0 = v[0];
    c_t<T> p1 = mk<T>(x0.x + c1 * a1.x + c2 * a2.x, x0.y + c1 * a1.y + c2 * a2.y);
    c_t<T> p2 = mk<T>(x0.x + c2 * a1.x + c1 * a2.x, x0.y + c2 * a1.y + c1 * a2.y);
    c_t<T> q1 = cmul_i<SIGN>(mk<T>(s1 * b1.x + s2 * b2.x, s1 * b1.y + s2 * b2.y));
    c_t<T> q2 = cmul_i<SIGN>(mk<T>(s2 * b1.x - s1 * b2.x, s2 * b1.y - s1 * b2.y));
    v[0] = cadd(x0, cadd(a1, a2));
    v[1] = cadd(p1, q1);
    v[4] = csub(p1, q1);
    v[2] = cadd(p2, q2);
    v[3] = csub(p2, q2);
}

template <typename T, int SIGN>
__device__ __forceinline__ void dft8(c_t<T>* v) {
    // Split into even and odd samples, 4-point DFTs, then combine with W8^m.
    c_t<T> e[4] = {v[0], v[2], v[4], v[6]};
    c_t<T> o[4] = {v[1], v[3], v[5], v[7]};
    dft4<T, SIGN>(e);
    dft4<T, SIGN>(o);
    const T r = T(0.70710678118654752440084436210485);  // 1/sqrt(2)
    // W8^1 = (1 + SIGN i)/sqrt2, W8^2 = SIGN i, W8^3 = (-1 + SIGN i)/sqrt2
    c_t<T> w1 = mk<T>(r * (o[1].x - SIGN * o[1].y), r * (o[1].y + SIGN * o[1].x));
    c_t<T> w2 = cmul_i<SIGN>(o[2]);
    c_t<T> w3 = mk<T>(r * (-o[3].x - SIGN * o[3].y), r * (-o[3].y + SIGN * o[3].x));
    v[0] = cadd(e[0], o[0]);
    v[4] = csub(e[0], o[0]);
    v[1] = cadd(e[1], w1);
    v[5] = csub(e[1], w1);
    v[2] = cadd(e[2], w2);
    v[6] = csub(e[2], w2);
    v[3] = cadd(e[3], w3);
    v[7] = csub(e[3], w3);
}

template <typename T, int SIGN, int R>
__device__ __forceinline__ void stockham_pass(const c_t<T>* __restrict__ src, c_t<T>* __restrict__ dst,
                                              int nlines, int ls, int n, int Ns,
                                              const c_t<T>* __restrict__ tw) {
    const int nb = n / R;             // butterflies per line
    const int twstep = n / (Ns * R);  // table stride of this pass's root
    const int total = nlines * nb;
    for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
        const int l = idx / nb;
        const int j = idx - l * nb;
        const int k = j % Ns;
        const c_t<T>* s = src + l * ls + j;
        c_t<T> v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = s[r * nb];
        if (k != 0) {
#pragma unroll
            for (int r = 1; r < R; ++r) {
                c_t<T> w = tw[r * k * twstep];
                v[r] = (SIGN > 0) ? cmul(v[r], w) : cmulc(v[r], w);
            }
        }
        if (R == 2) dft2<T, SIGN>(v);
        if (R == 3) dft3<T, SIGN>(v);
        if (R == 4) dft4<T, SIGN>(v);
        if (R == 5) dft5<T, SIGN>(v);
        if (R == 8) dft8<T, SIGN>(v);
        c_t<T>* d = dst + l * ls + (j - k) * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) d[r * Ns] = v[r];
    }
}

// Transform `nlines` lines of length plan.n, line l at a[l * ls].  The caller
// must have synchronised after writing `a`.  Returns the buffer (a or b) that
// holds the result; the block is synchronised on return.  tw points at this
// length's table W[e] = exp(+2 pi i e / n).
template <typename T, int SIGN>
__device__ c_t<T>* fft_lines(c_t<T>* a, c_t<T>* b, int nlines, int ls, const FftPlan& plan,
                             const c_t<T>* __restrict__ tw) {
    int Ns = 1;
    const int n = plan.n;
    for (int p = 0; p < plan.npass; ++p) {
        const int R = plan.radix[p];
        switch (R) {
            case 2: stockham_pass<T, SIGN, 2>(a, b, nlines, ls, n, Ns, tw); break;
            case 3: stockham_pass<T, SIGN, 3>(a, b, nlines, ls, n, Ns, tw); break;
            case 4: stockham_pass<T, SIGN, 4>(a, b, nlines, ls, n, Ns, tw); break;
            case 5: stockham_pass<T, SIGN, 5>(a, b, nlines, ls, n, Ns, tw); break;
            default: stockham_pass<T, SIGN, 8>(a, b, nlines, ls, n, Ns, tw); break;
        }
        __syncthreads();
        c_t<T>* t = a; a = b; b = t;
        Ns *= R;
    }
    return a;
}

}  // namespace jdft
