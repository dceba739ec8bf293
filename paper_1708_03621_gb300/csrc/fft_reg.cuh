// Register-resident line FFTs of compile-time length N, for the plane pass.
//
// A line of N complex values is split over TL consecutive lanes of one warp;
// each lane holds E = N / TL values in registers.  The transform is a
// Stockham autosort FFT with a compile-time radix list Rad<R0, R1, ...>:
// stage s (span NS = R0 ... R_{s-1}, radix R) has N/R butterflies; lane t
// owns butterflies j = t + TL u (u < E/R), reads inputs j + r N/R, multiplies
// input r by W_N^{SIGN r k N/(NS R)} (k = j mod NS), takes the R-point DFT in
// registers and produces outputs (j - k) R + k + r NS.  Between stages the
// values move through a warp-private scratch line with __syncwarp; no block
// barrier is involved.  Unnormalised: y_m = sum_t x_t exp(SIGN 2 pi i t m / N).
#pragma once

#include "fft.cuh"

namespace jdft {

template <int... R>
struct Rad {};

// Scratch lines are padded with one element after every 16 (and lines are
// N + N/16 apart): the stage exchanges write index 16 t + r from lane t, which
// without the pad would put every lane of a warp on the same bank.
__host__ __device__ constexpr int padx(int idx) { return idx + (idx >> 4); }
__host__ __device__ constexpr int padded_line(int N) { return N + (N >> 4); }

template <typename T, int SIGN>
__device__ __forceinline__ void dft16(c_t<T>* v) {
    // 16 = 4 x 4: DFT4 over n2 (stride 4), twiddle W16^{n1 k1}, DFT4 over n1.
    const T c1 = T(0.92387953251128675612818318939679);  // cos(pi/8)
    const T s1 = T(0.38268343236508977172845998403040);  // sin(pi/8)
    const T h = T(0.70710678118654752440084436210485);   // cos(pi/4)
    c_t<T> a[4][4];
#pragma unroll
    for (int n1 = 0; n1 < 4; ++n1) {
        c_t<T> w[4] = {v[n1], v[n1 + 4], v[n1 + 8], v[n1 + 12]};
        dft4<T, SIGN>(w);
#pragma unroll
        for (int k1 = 0; k1 < 4; ++k1) a[n1][k1] = w[k1];
    }
    // twiddles W16^{n1 k1} = exp(SIGN 2 pi i n1 k1 / 16); table of cos/sin for e = n1 k1 in 0..9
    auto tw = [&](c_t<T> x, int e) -> c_t<T> {
        T c, s;
        switch (e) {
            case 0: return x;
            case 1: c = c1; s = s1; break;
            case 2: c = h; s = h; break;
            case 3: c = s1; s = c1; break;
            case 4: c = T(0); s = T(1); break;
            case 6: c = -h; s = h; break;
            default: c = -c1; s = -s1; break;  // e = 9: cos(9 pi/8), sin(9 pi/8)
        }
        s = SIGN > 0 ? s : -s;
        return mk<T>(x.x * c - x.y * s, x.x * s + x.y * c);
    };
#pragma unroll
    for (int n1 = 1; n1 < 4; ++n1)
#pragma unroll
        for (int k1 = 1; k1 < 4; ++k1) a[n1][k1] = tw(a[n1][k1], n1 * k1);
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) {
        c_t<T> w[4] = {a[0][k1], a[1][k1], a[2][k1], a[3][k1]};
        dft4<T, SIGN>(w);
#pragma unroll
        for (int k2 = 0; k2 < 4; ++k2) v[k1 + 4 * k2] = w[k2];
    }
}

template <typename T, int SIGN, int R>
__device__ __forceinline__ void dft_r(c_t<T>* v) {
    if constexpr (R == 2) dft2<T, SIGN>(v);
    else if constexpr (R == 3) dft3<T, SIGN>(v);
    else if constexpr (R == 4) dft4<T, SIGN>(v);
    else if constexpr (R == 5) dft5<T, SIGN>(v);
    else if constexpr (R == 8) dft8<T, SIGN>(v);
    else if constexpr (R == 16) dft16<T, SIGN>(v);
}

template <int... R>
struct RadInfo;
template <>
struct RadInfo<> {
    static constexpr int prod = 1;
    static constexpr int lcm = 1;
};
constexpr int gcd_c(int a, int b) { return b == 0 ? a : gcd_c(b, a % b); }
template <int R, int... Rest>
struct RadInfo<R, Rest...> {
    static constexpr int prod = R * RadInfo<Rest...>::prod;
    static constexpr int lcm = R / gcd_c(R, RadInfo<Rest...>::lcm) * RadInfo<Rest...>::lcm;
};

// Line geometry for length N with radices R...: E values per lane, TL lanes per line.
template <int N, int E>
struct LineShape {
    static constexpr int TL = N / E;
    static constexpr int LPW = 32 / TL;  // lines per warp
    static_assert(N % E == 0 && 32 % (N / E) == 0, "lanes per line must divide the warp");
};

// Twiddles w[r] = W[r b], r = 1 .. R-1 (r b < N): the table is read at the
// powers of two r = 1, 2, 4, 8 and the other w[r] are products
// w[r] = w[r - lowbit(r)] w[lowbit(r)] (at most three roundings), which moves
// work from the shared-memory pipe to the FMA pipe.
template <typename T, int R>
__device__ __forceinline__ void stage_twiddles(c_t<T>* w, int b, const c_t<T>* __restrict__ W) {
#pragma unroll
    for (int r = 1; r < R; ++r) {
        const int low = r & (-r);
        if (low == r) w[r] = W[r * b];
        else w[r] = cmul(w[r - low], w[low]);
    }
}

// One stage: v holds the inputs of this lane's butterflies, v[u*R + r].
template <typename T, int N, int TL, int E, int SIGN, int NS, int R>
__device__ __forceinline__ void stage_compute(c_t<T>* v, int t, const c_t<T>* __restrict__ W) {
    constexpr int NB = E / R;
#pragma unroll
    for (int u = 0; u < NB; ++u) {
        const int j = t + TL * u;
        const int k = j % NS;
        if (NS > 1 && k != 0) {
            c_t<T> w[R];
            stage_twiddles<T, R>(w, k * (N / (NS * R)), W);
#pragma unroll
            for (int r = 1; r < R; ++r) v[u * R + r] = SIGN > 0 ? cmul(v[u * R + r], w[r]) : cmulc(v[u * R + r], w[r]);
        }
        dft_r<T, SIGN, R>(v + u * R);
    }
}

// Adjoint of the stage (NS, R) of the transform with sign -SIGN2: the R-point
// DFT with sign SIGN2 on this lane's butterfly outputs v[u*R + r], then the
// conjugate twiddles.  On return v[u*R + r] holds the stage's input position
// j + r N/R (j = t + TL u).
template <typename T, int N, int TL, int E, int SIGN2, int NS, int R>
__device__ __forceinline__ void stage_adjoint(c_t<T>* v, int t, const c_t<T>* __restrict__ W) {
    constexpr int NB = E / R;
#pragma unroll
    for (int u = 0; u < NB; ++u) {
        dft_r<T, SIGN2, R>(v + u * R);
        const int j = t + TL * u;
        const int k = j % NS;
        if (NS > 1 && k != 0) {
            c_t<T> w[R];
            stage_twiddles<T, R>(w, k * (N / (NS * R)), W);
#pragma unroll
            for (int r = 1; r < R; ++r)
                v[u * R + r] = SIGN2 > 0 ? cmul(v[u * R + r], w[r]) : cmulc(v[u * R + r], w[r]);
        }
    }
}

// Output index of value v[u*R + r] after the stage (NS, R).
template <int TL, int NS, int R>
__device__ __forceinline__ int stage_out_index(int t, int u, int r) {
    const int j = t + TL * u;
    const int k = j % NS;
    return (j - k) * R + k + r * NS;
}

template <typename T, int N, int TL, int E, int SIGN, int NS, int R, int... Rest>
struct StageRunner {
    // Runs this stage and the rest; on return v holds the last stage's outputs.
    static __device__ __forceinline__ void run(c_t<T>* v, int t, c_t<T>* scr, const c_t<T>* __restrict__ W) {
        stage_compute<T, N, TL, E, SIGN, NS, R>(v, t, W);
        if constexpr (sizeof...(Rest) > 0) {
            constexpr int R2 = RadInfo<Rest...>::prod;  // unused, keeps the pack named
            (void)R2;
            __syncwarp();
#pragma unroll
            for (int u = 0; u < E / R; ++u)
#pragma unroll
                for (int r = 0; r < R; ++r) scr[padx(stage_out_index<TL, NS, R>(t, u, r))] = v[u * R + r];
            __syncwarp();
            load_next<Rest...>(v, t, scr);
            StageRunner<T, N, TL, E, SIGN, NS * R, Rest...>::run(v, t, scr, W);
        }
    }
    template <int R2, int... Rest2>
    static __device__ __forceinline__ void load_next(c_t<T>* v, int t, const c_t<T>* scr) {
#pragma unroll
        for (int u = 0; u < E / R2; ++u)
#pragma unroll
            for (int r = 0; r < R2; ++r) v[u * R2 + r] = scr[padx(t + TL * u + r * (N / R2))];
    }
};

template <int R, int... Rest>
struct FirstRadix {
    static constexpr int value = R;
};

// The transform with sign SIGN2 as the adjoint of the sign -SIGN2 flow graph
// (stages (NS, R), (NS R, Rest...)): the later stages first, then an exchange
// from their input positions to this stage's output grouping, then this
// stage's adjoint.
template <typename T, int N, int TL, int E, int SIGN2, int NS, int R, int... Rest>
struct AdjRunner {
    static __device__ __forceinline__ void run(c_t<T>* v, int t, c_t<T>* scr, const c_t<T>* __restrict__ W) {
        if constexpr (sizeof...(Rest) > 0) {
            AdjRunner<T, N, TL, E, SIGN2, NS * R, Rest...>::run(v, t, scr, W);
            constexpr int Rn = FirstRadix<Rest...>::value;
            __syncwarp();
#pragma unroll
            for (int u = 0; u < E / Rn; ++u)
#pragma unroll
                for (int r = 0; r < Rn; ++r) scr[padx(t + TL * u + r * (N / Rn))] = v[u * Rn + r];
            __syncwarp();
#pragma unroll
            for (int u = 0; u < E / R; ++u)
#pragma unroll
                for (int r = 0; r < R; ++r) v[u * R + r] = scr[padx(stage_out_index<TL, NS, R>(t, u, r))];
        }
        stage_adjoint<T, N, TL, E, SIGN2, NS, R>(v, t, W);
    }
};

// Input index of value v[u*R + r] of the first stage with radix R.
template <int N, int TL, int R>
__device__ __forceinline__ int first_in_index(int t, int u, int r) {
    return t + TL * u + r * (N / R);
}

// Output index of v[e] after all stages of Rad<R...>.
template <int N, int TL, int NS, int R, int... Rest>
struct LastIndex {
    static __device__ __forceinline__ int of(int t, int e) {
        if constexpr (sizeof...(Rest) == 0) return stage_out_index<TL, NS, R>(t, e / R, e % R);
        else return LastIndex<N, TL, NS * R, Rest...>::of(t, e);
    }
};

template <typename T, int N, int E, int SIGN, class RadList>
struct LineFFT;

template <typename T, int N, int E, int SIGN, int R0, int... R>
struct LineFFT<T, N, E, SIGN, Rad<R0, R...>> {
    static constexpr int TL = N / E;
    static_assert(RadInfo<R0, R...>::prod == N, "radices must multiply to N");
    static_assert(E % RadInfo<R0, R...>::lcm == 0, "E must be a multiple of every radix");
    // v[u*R0 + r] must hold input first_in(t, u, r); on return v[e] holds output out(t, e).
    static __device__ __forceinline__ void run(c_t<T>* v, int t, c_t<T>* scr, const c_t<T>* __restrict__ W) {
        StageRunner<T, N, TL, E, SIGN, 1, R0, R...>::run(v, t, scr, W);
    }
    // The transform of sign -SIGN from the layout run() leaves: v[e] must hold
    // input out(t, e); on return v[e] holds output in(t, e).
    static __device__ __forceinline__ void run_adjoint(c_t<T>* v, int t, c_t<T>* scr, const c_t<T>* __restrict__ W) {
        AdjRunner<T, N, TL, E, -SIGN, 1, R0, R...>::run(v, t, scr, W);
    }
    static __device__ __forceinline__ int in_index(int t, int e) {
        return first_in_index<N, TL, R0>(t, e / R0, e % R0);
    }
    static __device__ __forceinline__ int out_index(int t, int e) { return LastIndex<N, TL, 1, R0, R...>::of(t, e); }
};

}  // namespace jdft
