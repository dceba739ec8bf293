// Register-resident line FFTs on pairs of bands with packed FP32 arithmetic.
//
// A "band pair" holds the same complex entry of two bands: x = (Re_0, Re_1)
// and y = (Im_0, Im_1), each a pair of FP32 values in one 64-bit register.
// Every add, subtract, multiply and fused multiply-add of the transform is
// the same for both bands, so it is issued once as a packed two-wide FP32
// instruction (add/sub/mul/fma .rn.f32x2), which halves the instruction count
// of the arithmetic against one band at a time.  The transforms have the
// structure of fft_reg.cuh (Stockham stages over TL lanes of a warp, E pairs
// per lane, exchanges through a warp-private scratch line) and give, for each
// band, the same unnormalised sums y_m = sum_t x_t exp(SIGN 2 pi i t m / N).
//
// Exchanges move the x and the y halves through a scratch line of float2
// (one 8-byte pair per element) one after the other, which keeps the
// scratch at the size of a one-band line.
#pragma once

#include <cstdint>

#include "fft_reg.cuh"

namespace jdft {

// ---- packed FP32 pairs --------------------------------------------------------
// Device code issues the packed instructions; the host versions (plain FP32
// arithmetic on the two halves) serve CPU checks of the butterflies.
struct f2x {
    unsigned long long v;
};

__host__ __device__ __forceinline__ f2x p_pack(float lo, float hi) {
    f2x r;
#ifdef __CUDA_ARCH__
    asm("mov.b64 %0, {%1, %2};" : "=l"(r.v) : "f"(lo), "f"(hi));
#else
    unsigned int a, b;
    __builtin_memcpy(&a, &lo, 4);
    __builtin_memcpy(&b, &hi, 4);
    r.v = (unsigned long long)a | ((unsigned long long)b << 32);
#endif
    return r;
}
__host__ __device__ __forceinline__ void p_unpack(f2x a, float& lo, float& hi) {
#ifdef __CUDA_ARCH__
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(a.v));
#else
    const unsigned int x = (unsigned int)(a.v & 0xffffffffull), y = (unsigned int)(a.v >> 32);
    __builtin_memcpy(&lo, &x, 4);
    __builtin_memcpy(&hi, &y, 4);
#endif
}
__host__ __device__ __forceinline__ f2x p_dup(float a) { return p_pack(a, a); }

#ifdef __CUDA_ARCH__
#define JDFT_PAIR_OP2(NAME, PTX, HOSTOP)                                               \
    __host__ __device__ __forceinline__ f2x NAME(f2x a, f2x b) {                       \
        f2x r;                                                                         \
        asm(PTX " %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));                      \
        return r;                                                                      \
    }
#else
#define JDFT_PAIR_OP2(NAME, PTX, HOSTOP)                                               \
    __host__ __device__ __forceinline__ f2x NAME(f2x a, f2x b) {                       \
        float a0, a1, b0, b1;                                                          \
        p_unpack(a, a0, a1);                                                           \
        p_unpack(b, b0, b1);                                                           \
        return p_pack(a0 HOSTOP b0, a1 HOSTOP b1);                                     \
    }
#endif
JDFT_PAIR_OP2(p_add, "add.rn.f32x2", +)
JDFT_PAIR_OP2(p_sub, "sub.rn.f32x2", -)
JDFT_PAIR_OP2(p_mul, "mul.rn.f32x2", *)
#undef JDFT_PAIR_OP2

// a * b + c
__host__ __device__ __forceinline__ f2x p_fma(f2x a, f2x b, f2x c) {
    f2x r;
#ifdef __CUDA_ARCH__
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r.v) : "l"(a.v), "l"(b.v), "l"(c.v));
#else
    float a0, a1, b0, b1, c0, c1;
    p_unpack(a, a0, a1);
    p_unpack(b, b0, b1);
    p_unpack(c, c0, c1);
    r = p_pack(__builtin_fmaf(a0, b0, c0), __builtin_fmaf(a1, b1, c1));
#endif
    return r;
}
__host__ __device__ __forceinline__ f2x p_zero() { return p_pack(0.f, 0.f); }

// Constant pairs of the butterflies, kept in the constant bank so that no
// register holds them and no instruction builds them (device code); the host
// versions serve CPU checks.
enum PairConst { PC_C1, PC_S1, PC_H, PC_MC1, PC_MS1, PC_MH, PC_MHALF, PC_R3, PC_MR3, PC_COUNT };
static __constant__ unsigned long long kPairConst[PC_COUNT] = {
    0x3f6c835e3f6c835eull,  // cos(pi/8)
    0x3ec3ef153ec3ef15ull,  // sin(pi/8)
    0x3f3504f33f3504f3ull,  // 1/sqrt(2)
    0xbf6c835ebf6c835eull,  // -cos(pi/8)
    0xbec3ef15bec3ef15ull,  // -sin(pi/8)
    0xbf3504f3bf3504f3ull,  // -1/sqrt(2)
    0xbf000000bf000000ull,  // -1/2
    0x3f5db3d73f5db3d7ull,  // sqrt(3)/2
    0xbf5db3d7bf5db3d7ull,  // -sqrt(3)/2
};
__host__ __device__ __forceinline__ f2x pconst(int i) {
#ifdef __CUDA_ARCH__
    return f2x{kPairConst[i]};
#else
    const float v[PC_COUNT] = {0.92387953251128675613f, 0.38268343236508977173f, 0.70710678118654752440f,
                               -0.92387953251128675613f, -0.38268343236508977173f, -0.70710678118654752440f,
                               -0.5f, 0.86602540378443864676f, -0.86602540378443864676f};
    return p_dup(v[i]);
#endif
}

// The same complex entry of two bands.
struct cpair {
    f2x x, y;
};

__host__ __device__ __forceinline__ cpair cp_add(cpair a, cpair b) { return {p_add(a.x, b.x), p_add(a.y, b.y)}; }
__host__ __device__ __forceinline__ cpair cp_sub(cpair a, cpair b) { return {p_sub(a.x, b.x), p_sub(a.y, b.y)}; }
__host__ __device__ __forceinline__ cpair cp_zero() { return {p_zero(), p_zero()}; }
__host__ __device__ __forceinline__ cpair cp_scale(cpair a, f2x s) { return {p_mul(a.x, s), p_mul(a.y, s)}; }

// Twiddle table entry W[e] = exp(+2 pi i e / N) held as (c, c, s, s): both
// halves of a pair multiply by the same root.
struct tw2 {
    f2x c, s;
};

// v * w (SIGN > 0) or v * conj(w) (SIGN < 0) for a twiddle w = (c, s).
template <int SIGN>
__host__ __device__ __forceinline__ cpair cp_twiddle(cpair v, tw2 w) {
    if constexpr (SIGN > 0) {
        return {p_sub(p_mul(v.x, w.c), p_mul(v.y, w.s)), p_fma(v.x, w.s, p_mul(v.y, w.c))};
    } else {
        return {p_fma(v.x, w.c, p_mul(v.y, w.s)), p_sub(p_mul(v.y, w.c), p_mul(v.x, w.s))};
    }
}
// Product of two roots (both as (c, c, s, s)).
__host__ __device__ __forceinline__ tw2 tw_mul(tw2 a, tw2 b) {
    return {p_sub(p_mul(a.c, b.c), p_mul(a.s, b.s)), p_fma(a.c, b.s, p_mul(a.s, b.c))};
}

// ---- R-point DFTs of pairs in registers: out[m] = sum_r v[r] exp(SIGN 2 pi i r m / R)
template <int SIGN>
__host__ __device__ __forceinline__ void pdft2(cpair* v) {
    const cpair a = v[0], b = v[1];
    v[0] = cp_add(a, b);
    v[1] = cp_sub(a, b);
}

template <int SIGN>
__host__ __device__ __forceinline__ void pdft4(cpair* v) {
    const cpair y0 = cp_add(v[0], v[2]), y1 = cp_sub(v[0], v[2]);
    const cpair y2 = cp_add(v[1], v[3]), d = cp_sub(v[1], v[3]);
    v[0] = cp_add(y0, y2);
    v[2] = cp_sub(y0, y2);
    // y3 = SIGN i d = (-SIGN d.y, SIGN d.x), added to and subtracted from y1
    if constexpr (SIGN > 0) {
        v[1] = {p_sub(y1.x, d.y), p_add(y1.y, d.x)};
        v[3] = {p_add(y1.x, d.y), p_sub(y1.y, d.x)};
    } else {
        v[1] = {p_add(y1.x, d.y), p_sub(y1.y, d.x)};
        v[3] = {p_sub(y1.x, d.y), p_add(y1.y, d.x)};
    }
}

template <int SIGN>
__host__ __device__ __forceinline__ void pdft3(cpair* v) {
    const cpair t1 = cp_add(v[1], v[2]), d = cp_sub(v[1], v[2]);
    const cpair m = {p_fma(t1.x, pconst(PC_MHALF), v[0].x), p_fma(t1.y, pconst(PC_MHALF), v[0].y)};
    v[0] = cp_add(v[0], t1);
    // t2 = SIGN i h d = (-SIGN h d.y, SIGN h d.x), h = sqrt(3)/2
    const f2x ph = pconst(SIGN > 0 ? PC_R3 : PC_MR3), mh = pconst(SIGN > 0 ? PC_MR3 : PC_R3);
    v[1] = {p_fma(d.y, mh, m.x), p_fma(d.x, ph, m.y)};
    v[2] = {p_fma(d.y, ph, m.x), p_fma(d.x, mh, m.y)};
}

template <int SIGN>
__host__ __device__ __forceinline__ void pdft8(cpair* v) {
    cpair e[4] = {v[0], v[2], v[4], v[6]};
    cpair o[4] = {v[1], v[3], v[5], v[7]};
    pdft4<SIGN>(e);
    pdft4<SIGN>(o);
    const f2x pr = pconst(PC_H), mr = pconst(PC_MH);  // +-1/sqrt(2)
    v[0] = cp_add(e[0], o[0]);
    v[4] = cp_sub(e[0], o[0]);
    // W8^1 o1 = r (o1.x - SIGN o1.y, o1.y + SIGN o1.x)
    {
        const f2x a = SIGN > 0 ? p_sub(o[1].x, o[1].y) : p_add(o[1].x, o[1].y);
        const f2x b = SIGN > 0 ? p_add(o[1].y, o[1].x) : p_sub(o[1].y, o[1].x);
        v[1] = {p_fma(a, pr, e[1].x), p_fma(b, pr, e[1].y)};
        v[5] = {p_fma(a, mr, e[1].x), p_fma(b, mr, e[1].y)};
    }
    // W8^2 o2 = SIGN i o2 = (-SIGN o2.y, SIGN o2.x)
    if constexpr (SIGN > 0) {
        v[2] = {p_sub(e[2].x, o[2].y), p_add(e[2].y, o[2].x)};
        v[6] = {p_add(e[2].x, o[2].y), p_sub(e[2].y, o[2].x)};
    } else {
        v[2] = {p_add(e[2].x, o[2].y), p_sub(e[2].y, o[2].x)};
        v[6] = {p_sub(e[2].x, o[2].y), p_add(e[2].y, o[2].x)};
    }
    // W8^3 o3 = r (-o3.x - SIGN o3.y, -o3.y + SIGN o3.x) = (-r a, SIGN r b)
    {
        const f2x a = SIGN > 0 ? p_add(o[3].x, o[3].y) : p_sub(o[3].x, o[3].y);
        const f2x b = SIGN > 0 ? p_sub(o[3].x, o[3].y) : p_add(o[3].x, o[3].y);
        const f2x sr = SIGN > 0 ? pr : mr, msr = SIGN > 0 ? mr : pr;
        v[3] = {p_fma(a, mr, e[3].x), p_fma(b, sr, e[3].y)};
        v[7] = {p_fma(a, pr, e[3].x), p_fma(b, msr, e[3].y)};
    }
}

// PIN: the inputs v[4] .. v[11] are zero (a line whose nonzero values lie in
// the central quarter of the box on either side of the origin); the first
// layer's 4-point DFTs then have two inputs each.  POUT: only the outputs
// v[0..3] and v[12..15] are wanted; the last layer computes only those and
// leaves the others undefined.
template <int SIGN, bool PIN = false, bool POUT = false>
__host__ __device__ __forceinline__ void pdft16(cpair* v) {
    // 16 = 4 x 4: DFT4 over n2 (stride 4), twiddle W16^{n1 k1}, DFT4 over n1.
    cpair a[4][4];
#pragma unroll
    for (int n1 = 0; n1 < 4; ++n1) {
        if constexpr (PIN) {
            // out[k] = w0 + w3 (SIGN i)^{3k}: w0 + w3, w0 - SIGN i w3, w0 - w3, w0 + SIGN i w3
            const cpair w0 = v[n1], w3 = v[n1 + 12];
            a[n1][0] = cp_add(w0, w3);
            a[n1][2] = cp_sub(w0, w3);
            if constexpr (SIGN > 0) {
                a[n1][1] = {p_add(w0.x, w3.y), p_sub(w0.y, w3.x)};
                a[n1][3] = {p_sub(w0.x, w3.y), p_add(w0.y, w3.x)};
            } else {
                a[n1][1] = {p_sub(w0.x, w3.y), p_add(w0.y, w3.x)};
                a[n1][3] = {p_add(w0.x, w3.y), p_sub(w0.y, w3.x)};
            }
        } else {
            cpair w[4] = {v[n1], v[n1 + 4], v[n1 + 8], v[n1 + 12]};
            pdft4<SIGN>(w);
#pragma unroll
            for (int k1 = 0; k1 < 4; ++k1) a[n1][k1] = w[k1];
        }
    }
    // x exp(SIGN 2 pi i e / 16) for e = n1 k1 in {1, 2, 3, 4, 6, 9}: (x.x c - x.y s, x.x s + x.y c)
    // with (c, s) = (C1, S1), (H, H), (S1, C1), (0, 1), (-H, H), (-C1, -S1) and s negated for SIGN < 0
    auto tw = [&](cpair x, int e) -> cpair {
        int c, s, ms;
        switch (e) {
            case 1: c = PC_C1; s = PC_S1; ms = PC_MS1; break;
            case 2: c = PC_H; s = PC_H; ms = PC_MH; break;
            case 3: c = PC_S1; s = PC_C1; ms = PC_MC1; break;
            case 4: {
                // SIGN i x = (-SIGN x.y, SIGN x.x)
                const f2x nx = p_sub(p_zero(), SIGN > 0 ? x.y : x.x);
                return SIGN > 0 ? cpair{nx, x.x} : cpair{x.y, nx};
            }
            case 6: c = PC_MH; s = PC_H; ms = PC_MH; break;
            default: c = PC_MC1; s = PC_MS1; ms = PC_S1; break;  // e = 9
        }
        if (SIGN < 0) {
            const int t = s;
            s = ms;
            ms = t;
        }
        return {p_fma(x.y, pconst(ms), p_mul(x.x, pconst(c))), p_fma(x.x, pconst(s), p_mul(x.y, pconst(c)))};
    };
#pragma unroll
    for (int n1 = 1; n1 < 4; ++n1)
#pragma unroll
        for (int k1 = 1; k1 < 4; ++k1) a[n1][k1] = tw(a[n1][k1], n1 * k1);
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) {
        if constexpr (POUT) {
            // outputs k2 = 0 and 3 of the 4-point DFT over n1
            const cpair y0 = cp_add(a[0][k1], a[2][k1]), y1 = cp_sub(a[0][k1], a[2][k1]);
            const cpair y2 = cp_add(a[1][k1], a[3][k1]), d = cp_sub(a[1][k1], a[3][k1]);
            v[k1] = cp_add(y0, y2);
            v[k1 + 12] = SIGN > 0 ? cpair{p_add(y1.x, d.y), p_sub(y1.y, d.x)} : cpair{p_sub(y1.x, d.y), p_add(y1.y, d.x)};
        } else {
            cpair w[4] = {a[0][k1], a[1][k1], a[2][k1], a[3][k1]};
            pdft4<SIGN>(w);
#pragma unroll
            for (int k2 = 0; k2 < 4; ++k2) v[k1 + 4 * k2] = w[k2];
        }
    }
}

template <int SIGN, int R, bool PIN = false, bool POUT = false>
__host__ __device__ __forceinline__ void pdft_r(cpair* v) {
    static_assert(R == 16 || !(PIN || POUT), "pruned butterflies exist for radix 16 only");
    if constexpr (R == 2) pdft2<SIGN>(v);
    else if constexpr (R == 3) pdft3<SIGN>(v);
    else if constexpr (R == 4) pdft4<SIGN>(v);
    else if constexpr (R == 8) pdft8<SIGN>(v);
    else if constexpr (R == 16) pdft16<SIGN, PIN, POUT>(v);
    else static_assert(R == 2 || R == 3 || R == 4 || R == 8 || R == 16, "radix not available for band pairs");
}

// Twiddles w[r] = W[r b], r = 1 .. R-1: table reads at the powers of two, the
// others as products w[r] = w[r - lowbit(r)] w[lowbit(r)].
template <int R>
__device__ __forceinline__ void pstage_twiddles(tw2* w, int b, const float4* __restrict__ W) {
#pragma unroll
    for (int r = 1; r < R; ++r) {
        const int low = r & (-r);
        if (low == r) {
            const float4 q = W[r * b];
            w[r] = {p_pack(q.x, q.y), p_pack(q.z, q.w)};
        } else {
            w[r] = tw_mul(w[r - low], w[low]);
        }
    }
}

template <int N, int TL, int E, int SIGN, int NS, int R, bool PIN = false>
__device__ __forceinline__ void pstage_compute(cpair* v, int t, const float4* __restrict__ W) {
    constexpr int NB = E / R;
#pragma unroll
    for (int u = 0; u < NB; ++u) {
        const int j = t + TL * u;
        const int k = j % NS;
        if (NS > 1 && k != 0) {
            tw2 w[R];
            pstage_twiddles<R>(w, k * (N / (NS * R)), W);
#pragma unroll
            for (int r = 1; r < R; ++r) v[u * R + r] = cp_twiddle<SIGN>(v[u * R + r], w[r]);
        }
        pdft_r<SIGN, R, PIN, false>(v + u * R);
    }
}

template <int N, int TL, int E, int SIGN2, int NS, int R, bool POUT = false>
__device__ __forceinline__ void pstage_adjoint(cpair* v, int t, const float4* __restrict__ W) {
    constexpr int NB = E / R;
#pragma unroll
    for (int u = 0; u < NB; ++u) {
        pdft_r<SIGN2, R, false, POUT>(v + u * R);
        const int j = t + TL * u;
        const int k = j % NS;
        if (NS > 1 && k != 0) {
            tw2 w[R];
            pstage_twiddles<R>(w, k * (N / (NS * R)), W);
#pragma unroll
            for (int r = 1; r < R; ++r) v[u * R + r] = cp_twiddle<SIGN2>(v[u * R + r], w[r]);
        }
    }
}

// Exchange through the scratch line: value v[i] goes to scratch slot
// dst(i), then v[i] is read back from slot src(i); the x halves first, then
// the y halves, through the same float2 line.
template <int E, class Dst, class Src>
__device__ __forceinline__ void pexchange(cpair* v, float2* scr, Dst dst, Src src) {
    __syncwarp();
#pragma unroll
    for (int i = 0; i < E; ++i) *reinterpret_cast<f2x*>(scr + padx(dst(i))) = v[i].x;
    __syncwarp();
#pragma unroll
    for (int i = 0; i < E; ++i) v[i].x = *reinterpret_cast<const f2x*>(scr + padx(src(i)));
    __syncwarp();
#pragma unroll
    for (int i = 0; i < E; ++i) *reinterpret_cast<f2x*>(scr + padx(dst(i))) = v[i].y;
    __syncwarp();
#pragma unroll
    for (int i = 0; i < E; ++i) v[i].y = *reinterpret_cast<const f2x*>(scr + padx(src(i)));
}

// PRUNE: the first stage (NS = 1) takes the pruned radix-16 butterflies
// (inputs outside the window are zero in run, outputs outside it unwanted in
// the adjoint).
template <int N, int TL, int E, int SIGN, int NS, bool PRUNE, int R, int... Rest>
struct PStageRunner {
    static __device__ __forceinline__ void run(cpair* v, int t, float2* scr, const float4* __restrict__ W) {
        pstage_compute<N, TL, E, SIGN, NS, R, PRUNE && NS == 1>(v, t, W);
        if constexpr (sizeof...(Rest) > 0) {
            constexpr int Rn = FirstRadix<Rest...>::value;
            pexchange<E>(
                v, scr, [&](int i) { return stage_out_index<TL, NS, R>(t, i / R, i % R); },
                [&](int i) { return t + TL * (i / Rn) + (i % Rn) * (N / Rn); });
            PStageRunner<N, TL, E, SIGN, NS * R, false, Rest...>::run(v, t, scr, W);
        }
    }
};

template <int N, int TL, int E, int SIGN2, int NS, bool PRUNE, int R, int... Rest>
struct PAdjRunner {
    static __device__ __forceinline__ void run(cpair* v, int t, float2* scr, const float4* __restrict__ W) {
        if constexpr (sizeof...(Rest) > 0) {
            PAdjRunner<N, TL, E, SIGN2, NS * R, false, Rest...>::run(v, t, scr, W);
            constexpr int Rn = FirstRadix<Rest...>::value;
            pexchange<E>(
                v, scr, [&](int i) { return t + TL * (i / Rn) + (i % Rn) * (N / Rn); },
                [&](int i) { return stage_out_index<TL, NS, R>(t, i / R, i % R); });
        }
        pstage_adjoint<N, TL, E, SIGN2, NS, R, PRUNE && NS == 1>(v, t, W);
    }
};

template <int N, int E, int SIGN, class RadList, bool WIN = false>
struct LineFFTP;

// Same lane layout and index maps as LineFFT<T, N, E, SIGN, Rad<R0, R...>>.
// WIN: the line's nonzero inputs of run() (and the wanted outputs of
// run_adjoint()) lie at positions -N/4 .. N/4 - 1 (mod N); with a first
// radix of 16 and E = 16, lane t holds positions t + (N/16) e, so that is
// e in 0..3 and 12..15 for every lane, and the first stage's butterflies are
// pruned to them.
template <int N, int E, int SIGN, int R0, int... R, bool WIN>
struct LineFFTP<N, E, SIGN, Rad<R0, R...>, WIN> {
    static constexpr int TL = N / E;
    static_assert(RadInfo<R0, R...>::prod == N, "radices must multiply to N");
    static_assert(E % RadInfo<R0, R...>::lcm == 0, "E must be a multiple of every radix");
    static_assert(!WIN || (R0 == 16 && E == 16), "the window pruning needs a first radix of 16 and E = 16");
    // whether value e of a lane can lie in the window
    static __host__ __device__ constexpr bool in_window(int e) { return !WIN || e < 4 || e >= 12; }
    static __device__ __forceinline__ void run(cpair* v, int t, float2* scr, const float4* __restrict__ W) {
        PStageRunner<N, TL, E, SIGN, 1, WIN, R0, R...>::run(v, t, scr, W);
    }
    static __device__ __forceinline__ void run_adjoint(cpair* v, int t, float2* scr, const float4* __restrict__ W) {
        PAdjRunner<N, TL, E, -SIGN, 1, WIN, R0, R...>::run(v, t, scr, W);
    }
    static __device__ __forceinline__ int in_index(int t, int e) {
        return first_in_index<N, TL, R0>(t, e / R0, e % R0);
    }
    static __device__ __forceinline__ int out_index(int t, int e) { return LastIndex<N, TL, 1, R0, R...>::of(t, e); }
};

}  // namespace jdft
