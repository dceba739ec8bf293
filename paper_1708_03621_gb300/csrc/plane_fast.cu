// Plane pass of the Hamiltonian chain with register-resident line FFTs, for
// the box shapes it is compiled for (the generic shared-memory Stockham plane
// kernels in chain.cu serve every other shape).
//
// One block per (z-plane j2, band); 8 warps.  Three phases with one block
// barrier between consecutive phases:
//   1. rows: inverse transform along axis 1 of the nrows i0-rows the sphere
//      touches; each row's input is read straight from the plane's disk
//      values (a row's columns are consecutive i1) and its output written to
//      the shared plane A[r][j1];
//   2. columns: for every j1, inverse transform along axis 0 of the column
//      A[.][j1] placed at slots (i0min + r) mod S0, multiply by V(j0, j1, j2),
//      forward transform, keep the nrows sphere slots, back into A;
//   3. rows: forward transform along axis 1, gather the disk values back.
// Lines are split over TL lanes of one warp (E values per lane); stages of a
// line exchange values through a warp-private scratch line with __syncwarp.
// (JDFTx paper, Sec. 2.1: the I, multiply, J chain of Listing 1 on
// temporaries; here the real-space box never leaves on-chip memory.)
#include <algorithm>
#include <cstdlib>

#include "chain.cuh"
#include "fft_reg.cuh"
#include "profile.cuh"
#include "tc_ptx.cuh"

namespace jdft {

constexpr int kFastThreads = 256;
constexpr int kFastWarps = kFastThreads / 32;
// z passes: warps per block (LPW columns each)
constexpr int kZWarps = 8;
constexpr int kZThreads = 32 * kZWarps;

// i mod N in [0, N) for either sign of i: one bit mask when N is a power of
// two (two's complement), else a remainder and a correction.
template <int N>
__device__ __forceinline__ int wrapn(int i) {
    if constexpr ((N & (N - 1)) == 0) {
        return i & (N - 1);
    } else {
        const int r = i % N;
        return r < 0 ? r + N : r;
    }
}

// Shared-memory layout of the register-FFT kernels.  A warp's 8-byte shared
// access is served in two halves of 16 lanes and a 16-byte access in four
// quarters of 8 lanes; lanes of one group that hit different addresses in the
// same bank slot (16 eight-byte or 8 sixteen-byte slots per 128 bytes) cost
// one wavefront each.  The constants below are the ones with the fewest such
// conflicts over every shared access of these kernels, counted access by
// access (plane_layout.py beside this package prints them); the 128^3 FP32
// plane pass has none.
//
// Lanes: a line of N values is split over TL = N / E lanes and a warp serves
// LPW = 32 / TL lines; lane l takes position l / LPW of line l % LPW, so a
// half-warp covers several lines at once and several consecutive rows or
// columns of the plane array.
template <int N, int E>
struct Lanes {
    static constexpr int TL = N / E, LPW = 32 / TL;
    static __device__ __forceinline__ int line(int lane) { return lane % LPW; }
    static __device__ __forceinline__ int pos(int lane) { return lane / LPW; }
};

// Elements between the LPW scratch lines of one warp (each line needs
// padded_line(N)).
template <typename T, int N>
struct ScratchSpacing;
#define JDFT_SCRATCH_SPACING(T, N, SP)                                                      \
    template <>                                                                             \
    struct ScratchSpacing<T, N> {                                                           \
        static constexpr int value = SP;                                                    \
        static_assert(SP >= padded_line(N), "scratch lines of one warp must not overlap"); \
    };
JDFT_SCRATCH_SPACING(float, 12, 13)
JDFT_SCRATCH_SPACING(float, 16, 17)
JDFT_SCRATCH_SPACING(float, 40, 43)
JDFT_SCRATCH_SPACING(float, 48, 54)
JDFT_SCRATCH_SPACING(float, 64, 68)
JDFT_SCRATCH_SPACING(float, 80, 86)
JDFT_SCRATCH_SPACING(float, 128, 140)
JDFT_SCRATCH_SPACING(float, 256, 280)
JDFT_SCRATCH_SPACING(double, 12, 13)
JDFT_SCRATCH_SPACING(double, 16, 17)
JDFT_SCRATCH_SPACING(double, 40, 43)
JDFT_SCRATCH_SPACING(double, 48, 51)
JDFT_SCRATCH_SPACING(double, 64, 70)
JDFT_SCRATCH_SPACING(double, 80, 85)
JDFT_SCRATCH_SPACING(double, 128, 138)
JDFT_SCRATCH_SPACING(double, 256, 276)
#undef JDFT_SCRATCH_SPACING

// Row stride (elements) of the plane array A of an S0 x S1 plane.
template <typename T, int N0, int N1>
struct PlaneStride;
#define JDFT_PLANE_STRIDE(T, N0, N1, LS)    \
    template <>                             \
    struct PlaneStride<T, N0, N1> {         \
        static constexpr int value = LS;    \
        static_assert(LS > N1, "row pad"); \
    };
JDFT_PLANE_STRIDE(float, 12, 12, 13)
JDFT_PLANE_STRIDE(float, 16, 12, 13)
JDFT_PLANE_STRIDE(float, 40, 40, 41)
JDFT_PLANE_STRIDE(float, 48, 48, 50)
JDFT_PLANE_STRIDE(float, 64, 64, 68)
JDFT_PLANE_STRIDE(float, 80, 80, 82)
JDFT_PLANE_STRIDE(float, 128, 128, 132)
JDFT_PLANE_STRIDE(float, 256, 128, 130)
JDFT_PLANE_STRIDE(double, 12, 12, 13)
JDFT_PLANE_STRIDE(double, 16, 12, 13)
JDFT_PLANE_STRIDE(double, 40, 40, 41)
JDFT_PLANE_STRIDE(double, 48, 48, 49)
JDFT_PLANE_STRIDE(double, 64, 64, 66)
JDFT_PLANE_STRIDE(double, 80, 80, 81)
JDFT_PLANE_STRIDE(double, 128, 128, 130)
JDFT_PLANE_STRIDE(double, 256, 128, 130)
#undef JDFT_PLANE_STRIDE

// Elements of warp-private scratch: the LPW lines of the axis that needs more.
template <typename T, int N0, int E0, int N1, int E1>
__host__ __device__ constexpr int warp_scratch() {
    return Lanes<N0, E0>::LPW * ScratchSpacing<T, N0>::value > Lanes<N1, E1>::LPW * ScratchSpacing<T, N1>::value
               ? Lanes<N0, E0>::LPW * ScratchSpacing<T, N0>::value
               : Lanes<N1, E1>::LPW * ScratchSpacing<T, N1>::value;
}

// Phase 1 / 3 helpers -------------------------------------------------------
template <typename T, int N1, int E1, class R1, int NW = kFastWarps>
__device__ __forceinline__ void rows_inverse_fast(const ChainGeom& g, const c_t<T>* __restrict__ plane, c_t<T>* A,
                                                  int lsA, c_t<T>* wscr, const c_t<T>* W1, int warp, int lane) {
    using F = LineFFT<T, N1, E1, +1, R1>;
    using LN = Lanes<N1, E1>;
    constexpr int LPW = LN::LPW;
    const int liw = LN::line(lane), t = LN::pos(lane);
    c_t<T>* scr = wscr + liw * ScratchSpacing<T, N1>::value;
    for (int base = warp * LPW; base < g.nrows; base += NW * LPW) {
        const int r = base + liw;
        const bool act = r < g.nrows;
        int cs = 0, cnt = 0, lo = 0;
        if (act) {
            cs = g.row_col_start[r];
            cnt = g.row_col_start[r + 1] - cs;
            lo = g.row_i1lo[r];
        }
        c_t<T> v[E1];
#pragma unroll
        for (int e = 0; e < E1; ++e) {
            const int off = wrapn<N1>(F::in_index(t, e) - lo);
            v[e] = (off < cnt) ? plane[cs + off] : mk<T>(T(0), T(0));
        }
        F::run(v, t, scr, W1);
        if (act) {
#pragma unroll
            for (int e = 0; e < E1; ++e) A[r * lsA + F::out_index(t, e)] = v[e];
        }
    }
}

template <typename T, int N1, int E1, class R1, int NW = kFastWarps>
__device__ __forceinline__ void rows_forward_fast(const ChainGeom& g, c_t<T>* __restrict__ plane, const c_t<T>* A,
                                                  int lsA, c_t<T>* wscr, const c_t<T>* W1, int warp, int lane) {
    using F = LineFFT<T, N1, E1, -1, R1>;
    using LN = Lanes<N1, E1>;
    constexpr int LPW = LN::LPW;
    const int liw = LN::line(lane), t = LN::pos(lane);
    c_t<T>* scr = wscr + liw * ScratchSpacing<T, N1>::value;
    for (int base = warp * LPW; base < g.nrows; base += NW * LPW) {
        const int r = base + liw;
        const bool act = r < g.nrows;
        c_t<T> v[E1];
#pragma unroll
        for (int e = 0; e < E1; ++e) v[e] = act ? A[r * lsA + F::in_index(t, e)] : mk<T>(T(0), T(0));
        F::run(v, t, scr, W1);
        if (act) {
            const int cs = g.row_col_start[r];
            const int cnt = g.row_col_start[r + 1] - cs;
            const int lo = g.row_i1lo[r];
#pragma unroll
            for (int e = 0; e < E1; ++e) {
                const int off = wrapn<N1>(F::out_index(t, e) - lo);
                if (off < cnt) plane[cs + off] = v[e];
            }
        }
    }
}

// Inverse transform of column j1 (sphere rows of A placed at their slots).
template <typename T, int N0, int E0, class R0>
__device__ __forceinline__ void column_inverse_fast(const ChainGeom& g, const c_t<T>* A, int lsA, int j1, bool act,
                                                    c_t<T>* v, int t, c_t<T>* scr, const c_t<T>* W0) {
    using F = LineFFT<T, N0, E0, +1, R0>;
#pragma unroll
    for (int e = 0; e < E0; ++e) {
        const int r = wrapn<N0>(F::in_index(t, e) - g.i0min);
        v[e] = (act && r < g.nrows) ? A[r * lsA + j1] : mk<T>(T(0), T(0));
    }
    F::run(v, t, scr, W0);
}

// The plane pass of H: rows inverse, columns inverse x V forward, rows forward.
template <typename T, int N0, int E0, class R0, int N1, int E1, class R1>
__global__ void __launch_bounds__(kFastThreads) plane_apply_fast_kernel(ChainGeom g, c_t<T>* __restrict__ colbuf,
                                                                        const T* __restrict__ Vp,
                                                                        const c_t<T>* __restrict__ tw0,
                                                                        const c_t<T>* __restrict__ tw1) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int lsA = PlaneStride<T, N0, N1>::value;
    constexpr int SCR = warp_scratch<T, N0, E0, N1, E1>();  // per-warp scratch (LPW lines)
    c_t<T>* W0 = reinterpret_cast<c_t<T>*>(smem_raw);
    c_t<T>* W1 = W0 + N0;
    c_t<T>* scr_all = W1 + N1;
    c_t<T>* A = scr_all + kFastWarps * SCR;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    c_t<T>* wscr = scr_all + warp * SCR;
    for (int i = threadIdx.x; i < N0; i += blockDim.x) W0[i] = tw0[i];
    for (int i = threadIdx.x; i < N1; i += blockDim.x) W1[i] = tw1[i];
    __syncthreads();
    const int j2 = blockIdx.x, b = blockIdx.y;
    c_t<T>* plane = colbuf + colbuf_index(g, b, j2, 0);

    rows_inverse_fast<T, N1, E1, R1>(g, plane, A, lsA, wscr, W1, warp, lane);
    __syncthreads();

    {
        using FI = LineFFT<T, N0, E0, +1, R0>;
        using LN = Lanes<N0, E0>;
        constexpr int LPW = LN::LPW;
        const int liw = LN::line(lane), t = LN::pos(lane);
        c_t<T>* scr = wscr + liw * ScratchSpacing<T, N0>::value;
        // every lane has a column when the rounds tile the plane exactly
        constexpr bool kAllCols = N1 % (kFastWarps * LPW) == 0;
        for (int base = warp * LPW; base < N1; base += kFastWarps * LPW) {
            const int j1 = base + liw;
            const bool act = kAllCols || j1 < N1;
            c_t<T> v[E0];
            column_inverse_fast<T, N0, E0, R0>(g, A, lsA, j1, act, v, t, scr, W0);
            const T* Vq = Vp + ((size_t)j2 * N1 + (act ? j1 : 0)) * N0;
#pragma unroll
            for (int e = 0; e < E0; ++e) v[e] = act ? cscale(v[e], Vq[FI::out_index(t, e)]) : mk<T>(T(0), T(0));
            // forward transform as the adjoint of the inverse: starts from the
            // layout the inverse left, ends in the layout it started from
            FI::run_adjoint(v, t, scr, W0);
            if (act) {
#pragma unroll
                for (int e = 0; e < E0; ++e) {
                    const int r = wrapn<N0>(FI::in_index(t, e) - g.i0min);
                    if (r < g.nrows) A[r * lsA + j1] = v[e];
                }
            }
        }
    }
    __syncthreads();

    rows_forward_fast<T, N1, E1, R1>(g, plane, A, lsA, wscr, W1, warp, lane);
}

// Density, FP32 blocks: block (j2, band group) accumulates f_b |psi_b|^2 in
// registers (each lane always owns the same (j0, j1) points) over its bands.
template <int N0, int E0, class R0, int N1, int E1, class R1, int NW>
__global__ void __launch_bounds__(32 * NW) plane_density_fast_kernel(ChainGeom g,
                                                                          const float2* __restrict__ colbuf, int nb,
                                                                          int bands_per_block,
                                                                          const double* __restrict__ f, double w,
                                                                          double* __restrict__ n_r,
                                                                          const float2* __restrict__ tw0,
                                                                          const float2* __restrict__ tw1) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int lsA = PlaneStride<float, N0, N1>::value;
    constexpr int SCR = warp_scratch<float, N0, E0, N1, E1>();
    using LN = Lanes<N0, E0>;
    constexpr int LPW = LN::LPW;
    constexpr int ROUNDS = (N1 + NW * LPW - 1) / (NW * LPW);
    constexpr bool kAllCols = N1 % (NW * LPW) == 0;  // every lane has a column in every round
    float2* W0 = reinterpret_cast<float2*>(smem_raw);
    float2* W1 = W0 + N0;
    float2* scr_all = W1 + N1;
    float2* A = scr_all + NW * SCR;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float2* wscr = scr_all + warp * SCR;
    for (int i = threadIdx.x; i < N0; i += blockDim.x) W0[i] = tw0[i];
    for (int i = threadIdx.x; i < N1; i += blockDim.x) W1[i] = tw1[i];
    __syncthreads();
    const int j2 = blockIdx.x;
    const int bA = blockIdx.y * bands_per_block, bB = min(nb, bA + bands_per_block);
    const int liw = LN::line(lane), t = LN::pos(lane);
    float acc[ROUNDS][E0];
#pragma unroll
    for (int k = 0; k < ROUNDS; ++k)
#pragma unroll
        for (int e = 0; e < E0; ++e) acc[k][e] = 0.f;
    for (int b = bA; b < bB; ++b) {
        const float fb = (float)f[b];
        rows_inverse_fast<float, N1, E1, R1, NW>(g, colbuf + colbuf_index(g, b, j2, 0), A, lsA, wscr, W1, warp,
                                                 lane);
        __syncthreads();
#pragma unroll
        for (int k = 0; k < ROUNDS; ++k) {
            const int j1 = warp * LPW + liw + k * NW * LPW;
            float2 v[E0];
            column_inverse_fast<float, N0, E0, R0>(g, A, lsA, j1, kAllCols || j1 < N1, v, t,
                                                   wscr + liw * ScratchSpacing<float, N0>::value, W0);
#pragma unroll
            for (int e = 0; e < E0; ++e) acc[k][e] += fb * (v[e].x * v[e].x + v[e].y * v[e].y);
        }
        __syncthreads();
    }
    using FI = LineFFT<float, N0, E0, +1, R0>;
    const bool atomic = gridDim.y > 1;
#pragma unroll
    for (int k = 0; k < ROUNDS; ++k) {
        const int j1 = warp * LPW + liw + k * NW * LPW;
        if (j1 >= N1) continue;
#pragma unroll
        for (int e = 0; e < E0; ++e) {
            const int j0 = FI::out_index(t, e);
            double* dst = n_r + ((size_t)j0 * N1 + j1) * g.S2 + j2;
            const double val = w * (double)acc[k][e];
            if (atomic) atomicAdd(dst, val);
            else *dst += val;
        }
    }
}

// Hamiltonian plane pass and density in one (FP32 blocks, 16 values per lane
// along axis 0).  A persistent block takes a contiguous range of the
// plane-major list of (z-plane j2, band) items, runs the plane pass of
// plane_apply_fast_kernel on each, and adds f_b |psi_b|^2 of the column
// inverse transforms (the psi_b(r) the pass forms anyway) to FP32 sums held
// in tensor memory: 128 columns per block, lane quadrant warp % 4, column half
// warp / 4, 16 columns per column round.  The sums go to n(r) with FP64
// atomics whenever the block's plane changes and at the end, about twice per
// block.
template <int N0, int E0, class R0, int N1, int E1, class R1>
__global__ void __launch_bounds__(kFastThreads, 2) plane_apply_density_fast_kernel(
    ChainGeom g, float2* __restrict__ colbuf, const float* __restrict__ Vp, int nb, const double* __restrict__ f,
    double w, double* __restrict__ n_r, const float2* __restrict__ tw0, const float2* __restrict__ tw1) {
    static_assert(E0 == 16, "the tensor-memory sums take 16 values per lane and round");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ uint32_t tslot;
    constexpr int lsA = PlaneStride<float, N0, N1>::value;
    constexpr int SCR = warp_scratch<float, N0, E0, N1, E1>();
    using LN = Lanes<N0, E0>;
    constexpr int LPW = LN::LPW;
    constexpr int ROUNDS = (N1 + kFastWarps * LPW - 1) / (kFastWarps * LPW);
    constexpr bool kAllCols = N1 % (kFastWarps * LPW) == 0;  // every lane has a column in every round
    static_assert(ROUNDS * 16 <= 64, "at most 64 sums per lane");
    using FI = LineFFT<float, N0, E0, +1, R0>;
    float2* W0 = reinterpret_cast<float2*>(smem_raw);
    float2* W1 = W0 + N0;
    float2* scr_all = W1 + N1;
    float2* A = scr_all + kFastWarps * SCR;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int liw = LN::line(lane), t = LN::pos(lane);
    float2* wscr = scr_all + warp * SCR;
    float2* scr = wscr + liw * ScratchSpacing<float, N0>::value;
    for (int i = threadIdx.x; i < N0; i += blockDim.x) W0[i] = tw0[i];
    for (int i = threadIdx.x; i < N1; i += blockDim.x) W1[i] = tw1[i];
    if (warp == 0) tc::tmem_alloc(&tslot, 128);
    tc::tc_fence_before_sync();
    __syncthreads();
    tc::tc_fence_after_sync();
    const uint32_t tb = tslot + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)((warp >> 2) * 64);
    const int64_t items = (int64_t)g.S2 * nb;
    const int64_t it0 = items * blockIdx.x / gridDim.x, it1 = items * (blockIdx.x + 1) / gridDim.x;
    auto flush = [&](int j2) {
#pragma unroll 1
        for (int k = 0; k < ROUNDS; ++k) {
            float acc[16];
            tc::tmem_ld16(tb + 16 * k, acc);
            const int j1 = warp * LPW + liw + k * kFastWarps * LPW;
            if (j1 < N1) {
#pragma unroll
                for (int e = 0; e < E0; ++e)
                    atomicAdd(n_r + ((size_t)FI::out_index(t, e) * N1 + j1) * g.S2 + j2, w * (double)acc[e]);
            }
        }
    };
    auto zero = [&]() {
        float z[16];
#pragma unroll
        for (int e = 0; e < 16; ++e) z[e] = 0.f;
#pragma unroll
        for (int k = 0; k < ROUNDS; ++k) tc::tmem_st16(tb + 16 * k, z);
        tc::tmem_wait_st();
    };
    int cur = -1;
    for (int64_t it = it0; it < it1; ++it) {
        const int j2 = (int)(it / nb), b = (int)(it - (int64_t)j2 * nb);
        if (j2 != cur) {
            if (cur >= 0) flush(cur);
            zero();
            cur = j2;
        }
        float2* plane = colbuf + colbuf_index(g, b, j2, 0);
        rows_inverse_fast<float, N1, E1, R1>(g, plane, A, lsA, wscr, W1, warp, lane);
        __syncthreads();
        const float fb = (float)f[b];
        // rolled: four copies of the two column transforms would overflow the instruction cache
#pragma unroll 1
        for (int k = 0; k < ROUNDS; ++k) {
            const int j1 = warp * LPW + liw + k * kFastWarps * LPW;
            const bool act = kAllCols || j1 < N1;
            // this round's sums are fetched while the column transform runs
            uint32_t sr[16];
            tc::tmem_ld16_issue(tb + 16 * k, sr);
            float2 v[E0];
            column_inverse_fast<float, N0, E0, R0>(g, A, lsA, j1, act, v, t, scr, W0);
            tc::tmem_wait_ld16(sr);
            float acc[16];
#pragma unroll
            for (int e = 0; e < E0; ++e)
                acc[e] = __uint_as_float(sr[e]) + fb * (v[e].x * v[e].x + v[e].y * v[e].y);
            tc::tmem_st16(tb + 16 * k, acc);
            const float* Vq = Vp + ((size_t)j2 * N1 + (act ? j1 : 0)) * N0;
#pragma unroll
            for (int e = 0; e < E0; ++e) v[e] = act ? cscale(v[e], Vq[FI::out_index(t, e)]) : mk<float>(0.f, 0.f);
            FI::run_adjoint(v, t, scr, W0);
            if (act) {
#pragma unroll
                for (int e = 0; e < E0; ++e) {
                    const int r = wrapn<N0>(FI::in_index(t, e) - g.i0min);
                    if (r < g.nrows) A[r * lsA + j1] = v[e];
                }
            }
        }
        tc::tmem_wait_st();
        __syncthreads();
        rows_forward_fast<float, N1, E1, R1>(g, plane, A, lsA, wscr, W1, warp, lane);
        __syncthreads();
    }
    if (cur >= 0) flush(cur);
    tc::tc_fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tslot, 128);
}

// z passes with register line FFTs: TL lanes per (i0, i1) column of the
// sphere, LPW columns per warp, 8 warps per block, one band per blockIdx.y.
// A column's plane waves have consecutive z-slots from pw_z of its first one
// (modulo S2), so a slot p holds sphere entry (p - z0) mod S2 when that is
// below the column's count.
template <typename T, int N2, int E2, class R2>
__global__ void __launch_bounds__(kZThreads) zpass_inverse_fast_kernel(ChainGeom g, const c_t<T>* __restrict__ C,
                                                                          int ldc, c_t<T>* __restrict__ colbuf,
                                                                          const c_t<T>* __restrict__ tw2) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    using F = LineFFT<T, N2, E2, +1, R2>;
    using LN = Lanes<N2, E2>;
    constexpr int LPW = LN::LPW;
    c_t<T>* W = reinterpret_cast<c_t<T>*>(smem_raw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int liw = LN::line(lane), t = LN::pos(lane);
    c_t<T>* scr = W + N2 + (warp * LPW + liw) * ScratchSpacing<T, N2>::value;
    for (int i = threadIdx.x; i < N2; i += blockDim.x) W[i] = tw2[i];
    __syncthreads();
    const int c = (blockIdx.x * kZWarps + warp) * LPW + liw;
    const int b = blockIdx.y;
    const bool act = c < g.ncols;
    int q0 = 0, cnt = 0, z0 = 0;
    if (act) {
        q0 = g.col_start[c];
        cnt = g.col_start[c + 1] - q0;
        z0 = g.pw_z[q0];
    }
    const c_t<T>* Cb = C + (size_t)b * ldc + q0;
    c_t<T> v[E2];
#pragma unroll
    for (int e = 0; e < E2; ++e) {
        const int off = wrapn<N2>(F::in_index(t, e) - z0);
        v[e] = off < cnt ? Cb[off] : mk<T>(T(0), T(0));
    }
    F::run(v, t, scr, W);
    if (act) {
#pragma unroll
        for (int e = 0; e < E2; ++e) colbuf[colbuf_index(g, b, F::out_index(t, e), c)] = v[e];
    }
}

// MODE 0: out = omega (kin C + scale y); MODE 1: out = scale y.
template <typename T, int N2, int E2, class R2, int MODE>
__global__ void __launch_bounds__(kZThreads) zpass_forward_fast_kernel(ChainGeom g,
                                                                          const c_t<T>* __restrict__ colbuf,
                                                                          const c_t<T>* __restrict__ C, int ldc,
                                                                          c_t<T>* __restrict__ out, int ldo,
                                                                          const T* __restrict__ kin, T omega, T scale,
                                                                          const c_t<T>* __restrict__ tw2) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    using F = LineFFT<T, N2, E2, -1, R2>;
    using LN = Lanes<N2, E2>;
    constexpr int LPW = LN::LPW;
    c_t<T>* W = reinterpret_cast<c_t<T>*>(smem_raw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int liw = LN::line(lane), t = LN::pos(lane);
    c_t<T>* scr = W + N2 + (warp * LPW + liw) * ScratchSpacing<T, N2>::value;
    for (int i = threadIdx.x; i < N2; i += blockDim.x) W[i] = tw2[i];
    __syncthreads();
    const int c = (blockIdx.x * kZWarps + warp) * LPW + liw;
    const int b = blockIdx.y;
    const bool act = c < g.ncols;
    c_t<T> v[E2];
#pragma unroll
    for (int e = 0; e < E2; ++e)
        v[e] = act ? colbuf[colbuf_index(g, b, F::in_index(t, e), c)] : mk<T>(T(0), T(0));
    F::run(v, t, scr, W);
    if (act) {
        const int q0 = g.col_start[c];
        const int cnt = g.col_start[c + 1] - q0;
        const int z0 = g.pw_z[q0];
#pragma unroll
        for (int e = 0; e < E2; ++e) {
            const int off = wrapn<N2>(F::out_index(t, e) - z0);
            if (off < cnt) {
                const int q = q0 + off;
                c_t<T> r;
                if (MODE == 0) {
                    const c_t<T> cq = C[(size_t)b * ldc + q];
                    const T kq = kin[q];
                    r = mk<T>(omega * (kq * cq.x + scale * v[e].x), omega * (kq * cq.y + scale * v[e].y));
                } else {
                    r = cscale(v[e], scale);
                }
                out[(size_t)b * ldo + q] = r;
            }
        }
    }
}

// The z passes of a k-batched chain: blockIdx.z selects the job (k-point),
// blockIdx.y the band, blockIdx.x the block of columns, as in the one-job
// kernels; blocks beyond a job's columns or bands return at once.
template <int N2, int E2, class R2>
__global__ void __launch_bounds__(kZThreads) zpass_inverse_batch_kernel(const KJob* __restrict__ jobs,
                                                                           const float2* __restrict__ tw2) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    using F = LineFFT<float, N2, E2, +1, R2>;
    using LN = Lanes<N2, E2>;
    constexpr int LPW = LN::LPW;
    const KJob& J = jobs[blockIdx.z];
    const ChainGeom& g = J.g;
    const int b = blockIdx.y;
    if (b >= J.nb || (int)blockIdx.x * kZWarps * LPW >= g.ncols) return;
    float2* W = reinterpret_cast<float2*>(smem_raw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int liw = LN::line(lane), t = LN::pos(lane);
    float2* scr = W + N2 + (warp * LPW + liw) * ScratchSpacing<float, N2>::value;
    for (int i = threadIdx.x; i < N2; i += blockDim.x) W[i] = tw2[i];
    __syncthreads();
    const int c = (blockIdx.x * kZWarps + warp) * LPW + liw;
    const bool act = c < g.ncols;
    int q0 = 0, cnt = 0, z0 = 0;
    if (act) {
        q0 = g.col_start[c];
        cnt = g.col_start[c + 1] - q0;
        z0 = g.pw_z[q0];
    }
    const float2* Cb = J.C + (size_t)b * J.ldc + q0;
    float2 v[E2];
#pragma unroll
    for (int e = 0; e < E2; ++e) {
        const int off = wrapn<N2>(F::in_index(t, e) - z0);
        v[e] = off < cnt ? Cb[off] : make_float2(0.f, 0.f);
    }
    F::run(v, t, scr, W);
    if (act) {
#pragma unroll
        for (int e = 0; e < E2; ++e) J.colbuf[colbuf_index(g, b, F::out_index(t, e), c)] = v[e];
    }
}

// HC = omega (kin C + scale y) for every job.
template <int N2, int E2, class R2>
__global__ void __launch_bounds__(kZThreads) zpass_forward_batch_kernel(const KJob* __restrict__ jobs, float omega,
                                                                           float scale,
                                                                           const float2* __restrict__ tw2) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    using F = LineFFT<float, N2, E2, -1, R2>;
    using LN = Lanes<N2, E2>;
    constexpr int LPW = LN::LPW;
    const KJob& J = jobs[blockIdx.z];
    const ChainGeom& g = J.g;
    const int b = blockIdx.y;
    if (b >= J.nb || (int)blockIdx.x * kZWarps * LPW >= g.ncols) return;
    float2* W = reinterpret_cast<float2*>(smem_raw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int liw = LN::line(lane), t = LN::pos(lane);
    float2* scr = W + N2 + (warp * LPW + liw) * ScratchSpacing<float, N2>::value;
    for (int i = threadIdx.x; i < N2; i += blockDim.x) W[i] = tw2[i];
    __syncthreads();
    const int c = (blockIdx.x * kZWarps + warp) * LPW + liw;
    const bool act = c < g.ncols;
    float2 v[E2];
#pragma unroll
    for (int e = 0; e < E2; ++e)
        v[e] = act ? J.colbuf[colbuf_index(g, b, F::in_index(t, e), c)] : make_float2(0.f, 0.f);
    F::run(v, t, scr, W);
    if (act) {
        const int q0 = g.col_start[c];
        const int cnt = g.col_start[c + 1] - q0;
        const int z0 = g.pw_z[q0];
#pragma unroll
        for (int e = 0; e < E2; ++e) {
            const int off = wrapn<N2>(F::out_index(t, e) - z0);
            if (off < cnt) {
                const int q = q0 + off;
                const float2 cq = J.C[(size_t)b * J.ldc + q];
                const float kq = J.kin[q];
                J.HC[(size_t)b * J.ldhc + q] =
                    make_float2(omega * (kq * cq.x + scale * v[e].x), omega * (kq * cq.y + scale * v[e].y));
            }
        }
    }
}

// Line shapes per compiled length: E values per lane and the radix list.
template <int N> struct FastCfg;
template <> struct FastCfg<12> { static constexpr int E = 12; using R = Rad<4, 3>; };
template <> struct FastCfg<16> { static constexpr int E = 16; using R = Rad<16>; };
template <> struct FastCfg<40> { static constexpr int E = 20; using R = Rad<2, 4, 5>; };
template <> struct FastCfg<48> { static constexpr int E = 12; using R = Rad<4, 4, 3>; };
template <> struct FastCfg<64> { static constexpr int E = 8; using R = Rad<8, 8>; };
template <> struct FastCfg<80> { static constexpr int E = 20; using R = Rad<4, 4, 5>; };
template <> struct FastCfg<128> { static constexpr int E = 16; using R = Rad<16, 8>; };
template <> struct FastCfg<256> { static constexpr int E = 16; using R = Rad<16, 16>; };

constexpr size_t kFastMaxSmem = 220 * 1024;

template <int N0, int N1>
static size_t fast_smem(const ChainGeom& g, size_t elem, int nw = kFastWarps) {
    constexpr int E0 = FastCfg<N0>::E, E1 = FastCfg<N1>::E;
    const bool dbl = elem == sizeof(double2);
    const int lsA = dbl ? PlaneStride<double, N0, N1>::value : PlaneStride<float, N0, N1>::value;
    const int scr = dbl ? warp_scratch<double, N0, E0, N1, E1>() : warp_scratch<float, N0, E0, N1, E1>();
    return ((size_t)N0 + N1 + (size_t)nw * scr + (size_t)g.nrows * lsA) * elem;
}

// Warps of a density block: enough that the per-lane accumulators of the
// plane (N0 N1 / (32 warps) values) stay at 32 or fewer where the shared
// memory allows (16 warps for 128 x 128), else the 8 of the apply kernel.
template <int N0, int N1>
struct DensityWarps {
    static constexpr int value = (N0 * N1 > 8192 && N0 <= 128) ? 16 : kFastWarps;
};

static bool fast_disabled() {
    const char* e = getenv("JDFT_FAST_PLANE");
    return e && e[0] == '0';
}

template <typename T, int N0, int N1>
static jdft_status apply_fast_impl(const ChainGeom& g, c_t<T>* colbuf, const T* Vp, int nb, const c_t<T>* tw_base,
                                   cudaStream_t st) {
    using C0 = FastCfg<N0>;
    using C1 = FastCfg<N1>;
    const size_t smem = fast_smem<N0, N1>(g, sizeof(c_t<T>));
    if (smem > kFastMaxSmem) return JDFT_ERR_UNSUPPORTED;
    auto kern = plane_apply_fast_kernel<T, N0, C0::E, typename C0::R, N1, C1::E, typename C1::R>;
    cudaError_t e = set_smem_attr((const void*)kern, smem);
    if (e != cudaSuccess) return set_error(JDFT_ERR_CUDA, std::string("plane_apply_fast: ") + cudaGetErrorString(e));
    {
        Trace tr_("plane_apply_fast", st);
        kern<<<dim3(g.S2, nb), kFastThreads, smem, st>>>(g, colbuf, Vp, tw_base + g.p0.tw_offset,
                                                         tw_base + g.p1.tw_offset);
    }
    return check_launch("plane_apply_fast");
}

template <int N0, int N1>
static jdft_status density_fast_impl(const ChainGeom& g, const float2* colbuf, const double* f, double w, double* n_r,
                                     int nb, const float2* tw_base, cudaStream_t st) {
    using C0 = FastCfg<N0>;
    using C1 = FastCfg<N1>;
    constexpr int NW = DensityWarps<N0, N1>::value;
    const size_t smem = fast_smem<N0, N1>(g, sizeof(float2), NW);
    if (smem > kFastMaxSmem) return JDFT_ERR_UNSUPPORTED;
    auto kern = plane_density_fast_kernel<N0, C0::E, typename C0::R, N1, C1::E, typename C1::R, NW>;
    cudaError_t e = set_smem_attr((const void*)kern, smem);
    if (e != cudaSuccess)
        return set_error(JDFT_ERR_CUDA, std::string("plane_density_fast: ") + cudaGetErrorString(e));
    // band groups so that the grid covers the GPU about four blocks deep
    int groups = std::max(1, std::min(nb, (4 * 152 + g.S2 - 1) / g.S2));
    const int per = (nb + groups - 1) / groups;
    groups = (nb + per - 1) / per;
    {
        Trace tr_("plane_density_fast", st);
        kern<<<dim3(g.S2, groups), 32 * NW, smem, st>>>(g, colbuf, nb, per, f, w, n_r, tw_base + g.p0.tw_offset,
                                                        tw_base + g.p1.tw_offset);
    }
    return check_launch("plane_density_fast");
}

template <typename T, int N2>
static size_t zpass_fast_smem() {
    constexpr int LPW = Lanes<N2, FastCfg<N2>::E>::LPW;
    return ((size_t)N2 + (size_t)kZWarps * LPW * ScratchSpacing<T, N2>::value) * sizeof(c_t<T>);
}

template <int N2>
static int zpass_fast_blocks(const ChainGeom& g) {
    constexpr int TL = N2 / FastCfg<N2>::E, LPW = 32 / TL;
    return (g.ncols + kZWarps * LPW - 1) / (kZWarps * LPW);
}

template <typename T, int N2>
static jdft_status zinv_fast_impl(const ChainGeom& g, const c_t<T>* C, int ldc, c_t<T>* colbuf, int nb,
                                  const c_t<T>* tw2, cudaStream_t st) {
    using C2 = FastCfg<N2>;
    auto kern = zpass_inverse_fast_kernel<T, N2, C2::E, typename C2::R>;
    const size_t smem = zpass_fast_smem<T, N2>();
    cudaError_t e = set_smem_attr((const void*)kern, smem);
    if (e != cudaSuccess) return set_error(JDFT_ERR_CUDA, std::string("zpass_inverse_fast: ") + cudaGetErrorString(e));
    {
        Trace tr_("zpass_inverse", st);
        kern<<<dim3(zpass_fast_blocks<N2>(g), nb), kZThreads, smem, st>>>(g, C, ldc, colbuf, tw2);
    }
    return check_launch("zpass_inverse_fast");
}

template <typename T, int MODE, int N2>
static jdft_status zfwd_fast_impl(const ChainGeom& g, const c_t<T>* colbuf, const c_t<T>* C, int ldc, c_t<T>* out,
                                  int ldo, int nb, const T* kin, T omega, T scale, const c_t<T>* tw2,
                                  cudaStream_t st) {
    using C2 = FastCfg<N2>;
    auto kern = zpass_forward_fast_kernel<T, N2, C2::E, typename C2::R, MODE>;
    const size_t smem = zpass_fast_smem<T, N2>();
    cudaError_t e = set_smem_attr((const void*)kern, smem);
    if (e != cudaSuccess) return set_error(JDFT_ERR_CUDA, std::string("zpass_forward_fast: ") + cudaGetErrorString(e));
    {
        Trace tr_("zpass_forward", st);
        kern<<<dim3(zpass_fast_blocks<N2>(g), nb), kZThreads, smem, st>>>(g, colbuf, C, ldc, out, ldo, kin, omega,
                                                                            scale, tw2);
    }
    return check_launch("zpass_forward_fast");
}

// Shared memory requested per fused block: at least 58 KB, so that no more
// than three blocks share an SM and their tensor-memory sums (128 columns
// each) fit in its 512 columns.
template <int N0, int N1>
static jdft_status apply_density_fast_impl(const ChainGeom& g, float2* colbuf, const float* Vp, int nb,
                                           const double* f, double w, double* n_r, const float2* tw_base,
                                           cudaStream_t st) {
    using C0 = FastCfg<N0>;
    using C1 = FastCfg<N1>;
    const size_t smem = std::max<size_t>(fast_smem<N0, N1>(g, sizeof(float2)), 58 * 1024);
    if (smem > kFastMaxSmem) return JDFT_ERR_UNSUPPORTED;
    auto kern = plane_apply_density_fast_kernel<N0, C0::E, typename C0::R, N1, C1::E, typename C1::R>;
    cudaError_t e = set_smem_attr((const void*)kern, smem);
    if (e != cudaSuccess)
        return set_error(JDFT_ERR_CUDA, std::string("plane_apply_density_fast: ") + cudaGetErrorString(e));
    const int64_t items = (int64_t)g.S2 * nb;
    // resident blocks per SM from the footprint: __launch_bounds__(256, 2)
    // holds registers to 128 a thread, so shared memory decides (228 KB per
    // SM, 1 KB of it reserved per block)
    const int resident = std::max(1, std::min(3, (int)((228u * 1024u) / (smem + 1024u))));
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int grid = (int)std::min<int64_t>(items, (int64_t)std::max(1, sms) * resident);
    {
        Trace tr_("plane_apply_density_fast", st);
        kern<<<grid, kFastThreads, smem, st>>>(g, colbuf, Vp, nb, f, w, n_r, tw_base + g.p0.tw_offset,
                                               tw_base + g.p1.tw_offset);
    }
    return check_launch("plane_apply_density_fast");
}

jdft_status launch_plane_apply_density_fast(const ChainGeom& g, float2* colbuf, const float* Vp, int nb,
                                            const double* f, double w, double* n_r, const float2* tw_base,
                                            cudaStream_t st) {
    if (fast_disabled()) return JDFT_ERR_UNSUPPORTED;
    if (g.S0 == 128 && g.S1 == 128) return apply_density_fast_impl<128, 128>(g, colbuf, Vp, nb, f, w, n_r, tw_base, st);
    if (g.S0 == 16 && g.S1 == 12) return apply_density_fast_impl<16, 12>(g, colbuf, Vp, nb, f, w, n_r, tw_base, st);
    return JDFT_ERR_UNSUPPORTED;
}

#define JDFT_FAST_LENGTHS(X) X(12) X(16) X(40) X(48) X(64) X(80) X(128) X(256)

template <typename T>
jdft_status launch_zpass_inverse_fast(const ChainGeom& g, const c_t<T>* C, int ldc, c_t<T>* colbuf, int nb,
                                      const c_t<T>* tw2, cudaStream_t st) {
    if (fast_disabled()) return JDFT_ERR_UNSUPPORTED;
#define JDFT_CASE(a) \
    if (g.S2 == a) return zinv_fast_impl<T, a>(g, C, ldc, colbuf, nb, tw2, st);
    JDFT_FAST_LENGTHS(JDFT_CASE)
#undef JDFT_CASE
    return JDFT_ERR_UNSUPPORTED;
}

template <typename T, int MODE>
jdft_status launch_zpass_forward_fast(const ChainGeom& g, const c_t<T>* colbuf, const c_t<T>* C, int ldc, c_t<T>* out,
                                      int ldo, int nb, const T* kin, T omega, T scale, const c_t<T>* tw2,
                                      cudaStream_t st) {
    if (fast_disabled()) return JDFT_ERR_UNSUPPORTED;
#define JDFT_CASE(a) \
    if (g.S2 == a) return zfwd_fast_impl<T, MODE, a>(g, colbuf, C, ldc, out, ldo, nb, kin, omega, scale, tw2, st);
    JDFT_FAST_LENGTHS(JDFT_CASE)
#undef JDFT_CASE
    return JDFT_ERR_UNSUPPORTED;
}

#define JDFT_ZFAST_INST(T)                                                                                         \
    template jdft_status launch_zpass_inverse_fast<T>(const ChainGeom&, const c_t<T>*, int, c_t<T>*, int,         \
                                                      const c_t<T>*, cudaStream_t);                               \
    template jdft_status launch_zpass_forward_fast<T, 0>(const ChainGeom&, const c_t<T>*, const c_t<T>*, int,     \
                                                         c_t<T>*, int, int, const T*, T, T, const c_t<T>*,        \
                                                         cudaStream_t);                                           \
    template jdft_status launch_zpass_forward_fast<T, 1>(const ChainGeom&, const c_t<T>*, const c_t<T>*, int,     \
                                                         c_t<T>*, int, int, const T*, T, T, const c_t<T>*,        \
                                                         cudaStream_t);
JDFT_ZFAST_INST(double)
JDFT_ZFAST_INST(float)
#undef JDFT_ZFAST_INST

#define JDFT_FAST_SHAPES(X) X(12, 12) X(16, 12) X(40, 40) X(48, 48) X(64, 64) X(80, 80) X(128, 128) X(256, 128)

template <typename T>
jdft_status launch_plane_apply_fast(const ChainGeom& g, c_t<T>* colbuf, const T* Vp, int nb, const c_t<T>* tw_base,
                                    cudaStream_t st) {
    if (fast_disabled()) return JDFT_ERR_UNSUPPORTED;
#define JDFT_CASE(a, b) \
    if (g.S0 == a && g.S1 == b) return apply_fast_impl<T, a, b>(g, colbuf, Vp, nb, tw_base, st);
    JDFT_FAST_SHAPES(JDFT_CASE)
#undef JDFT_CASE
    return JDFT_ERR_UNSUPPORTED;
}

jdft_status launch_plane_density_fast(const ChainGeom& g, const float2* colbuf, const double* f, double w,
                                      double* n_r, int nb, const float2* tw_base, cudaStream_t st) {
    if (fast_disabled()) return JDFT_ERR_UNSUPPORTED;
#define JDFT_CASE(a, b) \
    if (g.S0 == a && g.S1 == b) return density_fast_impl<a, b>(g, colbuf, f, w, n_r, nb, tw_base, st);
    JDFT_FAST_SHAPES(JDFT_CASE)
#undef JDFT_CASE
    return JDFT_ERR_UNSUPPORTED;
}

template jdft_status launch_plane_apply_fast<double>(const ChainGeom&, double2*, const double*, int, const double2*,
                                                     cudaStream_t);
template jdft_status launch_plane_apply_fast<float>(const ChainGeom&, float2*, const float*, int, const float2*,
                                                    cudaStream_t);

jdft_status launch_zpass_inverse_batch(const ChainGeom& g, const KJob* jobs, int njobs, int max_ncols, int max_nb,
                                       const float2* tw2, cudaStream_t st) {
    if (fast_disabled()) return JDFT_ERR_UNSUPPORTED;
#define JDFT_CASE(a)                                                                                             \
    if (g.S2 == a) {                                                                                             \
        using C2 = FastCfg<a>;                                                                                   \
        auto kern = zpass_inverse_batch_kernel<a, C2::E, typename C2::R>;                                        \
        const size_t smem = zpass_fast_smem<float, a>();                                                         \
        cudaError_t e = set_smem_attr((const void*)kern, smem);                                                  \
        if (e != cudaSuccess) return set_error(JDFT_ERR_CUDA, std::string("zpass_inverse_batch: ") + cudaGetErrorString(e)); \
        constexpr int CPB = kZWarps * (32 / (a / C2::E));                                                     \
        Trace tr_("zpass_inverse_batch", st);                                                                    \
        kern<<<dim3((max_ncols + CPB - 1) / CPB, max_nb, njobs), kZThreads, smem, st>>>(jobs, tw2);           \
        return check_launch("zpass_inverse_batch");                                                              \
    }
    JDFT_FAST_LENGTHS(JDFT_CASE)
#undef JDFT_CASE
    return JDFT_ERR_UNSUPPORTED;
}

jdft_status launch_zpass_forward_batch(const ChainGeom& g, const KJob* jobs, int njobs, int max_ncols, int max_nb,
                                       float omega, float scale, const float2* tw2, cudaStream_t st) {
    if (fast_disabled()) return JDFT_ERR_UNSUPPORTED;
#define JDFT_CASE(a)                                                                                             \
    if (g.S2 == a) {                                                                                             \
        using C2 = FastCfg<a>;                                                                                   \
        auto kern = zpass_forward_batch_kernel<a, C2::E, typename C2::R>;                                        \
        const size_t smem = zpass_fast_smem<float, a>();                                                         \
        cudaError_t e = set_smem_attr((const void*)kern, smem);                                                  \
        if (e != cudaSuccess) return set_error(JDFT_ERR_CUDA, std::string("zpass_forward_batch: ") + cudaGetErrorString(e)); \
        constexpr int CPB = kZWarps * (32 / (a / C2::E));                                                     \
        Trace tr_("zpass_forward_batch", st);                                                                    \
        kern<<<dim3((max_ncols + CPB - 1) / CPB, max_nb, njobs), kZThreads, smem, st>>>(jobs, omega, scale, tw2); \
        return check_launch("zpass_forward_batch");                                                              \
    }
    JDFT_FAST_LENGTHS(JDFT_CASE)
#undef JDFT_CASE
    return JDFT_ERR_UNSUPPORTED;
}

}  // namespace jdft
