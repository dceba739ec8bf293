// Hamiltonian plane pass and density of FP32 blocks, two bands at a time with
// packed FP32 arithmetic (fft_pair.cuh).
//
// The work items are (z-plane j2, band pair p): bands 2p and 2p + 1 share
// every index computation, every twiddle and every potential value, and each
// arithmetic instruction of their transforms is issued once, two-wide.  A
// persistent block takes a contiguous, balanced range of the plane-major item
// list and, per item:
//   1. rows: inverse transform along axis 1 of the nrows i0-rows the sphere
//      touches, read from both bands' disk columns, into the shared plane A
//      (one 16-byte entry (Re_0, Re_1, Im_0, Im_1) per point);
//   2. columns: for every j1, inverse transform along axis 0, add
//      f_0 |psi_0|^2 + f_1 |psi_1|^2 to FP32 sums held in tensor memory,
//      multiply by V(j0, j1, j2), forward transform (as the adjoint of the
//      inverse), keep the nrows sphere slots;
//   3. rows: forward transform along axis 1, gather the disk values back.
// The density sums go to n(r) with FP64 atomics when the block's plane
// changes and at the end.  (JDFTx paper, Sec. 2.1: the I, multiply, J chain of
// Listing 1 on temporaries, and the density of ElecVars, Sec. 2.1.)
#include <algorithm>
#include <cstdlib>
#include <vector>

#include "chain.cuh"
#include "fft_pair.cuh"
#include "profile.cuh"
#include "tc_ptx.cuh"

namespace jdft {

// i mod N in [0, N) for either sign of i.
template <int N>
__device__ __forceinline__ int pwrap(int i) {
    if constexpr ((N & (N - 1)) == 0) {
        return i & (N - 1);
    } else {
        const int r = i % N;
        return r < 0 ? r + N : r;
    }
}

// Lane roles as in the one-band kernels: a line of N values over TL = N / E
// lanes, LPW = 32 / TL lines per warp, lane l at position l / LPW of line
// l % LPW.
template <int N, int E>
struct PLanes {
    static constexpr int TL = N / E, LPW = 32 / TL;
    static __device__ __forceinline__ int line(int lane) { return lane % LPW; }
    static __device__ __forceinline__ int pos(int lane) { return lane / LPW; }
};

// Row stride of the pair plane A, in 16-byte entries.  In the column pass a
// quarter-warp (8 lanes, one 16-byte wavefront) reads 4 consecutive columns
// of 2 consecutive rows; a stride of 4 (mod 8) puts them in 8 distinct bank
// slots.
template <int N1>
struct PairStride {
    static constexpr int value = N1 + (12 - N1 % 8) % 8;  // smallest value >= N1 that is 4 (mod 8)
};

// Scratch line spacing (float2 elements) per length: the values of the
// one-band kernels, whose 8-byte accesses these exchanges repeat.
template <int N>
struct PScratch;
template <> struct PScratch<12> { static constexpr int value = 13; };
template <> struct PScratch<16> { static constexpr int value = 17; };
template <> struct PScratch<128> { static constexpr int value = 140; };

template <int N0, int E0, int N1, int E1>
__host__ __device__ constexpr int pair_warp_scratch() {
    return PLanes<N0, E0>::LPW * PScratch<N0>::value > PLanes<N1, E1>::LPW * PScratch<N1>::value
               ? PLanes<N0, E0>::LPW * PScratch<N0>::value
               : PLanes<N1, E1>::LPW * PScratch<N1>::value;
}

__device__ __forceinline__ cpair ld_pair(const ulonglong2* p) {
    const ulonglong2 q = *p;
    return {f2x{q.x}, f2x{q.y}};
}
__device__ __forceinline__ void st_pair(ulonglong2* p, cpair v) { *p = make_ulonglong2(v.x.v, v.y.v); }

// Rows pass, inverse: row r of both bands' disk values -> A[r][.].
template <int N1, int E1, class R1, int NW, bool WIN>
__device__ __forceinline__ void prows_inverse(const ChainGeom& g, const float2* __restrict__ p0,
                                              const float2* __restrict__ p1, ulonglong2* A, int lsA, float2* wscr,
                                              const float4* W1, int warp, int lane) {
    using F = LineFFTP<N1, E1, +1, R1, WIN>;
    using LN = PLanes<N1, E1>;
    constexpr int LPW = LN::LPW;
    const int liw = LN::line(lane), t = LN::pos(lane);
    float2* scr = wscr + liw * PScratch<N1>::value;
    for (int base = warp * LPW; base < g.nrows; base += NW * LPW) {
        const int r = base + liw;
        const bool act = r < g.nrows;
        int cs = 0, cnt = 0, lo = 0;
        if (act) {
            cs = g.row_col_start[r];
            cnt = g.row_col_start[r + 1] - cs;
            lo = g.row_i1lo[r];
        }
        cpair v[E1];
#pragma unroll
        for (int e = 0; e < E1; ++e) {
            const int off = pwrap<N1>(F::in_index(t, e) - lo);
            if (F::in_window(e) && off < cnt) {
                const float2 a = p0[cs + off], b = p1[cs + off];
                v[e] = {p_pack(a.x, b.x), p_pack(a.y, b.y)};
            } else {
                v[e] = cp_zero();
            }
        }
        F::run(v, t, scr, W1);
        if (act) {
#pragma unroll
            for (int e = 0; e < E1; ++e) st_pair(A + r * lsA + F::out_index(t, e), v[e]);
        }
    }
}

// Rows pass, forward: A[r][.] -> both bands' disk values of row r.  The
// transform runs as the adjoint of the inverse flow graph, so that with WIN
// its last stage is the pruned one.
template <int N1, int E1, class R1, int NW, bool WIN>
__device__ __forceinline__ void prows_forward(const ChainGeom& g, float2* __restrict__ p0, float2* __restrict__ p1,
                                              bool have1, const ulonglong2* A, int lsA, float2* wscr,
                                              const float4* W1, int warp, int lane) {
    using F = LineFFTP<N1, E1, +1, R1, WIN>;
    using LN = PLanes<N1, E1>;
    constexpr int LPW = LN::LPW;
    const int liw = LN::line(lane), t = LN::pos(lane);
    float2* scr = wscr + liw * PScratch<N1>::value;
    for (int base = warp * LPW; base < g.nrows; base += NW * LPW) {
        const int r = base + liw;
        const bool act = r < g.nrows;
        cpair v[E1];
#pragma unroll
        for (int e = 0; e < E1; ++e) v[e] = act ? ld_pair(A + r * lsA + F::out_index(t, e)) : cp_zero();
        F::run_adjoint(v, t, scr, W1);
        if (act) {
            const int cs = g.row_col_start[r];
            const int cnt = g.row_col_start[r + 1] - cs;
            const int lo = g.row_i1lo[r];
#pragma unroll
            for (int e = 0; e < E1; ++e) {
                const int off = pwrap<N1>(F::in_index(t, e) - lo);
                if (F::in_window(e) && off < cnt) {
                    float x0, x1, y0, y1;
                    p_unpack(v[e].x, x0, x1);
                    p_unpack(v[e].y, y0, y1);
                    p0[cs + off] = make_float2(x0, y0);
                    if (have1) p1[cs + off] = make_float2(x1, y1);
                }
            }
        }
    }
}

template <int N0, int E0, class R0, int N1, int E1, class R1, int NW>
struct PairPlane {
    static constexpr int lsA = PairStride<N1>::value;
    static constexpr int SCR = pair_warp_scratch<N0, E0, N1, E1>();  // float2 per warp
    static constexpr int LPW = PLanes<N0, E0>::LPW;
    static constexpr int ROUNDS = (N1 + NW * LPW - 1) / (NW * LPW);
    static constexpr int GROUPS = NW / 4;
    static constexpr int TM_USED = GROUPS * ROUNDS * 16;
    static constexpr uint32_t TM_COLS = TM_USED <= 32 ? 32 : TM_USED <= 64 ? 64 : TM_USED <= 128 ? 128 : 256;
    static_assert(NW % 4 == 0, "whole warp quadrants");
    static_assert(E0 == 16, "the tensor-memory sums take 16 values per lane and round");
    static_assert((NW * SCR) % 2 == 0, "the plane array starts on a 16-byte boundary");
    static size_t smem(int nrows) {
        return (size_t)(N0 + N1) * sizeof(float4) + (size_t)NW * SCR * sizeof(float2) +
               (size_t)nrows * lsA * sizeof(ulonglong2);
    }
};

// One (z-plane j2, band pair b0, b0 + 1) item of the plane pass: rows
// inverse, columns (inverse, density sums, x V, forward), rows forward, with a
// block barrier after each phase.  g: the item's sphere maps; colbuf: its
// column buffer of nb bands.
// SPIN: the pair is one spinor band's (up, down) components and the potential
// is V 1 + M . sigma, M's three fields in Mp (each in Vp's permuted layout).
template <int N0, int E0, class R0, int N1, int E1, class R1, int NW, bool DENS, bool WIN, bool SPIN = false>
__device__ __forceinline__ void pair_item(const ChainGeom& g, float2* __restrict__ colbuf, int nb,
                                          const double* __restrict__ f, const float* __restrict__ Vp, int j2, int b0,
                                          const float4* W0, const float4* W1, float2* wscr, float2* scr,
                                          ulonglong2* A, uint32_t tb, int warp, int lane,
                                          const float* __restrict__ Mp = nullptr) {
    using PP = PairPlane<N0, E0, R0, N1, E1, R1, NW>;
    using FI = LineFFTP<N0, E0, +1, R0, WIN>;
    using LN = PLanes<N0, E0>;
    constexpr int LPW = LN::LPW, ROUNDS = PP::ROUNDS, lsA = PP::lsA;
    constexpr bool kAllCols = N1 % (NW * LPW) == 0;
    const int liw = LN::line(lane), t = LN::pos(lane);
    const bool have1 = b0 + 1 < nb;
    float2* plane0 = colbuf + colbuf_index(g, b0, j2, 0);
    // a missing second band reads the first band's values and is never written
    float2* plane1 = have1 ? colbuf + colbuf_index(g, b0 + 1, j2, 0) : plane0;
    prows_inverse<N1, E1, R1, NW, WIN>(g, plane0, plane1, A, lsA, wscr, W1, warp, lane);
    __syncthreads();
    const f2x fb = DENS ? p_pack((float)f[b0], have1 ? (float)f[b0 + 1] : 0.f) : p_zero();
    // rolled: copies of the two column transforms would overflow the instruction cache
#pragma unroll 1
    for (int k = 0; k < ROUNDS; ++k) {
        const int j1 = warp * LPW + liw + k * NW * LPW;
        const bool act = kAllCols || j1 < N1;
        // this round's sums are fetched while the column transform runs
        uint32_t sr[16];
        if constexpr (DENS) tc::tmem_ld16_issue(tb + 16 * k, sr);
        cpair v[E0];
#pragma unroll
        for (int e = 0; e < E0; ++e) {
            const int r = pwrap<N0>(FI::in_index(t, e) - g.i0min);
            v[e] = (FI::in_window(e) && act && r < g.nrows) ? ld_pair(A + r * lsA + j1) : cp_zero();
        }
        FI::run(v, t, scr, W0);
        if constexpr (DENS) {
            tc::tmem_wait_ld16(sr);
            float acc[16];
#pragma unroll
            for (int e = 0; e < E0; ++e) {
                // (f_0 |psi_0|^2, f_1 |psi_1|^2), folded into one sum
                const f2x d = p_mul(p_fma(v[e].y, v[e].y, p_mul(v[e].x, v[e].x)), fb);
                float d0, d1;
                p_unpack(d, d0, d1);
                acc[e] = __uint_as_float(sr[e]) + d0 + d1;
            }
            tc::tmem_st16(tb + 16 * k, acc);
        }
        const float* Vq = Vp + ((size_t)j2 * N1 + (act ? j1 : 0)) * N0;
        if constexpr (SPIN) {
            // (up, down) <- [[V + M_z, M_x - i M_y], [M_x + i M_y, V - M_z]] (up, down)
            const size_t nbox = (size_t)g.S2 * N1 * N0;
            const float* Mq = Mp + ((size_t)j2 * N1 + (act ? j1 : 0)) * N0;
#pragma unroll
            for (int e = 0; e < E0; ++e) {
                const int o = FI::out_index(t, e);
                const float V = Vq[o], mx = Mq[o], my = Mq[nbox + o], mz = Mq[2 * nbox + o];
                float ru, rd, iu, id;
                p_unpack(v[e].x, ru, rd);
                p_unpack(v[e].y, iu, id);
                const float pru = (V + mz) * ru + mx * rd + my * id;
                const float piu = (V + mz) * iu + mx * id - my * rd;
                const float prd = (V - mz) * rd + mx * ru - my * iu;
                const float pid = (V - mz) * id + mx * iu + my * ru;
                v[e] = act ? cpair{p_pack(pru, prd), p_pack(piu, pid)} : cp_zero();
            }
        } else {
#pragma unroll
            for (int e = 0; e < E0; ++e) v[e] = act ? cp_scale(v[e], p_dup(Vq[FI::out_index(t, e)])) : cp_zero();
        }
        FI::run_adjoint(v, t, scr, W0);
        if (act) {
#pragma unroll
            for (int e = 0; e < E0; ++e) {
                const int r = pwrap<N0>(FI::in_index(t, e) - g.i0min);
                if (FI::in_window(e) && r < g.nrows) st_pair(A + r * lsA + j1, v[e]);
            }
        }
    }
    if constexpr (DENS) tc::tmem_wait_st();
    __syncthreads();
    prows_forward<N1, E1, R1, NW, WIN>(g, plane0, plane1, have1, A, lsA, wscr, W1, warp, lane);
    __syncthreads();
}

// DENS = false: the plane pass alone (no density, no tensor memory).  WIN:
// the sphere lies in the central quarter of the box along axes 0 and 1
// (LineFFTP's window), so the transforms prune their first-stage butterflies
// and the loads and stores outside it are skipped.
template <int N0, int E0, class R0, int N1, int E1, class R1, int NW, bool DENS, bool WIN, bool SPIN = false>
__global__ void __launch_bounds__(32 * NW, 1) plane_apply_density_pair_kernel(
    ChainGeom g, float2* __restrict__ colbuf, const float* __restrict__ Vp, int nb, const double* __restrict__ f,
    double w, double* __restrict__ n_r, const float2* __restrict__ tw0, const float2* __restrict__ tw1,
    const float* __restrict__ Mp) {
    using PP = PairPlane<N0, E0, R0, N1, E1, R1, NW>;
    using FI = LineFFTP<N0, E0, +1, R0, WIN>;
    using LN = PLanes<N0, E0>;
    constexpr int LPW = LN::LPW, ROUNDS = PP::ROUNDS;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ uint32_t tslot;
    float4* W0 = reinterpret_cast<float4*>(smem_raw);
    float4* W1 = W0 + N0;
    float2* scr_all = reinterpret_cast<float2*>(W1 + N1);
    ulonglong2* A = reinterpret_cast<ulonglong2*>(scr_all + NW * PP::SCR);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int liw = LN::line(lane), t = LN::pos(lane);
    float2* wscr = scr_all + warp * PP::SCR;
    float2* scr = wscr + liw * PScratch<N0>::value;
    for (int i = threadIdx.x; i < N0; i += blockDim.x) W0[i] = make_float4(tw0[i].x, tw0[i].x, tw0[i].y, tw0[i].y);
    for (int i = threadIdx.x; i < N1; i += blockDim.x) W1[i] = make_float4(tw1[i].x, tw1[i].x, tw1[i].y, tw1[i].y);
    if (DENS && warp == 0) tc::tmem_alloc(&tslot, PP::TM_COLS);
    tc::tc_fence_before_sync();
    __syncthreads();
    tc::tc_fence_after_sync();
    // this warp's tensor-memory lanes (quadrant warp % 4) and column group
    const uint32_t tb = tslot + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)((warp >> 2) * ROUNDS * 16);
    const int np = (nb + 1) / 2;
    const int64_t items = (int64_t)g.S2 * np;
    const int64_t it0 = items * blockIdx.x / gridDim.x, it1 = items * (blockIdx.x + 1) / gridDim.x;
    auto flush = [&](int j2) {
#pragma unroll 1
        for (int k = 0; k < ROUNDS; ++k) {
            float acc[16];
            tc::tmem_ld16(tb + 16 * k, acc);
            const int j1 = warp * LPW + liw + k * NW * LPW;
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
        const int j2 = (int)(it / np), p = (int)(it - (int64_t)j2 * np);
        if (DENS && j2 != cur) {
            if (cur >= 0) flush(cur);
            zero();
            cur = j2;
        }
        pair_item<N0, E0, R0, N1, E1, R1, NW, DENS, WIN, SPIN>(g, colbuf, nb, f, Vp, j2, 2 * p, W0, W1, wscr, scr, A,
                                                                tb, warp, lane, Mp);
    }
    if (DENS && cur >= 0) flush(cur);
    tc::tc_fence_before_sync();
    __syncthreads();
    if (DENS && warp == 0) tc::tmem_dealloc(tslot, PP::TM_COLS);
}

// The plane pass (no density) over the items of several k-points (or cells
// on the same box) in one persistent launch: the batch's item list is the
// concatenation of each job's (plane, band pair) items, jobs[k].item0 its
// first item.  A block takes a contiguous range of the list and copies the
// current job's description to shared memory whenever its range crosses
// into the next job.
template <int N0, int E0, class R0, int N1, int E1, class R1, int NW, bool WIN>
__global__ void __launch_bounds__(32 * NW, 1) plane_apply_pair_batch_kernel(const KJob* __restrict__ jobs, int njobs,
                                                                            int64_t items, const float* __restrict__ Vp,
                                                                            const float2* __restrict__ tw0,
                                                                            const float2* __restrict__ tw1) {
    using PP = PairPlane<N0, E0, R0, N1, E1, R1, NW>;
    using LN = PLanes<N0, E0>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ KJob sj;
    __shared__ int sk;
    float4* W0 = reinterpret_cast<float4*>(smem_raw);
    float4* W1 = W0 + N0;
    float2* scr_all = reinterpret_cast<float2*>(W1 + N1);
    ulonglong2* A = reinterpret_cast<ulonglong2*>(scr_all + NW * PP::SCR);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int liw = LN::line(lane);
    float2* wscr = scr_all + warp * PP::SCR;
    float2* scr = wscr + liw * PScratch<N0>::value;
    for (int i = threadIdx.x; i < N0; i += blockDim.x) W0[i] = make_float4(tw0[i].x, tw0[i].x, tw0[i].y, tw0[i].y);
    for (int i = threadIdx.x; i < N1; i += blockDim.x) W1[i] = make_float4(tw1[i].x, tw1[i].x, tw1[i].y, tw1[i].y);
    if (threadIdx.x == 0) sk = -1;
    __syncthreads();
    const int64_t it0 = items * blockIdx.x / gridDim.x, it1 = items * (blockIdx.x + 1) / gridDim.x;
    int64_t next = -1;  // first item of the job after the current one (-1: no job loaded yet)
    for (int64_t it = it0; it < it1; ++it) {
        if (next < 0 || it >= next) {
            // every thread is past the previous item's last barrier
            if (threadIdx.x == 0) {
                int k = sk < 0 ? 0 : sk;
                while (k + 1 < njobs && jobs[k + 1].item0 <= it) ++k;
                sk = k;
                sj = jobs[k];
            }
            __syncthreads();
            next = sk + 1 < njobs ? jobs[sk + 1].item0 : items;
        }
        const int64_t local = it - sj.item0;
        const int np = (sj.nb + 1) / 2;
        const int j2 = (int)(local / np), p = (int)(local - (int64_t)j2 * np);
        pair_item<N0, E0, R0, N1, E1, R1, NW, false, WIN>(sj.g, sj.colbuf, sj.nb, nullptr, Vp, j2, 2 * p, W0, W1,
                                                           wscr, scr, A, 0u, warp, lane);
    }
}

template <class R> struct FirstRadix16 { static constexpr bool value = false; };
template <int... R> struct FirstRadix16<Rad<16, R...>> { static constexpr bool value = true; };

template <int N> struct PairCfg;
template <> struct PairCfg<12> { static constexpr int E = 12; using R = Rad<4, 3>; };
template <> struct PairCfg<16> { static constexpr int E = 16; using R = Rad<16>; };
template <> struct PairCfg<128> { static constexpr int E = 16; using R = Rad<16, 8>; };

constexpr int kPairWarps = 16;

static bool pair_disabled() {
    const char* e = getenv("JDFT_PAIR_PLANE");
    return e && e[0] == '0';
}

// Whether the sphere lies in LineFFTP's window along axes 0 and 1: signed
// indices -S/4 .. S/4 - 1 (and the axis transforms are radix-16 first with
// 16 values a lane).
template <int N0, int N1>
static bool pair_window(const ChainGeom& g) {
    using C0 = PairCfg<N0>;
    using C1 = PairCfg<N1>;
    if (!(C0::E == 16 && C1::E == 16 && FirstRadix16<typename C0::R>::value && FirstRadix16<typename C1::R>::value))
        return false;
    return g.i0min >= -N0 / 4 && g.i0min + g.nrows - 1 <= N0 / 4 - 1 && g.i1min >= -N1 / 4 && g.i1max <= N1 / 4 - 1;
}

template <int N0, int N1, bool DENS, bool WIN, bool SPIN = false>
static jdft_status pair_impl(const ChainGeom& g, float2* colbuf, const float* Vp, int nb, const double* f, double w,
                             double* n_r, const float2* tw_base, cudaStream_t st, const float* Mp = nullptr) {
    using C0 = PairCfg<N0>;
    using C1 = PairCfg<N1>;
    using PP = PairPlane<N0, C0::E, typename C0::R, N1, C1::E, typename C1::R, kPairWarps>;
    const char* name = SPIN ? "plane_apply_spinor_pair" : DENS ? "plane_apply_density_pair" : "plane_apply_pair";
    const size_t smem = PP::smem(g.nrows);
    if (smem > 227 * 1024) return JDFT_ERR_UNSUPPORTED;
    auto kern = plane_apply_density_pair_kernel<N0, C0::E, typename C0::R, N1, C1::E, typename C1::R, kPairWarps,
                                                DENS, WIN, SPIN>;
    cudaError_t e = set_smem_attr((const void*)kern, smem);
    if (e != cudaSuccess) return set_error(JDFT_ERR_CUDA, std::string(name) + ": " + cudaGetErrorString(e));
    const int64_t items = (int64_t)g.S2 * ((nb + 1) / 2);
    // resident blocks per SM: shared memory (228 KB, 1 KB reserved per
    // block), threads (2048), tensor-memory columns (512)
    int resident = (int)((228u * 1024u) / (smem + 1024u));
    resident = std::min(resident, 2048 / (32 * kPairWarps));
    if (DENS) resident = std::min(resident, (int)(512 / PP::TM_COLS));
    resident = std::max(1, resident);
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int grid = (int)std::min<int64_t>(items, (int64_t)std::max(1, sms - g.reserve_sms) * resident);
    {
        Trace tr_(name, st);
        kern<<<grid, 32 * kPairWarps, smem, st>>>(g, colbuf, Vp, nb, f, w, n_r, tw_base + g.p0.tw_offset,
                                                  tw_base + g.p1.tw_offset, Mp);
    }
    return check_launch(name);
}

jdft_status launch_plane_apply_density_pair(const ChainGeom& g, float2* colbuf, const float* Vp, int nb,
                                            const double* f, double w, double* n_r, const float2* tw_base,
                                            cudaStream_t st) {
    if (pair_disabled() || g.one_band) return JDFT_ERR_UNSUPPORTED;
    if (g.S0 == 128 && g.S1 == 128)
        return pair_window<128, 128>(g) ? pair_impl<128, 128, true, true>(g, colbuf, Vp, nb, f, w, n_r, tw_base, st)
                                        : pair_impl<128, 128, true, false>(g, colbuf, Vp, nb, f, w, n_r, tw_base, st);
    if (g.S0 == 16 && g.S1 == 12) return pair_impl<16, 12, true, false>(g, colbuf, Vp, nb, f, w, n_r, tw_base, st);
    return JDFT_ERR_UNSUPPORTED;
}

jdft_status launch_plane_apply_pair_spinor(const ChainGeom& g, float2* colbuf, const float* Vp, const float* Mp,
                                           int nb, const float2* tw_base, cudaStream_t st) {
    if (nb % 2) return set_error(JDFT_ERR_ARG, "spinor plane pass needs whole (up, down) pairs");
    if (g.S0 == 128 && g.S1 == 128)
        return pair_window<128, 128>(g)
                   ? pair_impl<128, 128, false, true, true>(g, colbuf, Vp, nb, nullptr, 0.0, nullptr, tw_base, st, Mp)
                   : pair_impl<128, 128, false, false, true>(g, colbuf, Vp, nb, nullptr, 0.0, nullptr, tw_base, st, Mp);
    if (g.S0 == 16 && g.S1 == 12)
        return pair_impl<16, 12, false, false, true>(g, colbuf, Vp, nb, nullptr, 0.0, nullptr, tw_base, st, Mp);
    return JDFT_ERR_UNSUPPORTED;
}

jdft_status launch_plane_apply_pair(const ChainGeom& g, float2* colbuf, const float* Vp, int nb,
                                    const float2* tw_base, cudaStream_t st) {
    if (pair_disabled() || g.one_band) return JDFT_ERR_UNSUPPORTED;
    if (g.S0 == 128 && g.S1 == 128)
        return pair_window<128, 128>(g)
                   ? pair_impl<128, 128, false, true>(g, colbuf, Vp, nb, nullptr, 0.0, nullptr, tw_base, st)
                   : pair_impl<128, 128, false, false>(g, colbuf, Vp, nb, nullptr, 0.0, nullptr, tw_base, st);
    if (g.S0 == 16 && g.S1 == 12)
        return pair_impl<16, 12, false, false>(g, colbuf, Vp, nb, nullptr, 0.0, nullptr, tw_base, st);
    return JDFT_ERR_UNSUPPORTED;
}

template <int N0, int N1, bool WIN>
static jdft_status pair_batch_impl(const ChainGeom& g, const KJob* jobs, int njobs, int64_t items, int nrows_max,
                                   const float* Vp, const float2* tw_base, cudaStream_t st) {
    using C0 = PairCfg<N0>;
    using C1 = PairCfg<N1>;
    using PP = PairPlane<N0, C0::E, typename C0::R, N1, C1::E, typename C1::R, kPairWarps>;
    const size_t smem = PP::smem(nrows_max);
    if (smem > 227 * 1024) return JDFT_ERR_UNSUPPORTED;
    auto kern = plane_apply_pair_batch_kernel<N0, C0::E, typename C0::R, N1, C1::E, typename C1::R, kPairWarps, WIN>;
    cudaError_t e = set_smem_attr((const void*)kern, smem);
    if (e != cudaSuccess)
        return set_error(JDFT_ERR_CUDA, std::string("plane_apply_pair_batch: ") + cudaGetErrorString(e));
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int resident = std::max(1, std::min((int)((228u * 1024u) / (smem + 1024u)), 2048 / (32 * kPairWarps)));
    const int grid = (int)std::min<int64_t>(items, (int64_t)std::max(1, sms) * resident);
    {
        Trace tr_("plane_apply_pair_batch", st);
        kern<<<grid, 32 * kPairWarps, smem, st>>>(jobs, njobs, items, Vp, tw_base + g.p0.tw_offset,
                                                  tw_base + g.p1.tw_offset);
    }
    return check_launch("plane_apply_pair_batch");
}

bool plane_pair_batch_supported(const ChainGeom& g) {
    return !pair_disabled() && !g.one_band && ((g.S0 == 128 && g.S1 == 128) || (g.S0 == 16 && g.S1 == 12));
}

jdft_status launch_plane_apply_pair_batch(const std::vector<ChainGeom>& gs, const KJob* jobs, int64_t items,
                                          const float* Vp, const float2* tw_base, cudaStream_t st) {
    if (gs.empty() || !plane_pair_batch_supported(gs[0])) return JDFT_ERR_UNSUPPORTED;
    const ChainGeom& g = gs[0];
    int nrows_max = 0;
    bool win = true;
    for (const ChainGeom& x : gs) {
        nrows_max = std::max(nrows_max, x.nrows);
        if (g.S0 == 128) win = win && pair_window<128, 128>(x);
    }
    const int nj = (int)gs.size();
    if (g.S0 == 128)
        return win ? pair_batch_impl<128, 128, true>(g, jobs, nj, items, nrows_max, Vp, tw_base, st)
                   : pair_batch_impl<128, 128, false>(g, jobs, nj, items, nrows_max, Vp, tw_base, st);
    return pair_batch_impl<16, 12, false>(g, jobs, nj, items, nrows_max, Vp, tw_base, st);
}

}  // namespace jdft
