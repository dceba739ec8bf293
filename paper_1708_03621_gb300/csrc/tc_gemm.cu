// Complex GEMMs on the 5th-generation tensor cores with 3-term TF32 splitting
// (x = hi + lo, both TF32; x y ~ hi_x hi_y + hi_x lo_y + lo_x hi_y, FP32
// accumulation in tensor memory): the projector products P^dag C and
// P (D P^dag C) of the nonlocal pseudopotential term (JDFTx paper, Sec. 2.2)
// and the subspace matrices C^dag H C, C^dag O C of the band minimiser
// (Sec. 2.1, Minimize).
//
// Complex products become real ones by doubling K with the interleaved
// (re, im) storage: for conj(a) b, Re = sum a'.b'_re and Im = sum a'.b'_im
// with a' = (ar, ai), b'_re = (br, bi), b'_im = (bi, -br); for a b,
// b'_re = (br, -bi), b'_im = (bi, br).  A block of 512 threads computes a
// 128 x NT tile (NT = 32, 128, or 256 for BF16 operands): all threads stage a
// 32-deep (real) K chunk of A' (hi, lo) and B'_re, B'_im (hi, lo) into shared
// memory in the no-swizzle K-major
// core-matrix layout, one elected thread issues the tcgen05.mma (M = 128,
// N = NT, K = 8 per instruction, 6 per K step) and commits them to an
// mbarrier; two stages let the staging of chunk c+1 overlap the products of
// chunk c.  Accumulators (Re at columns [0, NT), Im at [NT, 2 NT)) stay in
// tensor memory until the epilogue reads them with tcgen05.ld.  Every wait is
// bounded by a run-time limit (g_tc_wait_ns, set by jdft_set_wait_limit).  A
// wait that gives up records JDFT_ERR_TIMEOUT in a device flag (read by
// jdft_device_status) and stops issuing products; the block then waits, under
// a fixed limit of its own, for the products it has already committed, skips
// the epilogue and only then frees its tensor memory.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdlib>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "gemm.cuh"
#include "minimize.cuh"
#include "profile.cuh"
#include "tc_ptx.cuh"

namespace jdft {

constexpr int TC_M = 128;
constexpr int TC_CPS = 16;          // complex K elements per stage
constexpr int TC_THREADS = 512;
constexpr int TC_WARPS = TC_THREADS / 32;
// Limit of one wait for a batch of products (run-time, per device; 2 s by
// default), and the fixed limit of the drain after a wait gave up.
__device__ unsigned long long g_tc_wait_ns = 2000000000ull;
constexpr unsigned long long TC_DRAIN_NS = 2000000000ull;

__device__ int g_tc_status = 0;

// Operand format: FMT 0 = TF32 (4-byte elements, kind::tf32, K = 8 per
// instruction), FMT 1 = BF16 (2-byte elements, kind::f16, K = 16).  A stage
// row holds 2 * CPS real values (CPS = 16 complex): 8 (TF32) or 4 (BF16) 16-byte core
// columns; 8-row groups are SBO bytes apart (their core matrices plus 16, so
// consecutive groups start on different banks); each instruction covers two
// core columns, so a stage takes KSTEPS = KG / 2 instructions per product.
template <int FMT, int CPS = TC_CPS>
struct Fmt {
    static constexpr int ELEM = FMT ? 2 : 4;
    static constexpr int PER16 = 16 / ELEM;                 // elements per 16-byte core row
    static constexpr int KG = 2 * CPS / PER16;              // core columns per row
    static constexpr int SBO = KG * 128 + 16;
    static constexpr int KSTEPS = KG / 2;
    static constexpr uint32_t IDESC_FMT = FMT ? 1u : 2u;
};

template <int FMT, int CPS>
__device__ __forceinline__ uint32_t core_off(int row, int k) {
    using F = Fmt<FMT, CPS>;
    return (uint32_t)((row >> 3) * F::SBO + (k / F::PER16) * 128 + (row & 7) * 16 + (k % F::PER16) * F::ELEM);
}

template <int NT, int FMT, int CPS = TC_CPS>
struct TcLayout {
    static constexpr int A_BYTES = (TC_M / 8) * Fmt<FMT, CPS>::SBO;
    static constexpr int B_BYTES = (NT / 8) * Fmt<FMT, CPS>::SBO;
    static constexpr int A_HI = 0, A_LO = A_BYTES;
    static constexpr int BR_HI = 2 * A_BYTES, BR_LO = BR_HI + B_BYTES;
    static constexpr int BI_HI = BR_LO + B_BYTES, BI_LO = BI_HI + B_BYTES;
    static constexpr int STAGE = 2 * A_BYTES + 4 * B_BYTES;
    static constexpr int SMEM = 2 * STAGE + 64;
    static constexpr uint32_t NCOLS =
        (2 * NT <= 32) ? 32 : (2 * NT <= 64) ? 64 : (2 * NT <= 128) ? 128 : (2 * NT <= 256) ? 256 : 512;
};

// Store the hi and lo parts of the complex value (x, y) at (row, k2), k2 even.
template <int FMT, int CPS>
__device__ __forceinline__ void put_split(char* buf, int off_hi, int off_lo, int row, int k2, float x, float y) {
    const uint32_t o = core_off<FMT, CPS>(row, k2);
    if constexpr (FMT == 0) {
        const float hx = tc::to_tf32(x), hy = tc::to_tf32(y);
        const float lx = tc::to_tf32(x - hx), ly = tc::to_tf32(y - hy);
        *reinterpret_cast<float2*>(buf + off_hi + o) = make_float2(hx, hy);
        *reinterpret_cast<float2*>(buf + off_lo + o) = make_float2(lx, ly);
    } else {
        const __nv_bfloat16 hx = __float2bfloat16_rn(x), hy = __float2bfloat16_rn(y);
        const __nv_bfloat16 lx = __float2bfloat16_rn(x - __bfloat162float(hx));
        const __nv_bfloat16 ly = __float2bfloat16_rn(y - __bfloat162float(hy));
        *reinterpret_cast<__nv_bfloat162*>(buf + off_hi + o) = __halves2bfloat162(hx, hy);
        *reinterpret_cast<__nv_bfloat162*>(buf + off_lo + o) = __halves2bfloat162(lx, ly);
    }
}

// Staging slots: the i-th value of a thread is (row, k) = (8 g + lane % 8,
// 4 q + lane / 8) with (g, q) = (it / 4, it % 4), it = warp + TC_WARPS i.  A
// warp access covers 8 rows x 4 consecutive complex k: whole 16-byte rows of
// two TF32 core matrices (or one BF16 core matrix), so the split stores are
// free of bank conflicts, and each row's 4 values are one 32-byte sector of
// the global operand.
template <int CPS>
__device__ __forceinline__ void stage_slot(int i, int warp, int lane, int& row, int& k) {
    constexpr int KQ = CPS / 4;  // quads of k per row
    const int it = warp + TC_WARPS * i;
    row = 8 * (it / KQ) + (lane & 7);
    k = 4 * (it % KQ) + (lane >> 3);
}

// out[m][n] = alpha sum_k conj(A[m][k]) B[n][k] (rows K-contiguous); FP64 atomics into out.
// The loads of a chunk go to registers first (load), the splits to shared
// memory after (store), so the next chunk's loads overlap the current
// chunk's products.
template <int NT, int FMT, int CPS_ = TC_CPS>
struct StageCN {
    static constexpr int CPS = CPS_;
    const float2* A; int lda; const float2* B; int ldb; int M, N, K;
    double2* out; int ldo; double alpha;
    static constexpr int PA = TC_M * CPS / TC_THREADS;  // complex values per thread
    static constexpr int PB = NT * CPS / TC_THREADS;
    struct Regs { float2 a[PA]; float2 b[PB]; };
    __device__ __forceinline__ void load(Regs& r, int m0, int n0, int kc0, int warp, int lane) const {
#pragma unroll
        for (int i = 0; i < PA; ++i) {
            int row, k;
            stage_slot<CPS>(i, warp, lane, row, k);
            const int m = m0 + row;
            r.a[i] = (m < M && kc0 + k < K) ? A[(size_t)m * lda + kc0 + k] : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int i = 0; i < PB; ++i) {
            int row, k;
            stage_slot<CPS>(i, warp, lane, row, k);
            const int n = n0 + row;
            r.b[i] = (n < N && kc0 + k < K) ? B[(size_t)n * ldb + kc0 + k] : make_float2(0.f, 0.f);
        }
    }
    __device__ __forceinline__ void store(const Regs& r, char* buf, int warp, int lane) const {
        using L = TcLayout<NT, FMT, CPS>;
#pragma unroll
        for (int i = 0; i < PA; ++i) {
            int row, k;
            stage_slot<CPS>(i, warp, lane, row, k);
            put_split<FMT, CPS>(buf, L::A_HI, L::A_LO, row, 2 * k, r.a[i].x, r.a[i].y);
        }
#pragma unroll
        for (int i = 0; i < PB; ++i) {
            int row, k;
            stage_slot<CPS>(i, warp, lane, row, k);
            const float2 b = r.b[i];
            put_split<FMT, CPS>(buf, L::BR_HI, L::BR_LO, row, 2 * k, b.x, b.y);
            put_split<FMT, CPS>(buf, L::BI_HI, L::BI_LO, row, 2 * k, b.y, -b.x);
        }
    }
    __device__ __forceinline__ void emit(int m, int n, float re, float im) const {
        if (m < M && n < N) {
            atomicAdd(&out[(size_t)m * ldo + n].x, alpha * (double)re);
            atomicAdd(&out[(size_t)m * ldo + n].y, alpha * (double)im);
        }
    }
    // columns n .. n + 15 of row m
    __device__ __forceinline__ void emit16(int m, int n, const float* re, const float* im) const {
#pragma unroll
        for (int j = 0; j < 16; ++j) emit(m, n + j, re[j], im[j]);
    }
};

// out[n][m] += sum_i A[i][m] Bm[i][n]  (A: K rows of length M; Bm row-major K x N); one writer per element.
// The operands are contiguous along M and N: a warp access reads 8
// consecutive rows of each of 4 k.
template <int NT, int FMT, int CPS_ = TC_CPS>
struct StageNN {
    static constexpr int CPS = CPS_;
    const float2* A; int lda; const float2* Bm; int ldb; int M, N, K;
    float2* out; int ldo; bool accumulate;
    static constexpr int PA = TC_M * CPS / TC_THREADS;
    static constexpr int PB = NT * CPS / TC_THREADS;
    struct Regs { float2 a[PA]; float2 b[PB]; };
    __device__ __forceinline__ void load(Regs& r, int m0, int n0, int kc0, int warp, int lane) const {
#pragma unroll
        for (int i = 0; i < PA; ++i) {
            int row, k;
            stage_slot<CPS>(i, warp, lane, row, k);
            const int m = m0 + row;
            r.a[i] = (m < M && kc0 + k < K) ? A[(size_t)(kc0 + k) * lda + m] : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int i = 0; i < PB; ++i) {
            int row, k;
            stage_slot<CPS>(i, warp, lane, row, k);
            const int n = n0 + row;
            r.b[i] = (n < N && kc0 + k < K) ? Bm[(size_t)(kc0 + k) * ldb + n] : make_float2(0.f, 0.f);
        }
    }
    __device__ __forceinline__ void store(const Regs& r, char* buf, int warp, int lane) const {
        using L = TcLayout<NT, FMT, CPS>;
#pragma unroll
        for (int i = 0; i < PA; ++i) {
            int row, k;
            stage_slot<CPS>(i, warp, lane, row, k);
            put_split<FMT, CPS>(buf, L::A_HI, L::A_LO, row, 2 * k, r.a[i].x, r.a[i].y);
        }
#pragma unroll
        for (int i = 0; i < PB; ++i) {
            int row, k;
            stage_slot<CPS>(i, warp, lane, row, k);
            const float2 b = r.b[i];
            put_split<FMT, CPS>(buf, L::BR_HI, L::BR_LO, row, 2 * k, b.x, -b.y);
            put_split<FMT, CPS>(buf, L::BI_HI, L::BI_LO, row, 2 * k, b.y, b.x);
        }
    }
    // columns n .. n + 15 of row m.  The 16 old values (accumulate) are all
    // loaded before the first store: the addresses are distinct and this thread
    // is their only writer, but the compiler cannot see that through ldo, and a
    // load-add-store per column would wait out 16 global latencies in turn.
    __device__ __forceinline__ void emit16(int m, int n, const float* re, const float* im) const {
        if (m >= M) return;
        float2 v[16];
#pragma unroll
        for (int j = 0; j < 16; ++j)
            v[j] = (accumulate && n + j < N) ? out[(size_t)(n + j) * ldo + m] : make_float2(0.f, 0.f);
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            if (n + j < N) {
                v[j].x += re[j];
                v[j].y += im[j];
                out[(size_t)(n + j) * ldo + m] = v[j];
            }
        }
    }
};

template <int NT, int FMT, class S>
__global__ void __launch_bounds__(TC_THREADS) tc_zgemm_kernel(S s, int nchunks, int chunks_per_split) {
    constexpr int CPS = S::CPS;
    using L = TcLayout<NT, FMT, CPS>;
    using F = Fmt<FMT, CPS>;
    extern __shared__ __align__(1024) char smem[];
    char* stage_buf[2] = {smem, smem + L::STAGE};
    uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + 2 * L::STAGE);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 2);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        tc::mbar_init(&mbar[0], 1);
        tc::mbar_init(&mbar[1], 1);
        tc::mbar_fence_init();
    }
    if (warp == 0) tc::tmem_alloc(tslot, L::NCOLS);
    tc::tc_fence_before_sync();
    __syncthreads();
    tc::tc_fence_after_sync();
    const uint32_t tmem = *tslot;
    const int m0 = blockIdx.x * TC_M, n0 = blockIdx.y * NT;
    const int c0 = blockIdx.z * chunks_per_split;
    const int c1 = min(nchunks, c0 + chunks_per_split);
    constexpr uint32_t idesc = tc::instr_desc(F::IDESC_FMT, TC_M, NT);
    const unsigned long long wait_ns = g_tc_wait_ns;
    int ok = 1;
    int it = 0;
    // two register sets: the loads of chunk c + 2 are issued right after the
    // products of chunk c, a full chunk before they are stored
    typename S::Regs regs0, regs1;
    if (c0 < c1) s.load(regs0, m0, n0, c0 * CPS, warp, lane);
    if (c0 + 1 < c1) s.load(regs1, m0, n0, (c0 + 1) * CPS, warp, lane);
    auto step = [&](typename S::Regs& regs, char* buf, uint64_t* bar) -> bool {
        if (it >= 2) {
            // the products issued from this buffer two chunks ago must be done before restaging it
            const int w = tc::mbar_wait_ns(bar, (uint32_t)(((it - 2) >> 1) & 1), wait_ns) ? 1 : 0;
            ok = __syncthreads_and(w);
            if (!ok) return false;
        }
        s.store(regs, buf, warp, lane);
        tc::fence_proxy_async_smem();
        __syncthreads();
        if (tid == 0) {
            tc::tc_fence_after_sync();
            const uint32_t base = tc::smem_addr(buf);
            constexpr uint32_t LBO = 128, SBO = F::SBO;
#pragma unroll
            for (int kk = 0; kk < F::KSTEPS; ++kk) {
                const uint32_t off = kk * 256;
                const uint64_t ahi = tc::smem_desc(base + L::A_HI + off, LBO, SBO);
                const uint64_t alo = tc::smem_desc(base + L::A_LO + off, LBO, SBO);
                const uint64_t brh = tc::smem_desc(base + L::BR_HI + off, LBO, SBO);
                const uint64_t brl = tc::smem_desc(base + L::BR_LO + off, LBO, SBO);
                const uint64_t bih = tc::smem_desc(base + L::BI_HI + off, LBO, SBO);
                const uint64_t bil = tc::smem_desc(base + L::BI_LO + off, LBO, SBO);
                const uint32_t acc = (it > 0 || kk > 0) ? 1u : 0u;
                if constexpr (FMT == 0) {
                    tc::mma_tf32(tmem, ahi, brh, idesc, acc);
                    tc::mma_tf32(tmem, ahi, brl, idesc, 1u);
                    tc::mma_tf32(tmem, alo, brh, idesc, 1u);
                    tc::mma_tf32(tmem + NT, ahi, bih, idesc, acc);
                    tc::mma_tf32(tmem + NT, ahi, bil, idesc, 1u);
                    tc::mma_tf32(tmem + NT, alo, bih, idesc, 1u);
                } else {
                    tc::mma_bf16(tmem, ahi, brh, idesc, acc);
                    tc::mma_bf16(tmem, ahi, brl, idesc, 1u);
                    tc::mma_bf16(tmem, alo, brh, idesc, 1u);
                    tc::mma_bf16(tmem + NT, ahi, bih, idesc, acc);
                    tc::mma_bf16(tmem + NT, ahi, bil, idesc, 1u);
                    tc::mma_bf16(tmem + NT, alo, bih, idesc, 1u);
                }
            }
            tc::mma_commit(bar);
        }
        const int c = c0 + it;
        if (c + 2 < c1) s.load(regs, m0, n0, (c + 2) * CPS, warp, lane);  // overlaps the products just issued
        ++it;
        return true;
    };
    while (c0 + it < c1) {
        if (!step(regs0, stage_buf[0], &mbar[0])) break;
        if (c0 + it >= c1) break;
        if (!step(regs1, stage_buf[1], &mbar[1])) break;
    }
    const int n = it;  // batches committed
    if (ok && n > 0) {
        // the last commit completes after every earlier product of this thread
        const int w = tc::mbar_wait_ns(&mbar[(n - 1) & 1], (uint32_t)(((n - 1) >> 1) & 1), wait_ns) ? 1 : 0;
        ok = __syncthreads_and(w);
    }
    if (!ok && n > 0) {
        // a wait gave up: nothing more is issued, but committed products may
        // still run and write this block's tensor memory (and read its
        // stages), so wait for the last of them before freeing anything
        tc::mbar_wait_ns(&mbar[(n - 1) & 1], (uint32_t)(((n - 1) >> 1) & 1), TC_DRAIN_NS);
        __syncthreads();
    }
    tc::tc_fence_after_sync();
    if (ok && n > 0) {
        // warp w reads tensor-memory lanes 32 (w % 4) .. + 31; the warp groups
        // w / 4 take the 16-column slices in turn
        const int quad = warp & 3, grp = warp >> 2;
        const int row = quad * 32 + lane;
        const uint32_t lane_base = tmem + ((uint32_t)(quad * 32) << 16);
#pragma unroll 1
        for (int col = grp * 16; col < NT; col += 16 * (TC_WARPS / 4)) {
            float re[16], im[16];
            tc::tmem_ld16(lane_base + col, re);
            tc::tmem_ld16(lane_base + NT + col, im);
            s.emit16(m0 + row, n0 + col, re, im);
        }
    }
    tc::tc_fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, L::NCOLS);
    if (!ok && tid == 0) atomicExch(&g_tc_status, (int)JDFT_ERR_TIMEOUT);
}

template <int NT, int FMT, class S>
static jdft_status tc_launch(const S& s, int M, int N, int K, int splits, const char* name, cudaStream_t st) {
    using L = TcLayout<NT, FMT, S::CPS>;
    static_assert(L::SMEM <= 227 * 1024, "tensor-core GEMM stages exceed shared memory");
    auto kern = tc_zgemm_kernel<NT, FMT, S>;
    cudaError_t e = set_smem_attr((const void*)kern, L::SMEM);
    if (e != cudaSuccess) return set_error(JDFT_ERR_CUDA, std::string(name) + ": " + cudaGetErrorString(e));
    const int nchunks = (K + S::CPS - 1) / S::CPS;
    splits = std::max(1, std::min(splits, nchunks));
    const int cps = (nchunks + splits - 1) / splits;
    splits = (nchunks + cps - 1) / cps;
    dim3 grid((M + TC_M - 1) / TC_M, (N + NT - 1) / NT, splits);
    {
        Trace tr_(name, st);
        kern<<<grid, TC_THREADS, L::SMEM, st>>>(s, nchunks, cps);
    }
    return check_launch(name);
}

// Split-K schedules chosen by jdft_autotune_gemm, per product shape (M, N, K,
// operand format); absent shapes use the default schedule.
namespace {
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int, int>, int> g_tune_cn;
}  // namespace

static int tuned_cn_splits(int M, int N, int K, int fmt) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune_cn.find(std::make_tuple(M, N, K, fmt));
    return it == g_tune_cn.end() ? 0 : it->second;
}

// Default split-K count of the 128-column C^dag B schedule and the smallest
// count the accuracy cap allows (at most 4096 complex K accumulate in tensor
// memory per block: the FP32 accumulation there loses precision in
// proportion to the number of accumulating products, about 6e-4 relative
// over 42 k complex K and 2e-5 over 1.6 k; the split partial sums meet in
// FP64).
static void cn_schedule(int M, int N, int K, int& dflt, int& capmin) {
    const int tiles = ((M + TC_M - 1) / TC_M) * ((N + 127) / 128);
    const int nck = (K + TC_CPS - 1) / TC_CPS;
    constexpr int kMaxChunks = 4096 / TC_CPS;
    capmin = (nck + kMaxChunks - 1) / kMaxChunks;
    dflt = std::max(std::min(nck / 4 + 1, (152 + tiles - 1) / tiles), capmin);
}

template <int FMT>
static jdft_status tc_cn(int M, int N, int K, const float2* A, int lda, const float2* B, int ldb, double2* out, int ldo,
                         double alpha, cudaStream_t st) {
    const int nchunks = (K + TC_CPS - 1) / TC_CPS;  // at the default stage depth
    if (N <= 32) {
        StageCN<32, FMT> s{A, lda, B, ldb, M, N, K, out, ldo, alpha};
        const int tiles = ((M + TC_M - 1) / TC_M) * ((N + 31) / 32);
        const int splits = std::max(std::min(nchunks / 4 + 1, (152 * 2 + tiles - 1) / tiles), (nchunks + 255) / 256);
        return tc_launch<32, FMT>(s, M, N, K, splits, "tc_zgemm_cn", st);
    }
    // 16 complex K per stage (32 for BF16, 256 contiguous bytes per operand
    // row, measured 10 % slower on the 256 x 256 x 62 759 products)
    StageCN<128, FMT, TC_CPS> s{A, lda, B, ldb, M, N, K, out, ldo, alpha};
    int splits, capmin;
    cn_schedule(M, N, K, splits, capmin);
    const int tuned = tuned_cn_splits(M, N, K, FMT);
    if (tuned > 0) splits = std::max(tuned, capmin);
    return tc_launch<128, FMT>(s, M, N, K, splits, "tc_zgemm_cn", st);
}

template <int FMT>
static jdft_status tc_nn(int M, int N, int K, const float2* A, int lda, const float2* Bm, int ldb, float2* out, int ldo,
                         bool accumulate, cudaStream_t st) {
    if (N <= 32) {
        StageNN<32, FMT> s{A, lda, Bm, ldb, M, N, K, out, ldo, accumulate};
        return tc_launch<32, FMT>(s, M, N, K, 1, "tc_zgemm_nn", st);
    }
    if constexpr (FMT == 1) {
        // BF16 and more than 128 columns: all 256 in one tile (N = 256 products,
        // all 512 tensor-memory columns), so each row of P or C is staged once
        if (N > 128 && N <= 256) {
            StageNN<256, FMT> s{A, lda, Bm, ldb, M, N, K, out, ldo, accumulate};
            return tc_launch<256, FMT>(s, M, N, K, 1, "tc_zgemm_nn", st);
        }
    }
    StageNN<128, FMT> s{A, lda, Bm, ldb, M, N, K, out, ldo, accumulate};
    return tc_launch<128, FMT>(s, M, N, K, 1, "tc_zgemm_nn", st);
}

jdft_status tc_zgemm_cn(int M, int N, int K, const float2* A, int lda, const float2* B, int ldb, double2* out, int ldo,
                        double alpha, bool bf16, cudaStream_t st) {
    if (M == 0 || N == 0 || K == 0) return JDFT_OK;
    return bf16 ? tc_cn<1>(M, N, K, A, lda, B, ldb, out, ldo, alpha, st)
                : tc_cn<0>(M, N, K, A, lda, B, ldb, out, ldo, alpha, st);
}

jdft_status tc_zgemm_nn_acc(int M, int N, int K, const float2* A, int lda, const float2* Bm, int ldb, float2* out,
                            int ldo, bool bf16, cudaStream_t st, bool accumulate) {
    if (M == 0 || N == 0) return JDFT_OK;
    if (K == 0) return accumulate ? JDFT_OK : zgemm_nn_acc<float>(M, N, 0, A, lda, Bm, ldb, out, ldo, st, false);
    return bf16 ? tc_nn<1>(M, N, K, A, lda, Bm, ldb, out, ldo, accumulate, st)
                : tc_nn<0>(M, N, K, A, lda, Bm, ldb, out, ldo, accumulate, st);
}

}  // namespace jdft

namespace jdft {

// ===========================================================================
// C^dag B products from operands split once into BF16 planes, staged by bulk
// asynchronous copies (TMA).
//
// A complex block X (rows of K values, FP32) is stored split into four planes
// of BF16 values: Re hi, Re lo, Im hi, Im lo, with x = hi + lo for
// hi = bf16(x), lo = bf16(x - hi).  The split copy is ordered by chunks of 16
// K: for each chunk, the four planes, each holding all rows (padded to a
// multiple of 128 with zeros; K padded to a multiple of 16 with zeros) in the
// no-swizzle K-major layout of the tensor cores (8-row x 8-value core
// matrices of 128 contiguous bytes; the two core matrices of a row group
// along K 128 bytes apart, row groups 256 bytes apart).  The rows a block
// needs from one plane of one chunk are then one contiguous copy.
//
// For out[m][n] += alpha sum_k conj(A[m][k]) B[n][k]:
//   Re = Ar.Br + Ai.Bi,  Im = Ar.Bi - Ai.Br,
// each real product as hi.hi + hi.lo + lo.hi (FP32 accumulation in tensor
// memory), the minus through the instruction descriptor's negate-A bit: 12
// MMAs of 128 x NT x 16 per 16 complex K.
//
// One block of 128 threads computes a 128 x NT tile over a range of K (split-K):
// thread 0 issues the copies of a 4-stage ring, thread 32 waits for a stage,
// issues its MMAs and commits them to the stage's "empty" barrier, and after
// the last stage to the accumulator barrier, which all four warps wait for
// before reading tensor memory (warp w: rows 32 w .. 32 w + 31).  The split-K
// partial tiles meet in one of two ways.  With a partial buffer, each block
// stores its FP32 tile (column-major, so a warp's store is 32 consecutive
// rows) and tcx_reduce_kernel sums the tiles of every output with compensated
// FP32 sums in a fixed order (deterministic; no atomics).  Without one, the epilogue adds the
// tile to the output with FP64 atomics, each warp's 32 x 16 slices passed
// through shared memory so that one atomic instruction covers 16 consecutive
// outputs of two rows.  Every wait is bounded by the run-time limit; a wait
// that gives up records JDFT_ERR_TIMEOUT, and the block waits (under the fixed
// drain limit) for the copies and products it already issued before freeing
// its tensor memory.
// ===========================================================================

constexpr int TCX_M = 128;
constexpr int TCX_KC = 16;  // complex K per stage: one instruction's K
constexpr int TCX_STAGES = 4;
constexpr int TCX_THREADS = 128;
constexpr int TCX_PLANE = TCX_M * TCX_KC * 2;  // bytes of 128 rows x 16 K of one plane

__host__ __device__ constexpr int tcx_rows_pad(int rows) { return (rows + TCX_M - 1) / TCX_M * TCX_M; }
__host__ __device__ constexpr int tcx_chunks(int K) { return (K + TCX_KC - 1) / TCX_KC; }

template <int NT>
struct TcxLayout {
    static constexpr int A_PL = TCX_PLANE;                 // bytes of one A plane in a stage
    static constexpr int B_PL = (NT / TCX_M) * TCX_PLANE;  // bytes of one B plane in a stage
    static constexpr int A_BYTES = 4 * A_PL;
    static constexpr int STAGE = 4 * A_PL + 4 * B_PL;
    static constexpr int BAR_OFF = TCX_STAGES * STAGE;
    static constexpr int SMEM = BAR_OFF + 256 + 1024;  // barriers, flags; 1 KB to align the ring
    static constexpr uint32_t NCOLS = 2 * NT <= 256 ? 256 : 512;
    static_assert(NT % TCX_M == 0, "B blocks are whole 128-row blocks");
};

// Element offset of (row r, k) of plane p in a split block of rp (padded) rows.
__device__ __forceinline__ size_t tcx_offset(int r, int k, int p, int rp) {
    const int kc = k >> 4, kk = k & 15;
    return ((size_t)(kc * 4 + p) * rp + (r & ~7)) * TCX_KC + (kk >> 3) * 64 + (r & 7) * 8 + (kk & 7);
}

// One thread per 16-byte row of a core matrix: 8 consecutive K values of one
// row (64 contiguous input bytes), their hi and lo parts of Re and Im written
// as one 16-byte store per plane.  Consecutive threads take consecutive rows
// of a row group, then the second K half, then the next row group, so a
// warp's stores to each plane are 512 contiguous bytes.
// TRANS: the split block's row r, value k is X[k * ld + r] (the split of the
// transpose, for the operands of the M-contiguous products); otherwise
// X[r * ld + k].  Consecutive threads then read consecutive r: coalesced too.
template <bool TRANS>
__global__ void split_planes_kernel(const float2* __restrict__ X, int ld, int rows, int K, int rows_pad, int nkc,
                                    __nv_bfloat16* __restrict__ out) {
    const int per_chunk = rows_pad * 2;  // 16-byte units per plane of one chunk
    const int64_t total = (int64_t)per_chunk * nkc;
    const size_t P = (size_t)rows_pad * TCX_KC;  // elements between planes of one chunk
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int kc = (int)(i / per_chunk), u = (int)(i - (int64_t)kc * per_chunk);
        const int r8 = u & 7, h = (u >> 3) & 1, g = u >> 4;
        const int r = g * 8 + r8, k0 = kc * TCX_KC + h * 8;
        float2 v[8];
        if constexpr (TRANS) {
            const float2* src = X + (size_t)k0 * ld + r;
#pragma unroll
            for (int j = 0; j < 8; ++j) v[j] = (r < rows && k0 + j < K) ? src[(size_t)j * ld] : make_float2(0.f, 0.f);
        } else {
            const float2* src = X + (size_t)r * ld + k0;
#pragma unroll
            for (int j = 0; j < 8; ++j) v[j] = (r < rows && k0 + j < K) ? src[j] : make_float2(0.f, 0.f);
        }
        uint32_t w[4][4];  // plane, 32-bit word (two BF16 values)
#pragma unroll
        for (int j = 0; j < 8; j += 2) {
            const __nv_bfloat16 hx0 = __float2bfloat16_rn(v[j].x), hx1 = __float2bfloat16_rn(v[j + 1].x);
            const __nv_bfloat16 hy0 = __float2bfloat16_rn(v[j].y), hy1 = __float2bfloat16_rn(v[j + 1].y);
            const __nv_bfloat162 hx = __halves2bfloat162(hx0, hx1), hy = __halves2bfloat162(hy0, hy1);
            const __nv_bfloat162 lx = __halves2bfloat162(__float2bfloat16_rn(v[j].x - __bfloat162float(hx0)),
                                                         __float2bfloat16_rn(v[j + 1].x - __bfloat162float(hx1)));
            const __nv_bfloat162 ly = __halves2bfloat162(__float2bfloat16_rn(v[j].y - __bfloat162float(hy0)),
                                                         __float2bfloat16_rn(v[j + 1].y - __bfloat162float(hy1)));
            w[0][j / 2] = *reinterpret_cast<const uint32_t*>(&hx);
            w[1][j / 2] = *reinterpret_cast<const uint32_t*>(&lx);
            w[2][j / 2] = *reinterpret_cast<const uint32_t*>(&hy);
            w[3][j / 2] = *reinterpret_cast<const uint32_t*>(&ly);
        }
        const size_t o = tcx_offset(r, k0, 0, rows_pad);
#pragma unroll
        for (int p = 0; p < 4; ++p)
            *reinterpret_cast<uint4*>(out + o + p * P) = make_uint4(w[p][0], w[p][1], w[p][2], w[p][3]);
    }
}

__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     tc::smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(tc::smem_addr(bar))
                 : "memory");
}

// Tile t of the upper triangle of an nt x nt grid of tiles, counted row by row
// ((0, 0) .. (0, nt - 1), (1, 1) ..): its tile row tm and column tn >= tm.
__host__ __device__ inline void tcx_upper_tile(int t, int nt, int& tm, int& tn) {
    tm = 0;
    while (t >= nt - tm) {
        t -= nt - tm;
        ++tm;
    }
    tn = tm + t;
}

template <int NT>
__global__ void __launch_bounds__(TCX_THREADS, 1)
    tcx_cn_kernel(const char* __restrict__ As, const char* __restrict__ Bs, int M, int N, int nkc, int cps,
                  double2* __restrict__ out, int ldo, double alpha, float2* __restrict__ part, int upper_nt) {
    // rows of the split blocks (padded to 128)
    const int rpA = (M + TCX_M - 1) / TCX_M * TCX_M, rpB = (N + TCX_M - 1) / TCX_M * TCX_M;
    using L = TcxLayout<NT>;
    extern __shared__ unsigned char smem_raw[];
    unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                                           ~(uintptr_t)1023);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + L::BAR_OFF);
    uint64_t* empty = full + TCX_STAGES;
    uint64_t* accbar = empty + TCX_STAGES;
    uint32_t* tslot = reinterpret_cast<uint32_t*>(accbar + 1);
    volatile int* flags = reinterpret_cast<volatile int*>(tslot + 1);  // 0: failed, 1: stages loaded, 2: committed
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // upper_nt > 0: the grid's x index runs over the upper-triangle tiles of an
    // upper_nt x upper_nt tile grid (a Hermitian product's other tiles are its mirror)
    int tm = blockIdx.x, tn = blockIdx.y;
    if (upper_nt > 0) tcx_upper_tile(blockIdx.x, upper_nt, tm, tn);
    const int m0 = tm * TCX_M, n0 = tn * NT;
    // B rows this block copies (the last column block may hold fewer than NT)
    const uint32_t bbytes = (uint32_t)min(NT, rpB - n0) * TCX_KC * 2;
    const int c0 = blockIdx.z * cps;
    const int nit = max(0, min(nkc, c0 + cps) - c0);
    if (tid == 0) {
        for (int s = 0; s < TCX_STAGES; ++s) {
            tc::mbar_init(&full[s], 1);
            tc::mbar_init(&empty[s], 1);
        }
        tc::mbar_init(accbar, 1);
        flags[0] = 0;
        flags[1] = 0;
        flags[2] = 0;
        tc::mbar_fence_init();
    }
    if (warp == 2) tc::tmem_alloc(tslot, L::NCOLS);
    tc::tc_fence_before_sync();
    __syncthreads();
    tc::tc_fence_after_sync();
    const uint32_t tmem = *tslot;
    const unsigned long long wait_ns = g_tc_wait_ns;
    if (tid == 0) {
        // producer: a stage is refilled once the products that read it are done
        int it = 0;
        for (; it < nit; ++it) {
            const int s = it % TCX_STAGES;
            const uint32_t par = (uint32_t)((it / TCX_STAGES) & 1);
            if (!tc::mbar_wait_ns(&empty[s], par ^ 1u, wait_ns)) {
                flags[0] = 1;
                break;
            }
            unsigned char* st = smem + s * L::STAGE;
            const int kc = c0 + it;
            tc::mbar_arrive_expect_tx(&full[s], (uint32_t)(4 * L::A_PL) + 4 * bbytes);
#pragma unroll
            for (int p = 0; p < 4; ++p) {
                bulk_load(st + p * L::A_PL, As + ((size_t)(kc * 4 + p) * rpA + m0) * (TCX_KC * 2), L::A_PL, &full[s]);
                bulk_load(st + L::A_BYTES + p * L::B_PL, Bs + ((size_t)(kc * 4 + p) * rpB + n0) * (TCX_KC * 2), bbytes,
                          &full[s]);
            }
        }
        flags[1] = it;
    } else if (tid == 32) {
        // MMA issuer
        constexpr uint32_t idesc = tc::instr_desc(1u, TCX_M, NT);
        constexpr uint32_t idesc_neg = idesc | (1u << 13);  // negate A
        int it = 0;
        for (; it < nit; ++it) {
            const int s = it % TCX_STAGES;
            const uint32_t par = (uint32_t)((it / TCX_STAGES) & 1);
            if (!tc::mbar_wait_ns(&full[s], par, wait_ns)) {
                flags[0] = 1;
                break;
            }
            tc::tc_fence_after_sync();
            const uint32_t base = tc::smem_addr(smem + s * L::STAGE);
            uint64_t a[4], b[4];
#pragma unroll
            for (int p = 0; p < 4; ++p) {
                a[p] = tc::smem_desc(base + p * L::A_PL, 128, 256);
                b[p] = tc::smem_desc(base + L::A_BYTES + p * L::B_PL, 128, 256);
            }
            const uint32_t acc = it > 0 ? 1u : 0u;
            const uint32_t re = tmem, im = tmem + NT;
            // planes: 0 Re hi, 1 Re lo, 2 Im hi, 3 Im lo
            tc::mma_bf16(re, a[0], b[0], idesc, acc);
            tc::mma_bf16(re, a[0], b[1], idesc, 1u);
            tc::mma_bf16(re, a[1], b[0], idesc, 1u);
            tc::mma_bf16(re, a[2], b[2], idesc, 1u);
            tc::mma_bf16(re, a[2], b[3], idesc, 1u);
            tc::mma_bf16(re, a[3], b[2], idesc, 1u);
            tc::mma_bf16(im, a[0], b[2], idesc, acc);
            tc::mma_bf16(im, a[0], b[3], idesc, 1u);
            tc::mma_bf16(im, a[1], b[2], idesc, 1u);
            tc::mma_bf16(im, a[2], b[0], idesc_neg, 1u);
            tc::mma_bf16(im, a[2], b[1], idesc_neg, 1u);
            tc::mma_bf16(im, a[3], b[0], idesc_neg, 1u);
            tc::mma_commit(&empty[s]);
        }
        flags[2] = it;
        if (it == nit && nit > 0) tc::mma_commit(accbar);
    }
    __syncthreads();
    const int loaded = flags[1], committed = flags[2];
    int ok = flags[0] == 0 && nit > 0;
    if (ok) {
        const int w = tc::mbar_wait_ns(accbar, 0u, wait_ns) ? 1 : 0;
        ok = __syncthreads_and(w);
    }
    if (!ok && nit > 0) {
        // drain before freeing anything: copies issued but never consumed, and
        // the last committed batch of products (batches complete in order)
        if (tid == 0) {
            for (int it = committed; it < loaded; ++it)
                tc::mbar_wait_ns(&full[it % TCX_STAGES], (uint32_t)((it / TCX_STAGES) & 1), TC_DRAIN_NS);
            if (committed > 0)
                tc::mbar_wait_ns(&empty[(committed - 1) % TCX_STAGES], (uint32_t)(((committed - 1) / TCX_STAGES) & 1),
                                 TC_DRAIN_NS);
            if (committed == nit) tc::mbar_wait_ns(accbar, 0u, TC_DRAIN_NS);
        }
        __syncthreads();
    }
    tc::tc_fence_after_sync();
    if (ok && part) {
        // the partial buffer is [tile][column pair][split][row], one 16-byte entry (Re, Im
        // of column 2 j, Re, Im of column 2 j + 1) per row, so that the splits of a column
        // pair are contiguous for the reduction
        const size_t tile = upper_nt > 0 ? (size_t)blockIdx.x : (size_t)blockIdx.y * gridDim.x + blockIdx.x;
        float4* P = reinterpret_cast<float4*>(part) + (tile * (NT / 2) * gridDim.z + blockIdx.z) * TCX_M + warp * 32 +
                    lane;
        const size_t jstride = (size_t)gridDim.z * TCX_M;
        const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll 1
        for (int col = 0; col < NT && n0 + col < N; col += 16) {
            float re[16], im[16];
            tc::tmem_ld16(lane_base + col, re);
            tc::tmem_ld16(lane_base + NT + col, im);
#pragma unroll
            for (int j = 0; j < 16; j += 2)
                P[(size_t)((col + j) / 2) * jstride] = make_float4(re[j], im[j], re[j + 1], im[j + 1]);
        }
    } else if (ok) {
        // each warp: its 32 rows in slices of 16 columns, transposed through
        // shared memory (the ring is free now) so that lanes 0-15 and 16-31
        // add to 16 consecutive outputs of one row each
        float2* T = reinterpret_cast<float2*>(smem) + warp * (32 * 17);
        const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
        const int c = lane & 15, rh = lane >> 4;
#pragma unroll 1
        for (int col = 0; col < NT && n0 + col < N; col += 16) {
            float re[16], im[16];
            tc::tmem_ld16(lane_base + col, re);
            tc::tmem_ld16(lane_base + NT + col, im);
#pragma unroll
            for (int j = 0; j < 16; ++j) T[lane * 17 + j] = make_float2(re[j], im[j]);
            __syncwarp();
            const int n = n0 + col + c;
#pragma unroll 4
            for (int i = 0; i < 16; ++i) {
                const int r = 2 * i + rh;
                const int m = m0 + warp * 32 + r;
                const float2 v = T[r * 17 + c];
                if (m < M && n < N) {
                    atomicAdd(&out[(size_t)m * ldo + n].x, alpha * (double)v.x);
                    atomicAdd(&out[(size_t)m * ldo + n].y, alpha * (double)v.y);
                }
            }
            __syncwarp();
        }
    }
    tc::tc_fence_before_sync();
    __syncthreads();
    if (warp == 2) tc::tmem_dealloc(tmem, L::NCOLS);
    if (!ok && nit > 0 && tid == 0) atomicExch(&g_tc_status, (int)JDFT_ERR_TIMEOUT);
}

// Compensated FP32 summation (Knuth's TwoSum): s + c carries the running sum
// of FP32 terms to twice the FP32 precision, with FP32 instructions only (the
// FP64 rate of the SMs is a small fraction of the FP32 rate).
struct Sum2 {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float x) {
        const float t = s + x;
        const float bp = t - s;
        c += (s - (t - bp)) + (x - bp);
        s = t;
    }
};

// out[m * ldo + n] += alpha sum_z (partial tile z of (m, n)) over the split-K
// partial tiles of tcx_cn_kernel ([tile][column pair][split][row] of 16-byte
// entries): block (column pair j of a tile, tile) with 128 x TCX_RZ
// threads; thread (r, q) sums the splits z = q, q + TCX_RZ, ... of columns 2 j
// and 2 j + 1 of row r with compensated FP32 sums, and the TCX_RZ sums of a
// row are combined in q order, so the result does not depend on timing.  The
// sums are formed to about 2^-44 of the sum of the terms' magnitudes, then
// rounded to FP64.  upper_nt > 0: the tiles are the upper triangle of an
// upper_nt x upper_nt tile grid of a Hermitian product, and each off-diagonal
// tile is also added, conjugated, at its mirror position.
constexpr int TCX_RZ = 8;
__global__ void __launch_bounds__(TCX_M* TCX_RZ)
    tcx_reduce_kernel(const float4* __restrict__ part, int splits, int tiles_m, int NT, int M, int N,
                      double2* __restrict__ out, int ldo, double alpha, int upper_nt) {
    __shared__ float4 sum[TCX_RZ][2][TCX_M];
    const int r = threadIdx.x, q = threadIdx.y;
    const int j = blockIdx.x, tile = blockIdx.y;
    const size_t zstride = TCX_M;
    const float4* p = part + ((size_t)tile * (NT / 2) + j) * (size_t)splits * TCX_M + r;
    Sum2 s[4];  // Re, Im of column 2 j; Re, Im of column 2 j + 1
    // eight loads in flight per thread, then their sums (absent splits add zeros)
    for (int z0 = q; z0 < splits; z0 += 8 * TCX_RZ) {
        float4 v[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int z = z0 + i * TCX_RZ;
            v[i] = z < splits ? p[(size_t)z * zstride] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            s[0].add(v[i].x);
            s[1].add(v[i].y);
            s[2].add(v[i].z);
            s[3].add(v[i].w);
        }
    }
    sum[q][0][r] = make_float4(s[0].s, s[0].c, s[1].s, s[1].c);
    sum[q][1][r] = make_float4(s[2].s, s[2].c, s[3].s, s[3].c);
    __syncthreads();
    // thread (r, 0) finishes column 2 j of row r, thread (r, 1) column 2 j + 1
    if (q >= 2) return;
    Sum2 x, y;
#pragma unroll
    for (int i = 0; i < TCX_RZ; ++i) {
        const float4 u = sum[i][q][r];
        x.add(u.x);
        x.add(u.y);
        y.add(u.z);
        y.add(u.w);
    }
    int tm = tile % tiles_m, tn = tile / tiles_m;
    if (upper_nt > 0) tcx_upper_tile(tile, upper_nt, tm, tn);
    const int m = tm * TCX_M + r, n = tn * NT + 2 * j + q;
    if (m < M && n < N) {
        const double re = alpha * ((double)x.s + (double)x.c), im = alpha * ((double)y.s + (double)y.c);
        double2* o = out + (size_t)m * ldo + n;
        o->x += re;
        o->y += im;
        if (upper_nt > 0 && tm != tn) {
            double2* t = out + (size_t)n * ldo + m;
            t->x += re;
            t->y -= im;
        }
    }
}

// out[n * ldo + m] (+)= sum_k A[m][k] B[n][k] from split blocks of A (M rows,
// K values: the split of the transpose of an M-contiguous operand) and B (N
// rows).  No conjugate: Re = Ar.Br - Ai.Bi, Im = Ar.Bi + Ai.Br.  One block
// covers a 128 x NT tile over all of K (K is a projector or band count, a few
// hundred at most), so the output is written once, without atomics: thread
// (warp w, lane l) owns output row m = m0 + 32 w + l and writes it for every
// column n, so a warp's stores to one band are 32 consecutive values.  Same
// ring, roles, waits and drain as tcx_cn_kernel.
template <int NT, bool ACC>
__global__ void __launch_bounds__(TCX_THREADS, 1)
    tcx_nn_kernel(const char* __restrict__ As, const char* __restrict__ Bs, int M, int N, int nkc,
                  float2* __restrict__ out, int ldo) {
    const int rpA = (M + TCX_M - 1) / TCX_M * TCX_M, rpB = (N + TCX_M - 1) / TCX_M * TCX_M;
    using L = TcxLayout<NT>;
    extern __shared__ unsigned char smem_raw[];
    unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                                           ~(uintptr_t)1023);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + L::BAR_OFF);
    uint64_t* empty = full + TCX_STAGES;
    uint64_t* accbar = empty + TCX_STAGES;
    uint32_t* tslot = reinterpret_cast<uint32_t*>(accbar + 1);
    volatile int* flags = reinterpret_cast<volatile int*>(tslot + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.x * TCX_M, n0 = blockIdx.y * NT;
    const uint32_t bbytes = (uint32_t)min(NT, rpB - n0) * TCX_KC * 2;
    const int nit = nkc;
    if (tid == 0) {
        for (int s = 0; s < TCX_STAGES; ++s) {
            tc::mbar_init(&full[s], 1);
            tc::mbar_init(&empty[s], 1);
        }
        tc::mbar_init(accbar, 1);
        flags[0] = 0;
        flags[1] = 0;
        flags[2] = 0;
        tc::mbar_fence_init();
    }
    if (warp == 2) tc::tmem_alloc(tslot, L::NCOLS);
    tc::tc_fence_before_sync();
    __syncthreads();
    tc::tc_fence_after_sync();
    const uint32_t tmem = *tslot;
    const unsigned long long wait_ns = g_tc_wait_ns;
    // accumulating: the old values of this thread's output row m, 64 columns at a
    // time; the first 64 are requested now, so their latency passes during the products
    const int m = m0 + warp * 32 + lane;
    constexpr int OG = ACC ? 64 : 1;
    float2 old[OG];
    auto load_old = [&](int col0) {
#pragma unroll
        for (int j = 0; j < OG; ++j) {
            const int n = n0 + col0 + j;
            old[j] = (m < M && n < N) ? out[(size_t)n * ldo + m] : make_float2(0.f, 0.f);
        }
    };
    if (ACC) load_old(0);
    if (tid == 0) {
        int it = 0;
        for (; it < nit; ++it) {
            const int s = it % TCX_STAGES;
            const uint32_t par = (uint32_t)((it / TCX_STAGES) & 1);
            if (!tc::mbar_wait_ns(&empty[s], par ^ 1u, wait_ns)) {
                flags[0] = 1;
                break;
            }
            unsigned char* st = smem + s * L::STAGE;
            tc::mbar_arrive_expect_tx(&full[s], (uint32_t)(4 * L::A_PL) + 4 * bbytes);
#pragma unroll
            for (int p = 0; p < 4; ++p) {
                bulk_load(st + p * L::A_PL, As + ((size_t)(it * 4 + p) * rpA + m0) * (TCX_KC * 2), L::A_PL, &full[s]);
                bulk_load(st + L::A_BYTES + p * L::B_PL, Bs + ((size_t)(it * 4 + p) * rpB + n0) * (TCX_KC * 2), bbytes,
                          &full[s]);
            }
        }
        flags[1] = it;
    } else if (tid == 32) {
        constexpr uint32_t idesc = tc::instr_desc(1u, TCX_M, NT);
        constexpr uint32_t idesc_neg = idesc | (1u << 13);  // negate A
        int it = 0;
        for (; it < nit; ++it) {
            const int s = it % TCX_STAGES;
            const uint32_t par = (uint32_t)((it / TCX_STAGES) & 1);
            if (!tc::mbar_wait_ns(&full[s], par, wait_ns)) {
                flags[0] = 1;
                break;
            }
            tc::tc_fence_after_sync();
            const uint32_t base = tc::smem_addr(smem + s * L::STAGE);
            uint64_t a[4], b[4];
#pragma unroll
            for (int p = 0; p < 4; ++p) {
                a[p] = tc::smem_desc(base + p * L::A_PL, 128, 256);
                b[p] = tc::smem_desc(base + L::A_BYTES + p * L::B_PL, 128, 256);
            }
            const uint32_t acc = it > 0 ? 1u : 0u;
            const uint32_t re = tmem, im = tmem + NT;
            // planes: 0 Re hi, 1 Re lo, 2 Im hi, 3 Im lo
            tc::mma_bf16(re, a[0], b[0], idesc, acc);
            tc::mma_bf16(re, a[0], b[1], idesc, 1u);
            tc::mma_bf16(re, a[1], b[0], idesc, 1u);
            tc::mma_bf16(re, a[2], b[2], idesc_neg, 1u);
            tc::mma_bf16(re, a[2], b[3], idesc_neg, 1u);
            tc::mma_bf16(re, a[3], b[2], idesc_neg, 1u);
            tc::mma_bf16(im, a[0], b[2], idesc, acc);
            tc::mma_bf16(im, a[0], b[3], idesc, 1u);
            tc::mma_bf16(im, a[1], b[2], idesc, 1u);
            tc::mma_bf16(im, a[2], b[0], idesc, 1u);
            tc::mma_bf16(im, a[2], b[1], idesc, 1u);
            tc::mma_bf16(im, a[3], b[0], idesc, 1u);
            tc::mma_commit(&empty[s]);
        }
        flags[2] = it;
        if (it == nit && nit > 0) tc::mma_commit(accbar);
    }
    __syncthreads();
    const int loaded = flags[1], committed = flags[2];
    int ok = flags[0] == 0 && nit > 0;
    if (ok) {
        const int w = tc::mbar_wait_ns(accbar, 0u, wait_ns) ? 1 : 0;
        ok = __syncthreads_and(w);
    }
    if (!ok && nit > 0) {
        if (tid == 0) {
            for (int it = committed; it < loaded; ++it)
                tc::mbar_wait_ns(&full[it % TCX_STAGES], (uint32_t)((it / TCX_STAGES) & 1), TC_DRAIN_NS);
            if (committed > 0)
                tc::mbar_wait_ns(&empty[(committed - 1) % TCX_STAGES], (uint32_t)(((committed - 1) / TCX_STAGES) & 1),
                                 TC_DRAIN_NS);
            if (committed == nit) tc::mbar_wait_ns(accbar, 0u, TC_DRAIN_NS);
        }
        __syncthreads();
    }
    tc::tc_fence_after_sync();
    if (ok) {
        const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
        if constexpr (ACC) {
            // groups of 64 columns: the group's old values were requested before its
            // four slices (one latency per group, the first one hidden)
#pragma unroll 1
            for (int g = 0; g < NT && n0 + g < N; g += 64) {
                if (g > 0) load_old(g);
#pragma unroll
                for (int q = 0; q < 64; q += 16) {
                    const int col = g + q;
                    if (n0 + col >= N) break;
                    float re[16], im[16];
                    tc::tmem_ld16(lane_base + col, re);
                    tc::tmem_ld16(lane_base + NT + col, im);
                    if (m < M) {
#pragma unroll
                        for (int j = 0; j < 16; ++j)
                            if (n0 + col + j < N)
                                out[(size_t)(n0 + col + j) * ldo + m] =
                                    make_float2(old[q + j].x + re[j], old[q + j].y + im[j]);
                    }
                }
            }
        } else {
#pragma unroll 1
            for (int col = 0; col < NT && n0 + col < N; col += 16) {
                float re[16], im[16];
                tc::tmem_ld16(lane_base + col, re);
                tc::tmem_ld16(lane_base + NT + col, im);
                if (m < M) {
#pragma unroll
                    for (int j = 0; j < 16; ++j)
                        if (n0 + col + j < N) out[(size_t)(n0 + col + j) * ldo + m] = make_float2(re[j], im[j]);
                }
            }
        }
    }
    tc::tc_fence_before_sync();
    __syncthreads();
    if (warp == 2) tc::tmem_dealloc(tmem, L::NCOLS);
    if (!ok && nit > 0 && tid == 0) atomicExch(&g_tc_status, (int)JDFT_ERR_TIMEOUT);
}

// Persistent X.Y products for N > 128 (tcx_nn with 256-column tiles): one
// block per SM walks a list of work items, so that the copies of an item's
// first stages overlap the previous item's epilogue and every block finishes
// at about the same time.  The list holds the r * P full tiles (128 rows x 256
// columns; P blocks, r = floor(tiles / P)) and then, when N is a multiple of
// 256, the remaining R tiles split into 2 R half tiles of 128 columns (else
// they stay whole); block p takes items p, p + P, p + 2P ...
// Roles: warps 0-3 drain tensor memory (warp w: rows 32 w .. 32 w + 31), warp
// 4 issues the copies of the 4-stage ring, warp 5 the MMAs.  The MMA warp
// starts an item once the four epilogue warps have released tensor memory
// (barrier tfree, 4 arrivals); the epilogue starts once the item's products
// have completed (barrier accfull).  Re accumulates at tensor-memory columns
// [0, nt), Im at [256, 256 + nt).  Every wait is bounded; a role whose wait
// gives up stops the others, and the block waits for its issued copies and
// products (drain limit) before freeing tensor memory.
constexpr int TCXP_THREADS = 192;

struct TcxItem {
    int m0, n0, nt;
};

// Tile t covers rows 128 (t / nblk) and columns 256 (t mod nblk) of the output.
__device__ __forceinline__ bool tcxp_item(int j, int full_tiles, int halves, int nblk, TcxItem& item) {
    const int idx = blockIdx.x + j * gridDim.x;
    int t = idx, half = -1;
    if (idx >= full_tiles) {
        const int h = idx - full_tiles;
        if (h >= halves) return false;
        t = full_tiles + h / 2;
        half = h & 1;
    }
    const int mt = t / nblk, nt = t - mt * nblk;
    item = {mt * TCX_M, nt * 256 + (half > 0 ? 128 : 0), half < 0 ? 256 : 128};
    return true;
}

__device__ __forceinline__ void tcxp_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_addr(bar)) : "memory");
}

template <bool ACC>
__global__ void __launch_bounds__(TCXP_THREADS, 1)
    tcx_nn_persist_kernel(const char* __restrict__ As, const char* __restrict__ Bs, int M, int N, int nkc,
                          float2* __restrict__ out, int ldo, int full_tiles, int halves) {
    const int rpA = (M + TCX_M - 1) / TCX_M * TCX_M, rpB = (N + TCX_M - 1) / TCX_M * TCX_M;
    const int nblk = (N + 255) / 256;
    using L = TcxLayout<256>;
    extern __shared__ unsigned char smem_raw[];
    unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                                           ~(uintptr_t)1023);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + L::BAR_OFF);
    uint64_t* empty = full + TCX_STAGES;
    uint64_t* accfull = empty + TCX_STAGES;
    uint64_t* tfree = accfull + 1;
    uint32_t* tslot = reinterpret_cast<uint32_t*>(tfree + 1);
    volatile int* flags = reinterpret_cast<volatile int*>(tslot + 1);  // 0: failed, 1: stages loaded, 2: committed
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        for (int s = 0; s < TCX_STAGES; ++s) {
            tc::mbar_init(&full[s], 1);
            tc::mbar_init(&empty[s], 1);
        }
        tc::mbar_init(accfull, 1);
        tc::mbar_init(tfree, 4);
        flags[0] = 0;
        flags[1] = 0;
        flags[2] = 0;
        tc::mbar_fence_init();
    }
    if (warp == 0) tc::tmem_alloc(tslot, L::NCOLS);
    tc::tc_fence_before_sync();
    __syncthreads();
    tc::tc_fence_after_sync();
    const uint32_t tmem = *tslot;
    const unsigned long long wait_ns = g_tc_wait_ns;
    TcxItem item;
    if (warp == 4) {
        if (lane == 0) {
            int it = 0;
            for (int j = 0; !flags[0] && tcxp_item(j, full_tiles, halves, nblk, item); ++j) {
                const uint32_t bbytes = (uint32_t)min(item.nt, rpB - item.n0) * TCX_KC * 2;
                for (int k = 0; k < nkc; ++k) {
                    const int s = it % TCX_STAGES;
                    const uint32_t par = (uint32_t)((it / TCX_STAGES) & 1);
                    if (!tc::mbar_wait_ns(&empty[s], par ^ 1u, wait_ns)) {
                        flags[0] = 1;
                        break;
                    }
                    unsigned char* st = smem + s * L::STAGE;
                    tc::mbar_arrive_expect_tx(&full[s], (uint32_t)(4 * L::A_PL) + 4 * bbytes);
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        bulk_load(st + q * L::A_PL, As + ((size_t)(k * 4 + q) * rpA + item.m0) * (TCX_KC * 2), L::A_PL,
                                  &full[s]);
                        bulk_load(st + L::A_BYTES + q * L::B_PL,
                                  Bs + ((size_t)(k * 4 + q) * rpB + item.n0) * (TCX_KC * 2), bbytes, &full[s]);
                    }
                    ++it;
                }
            }
            flags[1] = it;
        }
    } else if (warp == 5) {
        if (lane == 0) {
            constexpr uint32_t id256 = tc::instr_desc(1u, TCX_M, 256), id128 = tc::instr_desc(1u, TCX_M, 128);
            int it = 0;
            for (int j = 0; !flags[0] && tcxp_item(j, full_tiles, halves, nblk, item); ++j) {
                if (j > 0 && !tc::mbar_wait_ns(tfree, (uint32_t)((j - 1) & 1), wait_ns)) {
                    flags[0] = 1;
                    break;
                }
                tc::tc_fence_after_sync();
                const uint32_t idesc = item.nt == 256 ? id256 : id128;
                const uint32_t idesc_neg = idesc | (1u << 13);  // negate A
                bool fail = false;
                for (int k = 0; k < nkc; ++k) {
                    const int s = it % TCX_STAGES;
                    const uint32_t par = (uint32_t)((it / TCX_STAGES) & 1);
                    if (!tc::mbar_wait_ns(&full[s], par, wait_ns)) {
                        fail = true;
                        break;
                    }
                    tc::tc_fence_after_sync();
                    const uint32_t base = tc::smem_addr(smem + s * L::STAGE);
                    uint64_t a[4], b[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        a[q] = tc::smem_desc(base + q * L::A_PL, 128, 256);
                        b[q] = tc::smem_desc(base + L::A_BYTES + q * L::B_PL, 128, 256);
                    }
                    const uint32_t acc = k > 0 ? 1u : 0u;
                    const uint32_t re = tmem, im = tmem + 256;
                    // planes: 0 Re hi, 1 Re lo, 2 Im hi, 3 Im lo
                    tc::mma_bf16(re, a[0], b[0], idesc, acc);
                    tc::mma_bf16(re, a[0], b[1], idesc, 1u);
                    tc::mma_bf16(re, a[1], b[0], idesc, 1u);
                    tc::mma_bf16(re, a[2], b[2], idesc_neg, 1u);
                    tc::mma_bf16(re, a[2], b[3], idesc_neg, 1u);
                    tc::mma_bf16(re, a[3], b[2], idesc_neg, 1u);
                    tc::mma_bf16(im, a[0], b[2], idesc, acc);
                    tc::mma_bf16(im, a[0], b[3], idesc, 1u);
                    tc::mma_bf16(im, a[1], b[2], idesc, 1u);
                    tc::mma_bf16(im, a[2], b[0], idesc, 1u);
                    tc::mma_bf16(im, a[2], b[1], idesc, 1u);
                    tc::mma_bf16(im, a[3], b[0], idesc, 1u);
                    tc::mma_commit(&empty[s]);
                    ++it;
                }
                if (fail) {
                    flags[0] = 1;
                    break;
                }
                tc::mma_commit(accfull);
            }
            flags[2] = it;
        }
    } else {
        // epilogue: thread (warp w, lane l) owns output row m = m0 + 32 w + l of each item
        const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
        constexpr int OG = ACC ? 64 : 1;
        float2 old[OG];
        for (int j = 0; tcxp_item(j, full_tiles, halves, nblk, item); ++j) {
            const int m = item.m0 + warp * 32 + lane;
            auto load_old = [&](int col0) {
#pragma unroll
                for (int q = 0; q < OG; ++q) {
                    const int n = item.n0 + col0 + q;
                    old[q] = (m < M && n < N) ? out[(size_t)n * ldo + m] : make_float2(0.f, 0.f);
                }
            };
            if (ACC) load_old(0);  // requested while the item's products run
            int ok = 0;
            if (lane == 0) ok = tc::mbar_wait_ns(accfull, (uint32_t)(j & 1), wait_ns) ? 1 : 0;
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (!ok || flags[0]) {
                flags[0] = 1;
                break;
            }
            tc::tc_fence_after_sync();
#pragma unroll 1
            for (int g = 0; g < item.nt && item.n0 + g < N; g += 64) {
                if (ACC && g > 0) load_old(g);
#pragma unroll
                for (int q = 0; q < 64; q += 16) {
                    const int col = g + q;
                    if (item.n0 + col >= N) break;
                    float re[16], im[16];
                    tc::tmem_ld16(lane_base + col, re);
                    tc::tmem_ld16(lane_base + 256 + col, im);
                    if (m < M) {
#pragma unroll
                        for (int i = 0; i < 16; ++i) {
                            const int n = item.n0 + col + i;
                            if (n < N)
                                out[(size_t)n * ldo + m] = ACC ? make_float2(old[q + i].x + re[i], old[q + i].y + im[i])
                                                               : make_float2(re[i], im[i]);
                        }
                    }
                }
            }
            tc::tc_fence_before_sync();
            __syncwarp();
            if (lane == 0) tcxp_arrive(tfree);
        }
    }
    __syncthreads();
    const bool failed = flags[0] != 0;
    if (failed && tid == 0) {
        // drain: copies issued but never consumed, and the last committed batch of products
        const int loaded = flags[1], committed = flags[2];
        for (int it = committed; it < loaded; ++it)
            tc::mbar_wait_ns(&full[it % TCX_STAGES], (uint32_t)((it / TCX_STAGES) & 1), TC_DRAIN_NS);
        if (committed > 0)
            tc::mbar_wait_ns(&empty[(committed - 1) % TCX_STAGES], (uint32_t)(((committed - 1) / TCX_STAGES) & 1),
                             TC_DRAIN_NS);
    }
    tc::tc_fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, L::NCOLS);
    if (failed && tid == 0) atomicExch(&g_tc_status, (int)JDFT_ERR_TIMEOUT);
}

template <int NT, bool ACC>
static jdft_status launch_tcx_nn(int M, int N, int nkc, const void* Aplanes, const void* Bplanes, float2* out,
                                 int ldo, cudaStream_t st) {
    auto kern = tcx_nn_kernel<NT, ACC>;
    cudaError_t e = set_smem_attr((const void*)kern, TcxLayout<NT>::SMEM);
    if (e != cudaSuccess) return set_error(JDFT_ERR_CUDA, std::string("tcx_nn: ") + cudaGetErrorString(e));
    dim3 grid((M + TCX_M - 1) / TCX_M, (N + NT - 1) / NT);
    {
        Trace tr_("tcx_nn", st);
        kern<<<grid, TCX_THREADS, TcxLayout<NT>::SMEM, st>>>((const char*)Aplanes, (const char*)Bplanes, M, N, nkc,
                                                              out, ldo);
    }
    return check_launch("tcx_nn");
}

static bool getenv_zero(const char* name) {
    const char* e = getenv(name);
    return e && e[0] == '0';
}

template <bool ACC>
static jdft_status launch_tcx_nn_persist(int M, int N, int nkc, const void* Aplanes, const void* Bplanes, float2* out,
                                         int ldo, int blocks, int full_tiles, int halves, cudaStream_t st) {
    auto kern = tcx_nn_persist_kernel<ACC>;
    cudaError_t e = set_smem_attr((const void*)kern, TcxLayout<256>::SMEM);
    if (e != cudaSuccess) return set_error(JDFT_ERR_CUDA, std::string("tcx_nn: ") + cudaGetErrorString(e));
    {
        Trace tr_("tcx_nn", st);
        kern<<<blocks, TCXP_THREADS, TcxLayout<256>::SMEM, st>>>((const char*)Aplanes, (const char*)Bplanes, M, N, nkc,
                                                                 out, ldo, full_tiles, halves);
    }
    return check_launch("tcx_nn");
}

jdft_status tcx_nn(int M, int N, int K, const void* Aplanes, const void* Bplanes, float2* out, int ldo,
                   bool accumulate, cudaStream_t st) {
    if (M == 0 || N == 0) return JDFT_OK;
    const int nkc = tcx_chunks(K);
    if (N > 128) {
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const int tiles = (M + TCX_M - 1) / TCX_M * ((N + 255) / 256);
        if (tiles >= sms && !getenv_zero("JDFT_NN_PERSIST")) {
            const bool split = N % 256 == 0;
            const int full_tiles = split ? tiles / sms * sms : tiles;
            const int halves = 2 * (tiles - full_tiles);
            return accumulate ? launch_tcx_nn_persist<true>(M, N, nkc, Aplanes, Bplanes, out, ldo, sms, full_tiles,
                                                            halves, st)
                              : launch_tcx_nn_persist<false>(M, N, nkc, Aplanes, Bplanes, out, ldo, sms, full_tiles,
                                                             halves, st);
        }
        return accumulate ? launch_tcx_nn<256, true>(M, N, nkc, Aplanes, Bplanes, out, ldo, st)
                          : launch_tcx_nn<256, false>(M, N, nkc, Aplanes, Bplanes, out, ldo, st);
    }
    return accumulate ? launch_tcx_nn<128, true>(M, N, nkc, Aplanes, Bplanes, out, ldo, st)
                      : launch_tcx_nn<128, false>(M, N, nkc, Aplanes, Bplanes, out, ldo, st);
}

size_t tcx_split_bytes(int rows, int K) { return (size_t)tcx_rows_pad(rows) * tcx_chunks(K) * 4 * TCX_KC * 2; }

bool tcx_eligible(jdft_prec prec, int M, int N) { return prec == JDFT_BF16X3 && M > 32 && N > 32; }

jdft_status tcx_split(const float2* X, int ld, int rows, int K, void* planes, cudaStream_t st) {
    if (rows == 0 || K == 0) return JDFT_OK;
    const int nkc = tcx_chunks(K), rp = tcx_rows_pad(rows);
    const int64_t total = (int64_t)rp * 2 * nkc;
    const int grid = (int)std::min<int64_t>((total + 255) / 256, 152 * 16);
    {
        Trace tr_("split_planes", st);
        split_planes_kernel<false><<<grid, 256, 0, st>>>(X, ld, rows, K, rp, nkc, (__nv_bfloat16*)planes);
    }
    return check_launch("split_planes");
}

jdft_status tcx_split_t(const float2* X, int ld, int rows, int K, void* planes, cudaStream_t st) {
    if (rows == 0 || K == 0) return JDFT_OK;
    const int nkc = tcx_chunks(K), rp = tcx_rows_pad(rows);
    const int64_t total = (int64_t)rp * 2 * nkc;
    const int grid = (int)std::min<int64_t>((total + 255) / 256, 152 * 16);
    {
        Trace tr_("split_planes", st);
        split_planes_kernel<true><<<grid, 256, 0, st>>>(X, ld, rows, K, rp, nkc, (__nv_bfloat16*)planes);
    }
    return check_launch("split_planes");
}

// Split-K counts of tcx_cn chosen by jdft_autotune_gemm, per (M, N, K).
namespace {
std::map<std::tuple<int, int, int>, int> g_tune_tcx;
}  // namespace

static int tuned_tcx_splits(int M, int N, int K) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune_tcx.find(std::make_tuple(M, N, K));
    return it == g_tune_tcx.end() ? 0 : it->second;
}

// Tile width, K chunks per split and split count tcx_cn launches with for (M, N, K).
static void tcx_cn_config(int M, int N, int K, int& NT, int& cps, int& splits) {
    NT = N > 128 ? 256 : 128;
    const int nkc = tcx_chunks(K);
    const int tiles = ((M + TCX_M - 1) / TCX_M) * ((N + NT - 1) / NT);
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // one wave of blocks, and at most 4096 complex K accumulated per block
    const int capmin = (nkc + 4096 / TCX_KC - 1) / (4096 / TCX_KC);
    splits = std::max(capmin, std::min(nkc, std::max(1, sms / tiles)));
    const int tuned = tuned_tcx_splits(M, N, K);
    if (tuned > 0) splits = std::max(capmin, std::min(nkc, tuned));
    cps = (nkc + splits - 1) / splits;
    splits = (nkc + cps - 1) / cps;
}

size_t tcx_cn_partial_bytes(int M, int N, int K) {
    if (M == 0 || N == 0 || K == 0) return 0;
    int NT, cps, splits;
    tcx_cn_config(M, N, K, NT, cps, splits);
    const size_t tiles = (size_t)((M + TCX_M - 1) / TCX_M) * ((N + NT - 1) / NT);
    return ((size_t)splits * tiles * TCX_M * NT * sizeof(float2) + 255) / 256 * 256;
}

jdft_status tcx_cn(int M, int N, int K, const void* Aplanes, const void* Bplanes, double2* out, int ldo, double alpha,
                   cudaStream_t st, void* partials, size_t partial_bytes, bool hermitian) {
    if (M == 0 || N == 0 || K == 0) return JDFT_OK;
    if (hermitian && M == N && N > 128 && partials) {
        // the upper-triangle 128 x 128 tiles only, each over a share of K; the
        // reduction mirrors the off-diagonal ones
        const int nt = (N + TCX_M - 1) / TCX_M, tiles = nt * (nt + 1) / 2;
        const int nkc = tcx_chunks(K);
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const int capmin = (nkc + 4096 / TCX_KC - 1) / (4096 / TCX_KC);
        int splits = std::max(capmin, std::min(nkc, std::max(1, sms / tiles)));
        const int cps = (nkc + splits - 1) / splits;
        splits = (nkc + cps - 1) / cps;
        if ((size_t)splits * tiles * TCX_M * 128 * sizeof(float2) <= partial_bytes) {
            auto kern = tcx_cn_kernel<128>;
            cudaError_t e = set_smem_attr((const void*)kern, TcxLayout<128>::SMEM);
            if (e != cudaSuccess) return set_error(JDFT_ERR_CUDA, std::string("tcx_cn: ") + cudaGetErrorString(e));
            {
                Trace tr_("tcx_cn", st);
                kern<<<dim3(tiles, 1, splits), TCX_THREADS, TcxLayout<128>::SMEM, st>>>(
                    (const char*)Aplanes, (const char*)Bplanes, M, N, nkc, cps, out, ldo, alpha, (float2*)partials, nt);
            }
            jdft_status s = check_launch("tcx_cn");
            if (s != JDFT_OK) return s;
            {
                Trace tr_("tcx_reduce", st);
                tcx_reduce_kernel<<<dim3(64, tiles), dim3(TCX_M, TCX_RZ), 0, st>>>(
                    (const float4*)partials, splits, nt, 128, M, N, out, ldo, alpha, nt);
            }
            return check_launch("tcx_reduce");
        }
    }
    int NT, cps, splits;
    tcx_cn_config(M, N, K, NT, cps, splits);
    const bool wide = NT == 256;
    const int nkc = tcx_chunks(K);
    const int tiles_m = (M + TCX_M - 1) / TCX_M, tiles = tiles_m * ((N + NT - 1) / NT);
    float2* part = partials && partial_bytes >= tcx_cn_partial_bytes(M, N, K) ? (float2*)partials : nullptr;
    dim3 grid(tiles_m, (N + NT - 1) / NT, splits);
    if (wide) {
        auto kern = tcx_cn_kernel<256>;
        cudaError_t e = set_smem_attr((const void*)kern, TcxLayout<256>::SMEM);
        if (e != cudaSuccess) return set_error(JDFT_ERR_CUDA, std::string("tcx_cn: ") + cudaGetErrorString(e));
        Trace tr_("tcx_cn", st);
        kern<<<grid, TCX_THREADS, TcxLayout<256>::SMEM, st>>>((const char*)Aplanes, (const char*)Bplanes, M, N, nkc,
                                                               cps, out, ldo, alpha, part, 0);
    } else {
        auto kern = tcx_cn_kernel<128>;
        cudaError_t e = set_smem_attr((const void*)kern, TcxLayout<128>::SMEM);
        if (e != cudaSuccess) return set_error(JDFT_ERR_CUDA, std::string("tcx_cn: ") + cudaGetErrorString(e));
        Trace tr_("tcx_cn", st);
        kern<<<grid, TCX_THREADS, TcxLayout<128>::SMEM, st>>>((const char*)Aplanes, (const char*)Bplanes, M, N, nkc,
                                                               cps, out, ldo, alpha, part, 0);
    }
    jdft_status s = check_launch("tcx_cn");
    if (s != JDFT_OK || !part) return s;
    {
        Trace tr_("tcx_reduce", st);
        tcx_reduce_kernel<<<dim3(NT / 2, tiles), dim3(TCX_M, TCX_RZ), 0, st>>>((const float4*)part, splits, tiles_m, NT,
                                                                               M, N, out, ldo, alpha, 0);
    }
    return check_launch("tcx_reduce");
}

}  // namespace jdft

using namespace jdft;

extern "C" jdft_status jdft_device_status(void* stream) {
    clear_error();
    JDFT_CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
    int v = 0;
    JDFT_CUDA_TRY(cudaMemcpyFromSymbol(&v, g_tc_status, sizeof(int)));
    if (v != 0) {
        const int zero = 0;
        JDFT_CUDA_TRY(cudaMemcpyToSymbol(g_tc_status, &zero, sizeof(int)));
        return set_error((jdft_status)v, "a bounded device-side wait gave up (tensor-core product skipped)");
    }
    return mlp_device_status();
}

extern "C" jdft_status jdft_set_wait_limit(double seconds) {
    clear_error();
    JDFT_CHECK_ARG(seconds >= 0.0 && seconds <= 60.0, "wait limit must be in [0, 60] s");
    const unsigned long long ns = (unsigned long long)(seconds * 1e9);
    JDFT_CUDA_TRY(cudaMemcpyToSymbol(g_tc_wait_ns, &ns, sizeof(ns)));
    return JDFT_OK;
}

namespace jdft {
// Time tcx_cn on split copies of A and B for split-K counts around one wave
// of blocks and keep the fastest for (M, N, K).
static jdft_status autotune_tcx(int M, int N, int K, const float2* A, int lda, const float2* B, int ldb, int* splits,
                                cudaStream_t st) {
    const size_t sa = (tcx_split_bytes(M, K) + 255) / 256 * 256, sb = (tcx_split_bytes(N, K) + 255) / 256 * 256;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int NT = N > 128 ? 256 : 128;
    const int tiles = ((M + TCX_M - 1) / TCX_M) * ((N + NT - 1) / NT);
    const int wave = std::max(1, sms / tiles);
    std::vector<int> cand;
    for (int f : {25, 50, 75, 100, 150, 200}) {
        const int c = std::max(1, wave * f / 100);
        if (std::find(cand.begin(), cand.end(), c) == cand.end()) cand.push_back(c);
    }
    // the partial buffer of the largest candidate (the products are timed as
    // the library runs them, with partial tiles and the reduction)
    const int cmax = *std::max_element(cand.begin(), cand.end());
    const size_t ob = ((size_t)M * N * sizeof(double2) + 255) / 256 * 256;
    const size_t pb = ((size_t)std::max(cmax, tcx_chunks(K) / 256 + 1) * tiles * TCX_M * NT * sizeof(float2) + 255) /
                      256 * 256;
    char* mem = nullptr;
    JDFT_CUDA_TRY(cudaMalloc(&mem, sa + sb + ob + pb));
    double2* out = (double2*)(mem + sa + sb);
    void* part = mem + sa + sb + ob;
    jdft_status s = tcx_split(A, lda, M, K, mem, st);
    if (s == JDFT_OK) s = tcx_split(B, ldb, N, K, mem + sa, st);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const auto key = std::make_tuple(M, N, K);
    float best = 1e30f;
    int best_c = wave;
    for (int c : cand) {
        if (s != JDFT_OK) break;
        {
            std::lock_guard<std::mutex> lk(g_tune_mu);
            g_tune_tcx[key] = c;
        }
        // one untimed call, then three timed ones (the accumulated values are not used)
        s = tcx_cn(M, N, K, mem, mem + sa, out, N, 1.0, st, part, pb);
        cudaEventRecord(e0, st);
        for (int r = 0; r < 3 && s == JDFT_OK; ++r) s = tcx_cn(M, N, K, mem, mem + sa, out, N, 1.0, st, part, pb);
        cudaEventRecord(e1, st);
        if (s != JDFT_OK) break;
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) {
            best = ms;
            best_c = c;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamSynchronize(st);
    cudaFree(mem);
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune_tcx[key] = best_c;
    }
    if (s != JDFT_OK) return s;
    if (splits) *splits = best_c;
    return JDFT_OK;
}
}  // namespace jdft

extern "C" jdft_status jdft_autotune_gemm(int M, int N, int K, const void* A, int lda, const void* B, int ldb,
                                          jdft_prec prec, int* splits, void* stream) {
    clear_error();
    JDFT_CHECK_ARG(M >= 1 && N >= 1 && K >= 1 && A && B && lda >= K && ldb >= K, "bad arguments");
    if (splits) *splits = 0;
    if (prec != JDFT_TF32X3 && prec != JDFT_BF16X3) return JDFT_OK;  // only the tensor-core products have schedules
    const int fmt = prec == JDFT_BF16X3 ? 1 : 0;
    const bool bf16 = fmt == 1;
    cudaStream_t st = (cudaStream_t)stream;
    if (tcx_eligible(prec, M, N)) return autotune_tcx(M, N, K, (const float2*)A, lda, (const float2*)B, ldb, splits, st);
    if (N <= 32) return JDFT_OK;  // the 32-column schedule is fixed
    int dflt, capmin;
    cn_schedule(M, N, K, dflt, capmin);
    const int nck = (K + TC_CPS - 1) / TC_CPS;
    std::vector<int> cand;
    for (int f : {50, 75, 100, 150, 200}) {
        const int c = std::max(capmin, std::min(nck, dflt * f / 100));
        if (c >= 1 && std::find(cand.begin(), cand.end(), c) == cand.end()) cand.push_back(c);
    }
    double2* out = nullptr;
    JDFT_CUDA_TRY(cudaMalloc(&out, (size_t)M * N * sizeof(double2)));
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const auto key = std::make_tuple(M, N, K, fmt);
    float best = 1e30f;
    int best_c = dflt;
    jdft_status s = JDFT_OK;
    for (int c : cand) {
        {
            std::lock_guard<std::mutex> lk(g_tune_mu);
            g_tune_cn[key] = c;
        }
        // one untimed call, then three timed ones (the accumulated values are not used)
        s = tc_zgemm_cn(M, N, K, (const float2*)A, lda, (const float2*)B, ldb, out, N, 1.0, bf16, st);
        if (s != JDFT_OK) break;
        cudaEventRecord(e0, st);
        for (int r = 0; r < 3 && s == JDFT_OK; ++r)
            s = tc_zgemm_cn(M, N, K, (const float2*)A, lda, (const float2*)B, ldb, out, N, 1.0, bf16, st);
        cudaEventRecord(e1, st);
        if (s != JDFT_OK) break;
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) {
            best = ms;
            best_c = c;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune_cn[key] = best_c;
    }
    if (s != JDFT_OK) return s;
    if (splits) *splits = best_c;
    return JDFT_OK;
}
