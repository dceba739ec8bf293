// Learned per-coefficient preconditioner for the band minimiser: a
// 3 -> 64 -> 64 -> 1 network (SiLU, SiLU, softplus) with BF16 weights and FP32
// accumulation, trained on the GPU from residual/correction pairs that the
// Teter-preconditioned minimiser produces.  (The JDFTx paper's minimiser,
// Sec. 2.1 Minimize, uses a fixed preconditioner; the learned one replaces
// the Teter polynomial.)
//
// Parameters (4481 floats): W1 (64x3 row-major), b1 (64), W2 (64x64), b2 (64),
// W3 (64), b3.  Features of coefficient G of band b:
//   f1 = kin_G / T_b,  f2 = log(1 + T_b),  f3 = (h_b - min h) / T_b,
// T_b the band kinetic energy, h_b = (C^dag H C)_bb.  Training rows:
// (f1, f2, f3, a = |R|^2, q = Re(conj(R) t)); loss sum (K^2 a - 2 K q) / sum a.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "chain.cuh"
#include "gemm.cuh"
#include "minimize.cuh"
#include "profile.cuh"
#include "tc_ptx.cuh"

namespace jdft {

constexpr int HID = 64;
constexpr int NPARAM = 3 * HID + HID + HID * HID + HID + HID + 1;  // 4481
constexpr int OW1 = 0, OB1 = 3 * HID, OW2 = OB1 + HID, OB2 = OW2 + HID * HID, OW3 = OB2 + HID, OB3 = OW3 + HID;

}  // namespace jdft

struct jdft_mlp_s {
    float* master = nullptr;          // FP32 parameters (device)
    __nv_bfloat16* wb = nullptr;      // BF16 copy used by the kernels
    float* m = nullptr;               // Adam moments
    float* v = nullptr;
    int step = 0;
};

namespace jdft {

__device__ __forceinline__ float sigmoidf_(float z) {
    const float e = expf(-fabsf(z));
    return z >= 0.f ? 1.f / (1.f + e) : e / (1.f + e);
}
__device__ __forceinline__ float siluf_(float z) { return z * sigmoidf_(z); }
// SiLU from the hardware exponential and an approximate quotient (a few ulp),
// for inference: the network's output only shapes search directions, and 128
// activations per coefficient make the IEEE forms the kernel's largest cost.
__device__ __forceinline__ float siluf_fast_(float z) {
    const float e = __expf(-fabsf(z));
    return z * __fdividef(z >= 0.f ? 1.f : e, 1.f + e);
}
__device__ __forceinline__ float dsiluf_(float z) {
    const float s = sigmoidf_(z);
    return s * (1.f + z * (1.f - s));
}
__device__ __forceinline__ float softplusf_(float z) { return fmaxf(z, 0.f) + log1pf(expf(-fabsf(z))); }

// Per-band features: bf[2b] = 1/T_b, bf[2b+1] = log(1 + T_b), bf[2nb + b] = (h_b - min h)/T_b.
__global__ void band_features_kernel(int nb, const double* __restrict__ Tb, const double2* __restrict__ Hs,
                                     float* __restrict__ bf) {
    __shared__ double hmin;
    if (threadIdx.x == 0) {
        double m = 1e300;
        for (int b = 0; b < nb; ++b) m = fmin(m, Hs[(size_t)b * nb + b].x);
        hmin = m;
    }
    __syncthreads();
    for (int b = threadIdx.x; b < nb; b += blockDim.x) {
        const double t = Tb[b];
        bf[2 * b] = (float)(1.0 / t);
        bf[2 * b + 1] = (float)log1p(t);
        bf[2 * nb + b] = (float)((Hs[(size_t)b * nb + b].x - hmin) / t);
    }
}

// ---------------------------------------------------------------------------
// Inference with the hidden layer on the tensor cores.  A block of 128
// threads takes tiles of 128 rows (one row per thread and tensor-memory lane):
// each thread forms its row's layer-1 activations h (FP32, SiLU) and writes
// them as h = hi + mid + lo in BF16 (h to about 2^-24 relative, as in FP32)
// into three 128 x 64 K-major tiles in shared memory; one thread issues the
// hidden layer a2 = W2 h as 12 tcgen05.mma (M = 128, N = 64, K = 16 each:
// each tile times the BF16 weights, FP32 accumulation in 64 tensor-memory
// columns) and commits them to
// an mbarrier; every thread then reads its row's 64 sums, adds b2, applies
// SiLU, the output layer and softplus.  The wait is bounded; one that gives
// up records JDFT_ERR_TIMEOUT (jdft_device_status) and stops the block after
// waiting for the products already issued.
// ---------------------------------------------------------------------------
constexpr int MT = 128;                      // rows per tile = threads per block
constexpr int MT_ATILE = MT * HID * 2;       // bytes of one BF16 activation tile (16 KB)
constexpr int MT_BTILE = HID * HID * 2;      // bytes of the BF16 W2 tile (8 KB)
constexpr unsigned long long MLP_WAIT_NS = 2000000000ull;
__device__ int g_mlp_status = 0;

// Byte offset of (row r, k) in a K-major tile of 64 values per row: 8-row x
// 8-value core matrices of 128 bytes, K-adjacent ones 128 bytes apart, 8-row
// groups 1024 bytes apart.
__device__ __forceinline__ uint32_t mlp_core_off(int r, int k) {
    return (uint32_t)((r >> 3) * 1024 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

__device__ __forceinline__ uint32_t bf2_bits(float a, float b) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<const uint32_t*>(&v);
}

// MODE 0: K[r] for feature triples feats[3 r ..]; MODE 1: KG = K G for every
// coefficient of an (npw x nb) block (features from kin and the band features).
// The inference kernel keeps W1, b1 ([0, OW2) of the parameters) and b2, W3, b3
// ([OB2, NPARAM)) in shared memory as FP32, at these offsets.
constexpr int MLP_WSMALL = OW2 + (NPARAM - OB2);
constexpr int WS_OB2 = OW2, WS_OW3 = OW2 + (OW3 - OB2), WS_OB3 = OW2 + (OB3 - OB2);

template <int MODE, typename T>
__global__ void __launch_bounds__(MT) mlp_tc_kernel(int64_t rows, const float* __restrict__ feats,
                                                    float* __restrict__ Kout, int npw, int nb,
                                                    const c_t<T>* __restrict__ G, int ldg, c_t<T>* __restrict__ KG,
                                                    int ldk, const double* __restrict__ kin,
                                                    const float* __restrict__ bf,
                                                    const __nv_bfloat16* __restrict__ wb) {
    extern __shared__ __align__(1024) unsigned char sraw[];
    unsigned char* sm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(sraw) + 1023) & ~(uintptr_t)1023);
    unsigned char* Ahi = sm;
    unsigned char* Amid = sm + MT_ATILE;
    unsigned char* Alo = sm + 2 * MT_ATILE;
    unsigned char* Bt = sm + 3 * MT_ATILE;
    // the CUDA-core layers' parameters: W1, b1, b2, W3, b3 (W2 is the B operand)
    float* w = reinterpret_cast<float*>(Bt + MT_BTILE);
    uint64_t* bar = reinterpret_cast<uint64_t*>(w + MLP_WSMALL + 3);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 1);
    const int tid = threadIdx.x, warp = tid >> 5;
    for (int i = tid; i < MLP_WSMALL; i += MT)
        w[i] = __bfloat162float(wb[i < OW2 ? i : i - OW2 + OB2]);  // [0, OW2) then [OB2, NPARAM)
    // W2 as the B operand: row j (output), K = i (input)
    for (int e = tid; e < HID * HID / 2; e += MT) {
        const int j = (2 * e) / HID, i = (2 * e) % HID;
        *reinterpret_cast<__nv_bfloat162*>(Bt + mlp_core_off(j, i)) =
            __halves2bfloat162(wb[OW2 + HID * j + i], wb[OW2 + HID * j + i + 1]);
    }
    if (tid == 0) {
        tc::mbar_init(bar, 1);
        tc::mbar_fence_init();
    }
    if (warp == 0) tc::tmem_alloc(tslot, 64);
    tc::fence_proxy_async_smem();
    tc::tc_fence_before_sync();
    __syncthreads();
    tc::tc_fence_after_sync();
    const uint32_t tmem = *tslot;
    const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
    constexpr uint32_t idesc = tc::instr_desc(1u, MT, HID);
    const int64_t tiles = (rows + MT - 1) / MT;
    int ok = 1;
    uint32_t phase = 0;
    for (int64_t tl = blockIdx.x; tl < tiles && ok; tl += gridDim.x) {
        const int64_t r = tl * MT + tid;
        const bool act = r < rows;
        float f0 = 0.f, f1 = 0.f, f2 = 0.f;
        int64_t b = 0, gq = 0;
        if (act) {
            if constexpr (MODE == 0) {
                f0 = feats[3 * r];
                f1 = feats[3 * r + 1];
                f2 = feats[3 * r + 2];
            } else {
                b = r / npw;
                gq = r - b * npw;
                f0 = (float)kin[gq] * bf[2 * b];
                f1 = bf[2 * b + 1];
                f2 = bf[2 * nb + b];
            }
        }
        // layer 1 -> the hi / lo activation tiles, 8 values (16 bytes) at a time
#pragma unroll 1
        for (int k0 = 0; k0 < HID; k0 += 8) {
            float h[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int i = k0 + q;
                h[q] = siluf_fast_(w[OW1 + 3 * i] * f0 + w[OW1 + 3 * i + 1] * f1 + w[OW1 + 3 * i + 2] * f2 +
                                   w[OB1 + i]);
            }
            uint32_t hi[4], mid[4], lo[4];
#pragma unroll
            for (int q = 0; q < 8; q += 2) {
                const __nv_bfloat162 hh = __floats2bfloat162_rn(h[q], h[q + 1]);
                const float r0 = h[q] - __low2float(hh), r1 = h[q + 1] - __high2float(hh);
                const __nv_bfloat162 mm = __floats2bfloat162_rn(r0, r1);
                hi[q / 2] = *reinterpret_cast<const uint32_t*>(&hh);
                mid[q / 2] = *reinterpret_cast<const uint32_t*>(&mm);
                lo[q / 2] = bf2_bits(r0 - __low2float(mm), r1 - __high2float(mm));
            }
            const uint32_t o = mlp_core_off(tid, k0);
            *reinterpret_cast<uint4*>(Ahi + o) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
            *reinterpret_cast<uint4*>(Amid + o) = make_uint4(mid[0], mid[1], mid[2], mid[3]);
            *reinterpret_cast<uint4*>(Alo + o) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
        }
        tc::fence_proxy_async_smem();
        tc::tc_fence_before_sync();
        __syncthreads();
        if (tid == 0) {
            tc::tc_fence_after_sync();
            const uint32_t ah = tc::smem_addr(Ahi), am = tc::smem_addr(Amid), al = tc::smem_addr(Alo);
            const uint32_t bb = tc::smem_addr(Bt);
#pragma unroll
            for (int s = 0; s < HID / 16; ++s) {
                const uint64_t db = tc::smem_desc(bb + s * 256, 128, 1024);
                tc::mma_bf16(tmem, tc::smem_desc(ah + s * 256, 128, 1024), db, idesc, s > 0 ? 1u : 0u);
                tc::mma_bf16(tmem, tc::smem_desc(am + s * 256, 128, 1024), db, idesc, 1u);
                tc::mma_bf16(tmem, tc::smem_desc(al + s * 256, 128, 1024), db, idesc, 1u);
            }
            tc::mma_commit(bar);
        }
        const int w_ok = tc::mbar_wait_ns(bar, phase, MLP_WAIT_NS) ? 1 : 0;
        ok = __syncthreads_and(w_ok);
        if (!ok) {
            // the products may still run: wait for them (fixed limit) before leaving
            tc::mbar_wait_ns(bar, phase, MLP_WAIT_NS);
            if (tid == 0) atomicExch(&g_mlp_status, (int)JDFT_ERR_TIMEOUT);
            break;
        }
        phase ^= 1u;
        tc::tc_fence_after_sync();
        float z = w[WS_OB3];
#pragma unroll 1
        for (int c = 0; c < HID; c += 16) {
            float acc[16];
            tc::tmem_ld16(lane_base + c, acc);
#pragma unroll
            for (int q = 0; q < 16; ++q) z += w[WS_OW3 + c + q] * siluf_fast_(acc[q] + w[WS_OB2 + c + q]);
        }
        const float Kv = softplusf_(z);
        if (act) {
            if constexpr (MODE == 0) {
                Kout[r] = Kv;
            } else {
                const c_t<T> v = G[b * ldg + gq];
                KG[b * ldk + gq] = mk<T>((T)(Kv * v.x), (T)(Kv * v.y));
            }
        }
        tc::tc_fence_before_sync();
        __syncthreads();  // every lane's tensor-memory reads and tile reads are done before the next tile
    }
    tc::tc_fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, 64);
}

constexpr size_t MLP_TC_SMEM = 1024 + 3 * MT_ATILE + MT_BTILE + (MLP_WSMALL + 3) * sizeof(float) + 64;

// Persistent grid of the tensor-core inference kernel: two blocks per SM
// (shared memory; their 64 tensor-memory columns each fit easily).
static int mlp_tc_grid(int64_t rows) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t tiles = (rows + MT - 1) / MT;
    // three blocks per SM: shared memory (about 59 KB each) and tensor memory (64 columns each) allow it
    return (int)std::max<int64_t>(1, std::min<int64_t>(tiles, (int64_t)std::max(1, sms) * 3));
}

jdft_status mlp_device_status() {
    int v = 0;
    JDFT_CUDA_TRY(cudaMemcpyFromSymbol(&v, g_mlp_status, sizeof(int)));
    if (v != 0) {
        const int zero = 0;
        JDFT_CUDA_TRY(cudaMemcpyToSymbol(g_mlp_status, &zero, sizeof(int)));
        return set_error((jdft_status)v, "a bounded device-side wait gave up (preconditioner network)");
    }
    return JDFT_OK;
}

// ---------------------------------------------------------------------------
// Training: loss and gradient over rows.  128 rows per tile, one row per
// thread; persistent blocks keep their share of the W2 gradient in registers
// across tiles and add everything to the global FP32 gradient once.
// ---------------------------------------------------------------------------
constexpr int TR = 128;       // rows per tile = threads per block
constexpr int LD = HID + 1;   // padded row stride of the activation tiles
constexpr int NSMALL = 449;   // W1 (192), b1 (64), b2 (64), W3 (64), unused, b3 at 448

__global__ void __launch_bounds__(TR) mlp_grad_kernel(int64_t rows, const float* __restrict__ data,
                                                      const __nv_bfloat16* __restrict__ wb,
                                                      const double* __restrict__ suma, float* __restrict__ grad,
                                                      double* __restrict__ loss) {
    extern __shared__ __align__(16) float sm[];
    float* w = sm;                        // NPARAM
    float* H1 = w + NPARAM + 3;           // TR x LD   silu(a1)
    float* A1 = H1 + TR * LD;             // TR x LD   a1, then da1
    float* A2 = A1 + TR * LD;             // TR x LD   a2, then da2
    float* F = A2 + TR * LD;              // TR x 3
    float* gsm = F + 3 * TR;              // NSMALL small-parameter gradients
    for (int i = threadIdx.x; i < NPARAM; i += blockDim.x) w[i] = __bfloat162float(wb[i]);
    for (int i = threadIdx.x; i < NSMALL; i += blockDim.x) gsm[i] = 0.f;
    const float inv = (float)(1.0 / *suma);
    float gW2[HID * HID / TR];            // entries e = tid + TR k of W2's gradient
#pragma unroll
    for (int k = 0; k < HID * HID / TR; ++k) gW2[k] = 0.f;
    double lsum = 0.0;
    const int r = threadIdx.x;
    __syncthreads();
    for (int64_t t0 = (int64_t)blockIdx.x * TR; t0 < rows; t0 += (int64_t)gridDim.x * TR) {
        const int64_t row = t0 + r;
        const bool live = row < rows;
        float f0 = 0.f, f1 = 0.f, f2 = 0.f, a = 0.f, q = 0.f;
        if (live) {
            const float* d = data + 5 * row;
            f0 = d[0]; f1 = d[1]; f2 = d[2]; a = d[3]; q = d[4];
        }
        F[3 * r] = f0; F[3 * r + 1] = f1; F[3 * r + 2] = f2;
        float h1[HID];
#pragma unroll
        for (int i = 0; i < HID; ++i) {
            const float z1 = w[OW1 + 3 * i] * f0 + w[OW1 + 3 * i + 1] * f1 + w[OW1 + 3 * i + 2] * f2 + w[OB1 + i];
            A1[r * LD + i] = z1;
            h1[i] = siluf_(z1);
            H1[r * LD + i] = h1[i];
        }
        float z = w[OB3];
        for (int j = 0; j < HID; ++j) {
            float acc = w[OB2 + j];
#pragma unroll
            for (int i = 0; i < HID; ++i) acc += w[OW2 + HID * j + i] * h1[i];
            A2[r * LD + j] = acc;
            z += w[OW3 + j] * siluf_(acc);
        }
        const float K = softplusf_(z);
        float dz = 0.f;
        if (live) {
            lsum += ((double)K * K * a - 2.0 * K * q) * (double)inv;
            dz = (2.f * K * a - 2.f * q) * inv * sigmoidf_(z);
        }
        // da2 = dz W3 silu'(a2); gradients of W3, b2, b3
        for (int j = 0; j < HID; ++j) {
            const float a2 = A2[r * LD + j];
            const float da2 = dz * w[OW3 + j] * dsiluf_(a2);
            A2[r * LD + j] = da2;
            if (dz != 0.f) {
                atomicAdd(&gsm[320 + j], dz * siluf_(a2));
                atomicAdd(&gsm[256 + j], da2);
            }
        }
        if (dz != 0.f) atomicAdd(&gsm[448], dz);
        __syncthreads();
        // da1 = (W2^T da2) silu'(a1)
        for (int i = 0; i < HID; ++i) {
            float acc = 0.f;
#pragma unroll 8
            for (int j = 0; j < HID; ++j) acc += w[OW2 + HID * j + i] * A2[r * LD + j];
            A1[r * LD + i] = acc * dsiluf_(A1[r * LD + i]);
        }
        __syncthreads();
        // reductions over the tile's rows: W2 (registers), W1 and b1 (one owner thread each)
#pragma unroll 4
        for (int k = 0; k < HID * HID / TR; ++k) {
            const int e = threadIdx.x + TR * k;
            const int j = e / HID, i = e % HID;
            float acc = 0.f;
            for (int rr = 0; rr < TR; ++rr) acc += A2[rr * LD + j] * H1[rr * LD + i];
            gW2[k] += acc;
        }
        for (int e = threadIdx.x; e < 3 * HID + HID; e += TR) {
            float acc = 0.f;
            if (e < 3 * HID) {
                const int i = e / 3, c = e % 3;
                for (int rr = 0; rr < TR; ++rr) acc += A1[rr * LD + i] * F[3 * rr + c];
            } else {
                const int i = e - 3 * HID;
                for (int rr = 0; rr < TR; ++rr) acc += A1[rr * LD + i];
            }
            gsm[e] += acc;
        }
        __syncthreads();
    }
    // flush: W1 and b1 are contiguous at the start of the parameter vector
    for (int e = threadIdx.x; e < 3 * HID + HID; e += TR) atomicAdd(&grad[OW1 + e], gsm[e]);
    for (int j = threadIdx.x; j < HID; j += TR) {
        atomicAdd(&grad[OB2 + j], gsm[256 + j]);
        atomicAdd(&grad[OW3 + j], gsm[320 + j]);
    }
    if (threadIdx.x == 0) atomicAdd(&grad[OB3], gsm[448]);
#pragma unroll
    for (int k = 0; k < HID * HID / TR; ++k) atomicAdd(&grad[OW2 + threadIdx.x + TR * k], gW2[k]);
    __shared__ double red[TR / 32];
    for (int o = 16; o > 0; o >>= 1) lsum += __shfl_down_sync(0xffffffffu, lsum, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = lsum;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < TR / 32; ++i) s += red[i];
        atomicAdd(loss, s);
    }
}

__global__ void sum_a_kernel(int64_t rows, const float* __restrict__ data, double* out) {
    double acc = 0.0;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < rows; r += (int64_t)gridDim.x * blockDim.x)
        acc += data[5 * r + 3];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(out, acc);
}

__global__ void adam_kernel(float* __restrict__ p, __nv_bfloat16* __restrict__ wb, float* __restrict__ m,
                            float* __restrict__ v, const float* __restrict__ g, float lr, float b1, float b2, float eps,
                            float c1, float c2) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < NPARAM; i += gridDim.x * blockDim.x) {
        const float gi = g[i];
        m[i] = b1 * m[i] + (1.f - b1) * gi;
        v[i] = b2 * v[i] + (1.f - b2) * gi * gi;
        p[i] -= lr * (m[i] / c1) / (sqrtf(v[i] / c2) + eps);
        wb[i] = __float2bfloat16_rn(p[i]);
    }
}

__global__ void to_bf16_kernel(const float* __restrict__ p, __nv_bfloat16* __restrict__ wb) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < NPARAM; i += gridDim.x * blockDim.x)
        wb[i] = __float2bfloat16_rn(p[i]);
}

// Training rows from a snapshot: coefficients i = offset + r*stride of the
// band-major block give (f1, f2, f3, |G|^2, Re(conj(G) t)).
__global__ void make_rows_kernel(int npw, int nb, const double2* __restrict__ G, const double2* __restrict__ Tt,
                                 const double* __restrict__ kin, const float* __restrict__ bf, int64_t stride,
                                 int64_t offset, int64_t nrows, float* __restrict__ out) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < nrows; r += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = offset + r * stride;
        const int64_t b = i / npw, g = i - b * npw;
        const double2 x = G[b * npw + g], t = Tt[b * npw + g];
        float* o = out + 5 * r;
        o[0] = (float)kin[g] * bf[2 * b];
        o[1] = bf[2 * b + 1];
        o[2] = bf[2 * nb + b];
        o[3] = (float)(x.x * x.x + x.y * x.y);
        o[4] = (float)(x.x * t.x + x.y * t.y);
    }
}

// Tb[b] = Omega sum_G kin |C_Gb|^2 (one block per band)
__global__ void rows_band_kinetic_kernel(int npw, const double2* __restrict__ C, const double* __restrict__ kin,
                                         double omega, double* __restrict__ Tb) {
    const int b = blockIdx.x;
    double acc = 0.0;
    for (int g = threadIdx.x; g < npw; g += blockDim.x) {
        const double2 c = C[(size_t)b * npw + g];
        acc += kin[g] * (c.x * c.x + c.y * c.y);
    }
    __shared__ double red[8];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
        Tb[b] = omega * t;
    }
}

__global__ void rows_scale_kernel(int n, const double2* __restrict__ A, double alpha, double2* __restrict__ B) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x)
        B[e] = make_double2(alpha * A[e].x, alpha * A[e].y);
}

// sums[0] += a, sums[1] += q over the rows
__global__ void rows_sums_kernel(int64_t n, const float* __restrict__ rows, double* __restrict__ sums) {
    double a = 0.0, q = 0.0;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
        a += rows[5 * r + 3];
        q += rows[5 * r + 4];
    }
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        q += __shfl_down_sync(0xffffffffu, q, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&sums[0], a);
        atomicAdd(&sums[1], q);
    }
}

// q <- q * sum(a) / sum(q): the best constant K of the scaled rows is 1
__global__ void rows_normalize_kernel(int64_t n, float* __restrict__ rows, const double* __restrict__ sums) {
    const double s = sums[1] != 0.0 ? sums[0] / sums[1] : 1.0;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x)
        rows[5 * r + 4] = (float)(rows[5 * r + 4] * s);
}

static int grid_rows(int64_t rows, int per) {
    return (int)std::min<int64_t>(std::max<int64_t>((rows + per - 1) / per, 1), 152 * 8);
}

template <typename T>
jdft_status mlp_precondition(jdft_mlp_t mlp, int npw, int nb, const c_t<T>* G, int ldg, c_t<T>* KG, int ldk,
                             const double* kin, const double* Tb, const double2* Hs, float* bf, cudaStream_t st) {
    {
        Trace tr_("mlp_band_features", st);
        band_features_kernel<<<1, 256, 0, st>>>(nb, Tb, Hs, bf);
    }
    jdft_status s = check_launch("band_features");
    if (s != JDFT_OK) return s;
    {
        auto kern = mlp_tc_kernel<1, T>;
        cudaError_t e = set_smem_attr((const void*)kern, MLP_TC_SMEM);
        if (e != cudaSuccess) return set_error(JDFT_ERR_CUDA, std::string("mlp_precond: ") + cudaGetErrorString(e));
        const int64_t rows = (int64_t)npw * nb;
        Trace tr_("mlp_precond", st);
        kern<<<mlp_tc_grid(rows), MT, MLP_TC_SMEM, st>>>(rows, nullptr, nullptr, npw, nb, G, ldg, KG, ldk, kin, bf,
                                                         mlp->wb);
    }
    return check_launch("mlp_precond");
}
template jdft_status mlp_precondition<double>(jdft_mlp_t, int, int, const double2*, int, double2*, int, const double*,
                                              const double*, const double2*, float*, cudaStream_t);
template jdft_status mlp_precondition<float>(jdft_mlp_t, int, int, const float2*, int, float2*, int, const double*,
                                             const double*, const double2*, float*, cudaStream_t);

}  // namespace jdft

using namespace jdft;

extern "C" {

jdft_status jdft_mlp_create(const float* params, jdft_mlp_t* out) {
    clear_error();
    JDFT_CHECK_ARG(params && out, "null argument");
    jdft_mlp_s* m = new jdft_mlp_s();
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, NPARAM * (3 * sizeof(float)) + NPARAM * sizeof(__nv_bfloat16) + 256);
    if (e != cudaSuccess) {
        delete m;
        return set_error(JDFT_ERR_OOM, "jdft_mlp_create: cudaMalloc failed");
    }
    m->master = (float*)p;
    m->m = m->master + NPARAM;
    m->v = m->m + NPARAM;
    m->wb = (__nv_bfloat16*)(m->v + NPARAM);
    JDFT_CUDA_TRY(cudaMemcpy(m->master, params, NPARAM * sizeof(float), cudaMemcpyHostToDevice));
    JDFT_CUDA_TRY(cudaMemset(m->m, 0, 2 * NPARAM * sizeof(float)));
    {
        Trace tr_("mlp_to_bf16", 0);
        to_bf16_kernel<<<18, 256>>>(m->master, m->wb);
    }
    JDFT_CUDA_TRY(cudaDeviceSynchronize());
    *out = m;
    return JDFT_OK;
}

jdft_status jdft_mlp_destroy(jdft_mlp_t m) {
    if (!m) return JDFT_OK;
    cudaFree(m->master);
    delete m;
    return JDFT_OK;
}

jdft_status jdft_mlp_get_params(jdft_mlp_t m, float* params) {
    clear_error();
    JDFT_CHECK_ARG(m && params, "null argument");
    JDFT_CUDA_TRY(cudaMemcpy(params, m->master, NPARAM * sizeof(float), cudaMemcpyDeviceToHost));
    return JDFT_OK;
}

jdft_status jdft_mlp_forward(jdft_mlp_t m, int64_t rows, const float* feats, float* K, void* stream) {
    clear_error();
    JDFT_CHECK_ARG(m && rows >= 0 && (rows == 0 || (feats && K)), "bad arguments");
    if (rows == 0) return JDFT_OK;
    cudaStream_t st = (cudaStream_t)stream;
    {
        auto kern = mlp_tc_kernel<0, float>;
        cudaError_t e = set_smem_attr((const void*)kern, MLP_TC_SMEM);
        if (e != cudaSuccess) return set_error(JDFT_ERR_CUDA, std::string("mlp_forward: ") + cudaGetErrorString(e));
        Trace tr_("mlp_forward", st);
        kern<<<mlp_tc_grid(rows), MT, MLP_TC_SMEM, st>>>(rows, feats, K, 0, 0, nullptr, 0, nullptr, 0, nullptr,
                                                         nullptr, m->wb);
    }
    return check_launch("mlp_forward");
}

jdft_status jdft_mlp_loss_grad(jdft_mlp_t m, int64_t rows, const float* data, float* grad, double* loss,
                               void* stream) {
    clear_error();
    JDFT_CHECK_ARG(m && rows > 0 && data && grad && loss, "bad arguments");
    cudaStream_t st = (cudaStream_t)stream;
    double* suma = loss + 1;
    JDFT_CUDA_TRY(cudaMemsetAsync(loss, 0, 2 * sizeof(double), st));
    JDFT_CUDA_TRY(cudaMemsetAsync(grad, 0, NPARAM * sizeof(float), st));
    {
        Trace tr_("mlp_sum_a", st);
        sum_a_kernel<<<grid_rows(rows, 256), 256, 0, st>>>(rows, data, suma);
    }
    jdft_status s = check_launch("sum_a");
    if (s != JDFT_OK) return s;
    const size_t smem = (NPARAM + 3 + 3 * TR * LD + 3 * TR + NSMALL) * sizeof(float);
    JDFT_CUDA_TRY(set_smem_attr((const void*)mlp_grad_kernel, smem));
    const int tiles = (int)std::min<int64_t>((rows + TR - 1) / TR, 152 * 2);
    {
        Trace tr_("mlp_grad", st);
        mlp_grad_kernel<<<tiles, TR, smem, st>>>(rows, data, m->wb, suma, grad, loss);
    }
    return check_launch("mlp_grad");
}

jdft_status jdft_mlp_adam_step(jdft_mlp_t m, const float* grad, float lr, void* stream) {
    clear_error();
    JDFT_CHECK_ARG(m && grad && lr > 0, "bad arguments");
    cudaStream_t st = (cudaStream_t)stream;
    m->step += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - powf(b1, (float)m->step), c2 = 1.f - powf(b2, (float)m->step);
    {
        Trace tr_("mlp_adam", st);
        adam_kernel<<<18, 256, 0, st>>>(m->master, m->wb, m->m, m->v, grad, lr, b1, b2, 1e-8f, c1, c2);
    }
    return check_launch("mlp_adam");
}

jdft_status jdft_mlp_rows(jdft_basis_t b, int ik, const void* C, const void* Cstar, int nb, int64_t stride,
                          int64_t offset, float* rows_out, int64_t* nrows, void* stream) {
    clear_error();
    JDFT_CHECK_ARG(b && C && Cstar && nrows && nb >= 1 && stride >= 1 && offset >= 0, "bad arguments");
    JDFT_CHECK_ARG(ik >= 0 && ik < b->nk, "k-point index out of range");
    const int npw = b->ks[ik].npw;
    const int64_t total = (int64_t)npw * nb;
    const int64_t n = offset < total ? (total - offset + stride - 1) / stride : 0;
    if (!rows_out) { *nrows = n; return JDFT_OK; }
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<void*> bufs;
    auto alloc = [&](size_t bytes) -> void* {
        void* p = nullptr;
        if (cudaMalloc(&p, bytes) != cudaSuccess) return nullptr;
        bufs.push_back(p);
        return p;
    };
    auto done = [&](jdft_status r) {
        cudaStreamSynchronize(st);
        for (void* p : bufs) cudaFree(p);
        return r;
    };
    const size_t blk = (size_t)nb * npw * sizeof(double2);
    double2* HC = (double2*)alloc(blk);
    double2* G = (double2*)alloc(blk);
    double2* Tt = (double2*)alloc(blk);
    double2* Hs = (double2*)alloc((size_t)nb * nb * sizeof(double2));
    double2* M = (double2*)alloc((size_t)nb * nb * sizeof(double2));
    double2* Bm = (double2*)alloc((size_t)nb * nb * sizeof(double2));
    double* Tb = (double*)alloc(nb * sizeof(double));
    float* bf = (float*)alloc(3 * (size_t)nb * sizeof(float));
    double* sums = (double*)alloc(2 * sizeof(double));
    if (!HC || !G || !Tt || !Hs || !M || !Bm || !Tb || !bf || !sums)
        return done(set_error(JDFT_ERR_OOM, "jdft_mlp_rows"));
    const double2* Cd = (const double2*)C;
    const double2* Cs = (const double2*)Cstar;
    jdft_status s;
    // residual block G = HC - Omega C (C^dag H C)
    if ((s = jdft_apply_H(b, ik, Cd, npw, HC, npw, nb, JDFT_FP64, stream))) return done(s);
    if (cudaMemsetAsync(Hs, 0, (size_t)nb * nb * sizeof(double2), st) != cudaSuccess)
        return done(set_error(JDFT_ERR_CUDA, "memset"));
    if ((s = zgemm_cn<double>(nb, nb, npw, Cd, npw, HC, npw, Hs, nb, 1.0, st))) return done(s);
    if (cudaMemcpyAsync(G, HC, blk, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return done(set_error(JDFT_ERR_CUDA, "copy"));
    {
        Trace tr_("mlp_rows_scale", st);
        rows_scale_kernel<<<grid_rows((int64_t)nb * nb, 256), 256, 0, st>>>(nb * nb, Hs, -b->omega, Bm);
    }
    if ((s = check_launch("rows_scale"))) return done(s);
    if ((s = zgemm_nn_acc<double>(npw, nb, nb, Cd, npw, Bm, nb, G, npw, st))) return done(s);
    // target t = C - C* (Omega C*^dag C)
    if (cudaMemsetAsync(M, 0, (size_t)nb * nb * sizeof(double2), st) != cudaSuccess)
        return done(set_error(JDFT_ERR_CUDA, "memset"));
    if ((s = zgemm_cn<double>(nb, nb, npw, Cs, npw, Cd, npw, M, nb, -b->omega, st))) return done(s);
    if (cudaMemcpyAsync(Tt, Cd, blk, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return done(set_error(JDFT_ERR_CUDA, "copy"));
    if ((s = zgemm_nn_acc<double>(npw, nb, nb, Cs, npw, M, nb, Tt, npw, st))) return done(s);
    // features
    {
        Trace tr_("mlp_rows_band_kinetic", st);
        rows_band_kinetic_kernel<<<nb, 256, 0, st>>>(npw, Cd, b->ks[ik].kin, b->omega, Tb);
    }
    if ((s = check_launch("rows_band_kinetic"))) return done(s);
    {
        Trace tr_("mlp_band_features", st);
        band_features_kernel<<<1, 256, 0, st>>>(nb, Tb, Hs, bf);
    }
    if ((s = check_launch("band_features"))) return done(s);
    if (n > 0) {
        Trace tr_("mlp_make_rows", st);
        make_rows_kernel<<<grid_rows(n, 256), 256, 0, st>>>(npw, nb, G, Tt, b->ks[ik].kin, bf, stride, offset, n,
                                                           rows_out);
    }
    if ((s = check_launch("make_rows"))) return done(s);
    if (n > 0) {
        if (cudaMemsetAsync(sums, 0, 2 * sizeof(double), st) != cudaSuccess)
            return done(set_error(JDFT_ERR_CUDA, "memset"));
        {
            Trace tr_("mlp_rows_sums", st);
            rows_sums_kernel<<<grid_rows(n, 256), 256, 0, st>>>(n, rows_out, sums);
        }
        if ((s = check_launch("rows_sums"))) return done(s);
        {
            Trace tr_("mlp_rows_normalize", st);
            rows_normalize_kernel<<<grid_rows(n, 256), 256, 0, st>>>(n, rows_out, sums);
        }
        if ((s = check_launch("rows_normalize"))) return done(s);
    }
    *nrows = n;
    return done(JDFT_OK);
}

}  // extern "C"
