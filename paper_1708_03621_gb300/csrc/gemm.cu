// Complex GEMMs on the CUDA cores (FP64 and FP32): the projector products
// P^dag C and P (D B) of the nonlocal pseudopotential term (JDFTx paper,
// Sec. 2.2, pseudopotentials), and the subspace matrices C^dag H C and
// C^dag O C of the band minimiser (Sec. 2.1, Minimize; O diagonal in the
// plane-wave basis).
#include <algorithm>

#include <type_traits>

#include "gemm.cuh"
#include "profile.cuh"

namespace jdft {

// ---------------------------------------------------------------------------
// C^dag-style product with split K.  Tile 32 x 32 outputs, 16-deep K slices,
// 256 threads, 2 x 2 outputs per thread.  Each split adds its partial sum to
// the FP64 output with atomics.
// ---------------------------------------------------------------------------
constexpr int CN_BM = 32, CN_BN = 32, CN_BK = 16;

template <typename T>
__global__ void __launch_bounds__(256) zgemm_cn_kernel(int M, int N, int K, int kchunk, const c_t<T>* __restrict__ A,
                                                       int lda, const c_t<T>* __restrict__ B, int ldb,
                                                       double2* __restrict__ out, int ldo, double scale) {
    __shared__ c_t<T> As[CN_BK][CN_BM + 1];
    __shared__ c_t<T> Bs[CN_BK][CN_BN + 1];
    const int m0 = blockIdx.x * CN_BM, n0 = blockIdx.y * CN_BN;
    const int kA = blockIdx.z * kchunk, kB = min(K, kA + kchunk);
    const int tm = threadIdx.x / 16, tn = threadIdx.x % 16;
    c_t<T> acc[2][2];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j) acc[i][j] = mk<T>(T(0), T(0));
    for (int k0 = kA; k0 < kB; k0 += CN_BK) {
        for (int e = threadIdx.x; e < CN_BM * CN_BK; e += 256) {
            const int r = e / CN_BK, kk = e % CN_BK;
            const int m = m0 + r, k = k0 + kk;
            As[kk][r] = (m < M && k < kB) ? A[(size_t)m * lda + k] : mk<T>(T(0), T(0));
            const int n = n0 + r;
            Bs[kk][r] = (n < N && k < kB) ? B[(size_t)n * ldb + k] : mk<T>(T(0), T(0));
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < CN_BK; ++kk) {
            c_t<T> a[2] = {As[kk][tm], As[kk][tm + 16]};
            c_t<T> b[2] = {Bs[kk][tn], Bs[kk][tn + 16]};
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    // conj(a) * b
                    acc[i][j].x += a[i].x * b[j].x + a[i].y * b[j].y;
                    acc[i][j].y += a[i].x * b[j].y - a[i].y * b[j].x;
                }
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const int m = m0 + tm + 16 * i, n = n0 + tn + 16 * j;
            if (m < M && n < N) {
                atomicAdd(&out[(size_t)m * ldo + n].x, scale * (double)acc[i][j].x);
                atomicAdd(&out[(size_t)m * ldo + n].y, scale * (double)acc[i][j].y);
            }
        }
}

template <typename T>
jdft_status zgemm_cn(int M, int N, int K, const c_t<T>* A, int lda, const c_t<T>* B, int ldb, double2* out, int ldo,
                     double scale, cudaStream_t st) {
    if (M == 0 || N == 0 || K == 0) return JDFT_OK;
    const int tiles = ((M + CN_BM - 1) / CN_BM) * ((N + CN_BN - 1) / CN_BN);
    // enough K splits for ~4 blocks per SM, each at least 64 deep
    int splits = std::max(1, (152 * 4 + tiles - 1) / tiles);
    splits = std::min(splits, std::max(1, K / 64));
    int kchunk = (K + splits - 1) / splits;
    kchunk = (kchunk + CN_BK - 1) / CN_BK * CN_BK;
    splits = (K + kchunk - 1) / kchunk;
    dim3 grid((M + CN_BM - 1) / CN_BM, (N + CN_BN - 1) / CN_BN, splits);
    {
        Trace tr_("zgemm_cn", st);
        zgemm_cn_kernel<T><<<grid, 256, 0, st>>>(M, N, K, kchunk, A, lda, B, ldb, out, ldo, scale);
    }
    return check_launch("zgemm_cn");
}

// ---------------------------------------------------------------------------
// out[n][m] += sum_i A[i][m] Bm[i][n]: tile 64 (m) x 16 (n), 16-deep i slices,
// each thread one m and 4 n.
// ---------------------------------------------------------------------------
constexpr int NN_BM = 64, NN_BN = 16, NN_BK = 16;

template <typename T>
__global__ void __launch_bounds__(256) zgemm_nn_kernel(int M, int N, int K, const c_t<T>* __restrict__ A, int lda,
                                                       const c_t<T>* __restrict__ Bm, int ldb, c_t<T>* __restrict__ out,
                                                       int ldo, bool accumulate) {
    __shared__ c_t<T> As[NN_BK][NN_BM];
    __shared__ c_t<T> Bs[NN_BK][NN_BN];
    const int m0 = blockIdx.x * NN_BM, n0 = blockIdx.y * NN_BN;
    const int tm = threadIdx.x % NN_BM, tq = threadIdx.x / NN_BM;  // tq in 0..3
    c_t<T> acc[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[j] = mk<T>(T(0), T(0));
    for (int k0 = 0; k0 < K; k0 += NN_BK) {
        for (int e = threadIdx.x; e < NN_BK * NN_BM; e += 256) {
            const int kk = e / NN_BM, r = e % NN_BM;
            const int m = m0 + r, k = k0 + kk;
            As[kk][r] = (m < M && k < K) ? A[(size_t)k * lda + m] : mk<T>(T(0), T(0));
        }
        for (int e = threadIdx.x; e < NN_BK * NN_BN; e += 256) {
            const int kk = e / NN_BN, c = e % NN_BN;
            const int n = n0 + c, k = k0 + kk;
            Bs[kk][c] = (n < N && k < K) ? Bm[(size_t)k * ldb + n] : mk<T>(T(0), T(0));
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < NN_BK; ++kk) {
            const c_t<T> a = As[kk][tm];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const c_t<T> b = Bs[kk][tq * 4 + j];
                acc[j].x += a.x * b.x - a.y * b.y;
                acc[j].y += a.x * b.y + a.y * b.x;
            }
        }
        __syncthreads();
    }
    const int m = m0 + tm;
    if (m < M) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int n = n0 + tq * 4 + j;
            if (n < N) out[(size_t)n * ldo + m] = accumulate ? cadd(out[(size_t)n * ldo + m], acc[j]) : acc[j];
        }
    }
}

template <typename T>
jdft_status zgemm_nn_acc(int M, int N, int K, const c_t<T>* A, int lda, const c_t<T>* Bm, int ldb, c_t<T>* out,
                         int ldo, cudaStream_t st, bool accumulate) {
    if (M == 0 || N == 0) return JDFT_OK;
    if (K == 0) {
        if (!accumulate)
            for (int n = 0; n < N; ++n)
                JDFT_CUDA_TRY(cudaMemsetAsync(out + (size_t)n * ldo, 0, (size_t)M * sizeof(c_t<T>), st));
        return JDFT_OK;
    }
    dim3 grid((M + NN_BM - 1) / NN_BM, (N + NN_BN - 1) / NN_BN);
    {
        Trace tr_("zgemm_nn", st);
        zgemm_nn_kernel<T><<<grid, 256, 0, st>>>(M, N, K, A, lda, Bm, ldb, out, ldo, accumulate);
    }
    return check_launch("zgemm_nn");
}

// Bd[i][b] = sum_j D[i][j] Bc[j][b], rounded to the product type; D as ELL
// rows (w entries of column index and value per row).
template <typename T>
__global__ void dmul_kernel(int nproj, int nb, int w, const int* __restrict__ Dcol, const double* __restrict__ Dval,
                            const double2* __restrict__ Bc, c_t<T>* __restrict__ Bd) {
    const int total = nproj * nb;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
        const int i = e / nb, b = e % nb;
        double re = 0.0, im = 0.0;
        for (int q = 0; q < w; ++q) {
            const double d = Dval[(size_t)i * w + q];
            const double2 x = Bc[(size_t)Dcol[(size_t)i * w + q] * nb + b];
            re += d * x.x;
            im += d * x.y;
        }
        Bd[e] = mk<T>((T)re, (T)im);
    }
}

bool gemm_nn_inplace_ok(jdft_prec prec, int N) {
    if (prec == JDFT_BF16X3) return N <= 256;
    if (prec == JDFT_TF32X3) return N <= 128;
    return false;  // the CUDA-core products tile N in 16-column blocks
}

size_t nonlocal_workspace_bytes(int nproj, int nb, size_t elem, int npw, jdft_prec prec, bool split_c,
                                bool partials) {
    if (nproj == 0) return 0;
    const size_t a = ((size_t)nproj * nb * sizeof(double2) + 255) / 256 * 256;
    const size_t b = ((size_t)nproj * nb * elem + 255) / 256 * 256;
    const size_t c = split_c && tcx_eligible(prec, nproj, nb) ? (tcx_split_bytes(nb, npw) + 255) / 256 * 256 : 0;
    // the split of (D P^dag C)'s transpose for P (D P^dag C) on split operands
    const size_t d = tcx_eligible(prec, nproj, nb) ? (tcx_split_bytes(nb, nproj) + 255) / 256 * 256 : 0;
    const size_t e = partials && tcx_eligible(prec, nproj, nb) ? tcx_cn_partial_bytes(nproj, nb, npw) : 0;
    return a + b + c + d + e;
}

template <typename T>
static const c_t<T>* proj_ptr(const KSphere& sp);
template <> const double2* proj_ptr<double>(const KSphere& sp) { return (const double2*)sp.P; }
template <> const float2* proj_ptr<float>(const KSphere& sp) { return (const float2*)sp.P32; }

template <typename T>
jdft_status nonlocal_accumulate(const KSphere& sp, const void* C, int ldc, void* HC, int ldhc, int nb,
                                jdft_prec prec, void* work, cudaStream_t st, bool split_c, const void* Csplit,
                                bool partials) {
    if (sp.nproj == 0 || nb == 0) return JDFT_OK;
    double2* Bc = (double2*)work;
    const size_t abytes = ((size_t)sp.nproj * nb * sizeof(double2) + 255) / 256 * 256;
    const size_t bbytes = ((size_t)sp.nproj * nb * sizeof(c_t<T>) + 255) / 256 * 256;
    c_t<T>* Bd = (c_t<T>*)((char*)work + abytes);
    JDFT_CUDA_TRY(cudaMemsetAsync(Bc, 0, (size_t)sp.nproj * nb * sizeof(double2), st));
    jdft_status s;
    const bool split_ops = std::is_same<T, float>::value && (split_c || Csplit) && sp.Psplit &&
                           tcx_eligible(prec, sp.nproj, nb);
    const size_t cbytes = split_c && tcx_eligible(prec, sp.nproj, nb)
                              ? (tcx_split_bytes(nb, sp.npw) + 255) / 256 * 256 : 0;
    if (split_ops) {
        const void* Cs = Csplit;
        if (!Cs) {
            void* own = (char*)work + abytes + bbytes;
            if ((s = tcx_split((const float2*)C, ldc, nb, sp.npw, own, st))) return s;
            Cs = own;
        }
        const size_t dbytes = (tcx_split_bytes(nb, sp.nproj) + 255) / 256 * 256;
        void* part = partials ? (char*)work + abytes + bbytes + cbytes + dbytes : nullptr;
        s = tcx_cn(sp.nproj, nb, sp.npw, sp.Psplit, Cs, Bc, nb, 1.0, st, part,
                   partials ? tcx_cn_partial_bytes(sp.nproj, nb, sp.npw) : 0);
    } else {
        s = gemm_cn<T>(prec, sp.nproj, nb, sp.npw, proj_ptr<T>(sp), sp.npw, (const c_t<T>*)C, ldc, Bc, nb, 1.0, st);
    }
    if (s != JDFT_OK) return s;
    {
        Trace tr_("dmul", st);
        dmul_kernel<T><<<std::min(152 * 8, (sp.nproj * nb + 255) / 256), 256, 0, st>>>(sp.nproj, nb, sp.Dw, sp.Dcol,
                                                                                        sp.Dval, Bc, Bd);
    }
    if ((s = check_launch("dmul"))) return s;
    if (split_ops && sp.Psplit_t) {
        // HC += P (D P^dag C): P's transposed split (made with the projectors) and that of D P^dag C
        void* Bt = (char*)work + abytes + bbytes + cbytes;
        if ((s = tcx_split_t((const float2*)Bd, nb, nb, sp.nproj, Bt, st))) return s;
        return tcx_nn(sp.npw, nb, sp.nproj, sp.Psplit_t, Bt, (float2*)HC, ldhc, true, st);
    }
    return gemm_nn_acc<T>(prec, sp.npw, nb, sp.nproj, proj_ptr<T>(sp), sp.npw, Bd, nb, (c_t<T>*)HC, ldhc, st);
}

template <>
jdft_status gemm_cn<double>(jdft_prec, int M, int N, int K, const double2* A, int lda, const double2* B, int ldb,
                            double2* out, int ldo, double alpha, cudaStream_t st) {
    return zgemm_cn<double>(M, N, K, A, lda, B, ldb, out, ldo, alpha, st);
}
template <>
jdft_status gemm_cn<float>(jdft_prec prec, int M, int N, int K, const float2* A, int lda, const float2* B, int ldb,
                           double2* out, int ldo, double alpha, cudaStream_t st) {
    if (prec == JDFT_TF32X3 || prec == JDFT_BF16X3)
        return tc_zgemm_cn(M, N, K, A, lda, B, ldb, out, ldo, alpha, prec == JDFT_BF16X3, st);
    return zgemm_cn<float>(M, N, K, A, lda, B, ldb, out, ldo, alpha, st);
}
template <>
jdft_status gemm_nn_acc<double>(jdft_prec, int M, int N, int K, const double2* A, int lda, const double2* Bm, int ldb,
                                double2* out, int ldo, cudaStream_t st, bool accumulate) {
    return zgemm_nn_acc<double>(M, N, K, A, lda, Bm, ldb, out, ldo, st, accumulate);
}
template <>
jdft_status gemm_nn_acc<float>(jdft_prec prec, int M, int N, int K, const float2* A, int lda, const float2* Bm, int ldb,
                               float2* out, int ldo, cudaStream_t st, bool accumulate) {
    if (prec == JDFT_TF32X3 || prec == JDFT_BF16X3)
        return tc_zgemm_nn_acc(M, N, K, A, lda, Bm, ldb, out, ldo, prec == JDFT_BF16X3, st, accumulate);
    return zgemm_nn_acc<float>(M, N, K, A, lda, Bm, ldb, out, ldo, st, accumulate);
}

template jdft_status zgemm_cn<double>(int, int, int, const double2*, int, const double2*, int, double2*, int, double,
                                      cudaStream_t);
template jdft_status zgemm_cn<float>(int, int, int, const float2*, int, const float2*, int, double2*, int, double,
                                     cudaStream_t);
template jdft_status zgemm_nn_acc<double>(int, int, int, const double2*, int, const double2*, int, double2*, int,
                                          cudaStream_t, bool);
template jdft_status zgemm_nn_acc<float>(int, int, int, const float2*, int, const float2*, int, float2*, int,
                                         cudaStream_t, bool);
template jdft_status nonlocal_accumulate<double>(const KSphere&, const void*, int, void*, int, int, jdft_prec, void*,
                                                 cudaStream_t, bool, const void*, bool);
template jdft_status nonlocal_accumulate<float>(const KSphere&, const void*, int, void*, int, int, jdft_prec, void*,
                                                cudaStream_t, bool, const void*, bool);

}  // namespace jdft

using namespace jdft;

extern "C" jdft_status jdft_subspace(jdft_basis_t b, int ik, const void* C, int ldc, const void* HC, int ldhc, int nb,
                                     void* CHC, void* COC, jdft_prec prec, void* stream) {
    clear_error();
    JDFT_CHECK_ARG(b, "null basis");
    JDFT_CHECK_ARG(ik >= 0 && ik < b->nk, "k-point index out of range");
    JDFT_CHECK_ARG(nb >= 0, "nb must be >= 0");
    JDFT_CHECK_ARG(prec >= JDFT_FP64 && prec <= JDFT_BF16X3, "unknown precision");
    if (nb == 0) return JDFT_OK;
    const int npw = b->ks[ik].npw;
    JDFT_CHECK_ARG(C && ldc >= npw, "bad C block");
    JDFT_CHECK_ARG(!CHC || (HC && ldhc >= npw), "bad HC block");
    JDFT_CHECK_ARG(((uintptr_t)CHC % 16) == 0 && ((uintptr_t)COC % 16) == 0, "outputs must be 16-byte aligned");
    cudaStream_t st = (cudaStream_t)stream;
    jdft_status s = JDFT_OK;
    if (prec == JDFT_BF16X3 && tcx_eligible(prec, nb, nb)) {
        // split C (and HC) once into BF16 planes in the basis workspace; both
        // products read the split C
        // (and room for the products' split-K partial tiles after them)
        const size_t cb = (tcx_split_bytes(nb, npw) + 255) / 256 * 256;
        const size_t pb = tcx_cn_partial_bytes(nb, nb, npw);
        const size_t sb = CHC ? 2 * cb : cb;
        if ((s = ensure_workspace(b, sb + pb))) return s;
        char* ws = (char*)b->work.ptr;
        if ((s = tcx_split((const float2*)C, ldc, nb, npw, ws, st))) return s;
        if (CHC) {
            if ((s = tcx_split((const float2*)HC, ldhc, nb, npw, ws + cb, st))) return s;
            JDFT_CUDA_TRY(cudaMemsetAsync(CHC, 0, (size_t)nb * nb * sizeof(double2), st));
            if ((s = tcx_cn(nb, nb, npw, ws, ws + cb, (double2*)CHC, nb, 1.0, st, ws + sb, pb))) return s;
        }
        if (COC) {
            JDFT_CUDA_TRY(cudaMemsetAsync(COC, 0, (size_t)nb * nb * sizeof(double2), st));
            if ((s = tcx_cn(nb, nb, npw, ws, ws, (double2*)COC, nb, b->omega, st, ws + sb, pb, true)))
                return s;
        }
        return JDFT_OK;
    }
    if (CHC) {
        JDFT_CUDA_TRY(cudaMemsetAsync(CHC, 0, (size_t)nb * nb * sizeof(double2), st));
        s = (prec == JDFT_FP64)
                ? zgemm_cn<double>(nb, nb, npw, (const double2*)C, ldc, (const double2*)HC, ldhc, (double2*)CHC, nb,
                                   1.0, st)
                : gemm_cn<float>(prec, nb, nb, npw, (const float2*)C, ldc, (const float2*)HC, ldhc, (double2*)CHC, nb, 1.0,
                                  st);
        if (s != JDFT_OK) return s;
    }
    if (COC) {
        JDFT_CUDA_TRY(cudaMemsetAsync(COC, 0, (size_t)nb * nb * sizeof(double2), st));
        s = (prec == JDFT_FP64)
                ? zgemm_cn<double>(nb, nb, npw, (const double2*)C, ldc, (const double2*)C, ldc, (double2*)COC, nb,
                                   b->omega, st)
                : gemm_cn<float>(prec, nb, nb, npw, (const float2*)C, ldc, (const float2*)C, ldc, (double2*)COC, nb,
                                  b->omega, st);
    }
    return s;
}
