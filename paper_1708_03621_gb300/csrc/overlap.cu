// The augmented overlap of ultrasoft-type pseudopotentials and the
// generalised eigenproblem it makes.  The JDFTx paper lists ultrasoft
// pseudopotentials among its features (Sec. 2.2) and names the overlap
// operator O (Sec. 2.1); it prints no formula.
//
// Reading (shared with the test oracle only through the paper): with
// augmentation charges Q on the projectors P of the nonlocal term,
//   S C = Omega C + P Q P^dag C,
// band energies are the eigenvalues of the pencil (C^dag H C, C^dag S C), and
// orthonormal blocks satisfy C^dag S C = 1.
//
// Design: S C reuses the nonlocal term's projector products with Q in place
// of D (the same P^dag C, sparse Q rows, P X kernels and precisions); the
// generalised Rayleigh-Ritz and orthonormalisation reuse the FP64 overlap
// factorisation of jdft_orthonormalize_async with C^dag S C given as U.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <vector>

#include "common.cuh"
#include "gemm.cuh"
#include "profile.cuh"

namespace jdft {
namespace {

template <typename T>
__global__ void __launch_bounds__(256)
scale_rows_kernel(const c_t<T>* __restrict__ C, int ldc, c_t<T>* __restrict__ out, int ldo, int npw, int nb, T s) {
    const int64_t total = (int64_t)npw * nb;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = i / npw, g = i - r * npw;
        const c_t<T> v = C[r * ldc + g];
        out[r * ldo + g] = mk<T>(s * v.x, s * v.y);
    }
}

int grid_of(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 8)); }

bool is64(jdft_prec p) { return p == JDFT_FP64; }

// SC = Omega C (+ P Q P^dag C when the augmentation is set).
template <typename T>
jdft_status run_op_S(jdft_basis_s* b, int ik, const void* C, int ldc, void* SC, int ldsc, int nb, jdft_prec prec,
                     cudaStream_t st) {
    const KSphere& sp = b->ks[ik];
    {
        Trace tr_("overlap_scale", st);
        scale_rows_kernel<T><<<grid_of((int64_t)sp.npw * nb), 256, 0, st>>>(
            (const c_t<T>*)C, ldc, (c_t<T>*)SC, ldsc, sp.npw, nb, (T)b->omega);
    }
    jdft_status s = check_launch("overlap_scale");
    if (s || !sp.Q) return s;
    KSphere aug = sp;          // the projectors of the nonlocal term, Q in place of D
    aug.D = sp.Q;
    aug.Dw = sp.Qw;
    aug.Dcol = sp.Qcol;
    aug.Dval = sp.Qval;
    if ((s = ensure_workspace(b, nonlocal_workspace_bytes(sp.nproj, nb, sizeof(c_t<T>), sp.npw, prec, false, false))))
        return s;
    s = nonlocal_accumulate<T>(aug, C, ldc, SC, ldsc, nb, prec, b->work.ptr, st);
    aug.iG.clear();
    return s;
}


// ---------------------------------------------------------------------------
// Generalised band minimiser (FP64): small kernels
// ---------------------------------------------------------------------------

constexpr int kDotBlocks = 304;

// partial[blockIdx.x] = Re sum conj(x) y over nb rows of npw (row strides ldx, ldy).
__global__ void __launch_bounds__(256)
gdot_kernel(int npw, int nb, const double2* __restrict__ x, int ldx, const double2* __restrict__ y, int ldy,
            double* __restrict__ partial) {
    double acc = 0.0;
    const int64_t total = (int64_t)npw * nb;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = i / npw, g = i - r * npw;
        const double2 a = x[r * ldx + g], b = y[r * ldy + g];
        acc += a.x * b.x + a.y * b.y;
    }
    __shared__ double red[32];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        partial[blockIdx.x] = t;
    }
}

// out[slot] = sum of n partials (one block, fixed order).
__global__ void __launch_bounds__(256)
gsum_kernel(const double* __restrict__ partial, int n, double* __restrict__ out) {
    double acc = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) acc += partial[i];
    __shared__ double red[32];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        *out = t;
    }
}

// z = a x + b y on nb rows (all with row stride ld).
__global__ void __launch_bounds__(256)
gaxpby_kernel(int npw, int nb, double a, const double2* __restrict__ x, double b, const double2* __restrict__ y,
              double2* __restrict__ z, int ld) {
    const int64_t total = (int64_t)npw * nb;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = i / npw, g = i - r * npw;
        const double2 u = x[r * ld + g];
        const double2 v = y ? y[r * ld + g] : make_double2(0.0, 0.0);
        z[r * ld + g] = make_double2(a * u.x + b * v.x, a * u.y + b * v.y);
    }
}

// Small nb x nb matrices (one block): Hermitian part in place and its trace;
// out = -A; trace of A B.
__global__ void __launch_bounds__(256)
ghermitize_kernel(int n, double2* A, double* trace) {
    double acc = 0.0;
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
        const int i = e / n, j = e - i * n;
        if (i < j) {
            const double2 a = A[i * n + j], b = A[j * n + i];
            const double2 m = make_double2(0.5 * (a.x + b.x), 0.5 * (a.y - b.y));
            A[i * n + j] = m;
            A[j * n + i] = make_double2(m.x, -m.y);
        } else if (i == j) {
            A[i * n + i].y = 0.0;
            acc += A[i * n + i].x;
        }
    }
    __shared__ double red[32];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        *trace = t;
    }
}

__global__ void __launch_bounds__(256)
gneg_kernel(int n, const double2* __restrict__ A, double2* __restrict__ out) {
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) out[e] = make_double2(-A[e].x, -A[e].y);
}

__global__ void __launch_bounds__(256)
gtrace_prod_kernel(int n, const double2* __restrict__ A, const double2* __restrict__ B, double* out) {
    double acc = 0.0;
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
        const int i = e / n, j = e - i * n;
        const double2 a = A[i * n + j], b = B[j * n + i];
        acc += a.x * b.x - a.y * b.y;
    }
    __shared__ double red[32];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        *out = t;
    }
}

// KG = K(x) G per coefficient, Teter's polynomial ratio with x = kin_G / T_b,
// T_b = Omega sum_G kin_G |C_Gb|^2 (one block per band: the sum, then the map).
__global__ void __launch_bounds__(256)
gteter_kernel(int npw, const double2* __restrict__ C, const double* __restrict__ kin, double omega,
              const double2* __restrict__ G, double2* __restrict__ KG, int ld) {
    const int b = blockIdx.x;
    const double2* Cb = C + (int64_t)b * ld;
    double acc = 0.0;
    for (int g = threadIdx.x; g < npw; g += blockDim.x) acc += kin[g] * (Cb[g].x * Cb[g].x + Cb[g].y * Cb[g].y);
    __shared__ double red[32];
    __shared__ double Tb;
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        Tb = omega * t;
    }
    __syncthreads();
    const double inv = 1.0 / Tb;
    for (int g = threadIdx.x; g < npw; g += blockDim.x) {
        const double x = kin[g] * inv;
        const double num = 27.0 + x * (18.0 + x * (12.0 + 8.0 * x));
        const double k = num / (num + 16.0 * x * x * x * x);
        const double2 v = G[(int64_t)b * ld + g];
        KG[(int64_t)b * ld + g] = make_double2(k * v.x, k * v.y);
    }
}

struct GenMin {
    jdft_basis_s* b;
    int ik, npw, nb;
    cudaStream_t st;
    double2 *C, *HC, *SC, *G, *KG, *KGp, *Gp, *d, *dp, *Hd, *Sd, *Y, *SY, *T;   // npw x nb blocks, ld = npw
    double2 *Hs, *M, *dSd, *U, *negM;                                             // nb x nb
    double *partial, *scal;
    int* status;

    jdft_status cn(const double2* A, const double2* Bm, double2* out) {   // out = A^dag B (nb x nb)
        JDFT_CUDA_TRY(cudaMemsetAsync(out, 0, (size_t)nb * nb * sizeof(double2), st));
        return gemm_cn<double>(JDFT_FP64, nb, nb, npw, A, npw, Bm, npw, out, nb, 1.0, st);
    }
    jdft_status nn_acc(const double2* A, const double2* Mm, double2* out) {   // out += A Mm
        return gemm_nn_acc<double>(JDFT_FP64, npw, nb, nb, A, npw, Mm, nb, out, npw, st, true);
    }
    jdft_status neg(const double2* A, double2* out) {
        {
            Trace tr_("gen_small", st);
            gneg_kernel<<<1, 256, 0, st>>>(nb, A, out);
        }
        return check_launch("gen_small");
    }
    // scal[slot] = Re sum conj(x) y
    jdft_status dot(const double2* x, const double2* y, int slot) {
        {
            Trace tr_("gen_dot", st);
            gdot_kernel<<<kDotBlocks, 256, 0, st>>>(npw, nb, x, npw, y, npw, partial);
            gsum_kernel<<<1, 256, 0, st>>>(partial, kDotBlocks, scal + slot);
        }
        return check_launch("gen_dot");
    }
    jdft_status axpby(double a, const double2* x, double bb, const double2* y, double2* z) {
        {
            Trace tr_("gen_axpby", st);
            gaxpby_kernel<<<grid_of((int64_t)npw * nb), 256, 0, st>>>(npw, nb, a, x, bb, y, z, npw);
        }
        return check_launch("gen_axpby");
    }
    jdft_status read(double* h, int n) {
        JDFT_CUDA_TRY(cudaMemcpyAsync(h, scal, n * sizeof(double), cudaMemcpyDeviceToHost, st));
        JDFT_CUDA_TRY(cudaStreamSynchronize(st));
        return JDFT_OK;
    }
    // X <- X - C (C^dag S X), with S X formed into T
    jdft_status project(double2* X) {
        jdft_status s = run_op_S<double>(b, ik, X, npw, T, npw, nb, JDFT_FP64, st);
        if (s) return s;
        if ((s = cn(C, T, M))) return s;
        if ((s = neg(M, negM))) return s;
        return nn_acc(C, negM, X);
    }
    // H C, S C and Hs = C^dag H C (Hermitian part), scal[0] = tr Hs
    jdft_status refresh(double2* Cx, double2* HCx, double2* SCx) {
        jdft_status s = jdft_apply_H(b, ik, Cx, npw, HCx, npw, nb, JDFT_FP64, st);
        if (s) return s;
        if ((s = run_op_S<double>(b, ik, Cx, npw, SCx, npw, nb, JDFT_FP64, st))) return s;
        if ((s = cn(Cx, HCx, Hs))) return s;
        {
            Trace tr_("gen_small", st);
            ghermitize_kernel<<<1, 256, 0, st>>>(nb, Hs, scal);
        }
        return check_launch("gen_small");
    }
    // Cx <- Cx L^{-dag} with U = Cx^dag (S Cx) given
    jdft_status orthonormalize(double2* Cx, const double2* SCx) {
        jdft_status s = cn(Cx, SCx, U);
        if (s) return s;
        return jdft_orthonormalize_async(b, ik, Cx, npw, nb, U, JDFT_FP64, status, st);
    }
};
}  // namespace
}  // namespace jdft

using namespace jdft;

extern "C" {

jdft_status jdft_set_augmentation(jdft_basis_t b, int ik, const double* Q, void* stream) {
    clear_error();
    JDFT_CHECK_ARG(b, "null basis");
    JDFT_CHECK_ARG(ik >= 0 && ik < b->nk, "k-point index out of range");
    KSphere& s = b->ks[ik];
    cudaStream_t st = (cudaStream_t)stream;
    if (s.Q) {
        JDFT_CUDA_TRY(cudaStreamSynchronize(st));
        cudaFree(s.Q); cudaFree(s.Qcol); cudaFree(s.Qval);
        s.Q = nullptr; s.Qcol = nullptr; s.Qval = nullptr; s.Qw = 0;
    }
    if (!Q) return JDFT_OK;
    JDFT_CHECK_ARG(s.nproj > 0, "set the projectors (jdft_set_projectors) before their augmentation");
    const int np = s.nproj;
    std::vector<double> h((size_t)np * np);
    JDFT_CUDA_TRY(cudaMemcpyAsync(h.data(), Q, h.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
    JDFT_CUDA_TRY(cudaStreamSynchronize(st));
    for (int i = 0; i < np; ++i)
        for (int j = 0; j < i; ++j)
            JDFT_CHECK_ARG(h[(size_t)i * np + j] == h[(size_t)j * np + i], "Q must be symmetric");
    int w = 1;
    for (int i = 0; i < np; ++i) {
        int c = 0;
        for (int j = 0; j < np; ++j) c += h[(size_t)i * np + j] != 0.0;
        w = std::max(w, c);
    }
    std::vector<int> col((size_t)np * w, 0);
    std::vector<double> val((size_t)np * w, 0.0);
    for (int i = 0; i < np; ++i) {
        int c = 0;
        for (int j = 0; j < np; ++j)
            if (h[(size_t)i * np + j] != 0.0) {
                col[(size_t)i * w + c] = j;
                val[(size_t)i * w + c] = h[(size_t)i * np + j];
                ++c;
            }
    }
    JDFT_CUDA_TRY(cudaMalloc(&s.Q, h.size() * sizeof(double)));
    JDFT_CUDA_TRY(cudaMalloc(&s.Qcol, col.size() * sizeof(int)));
    JDFT_CUDA_TRY(cudaMalloc(&s.Qval, val.size() * sizeof(double)));
    JDFT_CUDA_TRY(cudaMemcpy(s.Q, h.data(), h.size() * sizeof(double), cudaMemcpyHostToDevice));
    JDFT_CUDA_TRY(cudaMemcpy(s.Qcol, col.data(), col.size() * sizeof(int), cudaMemcpyHostToDevice));
    JDFT_CUDA_TRY(cudaMemcpy(s.Qval, val.data(), val.size() * sizeof(double), cudaMemcpyHostToDevice));
    s.Qw = w;
    return JDFT_OK;
}

jdft_status jdft_op_S(jdft_basis_t b, int ik, const void* C, int ldc, void* SC, int ldsc, int nb, jdft_prec prec,
                      void* stream) {
    clear_error();
    JDFT_CHECK_ARG(b && C && SC, "null argument");
    JDFT_CHECK_ARG(ik >= 0 && ik < b->nk, "k-point index out of range");
    JDFT_CHECK_ARG(nb >= 1, "nb must be >= 1");
    JDFT_CHECK_ARG(prec >= JDFT_FP64 && prec <= JDFT_BF16X3, "unknown precision");
    JDFT_CHECK_ARG(ldc >= b->ks[ik].npw && ldsc >= b->ks[ik].npw, "leading dimension below npw");
    JDFT_CHECK_ARG(C != SC, "C and SC must not overlap");
    cudaStream_t st = (cudaStream_t)stream;
    return is64(prec) ? run_op_S<double>(b, ik, C, ldc, SC, ldsc, nb, prec, st)
                      : run_op_S<float>(b, ik, C, ldc, SC, ldsc, nb, prec, st);
}

jdft_status jdft_subspace_generalized(jdft_basis_t b, int ik, const void* C, int ldc, const void* HC, int ldhc,
                                      int nb, void* CHC, void* CSC, double* eigs, void* stream) {
    clear_error();
    JDFT_CHECK_ARG(b && C && HC && CHC && CSC, "null argument");
    JDFT_CHECK_ARG(ik >= 0 && ik < b->nk, "k-point index out of range");
    const int npw = b->ks[ik].npw;
    JDFT_CHECK_ARG(nb >= 1 && nb <= npw, "bad band count");
    JDFT_CHECK_ARG(ldc >= npw && ldhc >= npw, "leading dimension below npw");
    cudaStream_t st = (cudaStream_t)stream;
    // scratch: S C, then copies of C and H C rotated to an S-orthonormal basis
    double2* wk = nullptr;
    const size_t blk = (size_t)nb * npw;
    JDFT_CUDA_TRY(cudaMalloc(&wk, (3 * blk + (size_t)nb * nb) * sizeof(double2) + 256));
    double2 *SCb = wk, *Cc = wk + blk, *Hc = wk + 2 * blk, *A = wk + 3 * blk;
    int* status = reinterpret_cast<int*>(A + (size_t)nb * nb);
    auto done = [&](jdft_status s_) {
        cudaStreamSynchronize(st);
        cudaFree(wk);
        return s_;
    };
    jdft_status s;
    if ((s = run_op_S<double>(b, ik, C, ldc, SCb, npw, nb, JDFT_FP64, st))) return done(s);
    if (cudaMemsetAsync(CHC, 0, (size_t)nb * nb * sizeof(double2), st) != cudaSuccess ||
        cudaMemsetAsync(CSC, 0, (size_t)nb * nb * sizeof(double2), st) != cudaSuccess ||
        cudaMemsetAsync(A, 0, (size_t)nb * nb * sizeof(double2), st) != cudaSuccess ||
        cudaMemsetAsync(status, 0, sizeof(int), st) != cudaSuccess)
        return done(set_error(JDFT_ERR_CUDA, "jdft_subspace_generalized: memset"));
    if ((s = gemm_cn<double>(JDFT_FP64, nb, nb, npw, (const double2*)C, ldc, (const double2*)HC, ldhc,
                             (double2*)CHC, nb, 1.0, st)))
        return done(s);
    if ((s = gemm_cn<double>(JDFT_FP64, nb, nb, npw, (const double2*)C, ldc, SCb, npw, (double2*)CSC, nb, 1.0, st)))
        return done(s);
    if (eigs) {
        // C' = C L^{-dag}, (HC)' = HC L^{-dag} with C^dag S C = L L^dag; eigenvalues of C'^dag (HC)'
        if (cudaMemcpy2DAsync(Cc, npw * sizeof(double2), C, (size_t)ldc * sizeof(double2), npw * sizeof(double2), nb,
                              cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
            cudaMemcpy2DAsync(Hc, npw * sizeof(double2), HC, (size_t)ldhc * sizeof(double2), npw * sizeof(double2), nb,
                              cudaMemcpyDeviceToDevice, st) != cudaSuccess)
            return done(set_error(JDFT_ERR_CUDA, "jdft_subspace_generalized: copies"));
        if ((s = jdft_orthonormalize_async(b, ik, Cc, npw, nb, CSC, JDFT_FP64, status, stream))) return done(s);
        if ((s = jdft_orthonormalize_async(b, ik, Hc, npw, nb, CSC, JDFT_FP64, status, stream))) return done(s);
        if ((s = gemm_cn<double>(JDFT_FP64, nb, nb, npw, Cc, npw, Hc, npw, A, nb, 1.0, st))) return done(s);
        int hs = 0;
        if (cudaMemcpyAsync(&hs, status, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return done(set_error(JDFT_ERR_CUDA, "jdft_subspace_generalized: status"));
        if (hs) return done(set_error(JDFT_ERR_NOT_POSDEF, "C^dag S C is not positive definite"));
        if ((s = jdft_subspace_eigs(nb, A, eigs, stream))) return done(s);
    }
    return done(JDFT_OK);
}

jdft_status jdft_orthonormalize_generalized(jdft_basis_t b, int ik, void* C, int ldc, int nb, void* stream) {
    clear_error();
    JDFT_CHECK_ARG(b && C, "null argument");
    JDFT_CHECK_ARG(ik >= 0 && ik < b->nk, "k-point index out of range");
    const int npw = b->ks[ik].npw;
    JDFT_CHECK_ARG(nb >= 1 && nb <= npw && ldc >= npw, "bad block shape");
    cudaStream_t st = (cudaStream_t)stream;
    double2* wk = nullptr;
    JDFT_CUDA_TRY(cudaMalloc(&wk, ((size_t)nb * npw + (size_t)nb * nb) * sizeof(double2) + 256));
    double2 *SCb = wk, *U = wk + (size_t)nb * npw;
    int* status = reinterpret_cast<int*>(U + (size_t)nb * nb);
    auto done = [&](jdft_status s_) {
        cudaStreamSynchronize(st);
        cudaFree(wk);
        return s_;
    };
    jdft_status s;
    if ((s = run_op_S<double>(b, ik, C, ldc, SCb, npw, nb, JDFT_FP64, st))) return done(s);
    if (cudaMemsetAsync(U, 0, (size_t)nb * nb * sizeof(double2), st) != cudaSuccess ||
        cudaMemsetAsync(status, 0, sizeof(int), st) != cudaSuccess)
        return done(set_error(JDFT_ERR_CUDA, "jdft_orthonormalize_generalized: memset"));
    if ((s = gemm_cn<double>(JDFT_FP64, nb, nb, npw, (const double2*)C, ldc, SCb, npw, U, nb, 1.0, st)))
        return done(s);
    if ((s = jdft_orthonormalize_async(b, ik, C, ldc, nb, U, JDFT_FP64, status, stream))) return done(s);
    int hs = 0;
    if (cudaMemcpyAsync(&hs, status, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return done(set_error(JDFT_ERR_CUDA, "jdft_orthonormalize_generalized: status"));
    if (hs) return done(set_error(JDFT_ERR_NOT_POSDEF, "C^dag S C is not positive definite"));
    return done(JDFT_OK);
}

jdft_status jdft_minimize_bands_generalized(jdft_basis_t b, int ik, void* C, int ldc, int nb,
                                           const jdft_min_opts* opts, double* eigs, jdft_min_report* report,
                                           void* stream) {
    clear_error();
    JDFT_CHECK_ARG(b && C && opts && report, "null argument");
    JDFT_CHECK_ARG(ik >= 0 && ik < b->nk, "k-point index out of range");
    const int npw = b->ks[ik].npw;
    JDFT_CHECK_ARG(nb >= 1 && nb <= npw && ldc >= npw, "bad block shape");
    JDFT_CHECK_ARG(opts->tol > 0 && opts->max_iter >= 1, "bad tolerance or iteration limit");
    JDFT_CHECK_ARG(opts->precond == JDFT_PRECOND_IDENTITY || opts->precond == JDFT_PRECOND_TETER,
                   "the generalised minimiser takes the identity or Teter preconditioner");
    JDFT_CHECK_ARG(opts->prec == JDFT_FP64, "the generalised minimiser runs in FP64");
    if (!b->have_V) return set_error(JDFT_ERR_ARG, "no potential set");
    cudaStream_t st = (cudaStream_t)stream;
    auto t0 = std::chrono::steady_clock::now();
    *report = jdft_min_report();
    const double f = opts->occupation > 0 ? opts->occupation : 2.0;
    const size_t blk = (size_t)npw * nb, sm = (size_t)nb * nb;
    double2* mem = nullptr;
    const size_t bytes = (14 * blk + 5 * sm) * sizeof(double2) + (kDotBlocks + 16) * sizeof(double) + 256;
    JDFT_CUDA_TRY(cudaMalloc(&mem, bytes));
    GenMin M;
    M.b = b; M.ik = ik; M.npw = npw; M.nb = nb; M.st = st;
    double2* q = mem;
    double2** blocks[] = {&M.C, &M.HC, &M.SC, &M.G, &M.KG, &M.KGp, &M.Gp, &M.d, &M.dp, &M.Hd, &M.Sd, &M.Y, &M.SY, &M.T};
    for (double2** pp : blocks) { *pp = q; q += blk; }
    M.Hs = q; q += sm; M.M = q; q += sm; M.dSd = q; q += sm; M.U = q; q += sm; M.negM = q; q += sm;
    M.partial = reinterpret_cast<double*>(q);
    M.scal = M.partial + kDotBlocks;
    M.status = reinterpret_cast<int*>(M.scal + 15);
    auto done = [&](jdft_status s_) {
        cudaStreamSynchronize(st);
        cudaFree(mem);
        return s_;
    };
    const double noise_ulp = 64.0 * 2.220446049250313e-16;
    jdft_status s;
    if (cudaMemsetAsync(M.status, 0, sizeof(int), st) != cudaSuccess ||
        cudaMemcpy2DAsync(M.C, npw * sizeof(double2), C, (size_t)ldc * sizeof(double2), npw * sizeof(double2), nb,
                          cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return done(set_error(JDFT_ERR_CUDA, "jdft_minimize_bands_generalized: set-up copies"));
    // S-orthonormal start
    if ((s = run_op_S<double>(b, ik, M.C, npw, M.SC, npw, nb, JDFT_FP64, st))) return done(s);
    if ((s = M.orthonormalize(M.C, M.SC))) return done(s);
    if ((s = M.refresh(M.C, M.HC, M.SC))) return done(s);
    double h[8];
    bool have_prev = false;
    double res = 0.0, E = 0.0;
    int it = 0;
    for (;; ++it) {
        // G = H C - S C Hs
        if ((s = M.axpby(1.0, M.HC, 0.0, nullptr, M.G))) return done(s);
        if ((s = M.neg(M.Hs, M.negM))) return done(s);
        if ((s = M.nn_acc(M.SC, M.negM, M.G))) return done(s);
        if ((s = M.dot(M.G, M.G, 1))) return done(s);
        if ((s = M.read(h, 2))) return done(s);
        E = f * h[0];
        res = std::sqrt(std::max(h[1], 0.0) / b->omega);
        if (res < opts->tol || it >= opts->max_iter) break;
        // preconditioned gradient
        if (opts->precond == JDFT_PRECOND_TETER) {
            {
                Trace tr_("gen_teter", st);
                gteter_kernel<<<nb, 256, 0, st>>>(npw, M.C, b->ks[ik].kin, b->omega, M.G, M.KG, npw);
            }
            if ((s = check_launch("gen_teter"))) return done(s);
        } else if ((s = M.axpby(1.0, M.G, 0.0, nullptr, M.KG))) {
            return done(s);
        }
        double beta = 0.0;
        if (have_prev) {
            // beta = <G, KG - KGp> / <Gp, KGp>, reset at < 0
            if ((s = M.axpby(1.0, M.KG, -1.0, M.KGp, M.T))) return done(s);
            if ((s = M.dot(M.G, M.T, 2)) || (s = M.dot(M.Gp, M.KGp, 3)) || (s = M.read(h, 4))) return done(s);
            beta = h[3] != 0.0 ? std::max(h[2] / h[3], 0.0) : 0.0;
        }
        // d = -KG + beta dp, S-orthogonal to C
        if ((s = M.axpby(-1.0, M.KG, beta, have_prev ? M.dp : nullptr, M.d))) return done(s);
        if ((s = M.project(M.d))) return done(s);
        if ((s = jdft_apply_H(b, ik, M.d, npw, M.Hd, npw, nb, JDFT_FP64, st))) return done(s);
        if ((s = M.dot(M.HC, M.d, 4)) || (s = M.read(h, 5))) return done(s);
        double a1 = 2.0 * h[4];
        if (a1 >= 0.0) {   // not a descent direction: restart along -KG
            if ((s = M.axpby(-1.0, M.KG, 0.0, nullptr, M.d)) || (s = M.project(M.d))) return done(s);
            if ((s = jdft_apply_H(b, ik, M.d, npw, M.Hd, npw, nb, JDFT_FP64, st))) return done(s);
            if ((s = M.dot(M.HC, M.d, 4)) || (s = M.read(h, 5))) return done(s);
            a1 = 2.0 * h[4];
        }
        if ((s = run_op_S<double>(b, ik, M.d, npw, M.Sd, npw, nb, JDFT_FP64, st))) return done(s);
        if ((s = M.cn(M.d, M.Sd, M.dSd))) return done(s);
        if ((s = M.dot(M.d, M.Hd, 5))) return done(s);
        {
            Trace tr_("gen_small", st);
            gtrace_prod_kernel<<<1, 256, 0, st>>>(nb, M.Hs, M.dSd, M.scal + 6);
        }
        if ((s = check_launch("gen_small")) || (s = M.read(h, 7))) return done(s);
        const double a2 = h[5] - h[6];
        double lam = a2 > 0.0 ? -a1 / (2.0 * a2) : 1.0;
        // the step: Y = C + lam d, S-orthonormalised; halved while the energy of the
        // new block exceeds E by more than rounding
        const double E0 = E;
        bool accepted = false;
        for (int tries = 0; tries < 30; ++tries) {
            if ((s = M.axpby(1.0, M.C, lam, M.d, M.Y)) || (s = M.axpby(1.0, M.SC, lam, M.Sd, M.SY))) return done(s);
            if ((s = M.orthonormalize(M.Y, M.SY))) return done(s);
            if ((s = M.refresh(M.Y, M.T, M.SY))) return done(s);    // H Y into T, S Y, Hs of Y
            if ((s = M.read(h, 1))) return done(s);
            const double E1 = f * h[0];
            if (E1 <= E0 + noise_ulp * std::fabs(E0) || tries == 29) {
                accepted = true;
                std::swap(M.C, M.Y);
                std::swap(M.HC, M.T);
                std::swap(M.SC, M.SY);
                break;
            }
            lam *= 0.5;
        }
        (void)accepted;
        std::swap(M.dp, M.d);
        std::swap(M.KGp, M.KG);
        std::swap(M.Gp, M.G);
        have_prev = true;
    }
    int hs = 0;
    if (cudaMemcpyAsync(&hs, M.status, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return done(set_error(JDFT_ERR_CUDA, "jdft_minimize_bands_generalized: status"));
    if (hs) return done(set_error(JDFT_ERR_NOT_POSDEF, "Y^dag S Y is not positive definite"));
    if (cudaMemcpy2DAsync(C, (size_t)ldc * sizeof(double2), M.C, npw * sizeof(double2), npw * sizeof(double2), nb,
                          cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return done(set_error(JDFT_ERR_CUDA, "jdft_minimize_bands_generalized: output copy"));
    if (eigs && (s = jdft_subspace_eigs(nb, M.Hs, eigs, stream))) return done(s);
    report->iterations = it;
    report->energy = E;
    report->residual = res;
    report->converged = res < opts->tol ? 1 : 0;
    s = done(JDFT_OK);
    report->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (!report->converged) return set_error(JDFT_ERR_NOT_CONVERGED, "generalised minimiser reached its limit");
    return s;
}

}  // extern "C"
