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

}  // extern "C"
