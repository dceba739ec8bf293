// Complex GEMMs of the projector term and the subspace matrices.
#pragma once

#include "common.cuh"

namespace jdft {

// out[m * ldo + n] += scale * sum_k conj(A[m * lda + k]) * B[n * ldb + k]   (complex128 out)
// Rows of A and B are K-contiguous (band-major blocks, projector-major P).
// `out` must be zeroed by the caller when a plain product is wanted; split-K
// partial sums are added with FP64 atomics.
template <typename T>
jdft_status zgemm_cn(int M, int N, int K, const c_t<T>* A, int lda, const c_t<T>* B, int ldb, double2* out, int ldo,
                     double scale, cudaStream_t st);

// out[n * ldo + m] += sum_i A[i * lda + m] * Bm[i * ldb + n]   (= instead of += when !accumulate)
// A: K rows of length M (projector-major P), Bm: K x N row-major, out band-major.
template <typename T>
jdft_status zgemm_nn_acc(int M, int N, int K, const c_t<T>* A, int lda, const c_t<T>* Bm, int ldb, c_t<T>* out,
                         int ldo, cudaStream_t st, bool accumulate = true);

// Tensor-core versions (FP32 inputs split into hi + lo, 3 products) of the two
// products above: TF32 pieces (bf16 = false) or BF16 pieces (bf16 = true).
jdft_status tc_zgemm_cn(int M, int N, int K, const float2* A, int lda, const float2* B, int ldb, double2* out, int ldo,
                        double alpha, bool bf16, cudaStream_t st);
jdft_status tc_zgemm_nn_acc(int M, int N, int K, const float2* A, int lda, const float2* Bm, int ldb, float2* out,
                            int ldo, bool bf16, cudaStream_t st, bool accumulate = true);

// BF16x3 products from operands split once into BF16 planes (tc_gemm.cu).
// A split block of `rows` rows of K complex values holds four planes of
// rows x tcx_ldk(K) BF16 values: Re hi, Re lo, Im hi, Im lo (x = hi + lo).
size_t tcx_split_bytes(int rows, int K);
// Whether tcx_cn serves this product (BF16x3, both dimensions above 32).
bool tcx_eligible(jdft_prec prec, int M, int N);
// Split rows of X (complex64, row stride ld) into planes (16-byte aligned, tcx_split_bytes).
jdft_status tcx_split(const float2* X, int ld, int rows, int K, void* planes, cudaStream_t st);
// The split block of the transpose: row r, value k taken from X[k * ld + r]
// (X: K rows of `rows` values), for operands contiguous along M or N.
jdft_status tcx_split_t(const float2* X, int ld, int rows, int K, void* planes, cudaStream_t st);
// out[n * ldo + m] (+)= sum_k A[m][k] B[n][k] (no conjugate) from split blocks
// of A (M rows of K) and B (N rows of K); K up to a few hundred (one block
// covers all of it); accumulate = false overwrites.  out may alias neither
// split block but may be the block A was split from.
jdft_status tcx_nn(int M, int N, int K, const void* Aplanes, const void* Bplanes, float2* out, int ldo,
                   bool accumulate, cudaStream_t st);
// out[m * ldo + n] += alpha sum_k conj(A[m][k]) B[n][k] from the split blocks
// of A (M rows) and B (N rows), split along K over one wave of blocks.  With
// `partials` (partial_bytes >= tcx_cn_partial_bytes(M, N, K), 16-byte
// aligned) the blocks' FP32 partial tiles are stored there and summed (with
// compensated FP32 sums, in a fixed order) by a second kernel; without, they
// are added to out with FP64 atomics.  Either way out accumulates, so zero it
// first for a product.  hermitian (M == N, with partials): the product is
// Hermitian by construction (C^dag O C, or C^dag H C with H C = H C exactly),
// so only the upper-triangle 128 x 128 tiles are formed and the reduction
// mirrors them; the partial tiles then need at most tcx_cn_partial_bytes.
size_t tcx_cn_partial_bytes(int M, int N, int K);
jdft_status tcx_cn(int M, int N, int K, const void* Aplanes, const void* Bplanes, double2* out, int ldo, double alpha,
                   cudaStream_t st, void* partials = nullptr, size_t partial_bytes = 0, bool hermitian = false);

// Precision dispatch: JDFT_TF32X3 and JDFT_BF16X3 run the tensor-core
// versions (T = float only), the other precisions the CUDA-core ones.
template <typename T>
jdft_status gemm_cn(jdft_prec prec, int M, int N, int K, const c_t<T>* A, int lda, const c_t<T>* B, int ldb,
                    double2* out, int ldo, double alpha, cudaStream_t st);
template <typename T>
jdft_status gemm_nn_acc(jdft_prec prec, int M, int N, int K, const c_t<T>* A, int lda, const c_t<T>* Bm, int ldb,
                        c_t<T>* out, int ldo, cudaStream_t st, bool accumulate = true);

// Whether gemm_nn_acc(prec, M, N, K, A, ...) may write its output over A
// (out == A, same leading dimension, K == N): true when one block computes
// all N output columns of its 128 rows (tensor-core products with N <= 256
// for BF16 operands, N <= 128 otherwise), since a block reads those rows of A
// for every k before its epilogue writes them and no other block touches them.
bool gemm_nn_inplace_ok(jdft_prec prec, int N);

// Workspace bytes the nonlocal term needs for nb bands (with split_c, room
// for the split copy of C that the BF16x3 projection P^dag C reads; with
// partials, room for that projection's split-K partial tiles).
size_t nonlocal_workspace_bytes(int nproj, int nb, size_t elem, int npw = 0, jdft_prec prec = JDFT_FP64,
                                bool split_c = false, bool partials = false);

// HC += P D P^dag C for the sphere's projectors (no-op when nproj == 0).
// split_c: take the projection from split operands (tcx_cn) when it is
// eligible, splitting C in the workspace, which must then hold
// nonlocal_workspace_bytes(..., true).
// Csplit: the caller's BF16 planes of C (tcx_split), used instead of a split
// of its own when the projection is eligible.
// partials: the workspace holds nonlocal_workspace_bytes(..., split_c, true)
// and the projection's split-K partial tiles go there (no atomics).
template <typename T>
jdft_status nonlocal_accumulate(const KSphere& sp, const void* C, int ldc, void* HC, int ldhc, int nb,
                                jdft_prec prec, void* work, cudaStream_t st, bool split_c = false,
                                const void* Csplit = nullptr, bool partials = false);

}  // namespace jdft
