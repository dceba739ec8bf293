// Blocked Cholesky + triangular inverse on many blocks (see chol.cu).
#pragma once

#include "common.cuh"

namespace jdft {

// double2 elements of workspace blocked_cholesky_winv needs for an n x n matrix.
size_t chol_work_elems(int n);

// U (n x n complex128 row-major, Hermitian positive definite) = L L^dag;
// W (n x n row-major, complex128 if fp64 else complex64) = L^{-dag}, factored
// in FP64 (in FP32 for complex64 W only when JDFT_CHOL_FP32=1).
// *status receives JDFT_ERR_NOT_POSDEF on a pivot below 1e-13 (FP64) or 2e-4
// (FP32) of the original diagonal (device word).
jdft_status blocked_cholesky_winv(int n, const double2* U, double2* work, void* W, bool fp64, int* status,
                                  cudaStream_t st);

}  // namespace jdft
