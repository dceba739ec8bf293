// Blocked FP64 Cholesky factorisation and triangular inverse of a Hermitian
// positive-definite n x n matrix on many blocks (the overlap U = Y^dag O Y of
// the band minimiser, JDFTx paper Sec. 2.1 Minimize; W = L^{-dag} makes
// Y W orthonormal).  FP64 units are scarce on this GPU (about 8 GFLOP/s per
// SM), so the work is spread over 32 x 32 tiles on separate blocks:
//   per diagonal block k:  factor L_kk and invert it (one block, shared memory);
//                          panel L_ik = A_ik L_kk^{-dag} (one block per i > k);
//                          trailing A_ij -= L_ik L_jk^dag (one block per i >= j > k)
//   inverse X = L^{-1}, block row by block row:
//                          S_ik = sum_{j=k}^{i-1} L_ij X_jk (one block per (k, j), FP64 atomics),
//                          X_ik = -L_ii^{-1} S_ik (one block per k)
//   W = X^dag in the caller's block type.
// The matrix is padded to a multiple of 32 with identity rows.
#include <algorithm>

#include "chol.cuh"
#include "profile.cuh"

namespace jdft {

constexpr int CB = 32;   // tile edge
constexpr int CT = 256;  // threads per block

size_t chol_work_elems(int n) {
    const size_t N = (size_t)((n + CB - 1) / CB) * CB;
    return 3 * N * N;  // L (N x N), X (N x N), S (N x N)
}

__device__ __forceinline__ double2 zmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a * conj(b)
__device__ __forceinline__ double2 zmulc(double2 a, double2 b) {
    return make_double2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}

// L = pad(U): lower triangle of U (both triangles copied; only the lower is used), identity on the pad.
__global__ void chol_init_kernel(int n, int N, const double2* __restrict__ U, double2* __restrict__ L,
                                 double2* __restrict__ X, int* status) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < N * N; e += gridDim.x * blockDim.x) {
        const int i = e / N, j = e % N;
        double2 v = make_double2(0.0, 0.0);
        if (i < n && j < n) v = U[(size_t)i * n + j];
        else if (i == j) v = make_double2(1.0, 0.0);
        L[e] = v;
        X[e] = make_double2(0.0, 0.0);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) *status = 0;
}

// Factor the diagonal tile k in shared memory and invert it; writes L_kk (lower) and X_kk = L_kk^{-1}.
// Right-looking: step j takes the pivot, scales column j and updates the
// trailing tile in parallel; the inverse is built row by row, every column of
// a row in parallel.
__global__ void __launch_bounds__(CT) chol_diag_kernel(int n, int N, int k, double2* __restrict__ L,
                                                       double2* __restrict__ X, const double2* __restrict__ U,
                                                       int* status) {
    __shared__ double2 a[CB][CB + 1];
    __shared__ double2 x[CB][CB + 1];
    __shared__ double piv;
    __shared__ int bad;
    const int r0 = k * CB;
    for (int e = threadIdx.x; e < CB * CB; e += CT) {
        const int i = e / CB, j = e % CB;
        a[i][j] = L[(size_t)(r0 + i) * N + r0 + j];
    }
    if (threadIdx.x == 0) bad = 0;
    __syncthreads();
    for (int j = 0; j < CB; ++j) {
        if (threadIdx.x == 0) {
            // a pivot that is not positive, or that lost all but ~1e-13 of the
            // original diagonal, means linearly dependent bands
            double d = a[j][j].x;
            const int g = r0 + j;
            const double ujj = g < n ? U[(size_t)g * n + g].x : 1.0;
            if (!(d > 1e-13 * ujj)) { bad = 1; d = 1.0; }
            piv = sqrt(d);
            a[j][j] = make_double2(piv, 0.0);
        }
        __syncthreads();
        const double ip = 1.0 / piv;
        for (int i = j + 1 + threadIdx.x; i < CB; i += CT) a[i][j] = make_double2(a[i][j].x * ip, a[i][j].y * ip);
        __syncthreads();
        const int w = CB - j - 1;
        for (int e = threadIdx.x; e < w * w; e += CT) {
            const int i = j + 1 + e / w, m = j + 1 + e % w;
            if (m <= i) {
                const double2 t = zmulc(a[i][j], a[m][j]);
                a[i][m].x -= t.x;
                a[i][m].y -= t.y;
            }
        }
        __syncthreads();
    }
    // X = L^{-1}: row i, all columns c <= i in parallel
    for (int i = 0; i < CB; ++i) {
        for (int c = threadIdx.x; c < CB; c += CT) {
            double2 s = make_double2(i == c ? 1.0 : 0.0, 0.0);
            if (c <= i) {
                for (int m = c; m < i; ++m) {
                    const double2 t = zmul(a[i][m], x[m][c]);
                    s.x -= t.x;
                    s.y -= t.y;
                }
                const double d = 1.0 / a[i][i].x;
                s = make_double2(s.x * d, s.y * d);
            } else {
                s = make_double2(0.0, 0.0);
            }
            x[i][c] = s;
        }
        __syncthreads();
    }
    for (int e = threadIdx.x; e < CB * CB; e += CT) {
        const int i = e / CB, j = e % CB;
        L[(size_t)(r0 + i) * N + r0 + j] = j <= i ? a[i][j] : make_double2(0.0, 0.0);
        X[(size_t)(r0 + i) * N + r0 + j] = x[i][j];
    }
    if (threadIdx.x == 0 && bad) *status = JDFT_ERR_NOT_POSDEF;
}

// Panel: L_ik = A_ik X_kk^dag for tile rows i > k (blockIdx.x = i - k - 1).
__global__ void __launch_bounds__(CT) chol_panel_kernel(int N, int k, double2* __restrict__ L,
                                                        const double2* __restrict__ X) {
    __shared__ double2 a[CB][CB + 1];
    __shared__ double2 xi[CB][CB + 1];
    const int i = k + 1 + blockIdx.x;
    const int ri = i * CB, rk = k * CB;
    for (int e = threadIdx.x; e < CB * CB; e += CT) {
        const int r = e / CB, c = e % CB;
        a[r][c] = L[(size_t)(ri + r) * N + rk + c];
        xi[r][c] = X[(size_t)(rk + r) * N + rk + c];
    }
    __syncthreads();
    // out[r][c] = sum_m a[r][m] conj(xi[c][m])
    for (int e = threadIdx.x; e < CB * CB; e += CT) {
        const int r = e / CB, c = e % CB;
        double2 s = make_double2(0.0, 0.0);
        for (int m = 0; m <= c; ++m) {  // xi is lower triangular
            const double2 t = zmulc(a[r][m], xi[c][m]);
            s.x += t.x;
            s.y += t.y;
        }
        L[(size_t)(ri + r) * N + rk + c] = s;
    }
}

// Trailing update: A_ij -= L_ik L_jk^dag for i >= j > k; blockIdx.x enumerates the pairs.
__global__ void __launch_bounds__(CT) chol_update_kernel(int N, int k, double2* __restrict__ L) {
    __shared__ double2 li[CB][CB + 1];
    __shared__ double2 lj[CB][CB + 1];
    // decode the lower-triangular pair index p -> (i, j), k < j <= i
    const int p = blockIdx.x;
    int ii = (int)((sqrt(8.0 * p + 1.0) - 1.0) * 0.5);
    while ((ii + 1) * (ii + 2) / 2 <= p) ++ii;
    while (ii * (ii + 1) / 2 > p) --ii;
    const int jj = p - ii * (ii + 1) / 2;
    const int i = k + 1 + ii, j = k + 1 + jj;
    const int rk = k * CB;
    for (int e = threadIdx.x; e < CB * CB; e += CT) {
        const int r = e / CB, c = e % CB;
        li[r][c] = L[(size_t)(i * CB + r) * N + rk + c];
        lj[r][c] = L[(size_t)(j * CB + r) * N + rk + c];
    }
    __syncthreads();
    for (int e = threadIdx.x; e < CB * CB; e += CT) {
        const int r = e / CB, c = e % CB;
        double2 s = make_double2(0.0, 0.0);
        for (int m = 0; m < CB; ++m) {
            const double2 t = zmulc(li[r][m], lj[c][m]);
            s.x += t.x;
            s.y += t.y;
        }
        double2* dst = &L[(size_t)(i * CB + r) * N + j * CB + c];
        dst->x -= s.x;
        dst->y -= s.y;
    }
}

// Inverse, block row i: S_ik += L_ij X_jk for every k <= j < i (blockIdx.x enumerates the (k, j) pairs).
__global__ void __launch_bounds__(CT) inv_accum_kernel(int N, int i, const double2* __restrict__ L,
                                                       const double2* __restrict__ X, double2* __restrict__ S) {
    __shared__ double2 l[CB][CB + 1];
    __shared__ double2 x[CB][CB + 1];
    const int p = blockIdx.x;  // pairs (k, j), 0 <= k <= j < i, enumerated by j then k
    int j = (int)((sqrt(8.0 * p + 1.0) - 1.0) * 0.5);
    while ((j + 1) * (j + 2) / 2 <= p) ++j;
    while (j * (j + 1) / 2 > p) --j;
    const int k = p - j * (j + 1) / 2;
    for (int e = threadIdx.x; e < CB * CB; e += CT) {
        const int r = e / CB, c = e % CB;
        l[r][c] = L[(size_t)(i * CB + r) * N + j * CB + c];
        x[r][c] = X[(size_t)(j * CB + r) * N + k * CB + c];
    }
    __syncthreads();
    for (int e = threadIdx.x; e < CB * CB; e += CT) {
        const int r = e / CB, c = e % CB;
        double2 s = make_double2(0.0, 0.0);
        for (int m = 0; m < CB; ++m) {
            const double2 t = zmul(l[r][m], x[m][c]);
            s.x += t.x;
            s.y += t.y;
        }
        double2* dst = &S[(size_t)(i * CB + r) * N + k * CB + c];
        atomicAdd(&dst->x, s.x);
        atomicAdd(&dst->y, s.y);
    }
}

// X_ik = -X_ii S_ik for every k < i (blockIdx.x = k).
__global__ void __launch_bounds__(CT) inv_finish_kernel(int N, int i, double2* __restrict__ X,
                                                        const double2* __restrict__ S) {
    __shared__ double2 d[CB][CB + 1];
    __shared__ double2 s_[CB][CB + 1];
    const int k = blockIdx.x;
    for (int e = threadIdx.x; e < CB * CB; e += CT) {
        const int r = e / CB, c = e % CB;
        d[r][c] = X[(size_t)(i * CB + r) * N + i * CB + c];
        s_[r][c] = S[(size_t)(i * CB + r) * N + k * CB + c];
    }
    __syncthreads();
    for (int e = threadIdx.x; e < CB * CB; e += CT) {
        const int r = e / CB, c = e % CB;
        double2 s = make_double2(0.0, 0.0);
        for (int m = 0; m <= r; ++m) {  // d lower triangular
            const double2 t = zmul(d[r][m], s_[m][c]);
            s.x += t.x;
            s.y += t.y;
        }
        X[(size_t)(i * CB + r) * N + k * CB + c] = make_double2(-s.x, -s.y);
    }
}

template <typename T>
__global__ void chol_out_kernel(int n, int N, const double2* __restrict__ X, c_t<T>* __restrict__ W) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n * n; e += gridDim.x * blockDim.x) {
        const int r = e / n, c = e % n;
        const double2 x = X[(size_t)c * N + r];  // W = X^dag
        W[e] = mk<T>((T)x.x, (T)(-x.y));
    }
}

jdft_status blocked_cholesky_winv(int n, const double2* U, double2* work, void* W, bool fp64, int* status,
                                  cudaStream_t st) {
    const int nb = (n + CB - 1) / CB;
    const int N = nb * CB;
    double2* L = work;
    double2* X = L + (size_t)N * N;
    double2* S = X + (size_t)N * N;
    const int g = (int)std::min<int64_t>(((int64_t)N * N + 255) / 256, 152 * 4);
    {
        Trace tr_("chol_init", st);
        chol_init_kernel<<<g, 256, 0, st>>>(n, N, U, L, X, status);
    }
    JDFT_CUDA_TRY(cudaMemsetAsync(S, 0, (size_t)N * N * sizeof(double2), st));
    for (int k = 0; k < nb; ++k) {
        {
            Trace tr_("chol_diag", st);
            chol_diag_kernel<<<1, CT, 0, st>>>(n, N, k, L, X, U, status);
        }
        const int m = nb - k - 1;
        if (m > 0) {
            {
                Trace tr_("chol_panel", st);
                chol_panel_kernel<<<m, CT, 0, st>>>(N, k, L, X);
            }
            {
                Trace tr_("chol_update", st);
                chol_update_kernel<<<m * (m + 1) / 2, CT, 0, st>>>(N, k, L);
            }
        }
    }
    for (int i = 1; i < nb; ++i) {
        {
            Trace tr_("chol_inv_accum", st);
            inv_accum_kernel<<<i * (i + 1) / 2, CT, 0, st>>>(N, i, L, X, S);
        }
        {
            Trace tr_("chol_inv_finish", st);
            inv_finish_kernel<<<i, CT, 0, st>>>(N, i, X, S);
        }
    }
    {
        Trace tr_("chol_out", st);
        if (fp64) chol_out_kernel<double><<<g, 256, 0, st>>>(n, N, X, (double2*)W);
        else chol_out_kernel<float><<<g, 256, 0, st>>>(n, N, X, (float2*)W);
    }
    return check_launch("blocked_cholesky_winv");
}

}  // namespace jdft
