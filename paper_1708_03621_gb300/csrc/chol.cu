// Blocked Cholesky factorisation and triangular inverse of a Hermitian
// positive-definite n x n matrix on many blocks (the overlap U = Y^dag O Y of
// the band minimiser, JDFTx paper Sec. 2.1 Minimize; W = L^{-dag} makes
// Y W orthonormal):
//   per diagonal tile k:  factor L_kk and invert it (one block, shared memory);
//                         panel L_ik = A_ik X_kk^dag for i > k;
//                         trailing A_ij -= L_ik L_jk^dag for i >= j > k
//   inverse X = L^{-1}, tile row by tile row:
//                         S_ik = sum_{j=k}^{i-1} L_ij X_jk (atomics over j),
//                         X_ik = -X_ii S_ik
//   W = X^dag in the caller's block type.
// Working precision S: FP64 for every block precision (W is rounded to the
// block type at the end); FP32 for FP32 blocks only on request
// (JDFT_CHOL_FP32=1).  FP64 units are scarce on this GPU (about two FP64 FMAs
// per clock per SM), so the FP64 work is spread over many blocks (the panel in
// 4-row slices, the trailing update in 8 x 8 output blocks), every complex
// multiply-add is 4 fused multiply-adds, and the diagonal tile factors and
// inverts in one loop over its columns.
// The matrix is padded to a multiple of 32 with identity rows.
#include <cooperative_groups.h>

#include <algorithm>
#include <vector>
#include <mutex>
#include <map>
#include <cstdlib>
#include <type_traits>

#include "chol.cuh"
#include "profile.cuh"

namespace jdft {

constexpr int CB = 32;   // tile edge
constexpr int CQ = 16;   // quadrant edge of the tile products
constexpr int CT = 256;  // threads per block

size_t chol_work_elems(int n) {
    const size_t N = (size_t)((n + CB - 1) / CB) * CB;
    return 3 * N * N + N;  // L, X, S (N x N each) and the diagonal of U, in double2 units
}

// A pivot below this fraction of the original diagonal means linearly
// dependent bands (in FP32 the rounding of the elimination alone reaches
// ~n eps |U_jj|).
template <typename S> struct PivotFloor;
template <> struct PivotFloor<double> { static constexpr double v = 1e-13; };
template <> struct PivotFloor<float> { static constexpr float v = 2e-4f; };

// Complex multiply-adds as two fused multiply-adds per part (4 instructions
// instead of the 6 of a product followed by an add).
__device__ __forceinline__ double fm(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float fm(float a, float b, float c) { return __fmaf_rn(a, b, c); }
template <typename V> __device__ __forceinline__ V cmac_conj(V acc, V p, V q) {  // acc + p conj(q)
    acc.x = fm(p.x, q.x, fm(p.y, q.y, acc.x));
    acc.y = fm(p.y, q.x, fm(-p.x, q.y, acc.y));
    return acc;
}
template <typename V> __device__ __forceinline__ V cmac(V acc, V p, V q) {  // acc + p q
    acc.x = fm(p.x, q.x, fm(-p.y, q.y, acc.x));
    acc.y = fm(p.x, q.y, fm(p.y, q.x, acc.y));
    return acc;
}
template <typename V> __device__ __forceinline__ V cmsub_conj(V acc, V p, V q) {  // acc - p conj(q)
    acc.x = fm(-p.x, q.x, fm(-p.y, q.y, acc.x));
    acc.y = fm(-p.y, q.x, fm(p.x, q.y, acc.y));
    return acc;
}
template <typename V> __device__ __forceinline__ V cmsub(V acc, V p, V q) {  // acc - p q
    acc.x = fm(-p.x, q.x, fm(p.y, q.y, acc.x));
    acc.y = fm(-p.x, q.y, fm(-p.y, q.x, acc.y));
    return acc;
}

// L = pad(U) (both triangles copied; only the lower is used), identity on the
// pad; X = S = 0; dg = the diagonal of U.
template <typename S>
__global__ void chol_init_kernel(int n, int N, const double2* __restrict__ U, c_t<S>* __restrict__ L,
                                 c_t<S>* __restrict__ X, c_t<S>* __restrict__ Sa, S* __restrict__ dg,
                                 int* status) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < N * N; e += gridDim.x * blockDim.x) {
        const int i = e / N, j = e % N;
        c_t<S> v = mk<S>(S(0), S(0));
        if (i < n && j < n) v = mk<S>((S)U[(size_t)i * n + j].x, (S)U[(size_t)i * n + j].y);
        else if (i == j) v = mk<S>(S(1), S(0));
        L[e] = v;
        X[e] = mk<S>(S(0), S(0));
        Sa[e] = mk<S>(S(0), S(0));
        if (i == j) dg[i] = v.x;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) *status = 0;
}

// Factor the diagonal tile k in shared memory and invert it; writes L_kk
// (lower) and X_kk = L_kk^{-1}.  Right-looking: step j subtracts
// a_ij conj(a_mj) / d_j from the trailing triangle with the unscaled column j
// (thread (i, m0) owns a_im for m = m0, m0 + 8, ...); the thread that updates
// a_{j+1,j+1} then takes the next pivot, so one barrier per column.  Columns
// are scaled by 1/L_jj at the end.  The inverse runs by columns, 8 threads per
// column summing over interleaved m.
template <typename S>
__global__ void __launch_bounds__(CT) chol_diag_kernel(int N, int k, c_t<S>* __restrict__ L, c_t<S>* __restrict__ X,
                                                       const S* __restrict__ dg, int* status) {
    using V = c_t<S>;
    __shared__ V a[CB][CB + 1];
    __shared__ S rp[CB];   // 1 / L_jj
    __shared__ S pv[CB];   // L_jj
    __shared__ S floor_[CB];
    __shared__ int bad;
    const int r0 = k * CB, tid = threadIdx.x;
    for (int e = tid; e < CB * CB; e += CT) {
        const int i = e / CB, j = e % CB;
        a[i][j] = L[(size_t)(r0 + i) * N + r0 + j];
    }
    if (tid < CB) floor_[tid] = PivotFloor<S>::v * dg[r0 + tid];
    if (tid == 0) bad = 0;
    __syncthreads();
    auto pivot = [&](int j) {
        S d = a[j][j].x;
        if (!(d > floor_[j])) { bad = 1; d = S(1); }
        const S p = sqrt(d);
        pv[j] = p;
        rp[j] = S(1) / p;
    };
    if (tid == 0) pivot(0);
    __syncthreads();
    const int i = tid >> 3, m0 = tid & 7;
    for (int j = 0; j < CB - 1; ++j) {
        if (i > j) {
            const S rd = rp[j] * rp[j];
            const V aij = cscale(a[i][j], rd);
#pragma unroll
            for (int q = 0; q < CB / 8; ++q) {
                const int m = m0 + 8 * q;
                if (m > j && m <= i) a[i][m] = csub(a[i][m], cmulc(aij, a[m][j]));
            }
            if (i == j + 1 && m0 == ((j + 1) & 7)) pivot(j + 1);
        }
        __syncthreads();
    }
    for (int e = tid; e < CB * CB; e += CT) {
        const int r = e / CB, c = e % CB;
        V v = mk<S>(S(0), S(0));
        if (r > c) v = cscale(a[r][c], rp[c]);
        else if (r == c) v = mk<S>(pv[r], S(0));
        a[r][c] = v;
        L[(size_t)(r0 + r) * N + r0 + c] = v;
    }
    __syncthreads();
    // X = L^{-1}: column c = tid / 8, thread sub holds X[m][c] for m = sub + 8 q
    {
        const int c = tid >> 3, sub = tid & 7;
        V xr[CB / 8];
#pragma unroll
        for (int q = 0; q < CB / 8; ++q) xr[q] = mk<S>(S(0), S(0));
        const int rstart = (tid >> 5) * 4;  // the warp's smallest column
        for (int r = rstart; r < CB; ++r) {
            V s = mk<S>(S(0), S(0));
#pragma unroll
            for (int q = 0; q < CB / 8; ++q) {
                const int m = sub + 8 * q;
                if (m >= c && m < r) s = cadd(s, cmul(a[r][m], xr[q]));
            }
#pragma unroll
            for (int o = 1; o < 8; o <<= 1) {
                s.x += __shfl_xor_sync(0xffffffffu, s.x, o);
                s.y += __shfl_xor_sync(0xffffffffu, s.y, o);
            }
            V xv = mk<S>(S(0), S(0));
            if (r >= c) xv = cscale(mk<S>((r == c ? S(1) : S(0)) - s.x, -s.y), rp[r]);
#pragma unroll
            for (int q = 0; q < CB / 8; ++q)
                if (r == sub + 8 * q) xr[q] = xv;
        }
#pragma unroll
        for (int q = 0; q < CB / 8; ++q) X[(size_t)(r0 + sub + 8 * q) * N + r0 + c] = xr[q];
    }
    if (tid == 0 && bad) *status = JDFT_ERR_NOT_POSDEF;
}

// 1/sqrt(d) for d > 0 in FP64: an FP32 estimate refined by two Newton steps
// y <- y (3 - d y^2) / 2 (each squares the relative error: ~1e-7 -> 1e-14 ->
// FP64 rounding), a handful of FP64 operations on the pivot's critical path.
__device__ __forceinline__ double rsqrt_newton(double d) {
    if (!(d > 1e-30 && d < 1e30)) return 1.0 / sqrt(d);  // outside the FP32 estimate's range
    double y = (double)rsqrtf((float)d);
    y = y * (1.5 - 0.5 * d * y * y);
    y = y * (1.5 - 0.5 * d * y * y);
    return y;
}

// FP64 diagonal tile.  FP64 warp instructions occupy the SM's FP64 units for
// the same time whatever the number of active lanes, so the work is packed
// into full warps, and the factor and the inverse X = L^{-1} share one loop
// over the columns j:
//  A: column j of L (l_ij = a_ij / L_jj, i > j) and row j of X (scaled by
//     1 / L_jj; its entries c <= j are then final) are formed;
//  B: the factor's trailing pairs (i, m), j < m <= i, lose l_ij conj(l_mj),
//     and the inverse's pairs (i, c), c <= j < i, lose l_ij x_jc: one pass
//     over both sets, 4 fused multiply-adds per pair.  The factor pairs come
//     from a table of the 528 lower-triangle pairs ordered by m ascending, so
//     the active ones are its last (31 - j)(32 - j) / 2 entries and the first
//     of them is (j + 1, j + 1): thread 0 updates it first and then takes the
//     next pivot while the others carry on.
// Two barriers per column (64 in all).
__global__ void __launch_bounds__(CT) chol_diag64_kernel(int N, int k, double2* __restrict__ L,
                                                         double2* __restrict__ X, const double* __restrict__ dg,
                                                         int* status) {
    constexpr int NPAIR = CB * (CB + 1) / 2;
    __shared__ double2 a[CB][CB + 1];
    __shared__ double2 x[CB][CB + 1];
    __shared__ unsigned short pr[NPAIR];
    __shared__ double rp[CB], pv[CB], fl[CB];
    __shared__ int bad;
    const int r0 = k * CB, tid = threadIdx.x;
    for (int e = tid; e < CB * CB; e += CT) {
        const int i = e / CB, j = e % CB;
        a[i][j] = L[(size_t)(r0 + i) * N + r0 + j];
        x[i][j] = make_double2(i == j ? 1.0 : 0.0, 0.0);
    }
    // pair table: m ascending, then i ascending; entry = i << 8 | m
    if (tid < CB) {
        const int m = tid;
        const int off = m * CB - m * (m - 1) / 2;  // pairs in the columns before m
        for (int i = m; i < CB; ++i) pr[off + i - m] = (unsigned short)(i << 8 | m);
        fl[tid] = PivotFloor<double>::v * dg[r0 + tid];
    }
    if (tid == 0) bad = 0;
    __syncthreads();
    auto pivot = [&](int j) {
        double d = a[j][j].x;
        if (!(d > fl[j])) { bad = 1; d = 1.0; }
        const double y = rsqrt_newton(d);
        rp[j] = y;      // 1 / L_jj
        pv[j] = d * y;  // L_jj = sqrt(d)
    };
    if (tid == 0) pivot(0);
    __syncthreads();
    for (int j = 0; j < CB; ++j) {
        const double r = rp[j];
        if (tid < CB) {
            if (tid > j) a[tid][j] = cscale(a[tid][j], r);
        } else if (tid < 2 * CB) {
            const int c = tid - CB;
            if (c <= j) x[j][c] = cscale(x[j][c], r);
        }
        __syncthreads();
        const int nf = (CB - 1 - j) * (CB - j) / 2;  // factor pairs
        const int w = j + 1, nx = (CB - 1 - j) * w;  // inverse pairs (i, c): w per row
        const int base = NPAIR - nf;
        // f / w for f < 256 by a float reciprocal: the error stays far below 0.5 / w
        const float rw = 1.0f / (float)w;
        for (int e = tid; e < nf + nx; e += CT) {
            if (e < nf) {
                const int p = pr[base + e], i = p >> 8, m = p & 0xff;
                a[i][m] = cmsub_conj(a[i][m], a[i][j], a[m][j]);
                if (e == 0) pivot(j + 1);
            } else {
                const int f = e - nf;
                const int q = (int)(((float)f + 0.5f) * rw);
                const int i = j + 1 + q, c = f - q * w;
                x[i][c] = cmsub(x[i][c], a[i][j], x[j][c]);
            }
        }
        __syncthreads();
    }
    for (int e = tid; e < CB * CB; e += CT) {
        const int r = e / CB, c = e % CB;
        double2 v = make_double2(0.0, 0.0);
        if (r > c) v = a[r][c];
        else if (r == c) v = make_double2(pv[r], 0.0);
        L[(size_t)(r0 + r) * N + r0 + c] = v;
        X[(size_t)(r0 + r) * N + r0 + c] = x[r][c];
    }
    if (tid == 0 && bad) *status = JDFT_ERR_NOT_POSDEF;
}

// Panel: L_ik = A_ik X_kk^dag for tile rows i > k (blockIdx.x = i - k - 1),
// rows [4 h, 4 h + 4) of the tile for blockIdx.y = h (a block overwrites only
// the rows it read; eight blocks share a tile row's FP64 work).
constexpr int PR = 4;  // panel rows per block
template <typename S>
__global__ void __launch_bounds__(CT) chol_panel_kernel(int N, int k, c_t<S>* __restrict__ L,
                                                        const c_t<S>* __restrict__ X) {
    using V = c_t<S>;
    __shared__ V a[PR][CB + 1];
    __shared__ V xk[CB][CB + 1];
    const int i = k + 1 + blockIdx.x, h = blockIdx.y;
    const int ri = i * CB + h * PR, rk = k * CB;
    for (int e = threadIdx.x; e < CB * CB; e += CT) {
        const int r = e / CB, c = e % CB;
        if (r < PR) a[r][c] = L[(size_t)(ri + r) * N + rk + c];
        xk[r][c] = X[(size_t)(rk + r) * N + rk + c];
    }
    __syncthreads();
    // out[r][c] = sum_{m <= c} a[r][m] conj(xk[c][m])  (xk lower triangular).
    // Warp w takes columns c = w + 8 q; lane (r, s) = (lane / 8, lane % 8)
    // sums m = s, s + 8, ... and three shuffles add the 8 partial sums.
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int r = lane >> 3, sg = lane & 7;
    for (int c = warp; c < CB; c += CT / 32) {
        V sum = mk<S>(S(0), S(0));
        for (int m = sg; m <= c; m += 8) sum = cmac_conj(sum, a[r][m], xk[c][m]);
#pragma unroll
        for (int o = 1; o < 8; o <<= 1) {
            sum.x += __shfl_xor_sync(0xffffffffu, sum.x, o);
            sum.y += __shfl_xor_sync(0xffffffffu, sum.y, o);
        }
        if (sg == 0) L[(size_t)(ri + r) * N + rk + c] = sum;
    }
}

// Quadrant (qr, qc) = (blockIdx.y >> 1, blockIdx.y & 1) of a tile product;
// thread (r, c) = (tid / 16, tid % 16) within the quadrant.
struct Quad {
    int qr, qc, r, c;
    __device__ Quad()
        : qr((int)(blockIdx.y >> 1) * CQ), qc((int)(blockIdx.y & 1) * CQ), r((int)threadIdx.x >> 4),
          c((int)threadIdx.x & 15) {}
};

// Lower-triangular pair index p -> (i, j), 0 <= j <= i.
__device__ __forceinline__ void tri_pair(int p, int& i, int& j) {
    int ii = (int)((sqrtf(8.0f * (float)p + 1.0f) - 1.0f) * 0.5f);
    while ((ii + 1) * (ii + 2) / 2 <= p) ++ii;
    while (ii * (ii + 1) / 2 > p) --ii;
    i = ii;
    j = p - ii * (ii + 1) / 2;
}

// Trailing update: A_ij -= L_ik L_jk^dag for i >= j > k; blockIdx.x
// enumerates the tile pairs, blockIdx.y = 4 br + bc the 8 x 8 output block
// (br, bc) of the tile (blocks above the diagonal of a diagonal tile return at
// once).  Warp w takes output row w of the block; lane (c, s) = (lane % 8,
// lane / 8) sums m = s, s + 4, ... and two shuffles add the 4 partial sums, so
// a tile pair's FP64 work is spread over 16 blocks.
constexpr int UB = 8;  // update output block edge
template <typename S>
__global__ void __launch_bounds__(CT) chol_update_kernel(int N, int k, c_t<S>* __restrict__ L) {
    using V = c_t<S>;
    __shared__ V li[UB][CB + 1];
    __shared__ V lj[UB][CB + 1];
    int ii, jj;
    tri_pair(blockIdx.x, ii, jj);
    const int i = k + 1 + ii, j = k + 1 + jj;
    const int br = (int)(blockIdx.y >> 2) * UB, bc = (int)(blockIdx.y & 3) * UB;
    if (i == j && bc > br) return;  // the whole block: upper part of a diagonal tile
    const int rk = k * CB;
    {
        const int r = threadIdx.x / CB, c = threadIdx.x % CB;  // UB x CB = CT elements
        li[r][c] = L[(size_t)(i * CB + br + r) * N + rk + c];
        lj[r][c] = L[(size_t)(j * CB + bc + r) * N + rk + c];
    }
    __syncthreads();
    const int r = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int c = lane & 7, sg = lane >> 3;
    V s = mk<S>(S(0), S(0));
#pragma unroll
    for (int m = sg; m < CB; m += 4) s = cmac_conj(s, li[r][m], lj[c][m]);
#pragma unroll
    for (int o = 8; o < 32; o <<= 1) {
        s.x += __shfl_xor_sync(0xffffffffu, s.x, o);
        s.y += __shfl_xor_sync(0xffffffffu, s.y, o);
    }
    if (sg == 0) {
        V* dst = &L[(size_t)(i * CB + br + r) * N + j * CB + bc + c];
        *dst = csub(*dst, s);
    }
}

// Inverse, tile row i: S_ik += L_ij X_jk for every k <= j < i (blockIdx.x enumerates the (j, k) pairs).
template <typename S>
__global__ void __launch_bounds__(CT) inv_accum_kernel(int N, int i, const c_t<S>* __restrict__ L,
                                                       const c_t<S>* __restrict__ X, c_t<S>* __restrict__ Sa) {
    using V = c_t<S>;
    __shared__ V l[CQ][CB + 1];
    __shared__ V x[CB][CQ + 1];
    int j, k;
    tri_pair(blockIdx.x, j, k);
    const Quad q;
    for (int e = threadIdx.x; e < CQ * CB; e += CT) {
        const int r = e / CB, c = e % CB;
        l[r][c] = L[(size_t)(i * CB + q.qr + r) * N + j * CB + c];
        const int r2 = e / CQ, c2 = e % CQ;
        x[r2][c2] = X[(size_t)(j * CB + r2) * N + k * CB + q.qc + c2];
    }
    __syncthreads();
    V s = mk<S>(S(0), S(0));
#pragma unroll 8
    for (int m = 0; m < CB; ++m) s = cmac(s, l[q.r][m], x[m][q.c]);
    V* dst = &Sa[(size_t)(i * CB + q.qr + q.r) * N + k * CB + q.qc + q.c];
    atomicAdd(&dst->x, s.x);
    atomicAdd(&dst->y, s.y);
}

// X_ik = -X_ii S_ik for every k < i (blockIdx.x = k).
template <typename S>
__global__ void __launch_bounds__(CT) inv_finish_kernel(int N, int i, c_t<S>* __restrict__ X,
                                                        const c_t<S>* __restrict__ Sa) {
    using V = c_t<S>;
    __shared__ V d[CQ][CB + 1];
    __shared__ V s_[CB][CQ + 1];
    const int k = blockIdx.x;
    const Quad q;
    for (int e = threadIdx.x; e < CQ * CB; e += CT) {
        const int r = e / CB, c = e % CB;
        d[r][c] = X[(size_t)(i * CB + q.qr + r) * N + i * CB + c];
        const int r2 = e / CQ, c2 = e % CQ;
        s_[r2][c2] = Sa[(size_t)(i * CB + r2) * N + k * CB + q.qc + c2];
    }
    __syncthreads();
    V s = mk<S>(S(0), S(0));
    const int rr = q.qr + q.r;  // row within the tile; X_ii is lower triangular
    for (int m = 0; m <= rr; ++m) s = cmac(s, d[q.r][m], s_[m][q.c]);
    X[(size_t)(i * CB + rr) * N + k * CB + q.qc + q.c] = mk<S>(-s.x, -s.y);
}

template <typename S, typename T>
__global__ void chol_out_kernel(int n, int N, const c_t<S>* __restrict__ X, c_t<T>* __restrict__ W) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n * n; e += gridDim.x * blockDim.x) {
        const int r = e / n, c = e % n;
        const c_t<S> x = X[(size_t)c * N + r];  // W = X^dag, rounded to the block type
        W[e] = mk<T>((T)x.x, (T)(-x.y));
    }
}

// ---------------------------------------------------------------------------
// FP32 factorisation of n <= 256 in one launch: a cluster of P = ceil(n/32)
// CTAs, CTA c holding block column c (rows 0 .. 32P-1, 32 columns) and its
// block column of X = L^{-1} in shared memory.  Step k: CTA k factors its
// diagonal tile (as chol_diag_kernel) and its panel L_ik = A_ik X_kk^dag; one
// cluster barrier; CTAs j > k subtract L_ik L_jk^dag from their block column,
// reading CTA k's panel through distributed shared memory.  Then each CTA
// forms its block column of X by block forward substitution,
// X_ic = -X_ii sum_{j=c}^{i-1} L_ij X_jc, with L_ij and X_ii read from the
// CTAs that hold them, and writes its 32 rows of W = X^dag.
// ---------------------------------------------------------------------------
constexpr int CLS = CB + 1;      // row stride of the block-column arrays (complex elements)
constexpr int CL_MAX = 8;        // portable cluster size: n <= 256

// JDFT_CHOL_FP32=1 factors the overlap of FP32 blocks in FP32 (read on every
// call; the default keeps FP64 for every precision); JDFT_CHOL_CLUSTER=0 then
// forces the multi-block path over the one-launch cluster one.
static bool fp32_factorisation() {
    const char* e = getenv("JDFT_CHOL_FP32");
    return e && e[0] == '1';
}
static bool cluster_disabled() {
    const char* e = getenv("JDFT_CHOL_CLUSTER");
    return e && e[0] == '0';
}

size_t chol_cluster_smem(int n) {
    const int NP = (n + CB - 1) / CB * CB;
    return (3 * (size_t)NP * CLS + (size_t)CB * CLS) * sizeof(float2);
}

// Factor the 32 x 32 tile A (stride lda, lower triangle used) in place into
// L (lower, zero above) and write X = L^{-1} (stride ldx); fl[j] = pivot floor.
__device__ void cl_factor_tile(float2* A, int lda, float2* X, int ldx, const float* fl, float* rp, float* pv,
                               int* bad) {
    const int tid = threadIdx.x;
    auto at = [&](int i, int j) -> float2& { return A[i * lda + j]; };
    auto pivot = [&](int j) {
        float d = at(j, j).x;
        if (!(d > fl[j])) { *bad = 1; d = 1.f; }
        const float p = sqrtf(d);
        pv[j] = p;
        rp[j] = 1.f / p;
    };
    if (tid == 0) pivot(0);
    __syncthreads();
    const int i = tid >> 3, m0 = tid & 7;
    for (int j = 0; j < CB - 1; ++j) {
        if (i > j) {
            const float2 aij = cscale(at(i, j), rp[j] * rp[j]);
#pragma unroll
            for (int q = 0; q < CB / 8; ++q) {
                const int m = m0 + 8 * q;
                if (m > j && m <= i) at(i, m) = csub(at(i, m), cmulc(aij, at(m, j)));
            }
            if (i == j + 1 && m0 == ((j + 1) & 7)) pivot(j + 1);
        }
        __syncthreads();
    }
    for (int e = tid; e < CB * CB; e += blockDim.x) {
        const int r = e / CB, c = e % CB;
        float2 v = make_float2(0.f, 0.f);
        if (r > c) v = cscale(at(r, c), rp[c]);
        else if (r == c) v = make_float2(pv[r], 0.f);
        at(r, c) = v;
    }
    __syncthreads();
    {
        const int c = tid >> 3, sub = tid & 7;
        float2 xr[CB / 8];
#pragma unroll
        for (int q = 0; q < CB / 8; ++q) xr[q] = make_float2(0.f, 0.f);
        const int rstart = (tid >> 5) * 4;
        for (int r = rstart; r < CB; ++r) {
            float2 s = make_float2(0.f, 0.f);
#pragma unroll
            for (int q = 0; q < CB / 8; ++q) {
                const int m = sub + 8 * q;
                if (m >= c && m < r) s = cadd(s, cmul(at(r, m), xr[q]));
            }
#pragma unroll
            for (int o = 1; o < 8; o <<= 1) {
                s.x += __shfl_xor_sync(0xffffffffu, s.x, o);
                s.y += __shfl_xor_sync(0xffffffffu, s.y, o);
            }
            float2 xv = make_float2(0.f, 0.f);
            if (r >= c) xv = cscale(make_float2((r == c ? 1.f : 0.f) - s.x, -s.y), rp[r]);
#pragma unroll
            for (int q = 0; q < CB / 8; ++q)
                if (r == sub + 8 * q) xr[q] = xv;
        }
#pragma unroll
        for (int q = 0; q < CB / 8; ++q) X[(sub + 8 * q) * ldx + c] = xr[q];
    }
    __syncthreads();
}

__global__ void __launch_bounds__(CT, 1) chol_cluster_kernel(int n, int NP, const double2* __restrict__ U,
                                                              float2* __restrict__ W, int* status) {
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    extern __shared__ __align__(16) float2 cls_sm[];
    float2* a = cls_sm;              // NP x CLS: block column `me` of A, then of L
    float2* x = a + NP * CLS;        // NP x CLS: block column `me` of X = L^{-1}
    float2* pc = x + NP * CLS;       // NP x CLS: local copy of remote rows (panel; L_ij, X_ii tiles)
    float2* t = pc + NP * CLS;       // CB x CLS: local copy of L_jk, then S_ic
    __shared__ float fl[CB], rp[CB], pv[CB];
    __shared__ int bad;
    const int me = (int)cl.block_rank();
    const int P = NP / CB;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    constexpr int NW = CT / 32;
    const int c0 = me * CB;
    for (int e = tid; e < NP * CB; e += CT) {
        const int r = e / CB, c = e % CB, gc = c0 + c;
        float2 v = make_float2(0.f, 0.f);
        if (r < n && gc < n) v = make_float2((float)U[(size_t)r * n + gc].x, (float)U[(size_t)r * n + gc].y);
        else if (r == gc) v = make_float2(1.f, 0.f);
        a[r * CLS + c] = v;
        x[r * CLS + c] = make_float2(0.f, 0.f);
    }
    if (tid < CB) {
        const int g = c0 + tid;
        fl[tid] = PivotFloor<float>::v * (g < n ? (float)U[(size_t)g * n + g].x : 1.f);
    }
    if (tid == 0) bad = 0;
    cl.sync();
    for (int k = 0; k < P; ++k) {
        if (me == k) {
            cl_factor_tile(a + c0 * CLS, CLS, x + c0 * CLS, CLS, fl, rp, pv, &bad);
            // panel: L_ik[r][c] = sum_{m <= c} A_ik[r][m] conj(X_kk[c][m]), a warp per row
            const float2* xk = x + c0 * CLS;
            for (int r = c0 + CB + warp; r < NP; r += NW) {
                float2 sum = make_float2(0.f, 0.f);
                for (int m = 0; m <= lane; ++m) sum = cadd(sum, cmulc(a[r * CLS + m], xk[lane * CLS + m]));
                __syncwarp();
                a[r * CLS + lane] = sum;
            }
        }
        cl.sync();
        if (me > k) {
            // rows c0 .. NP-1 of the panel L_{:,k}, copied in one pass (independent remote loads)
            const float2* rk = cl.map_shared_rank(a, k);
            for (int e = tid; e < (NP - c0) * CB; e += CT) {
                const int r = c0 + e / CB, c = e % CB;
                pc[r * CLS + c] = rk[r * CLS + c];
            }
            __syncthreads();
            // A_ij[r][lane] -= sum_m L_ik[r][m] conj(L_jk[lane][m]), a warp per row of block column me
            for (int r = c0 + warp; r < NP; r += NW) {
                float2 sum = make_float2(0.f, 0.f);
#pragma unroll 8
                for (int m = 0; m < CB; ++m) sum = cadd(sum, cmulc(pc[r * CLS + m], pc[(c0 + lane) * CLS + m]));
                a[r * CLS + lane] = csub(a[r * CLS + lane], sum);
            }
            __syncthreads();
        }
    }
    cl.sync();
    // X_ic for i > me: S = sum_{j=me}^{i-1} L_ij X_jc, X_ic = -X_ii S
    {
        const int r = tid >> 3, cb = tid & 7;
        for (int i = me + 1; i < P; ++i) {
            float2 acc[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[q] = make_float2(0.f, 0.f);
            // the tiles L_ij (j = me .. i-1, held by CTA j) and X_ii (held by CTA i), copied
            // in one pass into pc: tile j at rows CB j .., X_ii at rows CB i ..
            for (int j = me; j <= i; ++j) {
                const float2* src = j < i ? cl.map_shared_rank(a, j) : cl.map_shared_rank(x, i);
                for (int e = tid; e < CB * CB; e += CT) {
                    const int rr = e / CB, c = e % CB;
                    pc[(CB * j + rr) * CLS + c] = src[(CB * i + rr) * CLS + c];
                }
            }
            __syncthreads();
            for (int j = me; j < i; ++j) {
#pragma unroll 4
                for (int m = 0; m < CB; ++m) {
                    const float2 l = pc[(CB * j + r) * CLS + m];
#pragma unroll
                    for (int q = 0; q < 4; ++q) acc[q] = cadd(acc[q], cmul(l, x[(CB * j + m) * CLS + cb + 8 * q]));
                }
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) t[r * CLS + cb + 8 * q] = acc[q];
            __syncthreads();
            float2 o[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) o[q] = make_float2(0.f, 0.f);
            for (int m = 0; m <= r; ++m) {
                const float2 d = pc[(CB * i + r) * CLS + m];
#pragma unroll
                for (int q = 0; q < 4; ++q) o[q] = cadd(o[q], cmul(d, t[m * CLS + cb + 8 * q]));
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) x[(CB * i + r) * CLS + cb + 8 * q] = make_float2(-o[q].x, -o[q].y);
            __syncthreads();
        }
    }
    // rows c0 .. c0 + 31 of W = X^dag
    for (int e = tid; e < CB * n; e += CT) {
        const int cc = e / n, rr = e - cc * n;
        if (c0 + cc < n) {
            const float2 v = x[rr * CLS + cc];
            W[(size_t)(c0 + cc) * n + rr] = make_float2(v.x, -v.y);
        }
    }
    if (tid == 0 && bad) atomicExch(status, (int)JDFT_ERR_NOT_POSDEF);
    cl.sync();  // every CTA's shared memory stays in place until the others' remote reads are done
}

// One launch of chol_cluster_kernel; JDFT_ERR_UNSUPPORTED (nothing launched)
// when n is too large or the device cannot hold such a cluster.
static jdft_status run_cluster(int n, const double2* U, float2* W, int* status, cudaStream_t st) {
    const int P = (n + CB - 1) / CB;
    if (P > CL_MAX) return JDFT_ERR_UNSUPPORTED;
    const int NP = P * CB;
    const size_t smem = chol_cluster_smem(n);
    if (set_smem_attr((const void*)chol_cluster_kernel, smem) != cudaSuccess) {
        cudaGetLastError();
        return JDFT_ERR_UNSUPPORTED;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(P, 1, 1);
    cfg.blockDim = dim3(CT, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = P;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int clusters = 0;
    if (cudaOccupancyMaxActiveClusters(&clusters, (const void*)chol_cluster_kernel, &cfg) != cudaSuccess ||
        clusters < 1) {
        cudaGetLastError();
        return JDFT_ERR_UNSUPPORTED;
    }
    {
        Trace tr_("chol_cluster", st);
        cudaError_t e = cudaLaunchKernelEx(&cfg, chol_cluster_kernel, n, NP, U, W, status);
        if (e != cudaSuccess) return set_error(JDFT_ERR_CUDA, std::string("chol_cluster: ") + cudaGetErrorString(e));
    }
    return check_launch("chol_cluster");
}

// A second stream per device for the inverse rows (created once, non-blocking).
static cudaStream_t side_stream() {
    static std::mutex mu;
    static std::map<int, cudaStream_t> streams;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(mu);
    cudaStream_t& s = streams[dev];
    if (!s && cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) s = nullptr;
    return s;
}

// The factorisation runs on `st`; the inverse rows run on a side stream,
// row i as soon as factor step i has its diagonal tile (L_ij, j < i, and
// X_jj, j <= i, are final then), so they fill the SMs the one-block diagonal
// kernels leave idle.  The side stream forks from `st` after the set-up and
// joins it before W is written (also under stream capture).
template <typename S, typename T>
static jdft_status run_blocked(int n, const double2* U, double2* work, c_t<T>* W, int* status, cudaStream_t st) {
    const int nb = (n + CB - 1) / CB;
    const int N = nb * CB;
    c_t<S>* L = reinterpret_cast<c_t<S>*>(work);
    c_t<S>* X = L + (size_t)N * N;
    c_t<S>* Sa = X + (size_t)N * N;
    S* dg = reinterpret_cast<S*>(Sa + (size_t)N * N);
    const int g = (int)std::min<int64_t>(((int64_t)N * N + 255) / 256, 152 * 4);
    {
        Trace tr_("chol_init", st);
        chol_init_kernel<S><<<g, 256, 0, st>>>(n, N, U, L, X, Sa, dg, status);
    }
    cudaStream_t sb = nb > 1 ? side_stream() : nullptr;
    std::vector<cudaEvent_t> ev;
    if (sb) {
        ev.resize(nb + 1, nullptr);
        for (auto& e : ev)
            if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
                for (auto& f : ev)
                    if (f) cudaEventDestroy(f);
                ev.clear();
                sb = nullptr;
                break;
            }
    }
    cudaStream_t si = sb ? sb : st;  // stream of the inverse rows
    for (int k = 0; k < nb; ++k) {
        {
            Trace tr_("chol_diag", st);
            if constexpr (std::is_same<S, double>::value)
                chol_diag64_kernel<<<1, CT, 0, st>>>(N, k, L, X, dg, status);
            else
                chol_diag_kernel<S><<<1, CT, 0, st>>>(N, k, L, X, dg, status);
        }
        if (k >= 1) {
            // inverse row k: needs L rows <= k (panels 0 .. k-1 are done) and X_jj, j <= k
            if (sb) {
                JDFT_CUDA_TRY(cudaEventRecord(ev[k], st));
                JDFT_CUDA_TRY(cudaStreamWaitEvent(sb, ev[k], 0));
            }
            {
                Trace tr_("chol_inv_accum", si);
                inv_accum_kernel<S><<<dim3(k * (k + 1) / 2, 4), CT, 0, si>>>(N, k, L, X, Sa);
            }
            {
                Trace tr_("chol_inv_finish", si);
                inv_finish_kernel<S><<<dim3(k, 4), CT, 0, si>>>(N, k, X, Sa);
            }
        }
        const int m = nb - k - 1;
        if (m > 0) {
            {
                Trace tr_("chol_panel", st);
                chol_panel_kernel<S><<<dim3(m, CB / PR), CT, 0, st>>>(N, k, L, X);
            }
            {
                Trace tr_("chol_update", st);
                chol_update_kernel<S><<<dim3(m * (m + 1) / 2, (CB / UB) * (CB / UB)), CT, 0, st>>>(N, k, L);
            }
        }
    }
    jdft_status s = check_launch("blocked_cholesky_winv");
    if (sb) {
        // join: W needs every inverse row
        cudaEventRecord(ev[nb], sb);
        cudaStreamWaitEvent(st, ev[nb], 0);
        for (auto& e : ev) cudaEventDestroy(e);
    }
    if (s != JDFT_OK) return s;
    {
        Trace tr_("chol_out", st);
        chol_out_kernel<S, T><<<g, 256, 0, st>>>(n, N, X, W);
    }
    return check_launch("blocked_cholesky_winv");
}

jdft_status blocked_cholesky_winv(int n, const double2* U, double2* work, void* W, bool fp64, int* status,
                                  cudaStream_t st) {
    if (fp64) return run_blocked<double, double>(n, U, work, (double2*)W, status, st);
    if (!fp32_factorisation()) return run_blocked<double, float>(n, U, work, (float2*)W, status, st);
    if (!cluster_disabled()) {
        // the status word is cleared here (the multi-block path clears it in chol_init_kernel)
        JDFT_CUDA_TRY(cudaMemsetAsync(status, 0, sizeof(int), st));
        const jdft_status s = run_cluster(n, U, (float2*)W, status, st);
        if (s != JDFT_ERR_UNSUPPORTED) return s;
    }
    return run_blocked<float, float>(n, U, work, (float2*)W, status, st);
}

}  // namespace jdft
