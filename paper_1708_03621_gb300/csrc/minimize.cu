// Band minimisation on the GPU: orthonormalisation and subspace
// diagonalisation (small FP64 dense linear algebra), and the preconditioned
// all-band conjugate-gradient minimiser (JDFTx paper, Sec. 2.1 Minimize:
// nonlinear CG for variational minimisation; Sec. 2.2: variational
// electronic minimisation).  The paper prints no algorithm; the reading used:
//
//   C^dag O C = 1;  E = f tr(C^dag H C);  G = H C - O C (C^dag H C);
//   residual ||G||_F / sqrt(Omega);  K G per coefficient (Teter, identity or
//   a learned network), projected O-orthogonal to C;  Polak-Ribiere
//   direction d (beta reset at < 0), projected;  second-order line step from
//   a1 = 2 Re<HC, d>, a2 = Re<d, Hd> - Re tr(C^dag H C . d^dag O d), halved
//   while the new energy rises above E + 64 ulp;  Y = C + l d,
//   U = Y^dag O Y = L L^dag, C <- Y L^{-dag}, HC <- (HC + l Hd) L^{-dag}.
//
// Mixed precision: the bulk iterations can run with FP32 blocks (FFT chain,
// projector products and block GEMMs in FP32, accumulations of the small
// matrices and all small linear algebra in FP64); once the residual falls
// below a switch threshold, or stops improving, the state is promoted to
// FP64 and refined there to the requested tolerance.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <type_traits>
#include <vector>

#include "chain.cuh"
#include "chol.cuh"
#include "gemm.cuh"
#include "minimize.cuh"
#include "profile.cuh"

namespace jdft {

// ---------------------------------------------------------------------------
// Block kernels (a block is nb bands x npw, band-major, leading dimension ld).
// Grid: x strides over the plane waves of a band, y over the bands, so no
// thread divides an element index.  FP32 blocks compute in FP32 (the SMs'
// FP64 rate is a small fraction of it), with compensated FP32 sums where a
// reduction must keep FP64-like accuracy; FP64 blocks compute in FP64.
// ---------------------------------------------------------------------------
// s + c carries a running FP32 sum to twice the FP32 precision (Knuth's TwoSum).
struct CompSum {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float x) {
        const float t = s + x;
        const float bp = t - s;
        c += (s - (t - bp)) + (x - bp);
        s = t;
    }
    __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};

template <typename T>
__global__ void blk_axpby_kernel(int npw, int nb, double a, const c_t<T>* __restrict__ x, int ldx, double b,
                                 const c_t<T>* __restrict__ y, int ldy, c_t<T>* __restrict__ z, int ldz) {
    const T ar = (T)a, br = (T)b;
    for (int bb = blockIdx.y; bb < nb; bb += gridDim.y) {
        const c_t<T>* xb = x + (size_t)bb * ldx;
        const c_t<T>* yb = y ? y + (size_t)bb * ldy : nullptr;
        c_t<T>* zb = z + (size_t)bb * ldz;
        for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < npw; g += gridDim.x * blockDim.x) {
            const c_t<T> u = xb[g];
            c_t<T> r = mk<T>(ar * u.x, ar * u.y);
            if (yb) {
                const c_t<T> v = yb[g];
                r.x += br * v.x;
                r.y += br * v.y;
            }
            zb[g] = r;
        }
    }
}

// Block sum of a per-thread double into *out (one FP64 atomic per block).
__device__ __forceinline__ void block_sum_to(double acc, double* out) {
    __shared__ double red[32];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        acc = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
        if (threadIdx.x == 0) atomicAdd(out, acc);
    }
}

// out[slot] += Re sum conj(x) y over the whole block.
template <typename T>
__global__ void blk_dot_kernel(int npw, int nb, const c_t<T>* __restrict__ x, int ldx, const c_t<T>* __restrict__ y,
                               int ldy, double* __restrict__ out) {
    double acc = 0.0;
    CompSum cs;
    for (int bb = blockIdx.y; bb < nb; bb += gridDim.y) {
        const c_t<T>* xb = x + (size_t)bb * ldx;
        const c_t<T>* yb = y + (size_t)bb * ldy;
        for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < npw; g += gridDim.x * blockDim.x) {
            const c_t<T> u = xb[g], v = yb[g];
            if constexpr (std::is_same<T, float>::value)
                cs.add(fmaf(u.x, v.x, u.y * v.y));
            else
                acc += u.x * v.x + u.y * v.y;
        }
    }
    if constexpr (std::is_same<T, float>::value) acc = cs.value();
    block_sum_to(acc, out);
}

// Tb[b] = Omega sum_G kin[G] |C_Gb|^2 (one block per band).
template <typename T>
__global__ void band_kinetic_kernel(int npw, const c_t<T>* __restrict__ C, int ldc, const double* __restrict__ kin,
                                    const float* __restrict__ kin32, double omega, double* __restrict__ Tb) {
    const int b = blockIdx.x;
    double acc = 0.0;
    CompSum cs;
    for (int g = threadIdx.x; g < npw; g += blockDim.x) {
        const c_t<T> c = C[(size_t)b * ldc + g];
        if constexpr (std::is_same<T, float>::value)
            cs.add(kin32[g] * fmaf(c.x, c.x, c.y * c.y));
        else
            acc += kin[g] * (c.x * c.x + c.y * c.y);
    }
    if constexpr (std::is_same<T, float>::value) acc = cs.value();
    __shared__ double red[32];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        acc = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
        if (threadIdx.x == 0) Tb[b] = omega * acc;
    }
}

// KG = K(x) G with x = kin / Tb (Teter) or K = 1 (identity); in the block's precision.
template <typename T>
__global__ void precond_teter_kernel(int npw, int nb, const c_t<T>* __restrict__ G, int ldg, c_t<T>* __restrict__ KG,
                                     int ldk, const double* __restrict__ kin, const float* __restrict__ kin32,
                                     const double* __restrict__ Tb, int identity) {
    for (int bb = blockIdx.y; bb < nb; bb += gridDim.y) {
        const T rT = (T)(1.0 / Tb[bb]);
        const c_t<T>* gb = G + (size_t)bb * ldg;
        c_t<T>* kb = KG + (size_t)bb * ldk;
        for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < npw; g += gridDim.x * blockDim.x) {
            T k = (T)1;
            if (!identity) {
                T kg;
                if constexpr (std::is_same<T, float>::value)
                    kg = kin32[g];
                else
                    kg = kin[g];
                const T xx = kg * rT;
                const T num = (T)27 + xx * ((T)18 + xx * ((T)12 + (T)8 * xx));
                k = num / (num + (T)16 * xx * xx * xx * xx);
            }
            const c_t<T> v = gb[g];
            kb[g] = mk<T>(k * v.x, k * v.y);
        }
    }
}

// ---------------------------------------------------------------------------
// Small nb x nb matrices (complex128, row-major)
// ---------------------------------------------------------------------------
// A = (A + A^dag)/2; scal[0] = Re tr A
__global__ void hermitize_kernel(int n, double2* A, double* trace) {
    double acc = 0.0;
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
        const int i = e / n, j = e % n;
        if (i < j) {
            double2 a = A[i * n + j], b = A[j * n + i];
            double2 m = make_double2(0.5 * (a.x + b.x), 0.5 * (a.y - b.y));
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
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
        *trace = s;
    }
}

// out = alpha * A, converted to the block type
template <typename T>
__global__ void small_scale_kernel(int n, const double2* __restrict__ A, double alpha, c_t<T>* __restrict__ out) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n * n; e += gridDim.x * blockDim.x)
        out[e] = mk<T>((T)(alpha * A[e].x), (T)(alpha * A[e].y));
}

// *out = Re tr(A B) for Hermitian A, B: sum_ij A_ij B_ji = sum_ij A_ij conj(B_ij)
__global__ void trace_prod_kernel(int n, const double2* __restrict__ A, const double2* __restrict__ B, double* out) {
    double acc = 0.0;
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
        const int i = e / n, j = e % n;
        const double2 a = A[i * n + j], b = B[j * n + i];
        acc += a.x * b.x - a.y * b.y;
    }
    __shared__ double red[32];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
        *out = s;
    }
}

// One block: U = L L^dag (lower L, overwriting the work copy), then
// X = L^{-1} by forward substitution, W = X^dag (upper), written as the block
// type.  status = JDFT_ERR_NOT_POSDEF if a pivot is not positive.
template <typename T>
__global__ void cholesky_winv_kernel(int n, const double2* __restrict__ U, double2* __restrict__ L,
                                     double2* __restrict__ X, c_t<T>* __restrict__ W, int* status) {
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) L[e] = U[e];
    __syncthreads();
    __shared__ double piv;
    __shared__ int bad;
    if (threadIdx.x == 0) bad = 0;
    for (int j = 0; j < n; ++j) {
        // diagonal
        if (threadIdx.x == 0) {
            // a pivot that is not positive, or that lost all but ~1e-13 of the
            // diagonal to earlier columns, means linearly dependent bands
            const double ujj = L[j * n + j].x;
            double d = ujj;
            for (int k = 0; k < j; ++k) d -= L[j * n + k].x * L[j * n + k].x + L[j * n + k].y * L[j * n + k].y;
            if (!(d > 1e-13 * ujj)) { bad = 1; d = 1.0; }
            piv = sqrt(d);
            L[j * n + j] = make_double2(piv, 0.0);
        }
        __syncthreads();
        // column below the diagonal: L_ij = (U_ij - sum_k L_ik conj(L_jk)) / L_jj
        for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x) {
            double2 s = L[i * n + j];
            for (int k = 0; k < j; ++k) {
                const double2 a = L[i * n + k], b = L[j * n + k];
                s.x -= a.x * b.x + a.y * b.y;
                s.y -= a.y * b.x - a.x * b.y;
            }
            L[i * n + j] = make_double2(s.x / piv, s.y / piv);
        }
        __syncthreads();
    }
    // forward substitution, one column c of the identity per thread: L X = I
    for (int c = threadIdx.x; c < n; c += blockDim.x) {
        for (int i = 0; i < n; ++i) {
            if (i < c) { X[i * n + c] = make_double2(0.0, 0.0); continue; }
            double2 s = make_double2(i == c ? 1.0 : 0.0, 0.0);
            for (int k = c; k < i; ++k) {
                const double2 a = L[i * n + k], x = X[k * n + c];
                s.x -= a.x * x.x - a.y * x.y;
                s.y -= a.x * x.y + a.y * x.x;
            }
            const double d = L[i * n + i].x;
            X[i * n + c] = make_double2(s.x / d, s.y / d);
        }
    }
    __syncthreads();
    // W = X^dag
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
        const int i = e / n, j = e % n;
        const double2 x = X[j * n + i];
        W[e] = mk<T>((T)x.x, (T)(-x.y));
    }
    if (threadIdx.x == 0 && bad) *status = JDFT_ERR_NOT_POSDEF;
}

// Eigenvalues of a Hermitian matrix by cyclic Jacobi rotations (one block,
// in-place on A of size m x m, m even, round-robin pairs; indices >= n are a
// decoupled pad).  eigs receives the sorted diagonal.
__global__ void jacobi_eig_kernel(int n, int m, double2* A, int sweeps, double* eigs) {
    extern __shared__ __align__(16) unsigned char sm_raw[];
    double2* ph = reinterpret_cast<double2*>(sm_raw);   // m/2 phases
    double* cs = reinterpret_cast<double*>(ph + m / 2);  // m/2 cosines
    double* sn = cs + m / 2;                             // m/2 sines
    int* idx = reinterpret_cast<int*>(sn + m / 2);       // m tournament slots
    int* pp = idx + m;                                   // m/2 pair indices
    int* qq = pp + m / 2;
    for (int i = threadIdx.x; i < m; i += blockDim.x) idx[i] = i;
    __syncthreads();
    for (int sw = 0; sw < sweeps; ++sw) {
        for (int step = 0; step < m - 1; ++step) {
            for (int k = threadIdx.x; k < m / 2; k += blockDim.x) {
                int p = idx[k], q = idx[m - 1 - k];
                if (p > q) { int t = p; p = q; q = t; }
                pp[k] = p; qq[k] = q;
                double c = 1.0, s = 0.0;
                double2 e = make_double2(1.0, 0.0);
                if (q < n) {
                    const double2 apq = A[p * m + q];
                    const double ac = hypot(apq.x, apq.y);
                    if (ac > 1e-300) {
                        e = make_double2(apq.x / ac, apq.y / ac);
                        const double th = (A[q * m + q].x - A[p * m + p].x) / (2.0 * ac);
                        const double t = (th >= 0.0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
                        c = 1.0 / sqrt(t * t + 1.0);
                        s = t * c;
                    }
                }
                cs[k] = c; sn[k] = s; ph[k] = e;
            }
            __syncthreads();
            // columns: A[:,p] = c A_p - s conj(e) A_q ; A[:,q] = s A_p + c conj(e) A_q
            for (int w = threadIdx.x; w < (m / 2) * m; w += blockDim.x) {
                const int k = w / m, i = w % m;
                if (sn[k] == 0.0) continue;
                const int p = pp[k], q = qq[k];
                const double c = cs[k], s = sn[k];
                const double2 e = ph[k], a = A[i * m + p], b = A[i * m + q];
                const double2 eb = make_double2(e.x * b.x + e.y * b.y, e.x * b.y - e.y * b.x);  // conj(e) b
                A[i * m + p] = make_double2(c * a.x - s * eb.x, c * a.y - s * eb.y);
                A[i * m + q] = make_double2(s * a.x + c * eb.x, s * a.y + c * eb.y);
            }
            __syncthreads();
            // rows: A[p,:] = c A_p - s e A_q ; A[q,:] = s A_p + c e A_q
            for (int w = threadIdx.x; w < (m / 2) * m; w += blockDim.x) {
                const int k = w / m, j = w % m;
                if (sn[k] == 0.0) continue;
                const int p = pp[k], q = qq[k];
                const double c = cs[k], s = sn[k];
                const double2 e = ph[k], a = A[p * m + j], b = A[q * m + j];
                const double2 eb = make_double2(e.x * b.x - e.y * b.y, e.x * b.y + e.y * b.x);  // e b
                A[p * m + j] = make_double2(c * a.x - s * eb.x, c * a.y - s * eb.y);
                A[q * m + j] = make_double2(s * a.x + c * eb.x, s * a.y + c * eb.y);
            }
            __syncthreads();
            if (threadIdx.x == 0) {  // rotate the tournament: keep idx[0], shift the rest
                const int last = idx[m - 1];
                for (int i = m - 1; i > 1; --i) idx[i] = idx[i - 1];
                idx[1] = last;
            }
            __syncthreads();
        }
    }
    if (threadIdx.x == 0) {  // insertion sort of the n real diagonal entries
        for (int i = 0; i < n; ++i) eigs[i] = A[i * m + i].x;
        for (int i = 1; i < n; ++i) {
            const double v = eigs[i];
            int j = i - 1;
            while (j >= 0 && eigs[j] > v) { eigs[j + 1] = eigs[j]; --j; }
            eigs[j + 1] = v;
        }
    }
}

static int blocks_for(int64_t n) { return (int)std::min<int64_t>(std::max<int64_t>((n + 255) / 256, 1), 152 * 8); }
// Grid of the band-row kernels: about 8 blocks of 256 threads per SM, split
// between the plane waves of a band (x) and the bands (y).
static dim3 rows_grid(int npw, int nb) {
    const int bx = std::max(1, std::min((npw + 255) / 256, 32));
    const int by = std::max(1, std::min(nb, std::max(1, 152 * 8 / bx)));
    return dim3(bx, by);
}

template <typename T>
static jdft_status axpby(int npw, int nb, double a, const c_t<T>* x, int ldx, double b, const c_t<T>* y, int ldy,
                         c_t<T>* z, int ldz, cudaStream_t st) {
    {
        Trace tr_("blk_axpby", st);
        blk_axpby_kernel<T><<<rows_grid(npw, nb), 256, 0, st>>>(npw, nb, a, x, ldx, b, y, ldy, z, ldz);
    }
    return check_launch("blk_axpby");
}

template <typename T>
static jdft_status dot(int npw, int nb, const c_t<T>* x, int ldx, const c_t<T>* y, int ldy, double* out,
                       cudaStream_t st) {
    JDFT_CUDA_TRY(cudaMemsetAsync(out, 0, sizeof(double), st));
    {
        Trace tr_("blk_dot", st);
        blk_dot_kernel<T><<<rows_grid(npw, nb), 256, 0, st>>>(npw, nb, x, ldx, y, ldy, out);
    }
    return check_launch("blk_dot");
}

// work: chol_work_elems(n) double2 elements.  Small matrices factor in one
// block; larger ones use the blocked multi-block version.
jdft_status small_cholesky_winv(int n, const double2* U, double2* work, void* W, bool fp64, int* status,
                                cudaStream_t st) {
    if (n > 32) return blocked_cholesky_winv(n, U, work, W, fp64, status, st);
    Trace tr_("cholesky_winv", st);
    if (fp64)
        cholesky_winv_kernel<double><<<1, 256, 0, st>>>(n, U, work, work + (size_t)n * n, (double2*)W, status);
    else
        cholesky_winv_kernel<float><<<1, 256, 0, st>>>(n, U, work, work + (size_t)n * n, (float2*)W, status);
    return check_launch("cholesky_winv");
}

jdft_status small_jacobi_eigs(int n, const double2* A, double2* work, double* eigs, cudaStream_t st) {
    const int m = n + (n & 1);
    JDFT_CUDA_TRY(cudaMemsetAsync(work, 0, (size_t)m * m * sizeof(double2), st));
    JDFT_CUDA_TRY(cudaMemcpy2DAsync(work, m * sizeof(double2), A, n * sizeof(double2), n * sizeof(double2), n,
                                    cudaMemcpyDeviceToDevice, st));
    if (m > n) {
        const double2 pad = make_double2(1e300, 0.0);
        JDFT_CUDA_TRY(cudaMemcpyAsync(work + (size_t)n * m + n, &pad, sizeof pad, cudaMemcpyHostToDevice, st));
        JDFT_CUDA_TRY(cudaStreamSynchronize(st));
    }
    const size_t smem = (size_t)(m / 2) * (sizeof(double2) + 2 * sizeof(double) + 2 * sizeof(int)) +
                        (size_t)m * sizeof(int);
    const int sweeps = 14;
    {
        Trace tr_("jacobi_eig", st);
        jacobi_eig_kernel<<<1, 256, smem, st>>>(n, m, work, sweeps, eigs);
    }
    return check_launch("jacobi_eig");
}

// ---------------------------------------------------------------------------
// The minimiser state for one precision
// ---------------------------------------------------------------------------
struct DevBuf {
    void* p = nullptr;
    ~DevBuf() { if (p) cudaFree(p); }
};

template <typename T>
struct MinState {
    jdft_basis_s* b;
    int ik, nb, npw, ld;
    jdft_prec prec;
    cudaStream_t st;
    double omega, f;
    // blocks
    c_t<T> *C, *HC, *G, *KG, *KGp, *d, *dp, *Hd, *Y, *HY, *Cn, *HCn;
    // small
    double2 *Hs, *Hsn, *Pm, *dOd, *U, *lawork;
    c_t<T>* Bm;  // scaled small matrix in block type
    c_t<T>* W;
    double *Tb, *scal;
    float* bf;  // per-band features of the learned preconditioner
    int* status;
    DevBuf mem;
    const double* kin;
    const float* kin32;
    // split-operand (BF16x3) products of FP32 blocks: the BF16 planes of one
    // block (or of its transpose), of a second block, of the small matrix, and
    // the split-K partial tiles
    bool tcx = false;
    char *sp1 = nullptr, *sp2 = nullptr, *spw = nullptr, *spp = nullptr;
    size_t spp_bytes = 0;

    jdft_status alloc() {
        const size_t blk = (size_t)nb * ld * sizeof(c_t<T>);
        const size_t sm = (size_t)nb * nb * sizeof(double2);
        const int m = nb + (nb & 1);
        const size_t lab = std::max(2 * (size_t)m * m, chol_work_elems(nb)) * sizeof(double2);
        tcx = std::is_same<T, float>::value && tcx_eligible(prec, nb, nb);
        const size_t s1 = tcx ? std::max(tcx_split_bytes(nb, npw), tcx_split_bytes(npw, nb)) : 0;
        const size_t s2 = tcx ? tcx_split_bytes(nb, npw) : 0, sw = tcx ? tcx_split_bytes(nb, nb) : 0;
        spp_bytes = tcx ? tcx_cn_partial_bytes(nb, nb, npw) : 0;
        const size_t total = 12 * blk + 5 * sm + lab + 2 * (size_t)nb * nb * sizeof(c_t<T>) +
                             (size_t)nb * sizeof(double) + 64 * sizeof(double) + 64 + 3 * (size_t)nb * sizeof(float) +
                             s1 + s2 + sw + spp_bytes + 21 * 256;
        JDFT_CUDA_TRY(cudaMalloc(&mem.p, total));
        char* q = (char*)mem.p;
        auto take = [&](size_t n) { char* r = q; q += (n + 255) / 256 * 256; return (void*)r; };
        C = (c_t<T>*)take(blk); HC = (c_t<T>*)take(blk); G = (c_t<T>*)take(blk); KG = (c_t<T>*)take(blk);
        KGp = (c_t<T>*)take(blk); d = (c_t<T>*)take(blk); dp = (c_t<T>*)take(blk); Hd = (c_t<T>*)take(blk);
        Y = (c_t<T>*)take(blk); HY = (c_t<T>*)take(blk); Cn = (c_t<T>*)take(blk); HCn = (c_t<T>*)take(blk);
        Hs = (double2*)take(sm); Hsn = (double2*)take(sm); Pm = (double2*)take(sm); dOd = (double2*)take(sm);
        U = (double2*)take(sm); lawork = (double2*)take(lab);
        Bm = (c_t<T>*)take((size_t)nb * nb * sizeof(c_t<T>)); W = (c_t<T>*)take((size_t)nb * nb * sizeof(c_t<T>));
        Tb = (double*)take(nb * sizeof(double)); scal = (double*)take(64 * sizeof(double)); status = (int*)take(64);
        bf = (float*)take(3 * (size_t)nb * sizeof(float));
        if (tcx) {
            sp1 = (char*)take(s1);
            sp2 = (char*)take(s2);
            spw = (char*)take(sw);
            spp = (char*)take(spp_bytes);
        }
        JDFT_CUDA_TRY(cudaMemsetAsync(status, 0, sizeof(int), st));
        return JDFT_OK;
    }

    jdft_status applyH(const c_t<T>* X, c_t<T>* HX) {
        return jdft_apply_H(b, ik, X, ld, HX, ld, nb, prec, st);
    }
    // out (nb x nb complex128) = alpha X^dag Y
    jdft_status cn(const c_t<T>* X, const c_t<T>* Yb, double2* out, double alpha) {
        JDFT_CUDA_TRY(cudaMemsetAsync(out, 0, (size_t)nb * nb * sizeof(double2), st));
        if (tcx) {
            // X^dag X is Hermitian: its upper tiles only
            jdft_status s = tcx_split((const float2*)X, ld, nb, npw, sp1, st);
            if (s == JDFT_OK && Yb != X) s = tcx_split((const float2*)Yb, ld, nb, npw, sp2, st);
            if (s != JDFT_OK) return s;
            return tcx_cn(nb, nb, npw, sp1, Yb != X ? sp2 : sp1, out, nb, alpha, st, spp, spp_bytes, Yb == X);
        }
        return gemm_cn<T>(prec, nb, nb, npw, X, ld, Yb, ld, out, nb, alpha, st);
    }
    // Z (+)= X . S for a small block-type S, from split operands
    jdft_status tcx_times(const c_t<T>* X, const c_t<T>* S, c_t<T>* Z, bool accumulate) {
        jdft_status s = tcx_split_t((const float2*)X, ld, npw, nb, sp1, st);
        if (s == JDFT_OK) s = tcx_split_t((const float2*)S, nb, nb, nb, spw, st);
        if (s != JDFT_OK) return s;
        return tcx_nn(npw, nb, nb, sp1, spw, (float2*)Z, ld, accumulate, st);
    }
    // Z += X . (alpha A)   (A small complex128)
    jdft_status nn_acc(const c_t<T>* X, const double2* A, double alpha, c_t<T>* Z) {
        {
            Trace tr_("small_scale", st);
            small_scale_kernel<T><<<blocks_for((int64_t)nb * nb), 256, 0, st>>>(nb, A, alpha, Bm);
        }
        jdft_status s = check_launch("small_scale");
        if (s != JDFT_OK) return s;
        if (tcx) return tcx_times(X, Bm, Z, true);
        return gemm_nn_acc<T>(prec, npw, nb, nb, X, ld, Bm, nb, Z, ld, st);
    }
    // Z = X . W  (W already in block type)
    jdft_status rotate(const c_t<T>* X, c_t<T>* Z) {
        if (tcx) return tcx_times(X, W, Z, false);
        return gemm_nn_acc<T>(prec, npw, nb, nb, X, ld, W, nb, Z, ld, st, false);
    }
    jdft_status hermitize(double2* A, double* tr) {
        {
            Trace tr_("hermitize", st);
            hermitize_kernel<<<1, 256, 0, st>>>(nb, A, tr);
        }
        return check_launch("hermitize");
    }
    // X <- X - C (Omega C^dag X)
    jdft_status project(c_t<T>* X) {
        jdft_status s = cn(C, X, Pm, omega);
        if (s != JDFT_OK) return s;
        return nn_acc(C, Pm, -1.0, X);
    }
    jdft_status read_scal(double* host, int n) {
        JDFT_CUDA_TRY(cudaMemcpyAsync(host, scal, n * sizeof(double), cudaMemcpyDeviceToHost, st));
        JDFT_CUDA_TRY(cudaStreamSynchronize(st));
        return JDFT_OK;
    }
    jdft_status read_status() {
        int s = 0;
        JDFT_CUDA_TRY(cudaMemcpyAsync(&s, status, sizeof(int), cudaMemcpyDeviceToHost, st));
        JDFT_CUDA_TRY(cudaStreamSynchronize(st));
        if (s != 0) return set_error((jdft_status)s, "overlap matrix not positive definite in the minimiser");
        return JDFT_OK;
    }
    // Orthonormalise X -> C (Cholesky of Omega X^dag X), then HC = H C, Hs = C^dag HC.
    jdft_status start_from(const c_t<T>* X) {
        jdft_status s;
        if ((s = cn(X, X, U, omega))) return s;
        if ((s = small_cholesky_winv(nb, U, lawork, W, std::is_same<T, double>::value, status, st))) return s;
        if ((s = read_status())) return s;
        if ((s = rotate(X, C))) return s;
        if ((s = applyH(C, HC))) return s;
        if ((s = cn(C, HC, Hs, 1.0))) return s;
        return hermitize(Hs, scal + 0);
    }
};

// scal slots
enum { S_TR = 0, S_GG = 1, S_GKG = 2, S_GKGP = 3, S_A1 = 4, S_DHD = 5, S_HSDOD = 6, S_TRN = 7 };

template <typename T>
static jdft_status run_phase(MinState<T>& M, const jdft_min_opts& o, double stop_res, bool allow_stall_exit,
                             int max_iter, jdft_min_report* rep, double* res_out, double* E_out) {
    jdft_status s;
    const int npw = M.npw, nb = M.nb, ld = M.ld;
    cudaStream_t st = M.st;
    double h[8];
    double gkgp_prev = 0.0;
    bool have_prev = false;
    double best = 1e300;
    int stall = 0;
    // the learned preconditioner, while it passes its checks; Teter's after a failure
    auto use_mlp = [&]() { return o.precond == JDFT_PRECOND_MLP && !rep->precond_fallback; };
    double mlp_best = 1e300;
    int mlp_stall = 0;
    auto fall_back = [&]() {
        rep->precond_fallback = 1;
        have_prev = false;  // restart the conjugate directions
    };
    for (int it = 0;; ++it) {
        // gradient and residual
        if ((s = axpby<T>(npw, nb, 1.0, M.HC, ld, 0.0, nullptr, 0, M.G, ld, st))) return s;
        if ((s = M.nn_acc(M.C, M.Hs, -M.omega, M.G))) return s;
        if ((s = dot<T>(npw, nb, M.G, ld, M.G, ld, M.scal + S_GG, st))) return s;
        if ((s = M.read_scal(h, 2))) return s;
        const double E = M.f * h[S_TR];
        const double res = std::sqrt(std::max(h[S_GG], 0.0) / M.omega);
        *res_out = res;
        *E_out = E;
        if (res < stop_res) return JDFT_OK;
        if (allow_stall_exit) {
            if (res < 0.7 * best) { best = res; stall = 0; }
            else if (++stall >= 8) return JDFT_OK;
        }
        if (use_mlp()) {
            if (res < 0.7 * mlp_best) { mlp_best = res; mlp_stall = 0; }
            else if (++mlp_stall >= 40) fall_back();  // no progress with the network's directions
        }
        if (it >= max_iter || rep->iterations >= o.max_iter)
            return set_error(JDFT_ERR_NOT_CONVERGED, "band minimiser reached its iteration limit");
        rep->iterations++;
        // preconditioned gradient, projected
        {
            Trace tr_("band_kinetic", st);
            band_kinetic_kernel<T><<<nb, 256, 0, st>>>(npw, M.C, ld, M.kin, M.kin32, M.omega, M.Tb);
        }
        if ((s = check_launch("band_kinetic"))) return s;
        if (use_mlp()) {
            if ((s = mlp_precondition<T>(o.mlp, npw, nb, M.G, ld, M.KG, ld, M.kin, M.Tb, M.Hs, M.bf, st))) return s;
        } else {
            Trace tr_("precond_teter", st);
            precond_teter_kernel<T><<<rows_grid(npw, nb), 256, 0, st>>>(
                npw, nb, M.G, ld, M.KG, ld, M.kin, M.kin32, M.Tb, o.precond == JDFT_PRECOND_IDENTITY);
        }
        if ((s = check_launch("precondition"))) return s;
        if ((s = M.project(M.KG))) return s;
        // Polak-Ribiere
        if ((s = dot<T>(npw, nb, M.G, ld, M.KG, ld, M.scal + S_GKG, st))) return s;
        if (have_prev && (s = dot<T>(npw, nb, M.G, ld, M.KGp, ld, M.scal + S_GKGP, st))) return s;
        if ((s = M.read_scal(h, 4))) return s;
        if (use_mlp() && !(std::isfinite(h[S_GKG]) && h[S_GKG] > 0.0)) {
            // K G must be finite with G.(K G) > 0 (a positive preconditioner)
            fall_back();
            --rep->iterations;
            continue;
        }
        double beta = 0.0;
        if (have_prev && gkgp_prev != 0.0) beta = std::max(0.0, (h[S_GKG] - h[S_GKGP]) / gkgp_prev);
        const double gkg = h[S_GKG];
        for (int attempt = 0; attempt < 2; ++attempt) {
            if (beta > 0.0) {
                if ((s = axpby<T>(npw, nb, -1.0, M.KG, ld, beta, M.dp, ld, M.d, ld, st))) return s;
            } else {
                if ((s = axpby<T>(npw, nb, -1.0, M.KG, ld, 0.0, nullptr, 0, M.d, ld, st))) return s;
            }
            if ((s = M.project(M.d))) return s;
            if ((s = M.applyH(M.d, M.Hd))) return s;
            if ((s = dot<T>(npw, nb, M.HC, ld, M.d, ld, M.scal + S_A1, st))) return s;
            if ((s = dot<T>(npw, nb, M.d, ld, M.Hd, ld, M.scal + S_DHD, st))) return s;
            if ((s = M.cn(M.d, M.d, M.dOd, M.omega))) return s;
            {
                Trace tr_("trace_prod", st);
                trace_prod_kernel<<<1, 256, 0, st>>>(nb, M.Hs, M.dOd, M.scal + S_HSDOD);
            }
            if ((s = check_launch("trace_prod"))) return s;
            if ((s = M.read_scal(h, 7))) return s;
            if (2.0 * h[S_A1] < 0.0 || beta == 0.0) break;
            beta = 0.0;  // not a descent direction: restart along -KG
        }
        const double a1 = 2.0 * h[S_A1];
        const double a2 = h[S_DHD] - h[S_HSDOD];
        if (use_mlp() && !(std::isfinite(a1) && std::isfinite(a2) && a1 < 0.0)) {
            fall_back();  // not a finite descent direction even after the restart
            --rep->iterations;
            continue;
        }
        double lam = (a2 > 0.0) ? -a1 / (2.0 * a2) : 1.0;
        // error level of the computed energy: 64 ulp in FP64; with FP32 blocks,
        // 16 FP32 ulp for CUDA-core products, and for the 3-product tensor-core
        // splits their accuracy, 2e-5 relative (the FP32 accumulation of the
        // split products over long K; a tighter rule stops the cheap phase as
        // soon as the true decrease per step falls below it)
        const double rel = std::is_same<T, double>::value ? 64.0 * 2.220446049250313e-16
                           : (M.prec == JDFT_TF32X3 || M.prec == JDFT_BF16X3) ? 2e-5
                                                                             : 16.0 * 1.1920928955078125e-7;
        const double noise = rel * std::fabs(E);
        bool accepted = false;
        for (int tries = 0; tries < 30; ++tries) {
            if ((s = axpby<T>(npw, nb, 1.0, M.C, ld, lam, M.d, ld, M.Y, ld, st))) return s;
            if ((s = axpby<T>(npw, nb, 1.0, M.HC, ld, lam, M.Hd, ld, M.HY, ld, st))) return s;
            if ((s = M.cn(M.Y, M.Y, M.U, M.omega))) return s;
            if ((s = small_cholesky_winv(nb, M.U, M.lawork, M.W, std::is_same<T, double>::value, M.status, st)))
                return s;
            if ((s = M.read_status())) return s;
            if ((s = M.rotate(M.Y, M.Cn))) return s;
            if ((s = M.rotate(M.HY, M.HCn))) return s;
            if ((s = M.cn(M.Cn, M.HCn, M.Hsn, 1.0))) return s;
            if ((s = M.hermitize(M.Hsn, M.scal + S_TRN))) return s;
            if ((s = M.read_scal(h, 8))) return s;
            if (M.f * h[S_TRN] <= E + noise) { accepted = true; break; }
            lam *= 0.5;
        }
        if (!accepted && use_mlp()) {
            // no lower energy along the network's direction: Teter's from here on
            fall_back();
            --rep->iterations;
            continue;
        }
        if (!accepted) { *res_out = res; return JDFT_OK; }  // no lower energy along d: stationary to rounding
        std::swap(M.C, M.Cn);
        std::swap(M.HC, M.HCn);
        std::swap(M.Hs, M.Hsn);
        JDFT_CUDA_TRY(cudaMemcpyAsync(M.scal + S_TR, M.scal + S_TRN, sizeof(double), cudaMemcpyDeviceToDevice, st));
        std::swap(M.d, M.dp);
        std::swap(M.KG, M.KGp);
        gkgp_prev = gkg;
        have_prev = true;
    }
}

template <typename T>
static jdft_status setup_state(MinState<T>& M, jdft_basis_s* b, int ik, int nb, jdft_prec prec, double f,
                               cudaStream_t st) {
    M.b = b; M.ik = ik; M.nb = nb; M.npw = b->ks[ik].npw; M.ld = M.npw; M.prec = prec; M.st = st;
    M.omega = b->omega; M.f = f; M.kin = b->ks[ik].kin; M.kin32 = b->ks[ik].kin32;
    return M.alloc();
}

template <typename Src, typename Dst>
__global__ void convert_block_kernel(int npw, int nb, const c_t<Src>* __restrict__ a, int lda, c_t<Dst>* __restrict__ z,
                                     int ldz) {
    const int64_t total = (int64_t)npw * nb;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t bb = i / npw, g = i - bb * npw;
        const c_t<Src> v = a[bb * lda + g];
        z[bb * ldz + g] = mk<Dst>((Dst)v.x, (Dst)v.y);
    }
}

}  // namespace jdft

using namespace jdft;

extern "C" {

}  // extern "C"

namespace jdft {
// *dst = max(*dst, *src): a sticky status word for the asynchronous form.
__global__ void status_merge_kernel(const int* __restrict__ src, int* __restrict__ dst) {
    if (threadIdx.x == 0 && *src > *dst) *dst = *src;
}

// SMs the plane kernels leave to the overlap factorisation running beside them
// in jdft_hamiltonian_step (its kernels are small and latency-bound).
constexpr int kStepReserveSms = 4;

// sticky == nullptr: synchronous, the factorisation's status is returned;
// otherwise the status is merged into the device word *sticky and nothing waits.
template <typename T>
static jdft_status orthonormalize_impl(jdft_basis_s* b, int ik, void* C, int ldc, int nb, jdft_prec prec,
                                       cudaStream_t st, int* sticky = nullptr, const double2* Ugiven = nullptr) {
    const int npw = b->ks[ik].npw;
    const int m = nb + (nb & 1);
    const size_t sm = ((size_t)nb * nb * sizeof(double2) + 255) / 256 * 256;
    const size_t wbytes = ((size_t)nb * nb * sizeof(c_t<T>) + 255) / 256 * 256;
    const size_t lab = ((std::max(2 * (size_t)m * m, chol_work_elems(nb)) * sizeof(double2)) + 255) / 256 * 256;
    const size_t blk = ((size_t)nb * ldc * sizeof(c_t<T>) + 255) / 256 * 256;
    const bool split = !Ugiven && std::is_same<T, float>::value && tcx_eligible(prec, nb, nb);
    const size_t spl = split ? (tcx_split_bytes(nb, npw) + 255) / 256 * 256 : 0;
    const size_t pb = split ? tcx_cn_partial_bytes(nb, nb, npw) : 0;
    // the basis workspace (grown once) holds U, W, the factorisation scratch, a copy of C, a status
    // word and, for the split-operand overlap, the BF16 planes of C and the product's partial tiles
    jdft_status s = ensure_workspace(b, sm + wbytes + lab + blk + 256 + spl + pb);
    if (s != JDFT_OK) return s;
    char* q = (char*)b->work.ptr;
    double2* U = (double2*)q;
    c_t<T>* W = (c_t<T>*)(q + sm);
    double2* work = (double2*)(q + sm + wbytes);
    c_t<T>* tmp = (c_t<T>*)(q + sm + wbytes + lab);
    int* status = (int*)(q + sm + wbytes + lab + blk);
    JDFT_CUDA_TRY(cudaMemsetAsync(status, 0, sizeof(int), st));
    if (Ugiven) {
        U = const_cast<double2*>(Ugiven);  // read only
    } else {
        JDFT_CUDA_TRY(cudaMemsetAsync(U, 0, (size_t)nb * nb * sizeof(double2), st));
        if (split) {
            // the same split-operand product jdft_subspace forms C^dag O C with
            void* planes = q + sm + wbytes + lab + blk + 256;
            if ((s = tcx_split((const float2*)C, ldc, nb, npw, planes, st))) return s;
            if ((s = tcx_cn(nb, nb, npw, planes, planes, U, nb, b->omega, st, (char*)planes + spl, pb, true)))
                return s;
        } else if ((s = gemm_cn<T>(prec, nb, nb, npw, (const c_t<T>*)C, ldc, (const c_t<T>*)C, ldc, U, nb, b->omega,
                                   st))) {
            return s;
        }
    }
    if ((s = small_cholesky_winv(nb, U, work, W, std::is_same<T, double>::value, status, st))) return s;
    if (gemm_nn_inplace_ok(prec, nb)) {
        // C <- C W in place: each block reads its rows of C for every band before writing them
        if ((s = gemm_nn_acc<T>(prec, npw, nb, nb, (const c_t<T>*)C, ldc, W, nb, (c_t<T>*)C, ldc, st, false)))
            return s;
    } else {
        JDFT_CUDA_TRY(cudaMemcpyAsync(tmp, C, (size_t)nb * ldc * sizeof(c_t<T>), cudaMemcpyDeviceToDevice, st));
        if ((s = gemm_nn_acc<T>(prec, npw, nb, nb, tmp, ldc, W, nb, (c_t<T>*)C, ldc, st, false))) return s;
    }
    if (sticky) {
        {
            Trace tr_("status_merge", st);
            status_merge_kernel<<<1, 32, 0, st>>>(status, sticky);
        }
        return check_launch("status_merge");
    }
    int hs = 0;
    JDFT_CUDA_TRY(cudaMemcpyAsync(&hs, status, sizeof(int), cudaMemcpyDeviceToHost, st));
    JDFT_CUDA_TRY(cudaStreamSynchronize(st));
    if (hs) return set_error(JDFT_ERR_NOT_POSDEF, "C^dag O C is not positive definite");
    return JDFT_OK;
}
}  // namespace jdft

namespace jdft {

static size_t r256(size_t x) { return (x + 255) / 256 * 256; }

// Side stream and fork / join events of a basis (created on first use).
static jdft_status step_streams(jdft_basis_s* b) {
    if (!b->side) {
        JDFT_CUDA_TRY(cudaStreamCreateWithFlags(&b->side, cudaStreamNonBlocking));
        JDFT_CUDA_TRY(cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming));
        JDFT_CUDA_TRY(cudaEventCreateWithFlags(&b->ev_join, cudaEventDisableTiming));
    }
    return JDFT_OK;
}

// W = L^{-dag} of U = L L^dag (FP64 factorisation), in the basis's factor
// workspace (not the chain's), with its outcome merged into *sticky.
template <typename T>
static jdft_status overlap_factor(jdft_basis_s* b, const double2* U, int nb, int* sticky, cudaStream_t st,
                                  c_t<T>** W_out) {
    const int m = nb + (nb & 1);
    const size_t wbytes = r256((size_t)nb * nb * sizeof(c_t<T>));
    const size_t lab = r256(std::max(2 * (size_t)m * m, chol_work_elems(nb)) * sizeof(double2));
    jdft_status s = ensure_ws(b->fwork, wbytes + lab + 256);
    if (s != JDFT_OK) return s;
    char* q = (char*)b->fwork.ptr;
    c_t<T>* W = (c_t<T>*)q;
    double2* work = (double2*)(q + wbytes);
    int* status = (int*)(q + wbytes + lab);
    JDFT_CUDA_TRY(cudaMemsetAsync(status, 0, sizeof(int), st));
    if ((s = small_cholesky_winv(nb, U, work, W, std::is_same<T, double>::value, status, st))) return s;
    {
        Trace tr_("status_merge", st);
        status_merge_kernel<<<1, 32, 0, st>>>(status, sticky);
    }
    *W_out = W;
    return check_launch("status_merge");
}

// One pass of the hot path over a band block: C^dag O C from the input block;
// its FP64 factorisation on the basis's side stream (leaving reserve SMs free
// of the persistent plane kernel) while H C and n(r) run; C^dag H C; then
// C <- C L^{-dag} once the factor has joined.  Split-operand products share
// one BF16 split of C (and one of H C).
template <typename T>
static jdft_status hamiltonian_step_impl(jdft_basis_s* b, int ik, void* C, int ldc, void* HC, int ldhc, int nb,
                                         const double* f, double* n_r, double2* CHC, double2* COC, bool ortho,
                                         int* sticky, jdft_prec prec, cudaStream_t st) {
    const int npw = b->ks[ik].npw;
    const bool split = std::is_same<T, float>::value && tcx_eligible(prec, nb, nb);
    const size_t chain = r256(apply_H_density_workspace(b, ik, nb, prec, !split));
    const size_t cs = split ? r256(tcx_split_bytes(nb, npw)) : 0;
    const bool inplace = gemm_nn_inplace_ok(prec, nb);
    const size_t tmpb = inplace ? 0 : r256((size_t)nb * ldc * sizeof(c_t<T>));
    // layout: chain region, planes of C, planes of H C; the copy of C that a
    // rotation out of place needs reuses the start once the rest is done
    // the rotation's transposed splits of C and W reuse the start once the rest is done
    const size_t rot = split ? r256(tcx_split_bytes(npw, nb)) + r256(tcx_split_bytes(nb, nb)) : 0;
    // the split-K partial tiles of C^dag O C and C^dag H C follow the planes
    const size_t pb = split ? tcx_cn_partial_bytes(nb, nb, npw) : 0;
    jdft_status s = ensure_workspace(b, std::max(std::max(chain + 2 * cs + pb, tmpb), rot));
    if (s != JDFT_OK) return s;
    char* ws = (char*)b->work.ptr;
    void* Cs = ws + chain;
    void* HCs = ws + chain + cs;
    void* part = ws + chain + 2 * cs;
    const c_t<T>* Cc = (const c_t<T>*)C;
    JDFT_CUDA_TRY(cudaMemsetAsync(COC, 0, (size_t)nb * nb * sizeof(double2), st));
    if (split) {
        if ((s = tcx_split((const float2*)C, ldc, nb, npw, Cs, st))) return s;
        if ((s = tcx_cn(nb, nb, npw, Cs, Cs, COC, nb, b->omega, st, part, pb, true))) return s;
    } else if ((s = gemm_cn<T>(prec, nb, nb, npw, Cc, ldc, Cc, ldc, COC, nb, b->omega, st))) {
        return s;
    }
    c_t<T>* W = nullptr;
    if (ortho) {
        if ((s = step_streams(b))) return s;
        JDFT_CUDA_TRY(cudaEventRecord(b->ev_fork, st));
        JDFT_CUDA_TRY(cudaStreamWaitEvent(b->side, b->ev_fork, 0));
        if ((s = overlap_factor<T>(b, COC, nb, sticky, b->side, &W))) return s;
        JDFT_CUDA_TRY(cudaEventRecord(b->ev_join, b->side));
        b->reserve_sms = kStepReserveSms;
    }
    s = apply_H_density_with_split(b, ik, C, ldc, HC, ldhc, nb, f, n_r, prec, st, split ? Cs : nullptr);
    b->reserve_sms = 0;
    if (s != JDFT_OK) return s;
    JDFT_CUDA_TRY(cudaMemsetAsync(CHC, 0, (size_t)nb * nb * sizeof(double2), st));
    if (split) {
        if ((s = tcx_split((const float2*)HC, ldhc, nb, npw, HCs, st))) return s;
        // H C is this step's own H C, so C^dag H C is Hermitian up to rounding
        if ((s = tcx_cn(nb, nb, npw, Cs, HCs, CHC, nb, 1.0, st, part, pb, true))) return s;
    } else if ((s = gemm_cn<T>(prec, nb, nb, npw, Cc, ldc, (const c_t<T>*)HC, ldhc, CHC, nb, 1.0, st))) {
        return s;
    }
    if (!ortho) return JDFT_OK;
    JDFT_CUDA_TRY(cudaStreamWaitEvent(st, b->ev_join, 0));
    if (split) {
        // C <- C W from split operands: C's transpose (its planes take the
        // chain region, free now) and W's; the product writes C directly
        void* Ct = ws;
        void* Wt = ws + r256(tcx_split_bytes(npw, nb));
        if ((s = tcx_split_t((const float2*)C, ldc, npw, nb, Ct, st))) return s;
        if ((s = tcx_split_t((const float2*)W, nb, nb, nb, Wt, st))) return s;
        return tcx_nn(npw, nb, nb, Ct, Wt, (float2*)C, ldc, false, st);
    }
    if (inplace) return gemm_nn_acc<T>(prec, npw, nb, nb, Cc, ldc, W, nb, (c_t<T>*)C, ldc, st, false);
    c_t<T>* tmp = (c_t<T>*)ws;
    JDFT_CUDA_TRY(cudaMemcpyAsync(tmp, C, (size_t)nb * ldc * sizeof(c_t<T>), cudaMemcpyDeviceToDevice, st));
    return gemm_nn_acc<T>(prec, npw, nb, nb, tmp, ldc, W, nb, (c_t<T>*)C, ldc, st, false);
}
}  // namespace jdft

extern "C" {

jdft_status jdft_hamiltonian_step(jdft_basis_t b, int ik, void* C, int ldc, void* HC, int ldhc, int nb,
                                  const double* f, double* n_r, void* CHC, void* COC, int orthonormalize,
                                  int* status, jdft_prec prec, void* stream) {
    clear_error();
    JDFT_CHECK_ARG(b, "null basis");
    JDFT_CHECK_ARG(ik >= 0 && ik < b->nk, "k-point index out of range");
    JDFT_CHECK_ARG(prec >= JDFT_FP64 && prec <= JDFT_BF16X3, "unknown precision");
    JDFT_CHECK_ARG(nb >= 1, "nb must be >= 1");
    const int npw = b->ks[ik].npw;
    const uintptr_t align = prec == JDFT_FP64 ? 16 : 8;
    JDFT_CHECK_ARG(C && HC && f && n_r && CHC && COC, "null block, occupation, density or subspace pointer");
    JDFT_CHECK_ARG(ldc >= npw && ldhc >= npw, "leading dimension < npw");
    JDFT_CHECK_ARG((uintptr_t)C % align == 0 && (uintptr_t)HC % align == 0, "C or HC not aligned to its complex type");
    JDFT_CHECK_ARG((uintptr_t)CHC % 16 == 0 && (uintptr_t)COC % 16 == 0, "subspace outputs must be 16-byte aligned");
    JDFT_CHECK_ARG(!orthonormalize || status, "orthonormalize needs a status word");
    if (!b->have_V) return set_error(JDFT_ERR_ARG, "no potential set (call jdft_set_potential first)");
    cudaStream_t st = (cudaStream_t)stream;
    return prec == JDFT_FP64
               ? hamiltonian_step_impl<double>(b, ik, C, ldc, HC, ldhc, nb, f, n_r, (double2*)CHC, (double2*)COC,
                                               orthonormalize != 0, status, prec, st)
               : hamiltonian_step_impl<float>(b, ik, C, ldc, HC, ldhc, nb, f, n_r, (double2*)CHC, (double2*)COC,
                                              orthonormalize != 0, status, prec, st);
}

jdft_status jdft_orthonormalize(jdft_basis_t b, int ik, void* C, int ldc, int nb, jdft_prec prec, void* stream) {
    clear_error();
    JDFT_CHECK_ARG(b && C, "null argument");
    JDFT_CHECK_ARG(ik >= 0 && ik < b->nk, "k-point index out of range");
    JDFT_CHECK_ARG(nb >= 1 && ldc >= b->ks[ik].npw, "bad block shape");
    JDFT_CHECK_ARG(prec >= JDFT_FP64 && prec <= JDFT_BF16X3, "unknown precision");
    cudaStream_t st = (cudaStream_t)stream;
    return prec == JDFT_FP64 ? orthonormalize_impl<double>(b, ik, C, ldc, nb, prec, st)
                             : orthonormalize_impl<float>(b, ik, C, ldc, nb, prec, st);
}

jdft_status jdft_orthonormalize_async(jdft_basis_t b, int ik, void* C, int ldc, int nb, const void* U,
                                      jdft_prec prec, int* status, void* stream) {
    clear_error();
    JDFT_CHECK_ARG(b && C && status, "null argument");
    JDFT_CHECK_ARG(ik >= 0 && ik < b->nk, "k-point index out of range");
    JDFT_CHECK_ARG(nb >= 1 && ldc >= b->ks[ik].npw, "bad block shape");
    JDFT_CHECK_ARG(prec >= JDFT_FP64 && prec <= JDFT_BF16X3, "unknown precision");
    cudaStream_t st = (cudaStream_t)stream;
    const double2* Ug = (const double2*)U;
    return prec == JDFT_FP64 ? orthonormalize_impl<double>(b, ik, C, ldc, nb, prec, st, status, Ug)
                             : orthonormalize_impl<float>(b, ik, C, ldc, nb, prec, st, status, Ug);
}

jdft_status jdft_subspace_eigs(int nb, const void* A, double* eigs, void* stream) {
    clear_error();
    JDFT_CHECK_ARG(nb >= 1 && A && eigs, "bad arguments");
    const int m = nb + (nb & 1);
    DevBuf mem;
    JDFT_CUDA_TRY(cudaMalloc(&mem.p, (size_t)m * m * sizeof(double2)));
    cudaStream_t st = (cudaStream_t)stream;
    jdft_status s = small_jacobi_eigs(nb, (const double2*)A, (double2*)mem.p, eigs, st);
    if (s != JDFT_OK) return s;
    JDFT_CUDA_TRY(cudaStreamSynchronize(st));
    return JDFT_OK;
}

jdft_status jdft_minimize_bands(jdft_basis_t b, int ik, void* C, int ldc, int nb, const jdft_min_opts* opts,
                                double* eigs, jdft_min_report* report, void* stream) {
    clear_error();
    JDFT_CHECK_ARG(b && C && opts && report, "null argument");
    JDFT_CHECK_ARG(ik >= 0 && ik < b->nk, "k-point index out of range");
    const int npw = b->ks[ik].npw;
    JDFT_CHECK_ARG(nb >= 1 && nb <= npw && ldc >= npw, "bad block shape");
    JDFT_CHECK_ARG(opts->tol > 0 && opts->max_iter >= 1, "bad tolerance or iteration limit");
    JDFT_CHECK_ARG(opts->precond >= JDFT_PRECOND_IDENTITY && opts->precond <= JDFT_PRECOND_MLP, "bad preconditioner");
    JDFT_CHECK_ARG(opts->precond != JDFT_PRECOND_MLP || opts->mlp, "MLP preconditioner needs weights");
    if (!b->have_V) return set_error(JDFT_ERR_ARG, "no potential set");
    cudaStream_t st = (cudaStream_t)stream;
    const double f = opts->occupation > 0 ? opts->occupation : 2.0;
    *report = jdft_min_report();
    auto t0 = std::chrono::steady_clock::now();
    double res = 0.0, E = 0.0;
    jdft_status s;
    MinState<double> M64;
    if ((s = setup_state(M64, b, ik, nb, JDFT_FP64, f, st))) return s;
    JDFT_CUDA_TRY(cudaMemcpy2DAsync(M64.Y, (size_t)npw * sizeof(double2), C, (size_t)ldc * sizeof(double2),
                                    (size_t)npw * sizeof(double2), nb, cudaMemcpyDeviceToDevice, st));
    if (opts->prec != JDFT_FP64) {
        // bulk iterations with FP32 blocks, then promote
        MinState<float> M32;
        if ((s = setup_state(M32, b, ik, nb, opts->prec, f, st))) return s;
        {
            Trace tr_("convert_block", st);
            convert_block_kernel<double, float><<<blocks_for((int64_t)npw * nb), 256, 0, st>>>(npw, nb, M64.Y, npw,
                                                                                             M32.Y, npw);
        }
        if ((s = check_launch("convert_block"))) return s;
        if ((s = M32.start_from(M32.Y))) return s;
        const double sw = opts->switch_tol > 0 ? opts->switch_tol : 1e-4;
        s = run_phase<float>(M32, *opts, std::max(sw, opts->tol), true, opts->max_iter, report, &res, &E);
        if (s != JDFT_OK && s != JDFT_ERR_NOT_CONVERGED) return s;
        report->mixed_iterations = report->iterations;
        {
            Trace tr_("convert_block", st);
            convert_block_kernel<float, double><<<blocks_for((int64_t)npw * nb), 256, 0, st>>>(npw, nb, M32.C, npw,
                                                                                             M64.Y, npw);
        }
        if ((s = check_launch("convert_block"))) return s;
    }
    if ((s = M64.start_from(M64.Y))) return s;
    jdft_min_opts o64 = *opts;
    s = run_phase<double>(M64, o64, opts->tol, false, opts->max_iter, report, &res, &E);
    report->residual = res;
    report->energy = E;
    report->converged = (s == JDFT_OK && res < opts->tol) ? 1 : 0;
    if (s != JDFT_OK && s != JDFT_ERR_NOT_CONVERGED) return s;
    // outputs: converged block and subspace eigenvalues
    JDFT_CUDA_TRY(cudaMemcpy2DAsync(C, (size_t)ldc * sizeof(double2), M64.C, (size_t)npw * sizeof(double2),
                                    (size_t)npw * sizeof(double2), nb, cudaMemcpyDeviceToDevice, st));
    if (eigs) {
        jdft_status s2 = small_jacobi_eigs(nb, M64.Hs, M64.lawork, eigs, st);
        if (s2 != JDFT_OK) return s2;
    }
    JDFT_CUDA_TRY(cudaStreamSynchronize(st));
    report->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (!report->converged) return set_error(JDFT_ERR_NOT_CONVERGED, "band minimiser reached its iteration limit");
    return JDFT_OK;
}

}  // extern "C"
