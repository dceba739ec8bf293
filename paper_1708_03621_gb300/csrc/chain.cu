// The scatter -> inverse 3-D FFT -> x V(r) -> forward 3-D FFT -> gather chain
// of the Hamiltonian, and the operator entry points I, J, Idag, Jdag, O,
// apply_H and density (JDFTx paper, Sec. 2.1: I and J are Fourier transforms
// between reciprocal and real space; the pointwise multiply is the
// `epsilon * I(...)` of Listing 1; Sec. 2.1 also chains I -> multiply -> J on
// temporaries, which here becomes one plane pass with no box in memory).
//
// Organisation (per band, three kernels):
//   zpass_inverse  sphere coefficients of a group of (i0,i1) columns ->
//                  length-S2 inverse transforms -> column buffer
//   plane_*        one z-plane j2 per block: inverse along axis 1 for the rows
//                  the sphere touches, inverse along axis 0 for every j1,
//                  multiply by V (or accumulate |psi|^2), forward along axis
//                  0 keeping only those rows, forward along axis 1 keeping
//                  only the sphere's columns
//   zpass_forward  column buffer -> forward length-S2 transforms -> gather
//                  the sphere, add the kinetic term and scale by Omega
// Only the columns and rows the sphere touches are moved and transformed.
#include <algorithm>
#include <cstdlib>
#include <type_traits>

#include "chain.cuh"
#include "profile.cuh"
#include "gemm.cuh"

namespace jdft {

constexpr int kThreads = 256;

__device__ __forceinline__ int wrap(int i, int n) {
    int r = i % n;
    return r < 0 ? r + n : r;
}

template <typename T>
__device__ __forceinline__ void zero_fill(c_t<T>* p, int n) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) p[i] = mk<T>(T(0), T(0));
}

// ---------------------------------------------------------------------------
// z passes
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kThreads) zpass_inverse_kernel(ChainGeom g, const c_t<T>* __restrict__ C, int ldc,
                                                                 c_t<T>* __restrict__ colbuf, int cpb,
                                                                 const c_t<T>* __restrict__ tw) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int ls = g.S2 + 1;
    c_t<T>* buf0 = reinterpret_cast<c_t<T>*>(smem_raw);
    c_t<T>* buf1 = buf0 + cpb * ls;
    const int c0 = blockIdx.x * cpb;
    const int ncl = min(cpb, g.ncols - c0);
    const int b = blockIdx.y;
    zero_fill<T>(buf0, ncl * ls);
    __syncthreads();
    const int gA = g.col_start[c0], gB = g.col_start[c0 + ncl];
    const c_t<T>* Cb = C + (size_t)b * ldc;
    for (int q = gA + threadIdx.x; q < gB; q += blockDim.x) buf0[(g.pw_col[q] - c0) * ls + g.pw_z[q]] = Cb[q];
    __syncthreads();
    const c_t<T>* res = fft_lines<T, +1>(buf0, buf1, ncl, ls, g.p2, tw);
    for (int i = threadIdx.x; i < ncl * g.S2; i += blockDim.x) {
        const int j2 = i / ncl, cl = i - j2 * ncl;
        colbuf[colbuf_index(g, b, j2, c0 + cl)] = res[cl * ls + j2];
    }
}

template <typename T, int MODE>
__global__ void __launch_bounds__(kThreads) zpass_forward_kernel(ChainGeom g, const c_t<T>* __restrict__ colbuf,
                                                                 const c_t<T>* __restrict__ C, int ldc,
                                                                 c_t<T>* __restrict__ out, int ldo,
                                                                 const T* __restrict__ kin, T omega, T scale, int cpb,
                                                                 const c_t<T>* __restrict__ tw) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int ls = g.S2 + 1;
    c_t<T>* buf0 = reinterpret_cast<c_t<T>*>(smem_raw);
    c_t<T>* buf1 = buf0 + cpb * ls;
    const int c0 = blockIdx.x * cpb;
    const int ncl = min(cpb, g.ncols - c0);
    const int b = blockIdx.y;
    for (int i = threadIdx.x; i < ncl * g.S2; i += blockDim.x) {
        const int j2 = i / ncl, cl = i - j2 * ncl;
        buf0[cl * ls + j2] = colbuf[colbuf_index(g, b, j2, c0 + cl)];
    }
    __syncthreads();
    const c_t<T>* res = fft_lines<T, -1>(buf0, buf1, ncl, ls, g.p2, tw);
    const int gA = g.col_start[c0], gB = g.col_start[c0 + ncl];
    for (int q = gA + threadIdx.x; q < gB; q += blockDim.x) {
        c_t<T> y = res[(g.pw_col[q] - c0) * ls + g.pw_z[q]];
        c_t<T> r;
        if (MODE == 0) {
            c_t<T> c = C[(size_t)b * ldc + q];
            const T t = kin[q];
            r = mk<T>(omega * (t * c.x + scale * y.x), omega * (t * c.y + scale * y.y));
        } else {
            r = cscale(y, scale);
        }
        out[(size_t)b * ldo + q] = r;
    }
}

// ---------------------------------------------------------------------------
// Plane-pass stages.  Shared memory: A[nrows][S1 + 1] holds the plane after
// the axis-1 transforms of the sphere's rows; s0, s1 are G lines of
// max(S0, S1) + 1 each, the ping-pong pair of the transforms.
// ---------------------------------------------------------------------------
struct PlaneSmem {
    int lsA, lsS, G;
};

// Inverse along axis 1 of rows [0, nrows): disk values of this plane -> A.
// If jw > 0 only columns j1 in [ja, ja + jw) are kept, in A[r * lsA + j1 - ja].
template <typename T>
__device__ void rows_inverse(const ChainGeom& g, const c_t<T>* __restrict__ plane, c_t<T>* A, int lsA, c_t<T>* s0,
                             c_t<T>* s1, int lsS, int G, const c_t<T>* __restrict__ tw1, int ja, int jw) {
    for (int r0 = 0; r0 < g.nrows; r0 += G) {
        const int nl = min(G, g.nrows - r0);
        zero_fill<T>(s0, nl * lsS);
        __syncthreads();
        const int cA = g.row_col_start[r0], cB = g.row_col_start[r0 + nl];
        for (int c = cA + threadIdx.x; c < cB; c += blockDim.x) {
            const int sl = g.col_slot01[c];
            s0[((sl >> 16) - r0) * lsS + (sl & 0xffff)] = plane[c];
        }
        __syncthreads();
        const c_t<T>* res = fft_lines<T, +1>(s0, s1, nl, lsS, g.p1, tw1);
        const int w = jw > 0 ? jw : g.S1;
        for (int i = threadIdx.x; i < nl * w; i += blockDim.x) {
            const int l = i / w, t = i - l * w;
            A[(r0 + l) * lsA + t] = res[l * lsS + ja + t];
        }
        __syncthreads();
    }
}

// Forward along axis 1 of the rows in A, writing the disk values of this plane.
template <typename T>
__device__ void rows_forward(const ChainGeom& g, c_t<T>* __restrict__ plane, const c_t<T>* A, int lsA, c_t<T>* s0,
                             c_t<T>* s1, int lsS, int G, const c_t<T>* __restrict__ tw1) {
    for (int r0 = 0; r0 < g.nrows; r0 += G) {
        const int nl = min(G, g.nrows - r0);
        for (int i = threadIdx.x; i < nl * g.S1; i += blockDim.x) {
            const int l = i / g.S1, t = i - l * g.S1;
            s0[l * lsS + t] = A[(r0 + l) * lsA + t];
        }
        __syncthreads();
        const c_t<T>* res = fft_lines<T, -1>(s0, s1, nl, lsS, g.p1, tw1);
        const int cA = g.row_col_start[r0], cB = g.row_col_start[r0 + nl];
        for (int c = cA + threadIdx.x; c < cB; c += blockDim.x) {
            const int sl = g.col_slot01[c];
            plane[c] = res[((sl >> 16) - r0) * lsS + (sl & 0xffff)];
        }
        __syncthreads();
    }
}

// Place column values A[r][q0 + l] (r < nrows) at slot (i0min + r) mod S0 of
// line l, zeros elsewhere, and inverse-transform along axis 0.
template <typename T>
__device__ c_t<T>* column_inverse(const ChainGeom& g, const c_t<T>* A, int lsA, int q0, int nl, c_t<T>* s0,
                                  c_t<T>* s1, int lsS, const c_t<T>* __restrict__ tw0) {
    zero_fill<T>(s0, nl * lsS);
    __syncthreads();
    for (int i = threadIdx.x; i < nl * g.nrows; i += blockDim.x) {
        const int l = i / g.nrows, r = i - l * g.nrows;
        s0[l * lsS + wrap(g.i0min + r, g.S0)] = A[r * lsA + q0 + l];
    }
    __syncthreads();
    return fft_lines<T, +1>(s0, s1, nl, lsS, g.p0, tw0);
}

template <typename T>
__global__ void __launch_bounds__(kThreads) plane_apply_kernel(ChainGeom g, c_t<T>* __restrict__ colbuf,
                                                               const T* __restrict__ Vp, PlaneSmem sm,
                                                               const c_t<T>* __restrict__ tw0,
                                                               const c_t<T>* __restrict__ tw1) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    c_t<T>* A = reinterpret_cast<c_t<T>*>(smem_raw);
    c_t<T>* s0 = A + g.nrows * sm.lsA;
    c_t<T>* s1 = s0 + sm.G * sm.lsS;
    const int j2 = blockIdx.x, b = blockIdx.y;
    c_t<T>* plane = colbuf + colbuf_index(g, b, j2, 0);

    rows_inverse<T>(g, plane, A, sm.lsA, s0, s1, sm.lsS, sm.G, tw1, 0, 0);

    for (int q0 = 0; q0 < g.S1; q0 += sm.G) {
        const int nl = min(sm.G, g.S1 - q0);
        c_t<T>* res = column_inverse<T>(g, A, sm.lsA, q0, nl, s0, s1, sm.lsS, tw0);
        c_t<T>* other = (res == s0) ? s1 : s0;
        const T* Vq = Vp + ((size_t)j2 * g.S1 + q0) * g.S0;
        for (int i = threadIdx.x; i < nl * g.S0; i += blockDim.x) {
            const int l = i / g.S0, j0 = i - l * g.S0;
            res[l * sm.lsS + j0] = cscale(res[l * sm.lsS + j0], Vq[(size_t)l * g.S0 + j0]);
        }
        __syncthreads();
        const c_t<T>* out = fft_lines<T, -1>(res, other, nl, sm.lsS, g.p0, tw0);
        for (int i = threadIdx.x; i < nl * g.nrows; i += blockDim.x) {
            const int l = i / g.nrows, r = i - l * g.nrows;
            A[r * sm.lsA + q0 + l] = out[l * sm.lsS + wrap(g.i0min + r, g.S0)];
        }
        __syncthreads();
    }

    rows_forward<T>(g, plane, A, sm.lsA, s0, s1, sm.lsS, sm.G, tw1);
}

// Full-box inverse (operators I and Jdag): psi[b][(j0 S1 + j1) S2 + j2] = scale (I C)_j.
template <typename T>
__global__ void __launch_bounds__(kThreads) plane_inverse_full_kernel(ChainGeom g, const c_t<T>* __restrict__ colbuf,
                                                                      c_t<T>* __restrict__ psi, T scale, PlaneSmem sm,
                                                                      const c_t<T>* __restrict__ tw0,
                                                                      const c_t<T>* __restrict__ tw1) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    c_t<T>* A = reinterpret_cast<c_t<T>*>(smem_raw);
    c_t<T>* s0 = A + g.nrows * sm.lsA;
    c_t<T>* s1 = s0 + sm.G * sm.lsS;
    const int j2 = blockIdx.x, b = blockIdx.y;
    const c_t<T>* plane = colbuf + colbuf_index(g, b, j2, 0);
    rows_inverse<T>(g, plane, A, sm.lsA, s0, s1, sm.lsS, sm.G, tw1, 0, 0);
    const size_t N = (size_t)g.S0 * g.S1 * g.S2;
    c_t<T>* pb = psi + (size_t)b * N;
    for (int q0 = 0; q0 < g.S1; q0 += sm.G) {
        const int nl = min(sm.G, g.S1 - q0);
        const c_t<T>* res = column_inverse<T>(g, A, sm.lsA, q0, nl, s0, s1, sm.lsS, tw0);
        for (int i = threadIdx.x; i < nl * g.S0; i += blockDim.x) {
            const int j0 = i / nl, l = i - j0 * nl;
            pb[((size_t)j0 * g.S1 + q0 + l) * g.S2 + j2] = cscale(res[l * sm.lsS + j0], scale);
        }
        __syncthreads();
    }
}

// Full-box forward (operators J and Idag, before the z pass): box -> disk values of this plane.
template <typename T>
__global__ void __launch_bounds__(kThreads) plane_forward_full_kernel(ChainGeom g, const c_t<T>* __restrict__ psi,
                                                                      c_t<T>* __restrict__ colbuf, PlaneSmem sm,
                                                                      const c_t<T>* __restrict__ tw0,
                                                                      const c_t<T>* __restrict__ tw1) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    c_t<T>* A = reinterpret_cast<c_t<T>*>(smem_raw);
    c_t<T>* s0 = A + g.nrows * sm.lsA;
    c_t<T>* s1 = s0 + sm.G * sm.lsS;
    const int j2 = blockIdx.x, b = blockIdx.y;
    const size_t N = (size_t)g.S0 * g.S1 * g.S2;
    const c_t<T>* pb = psi + (size_t)b * N;
    for (int q0 = 0; q0 < g.S1; q0 += sm.G) {
        const int nl = min(sm.G, g.S1 - q0);
        for (int i = threadIdx.x; i < nl * g.S0; i += blockDim.x) {
            const int j0 = i / nl, l = i - j0 * nl;
            s0[l * sm.lsS + j0] = pb[((size_t)j0 * g.S1 + q0 + l) * g.S2 + j2];
        }
        __syncthreads();
        const c_t<T>* out = fft_lines<T, -1>(s0, s1, nl, sm.lsS, g.p0, tw0);
        for (int i = threadIdx.x; i < nl * g.nrows; i += blockDim.x) {
            const int l = i / g.nrows, r = i - l * g.nrows;
            A[r * sm.lsA + q0 + l] = out[l * sm.lsS + wrap(g.i0min + r, g.S0)];
        }
        __syncthreads();
    }
    rows_forward<T>(g, colbuf + colbuf_index(g, b, j2, 0), A, sm.lsA, s0, s1, sm.lsS, sm.G, tw1);
}

// Density: block (j2, j1-slab, band group) accumulates f_b |psi_b|^2 over its
// bands for j1 in [ja, ja + jw) in FP64 shared memory, then adds w times that
// to n_r (atomically when several band groups share a point).
template <typename T>
__global__ void __launch_bounds__(kThreads) plane_density_kernel(ChainGeom g, const c_t<T>* __restrict__ colbuf,
                                                                 int nb, int bands_per_block, int jw,
                                                                 const double* __restrict__ f, double w,
                                                                 double* __restrict__ n_r, PlaneSmem sm,
                                                                 const c_t<T>* __restrict__ tw0,
                                                                 const c_t<T>* __restrict__ tw1) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double* acc = reinterpret_cast<double*>(smem_raw);                      // [jw][S0]
    c_t<T>* A = reinterpret_cast<c_t<T>*>(acc + (((size_t)jw * g.S0 + 1) & ~(size_t)1));  // [nrows][jw + 1]
    c_t<T>* s0 = A + g.nrows * sm.lsA;
    c_t<T>* s1 = s0 + sm.G * sm.lsS;
    const int j2 = blockIdx.x;
    const int ja = blockIdx.y * jw;
    const int jwe = min(jw, g.S1 - ja);
    const int bA = blockIdx.z * bands_per_block, bB = min(nb, bA + bands_per_block);
    for (int i = threadIdx.x; i < jw * g.S0; i += blockDim.x) acc[i] = 0.0;
    __syncthreads();
    for (int b = bA; b < bB; ++b) {
        const double fb = f[b];
        rows_inverse<T>(g, colbuf + colbuf_index(g, b, j2, 0), A, sm.lsA, s0, s1, sm.lsS, sm.G, tw1, ja, jwe);
        for (int q0 = 0; q0 < jwe; q0 += sm.G) {
            const int nl = min(sm.G, jwe - q0);
            const c_t<T>* res = column_inverse<T>(g, A, sm.lsA, q0, nl, s0, s1, sm.lsS, tw0);
            for (int i = threadIdx.x; i < nl * g.S0; i += blockDim.x) {
                const int l = i / g.S0, j0 = i - l * g.S0;
                const c_t<T> z = res[l * sm.lsS + j0];
                acc[(q0 + l) * g.S0 + j0] += fb * ((double)z.x * (double)z.x + (double)z.y * (double)z.y);
            }
            __syncthreads();
        }
    }
    const bool atomic = gridDim.z > 1;
    for (int i = threadIdx.x; i < jwe * g.S0; i += blockDim.x) {
        const int j0 = i / jwe, l = i - j0 * jwe;
        double* dst = n_r + ((size_t)j0 * g.S1 + ja + l) * g.S2 + j2;
        const double v = w * acc[l * g.S0 + j0];
        if (atomic) atomicAdd(dst, v);
        else *dst += v;
    }
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
constexpr size_t kMaxSmem = 220 * 1024;

template <typename K>
static jdft_status prepare(K kernel, size_t smem, const char* name) {
    if (smem > kMaxSmem) return set_error(JDFT_ERR_UNSUPPORTED, std::string(name) + ": box too large for shared memory");
    cudaError_t e = set_smem_attr((const void*)kernel, smem);
    if (e != cudaSuccess) return set_error(JDFT_ERR_CUDA, std::string(name) + ": " + cudaGetErrorString(e));
    return JDFT_OK;
}

static int zpass_cpb(int S2, size_t elem) {
    int cpb = 16;
    while (cpb > 1 && 2 * (size_t)cpb * (S2 + 1) * elem > 96 * 1024) cpb /= 2;
    return cpb;
}

static PlaneSmem plane_layout(const ChainGeom& g, size_t elem, int lsA_width, size_t extra, int Gmax) {
    PlaneSmem sm;
    sm.lsA = lsA_width + 1;
    sm.lsS = std::max(g.S0, g.S1) + 1;
    sm.G = Gmax;
    while (sm.G > 1 && extra + ((size_t)g.nrows * sm.lsA + 2 * (size_t)sm.G * sm.lsS) * elem > kMaxSmem) sm.G /= 2;
    return sm;
}

static size_t plane_bytes(const ChainGeom& g, const PlaneSmem& sm, size_t elem) {
    return ((size_t)g.nrows * sm.lsA + 2 * (size_t)sm.G * sm.lsS) * elem;
}

template <typename T>
jdft_status launch_zpass_inverse(const ChainGeom& g, const c_t<T>* C, int ldc, c_t<T>* colbuf, int nb,
                                 const c_t<T>* tw_base, cudaStream_t st) {
    {
        // register-FFT kernel for the lengths it is compiled for, else the generic one
        const jdft_status fs = launch_zpass_inverse_fast<T>(g, C, ldc, colbuf, nb, tw_base + g.p2.tw_offset, st);
        if (fs != JDFT_ERR_UNSUPPORTED) return fs;
    }
    const int cpb = zpass_cpb(g.S2, sizeof(c_t<T>));
    const size_t smem = 2 * (size_t)cpb * (g.S2 + 1) * sizeof(c_t<T>);
    jdft_status s = prepare(zpass_inverse_kernel<T>, smem, "zpass_inverse");
    if (s != JDFT_OK) return s;
    dim3 grid((g.ncols + cpb - 1) / cpb, nb);
    {
        Trace tr_("zpass_inverse", st);
        zpass_inverse_kernel<T><<<grid, kThreads, smem, st>>>(g, C, ldc, colbuf, cpb, tw_base + g.p2.tw_offset);
    }
    return check_launch("zpass_inverse");
}

template <typename T, int MODE>
jdft_status launch_zpass_forward(const ChainGeom& g, const c_t<T>* colbuf, const c_t<T>* C, int ldc, c_t<T>* out,
                                 int ldo, int nb, const T* kin, T omega, T scale, const c_t<T>* tw_base,
                                 cudaStream_t st) {
    {
        const jdft_status fs = launch_zpass_forward_fast<T, MODE>(g, colbuf, C, ldc, out, ldo, nb, kin, omega, scale,
                                                                  tw_base + g.p2.tw_offset, st);
        if (fs != JDFT_ERR_UNSUPPORTED) return fs;
    }
    const int cpb = zpass_cpb(g.S2, sizeof(c_t<T>));
    const size_t smem = 2 * (size_t)cpb * (g.S2 + 1) * sizeof(c_t<T>);
    jdft_status s = prepare(zpass_forward_kernel<T, MODE>, smem, "zpass_forward");
    if (s != JDFT_OK) return s;
    dim3 grid((g.ncols + cpb - 1) / cpb, nb);
    {
        Trace tr_("zpass_forward", st);
        zpass_forward_kernel<T, MODE><<<grid, kThreads, smem, st>>>(g, colbuf, C, ldc, out, ldo, kin, omega, scale, cpb,
                                                                    tw_base + g.p2.tw_offset);
    }
    return check_launch("zpass_forward");
}

template <typename T>
jdft_status launch_plane_apply(const ChainGeom& g, c_t<T>* colbuf, const T* Vp, int nb, const c_t<T>* tw_base,
                               cudaStream_t st) {
    // band-pair or register-FFT kernel for the shapes they are compiled for, else the generic one
    jdft_status fs = JDFT_ERR_UNSUPPORTED;
    if constexpr (std::is_same<T, float>::value) fs = launch_plane_apply_pair(g, colbuf, Vp, nb, tw_base, st);
    if (fs == JDFT_ERR_UNSUPPORTED) fs = launch_plane_apply_fast<T>(g, colbuf, Vp, nb, tw_base, st);
    if (fs != JDFT_ERR_UNSUPPORTED) return fs;
    PlaneSmem sm = plane_layout(g, sizeof(c_t<T>), g.S1, 0, 16);
    const size_t smem = plane_bytes(g, sm, sizeof(c_t<T>));
    jdft_status s = prepare(plane_apply_kernel<T>, smem, "plane_apply");
    if (s != JDFT_OK) return s;
    dim3 grid(g.S2, nb);
    {
        Trace tr_("plane_apply", st);
        plane_apply_kernel<T><<<grid, kThreads, smem, st>>>(g, colbuf, Vp, sm, tw_base + g.p0.tw_offset,
                                                            tw_base + g.p1.tw_offset);
    }
    return check_launch("plane_apply");
}

template <typename T>
jdft_status launch_plane_inverse_full(const ChainGeom& g, const c_t<T>* colbuf, c_t<T>* psi, T scale, int nb,
                                      const c_t<T>* tw_base, cudaStream_t st) {
    PlaneSmem sm = plane_layout(g, sizeof(c_t<T>), g.S1, 0, 16);
    const size_t smem = plane_bytes(g, sm, sizeof(c_t<T>));
    jdft_status s = prepare(plane_inverse_full_kernel<T>, smem, "plane_inverse_full");
    if (s != JDFT_OK) return s;
    dim3 grid(g.S2, nb);
    {
        Trace tr_("plane_inverse_full", st);
        plane_inverse_full_kernel<T><<<grid, kThreads, smem, st>>>(g, colbuf, psi, scale, sm, tw_base + g.p0.tw_offset,
                                                                   tw_base + g.p1.tw_offset);
    }
    return check_launch("plane_inverse_full");
}

template <typename T>
jdft_status launch_plane_forward_full(const ChainGeom& g, const c_t<T>* psi, c_t<T>* colbuf, int nb,
                                      const c_t<T>* tw_base, cudaStream_t st) {
    PlaneSmem sm = plane_layout(g, sizeof(c_t<T>), g.S1, 0, 16);
    const size_t smem = plane_bytes(g, sm, sizeof(c_t<T>));
    jdft_status s = prepare(plane_forward_full_kernel<T>, smem, "plane_forward_full");
    if (s != JDFT_OK) return s;
    dim3 grid(g.S2, nb);
    {
        Trace tr_("plane_forward_full", st);
        plane_forward_full_kernel<T><<<grid, kThreads, smem, st>>>(g, psi, colbuf, sm, tw_base + g.p0.tw_offset,
                                                                   tw_base + g.p1.tw_offset);
    }
    return check_launch("plane_forward_full");
}

template <typename T>
jdft_status launch_plane_density(const ChainGeom& g, const c_t<T>* colbuf, const double* f, double w, double* n_r,
                                 int nb, const c_t<T>* tw_base, cudaStream_t st) {
    if constexpr (std::is_same<T, float>::value) {
        const jdft_status fs = launch_plane_density_fast(g, colbuf, f, w, n_r, nb, tw_base, st);
        if (fs != JDFT_ERR_UNSUPPORTED) return fs;
    }
    // Split j1 into slabs until accumulator + plane buffers fit.
    int nsplit = 1, jw = g.S1;
    PlaneSmem sm;
    size_t smem = 0;
    for (;;) {
        jw = (g.S1 + nsplit - 1) / nsplit;
        const size_t acc = (((size_t)jw * g.S0 + 1) & ~(size_t)1) * sizeof(double);
        sm = plane_layout(g, sizeof(c_t<T>), jw, acc, 8);
        smem = acc + plane_bytes(g, sm, sizeof(c_t<T>));
        if (smem <= kMaxSmem || jw == 1) break;
        ++nsplit;
    }
    nsplit = (g.S1 + jw - 1) / jw;
    jdft_status s = prepare(plane_density_kernel<T>, smem, "plane_density");
    if (s != JDFT_OK) return s;
    // Band groups so the grid covers the GPU about twice.
    const int planes = g.S2 * nsplit;
    int groups = std::max(1, std::min(nb, (2 * 152 + planes - 1) / planes));
    const int per = (nb + groups - 1) / groups;
    groups = (nb + per - 1) / per;
    dim3 grid(g.S2, nsplit, groups);
    {
        Trace tr_("plane_density", st);
        plane_density_kernel<T><<<grid, kThreads, smem, st>>>(g, colbuf, nb, per, jw, f, w, n_r, sm,
                                                              tw_base + g.p0.tw_offset, tw_base + g.p1.tw_offset);
    }
    return check_launch("plane_density");
}

#define JDFT_INSTANTIATE(T)                                                                                        \
    template jdft_status launch_zpass_inverse<T>(const ChainGeom&, const c_t<T>*, int, c_t<T>*, int, const c_t<T>*, \
                                                 cudaStream_t);                                                    \
    template jdft_status launch_zpass_forward<T, 0>(const ChainGeom&, const c_t<T>*, const c_t<T>*, int, c_t<T>*,   \
                                                    int, int, const T*, T, T, const c_t<T>*, cudaStream_t);         \
    template jdft_status launch_zpass_forward<T, 1>(const ChainGeom&, const c_t<T>*, const c_t<T>*, int, c_t<T>*,   \
                                                    int, int, const T*, T, T, const c_t<T>*, cudaStream_t);         \
    template jdft_status launch_plane_apply<T>(const ChainGeom&, c_t<T>*, const T*, int, const c_t<T>*,             \
                                               cudaStream_t);                                                      \
    template jdft_status launch_plane_inverse_full<T>(const ChainGeom&, const c_t<T>*, c_t<T>*, T, int,              \
                                                      const c_t<T>*, cudaStream_t);                                \
    template jdft_status launch_plane_forward_full<T>(const ChainGeom&, const c_t<T>*, c_t<T>*, int, const c_t<T>*, \
                                                      cudaStream_t);                                               \
    template jdft_status launch_plane_density<T>(const ChainGeom&, const c_t<T>*, const double*, double, double*,   \
                                                 int, const c_t<T>*, cudaStream_t);
JDFT_INSTANTIATE(double)
JDFT_INSTANTIATE(float)

// ---------------------------------------------------------------------------
// Entry-point helpers
// ---------------------------------------------------------------------------
static bool is_fp64(jdft_prec p) { return p == JDFT_FP64; }

static jdft_status check_prec(jdft_prec p) {
    if (p == JDFT_FP64 || p == JDFT_FP32 || p == JDFT_TF32X3 || p == JDFT_BF16X3) return JDFT_OK;
    return set_error(JDFT_ERR_ARG, "unknown precision");
}

static jdft_status check_common(const jdft_basis_s* b, int ik, int nb) {
    JDFT_CHECK_ARG(b, "null basis");
    JDFT_CHECK_ARG(ik >= 0 && ik < b->nk, "k-point index out of range");
    JDFT_CHECK_ARG(nb >= 0, "nb must be >= 0");
    return JDFT_OK;
}

static jdft_status check_block(const void* p, int ld, int npw, int nb, jdft_prec prec, const char* name) {
    if (nb == 0) return JDFT_OK;
    if (!p) return set_error(JDFT_ERR_ARG, std::string(name) + " is null");
    if (ld < npw) return set_error(JDFT_ERR_ARG, std::string(name) + ": leading dimension < npw");
    const uintptr_t align = is_fp64(prec) ? 16 : 8;
    if (((uintptr_t)p) % align) return set_error(JDFT_ERR_ARG, std::string(name) + " is not aligned to its complex type");
    return JDFT_OK;
}

// Bands per chunk so one chunk's column buffer stays near `budget` bytes.
static int chunk_bands(const ChainGeom& g, size_t elem, int nb, size_t budget) {
    const size_t per = (size_t)g.S2 * g.ncols * elem;
    int c = (int)std::max<size_t>(1, budget / per);
    return std::max(1, std::min(nb, c));
}

// Column-buffer bytes per chunk of bands.  The environment variable
// JDFT_CHUNK_MB overrides it (read on every call), then a value the
// autotuner stored in the basis, then 256 MB: measured on the 128^3,
// 256-band block, two chunks of 131 bands beat eight L2-sized ones (64 MB),
// since fewer, larger launches balance the persistent plane kernel better than
// L2 residency of the column buffer saves.
size_t chunk_budget(const jdft_basis_s* b) {
    const char* e = getenv("JDFT_CHUNK_MB");
    long long mb = e ? atoll(e) : 0;
    if (mb <= 0 && b) mb = b->chunk_mb;
    return (size_t)(mb > 0 ? mb : 256) << 20;
}

template <typename T>
static const c_t<T>* twiddles(const jdft_basis_s* b);
template <> const double2* twiddles<double>(const jdft_basis_s* b) { return b->tw64; }
template <> const float2* twiddles<float>(const jdft_basis_s* b) { return b->tw32; }

template <typename T>
static const T* potential(const jdft_basis_s* b);
template <> const double* potential<double>(const jdft_basis_s* b) { return b->V; }
template <> const float* potential<float>(const jdft_basis_s* b) { return b->V32; }

template <typename T>
static const T* kinetic(const KSphere& s);
template <> const double* kinetic<double>(const KSphere& s) { return s.kin; }
template <> const float* kinetic<float>(const KSphere& s) { return s.kin32; }

// psi = scale * I C
template <typename T>
static jdft_status run_inverse_full(jdft_basis_s* b, int ik, const void* C, int ldc, void* psi, int nb, T scale,
                                    cudaStream_t st) {
    const ChainGeom g = make_geom(b, ik);
    const int nc = chunk_bands(g, sizeof(c_t<T>), nb, chunk_budget(b));
    jdft_status s = ensure_workspace(b, (size_t)nc * g.S2 * g.ncols * sizeof(c_t<T>));
    if (s != JDFT_OK) return s;
    c_t<T>* colbuf = (c_t<T>*)b->work.ptr;
    for (int b0 = 0; b0 < nb; b0 += nc) {
        const int n = std::min(nc, nb - b0);
        if ((s = launch_zpass_inverse<T>(g, (const c_t<T>*)C + (size_t)b0 * ldc, ldc, colbuf, n, twiddles<T>(b), st)))
            return s;
        if ((s = launch_plane_inverse_full<T>(g, colbuf, (c_t<T>*)psi + (size_t)b0 * b->N, scale, n, twiddles<T>(b),
                                              st)))
            return s;
    }
    return JDFT_OK;
}

// C = scale * (forward transform of psi restricted to the sphere)
template <typename T>
static jdft_status run_forward_full(jdft_basis_s* b, int ik, const void* psi, void* C, int ldc, int nb, T scale,
                                    cudaStream_t st) {
    const ChainGeom g = make_geom(b, ik);
    const int nc = chunk_bands(g, sizeof(c_t<T>), nb, chunk_budget(b));
    jdft_status s = ensure_workspace(b, (size_t)nc * g.S2 * g.ncols * sizeof(c_t<T>));
    if (s != JDFT_OK) return s;
    c_t<T>* colbuf = (c_t<T>*)b->work.ptr;
    for (int b0 = 0; b0 < nb; b0 += nc) {
        const int n = std::min(nc, nb - b0);
        if ((s = launch_plane_forward_full<T>(g, (const c_t<T>*)psi + (size_t)b0 * b->N, colbuf, n, twiddles<T>(b),
                                              st)))
            return s;
        if ((s = launch_zpass_forward<T, 1>(g, colbuf, nullptr, 0, (c_t<T>*)C + (size_t)b0 * ldc, ldc, n, nullptr,
                                            T(0), scale, twiddles<T>(b), st)))
            return s;
    }
    return JDFT_OK;
}

template <typename T>
static jdft_status run_apply_H(jdft_basis_s* b, int ik, const void* C, int ldc, void* HC, int ldhc, int nb,
                               jdft_prec prec, cudaStream_t st) {
    const ChainGeom g = make_geom(b, ik);
    const KSphere& sp = b->ks[ik];
    const int nc = chunk_bands(g, sizeof(c_t<T>), nb, chunk_budget(b));
    const size_t colbytes = ((size_t)nc * g.S2 * g.ncols * sizeof(c_t<T>) + 255) / 256 * 256;
    const size_t nlbytes = nonlocal_workspace_bytes(sp.nproj, nb, sizeof(c_t<T>), sp.npw, prec, true, true);
    jdft_status s = ensure_workspace(b, colbytes + nlbytes);
    if (s != JDFT_OK) return s;
    c_t<T>* colbuf = (c_t<T>*)b->work.ptr;
    const T omega = (T)b->omega, invN = (T)(1.0 / (double)b->N);
    for (int b0 = 0; b0 < nb; b0 += nc) {
        const int n = std::min(nc, nb - b0);
        const c_t<T>* Cc = (const c_t<T>*)C + (size_t)b0 * ldc;
        c_t<T>* Hc = (c_t<T>*)HC + (size_t)b0 * ldhc;
        if ((s = launch_zpass_inverse<T>(g, Cc, ldc, colbuf, n, twiddles<T>(b), st))) return s;
        if ((s = launch_plane_apply<T>(g, colbuf, potential<T>(b), n, twiddles<T>(b), st))) return s;
        if ((s = launch_zpass_forward<T, 0>(g, colbuf, Cc, ldc, Hc, ldhc, n, kinetic<T>(sp), omega, invN,
                                            twiddles<T>(b), st)))
            return s;
    }
    if (sp.nproj > 0)
        return nonlocal_accumulate<T>(sp, C, ldc, HC, ldhc, nb, prec, (char*)b->work.ptr + colbytes, st, true, nullptr,
                                      true);
    return JDFT_OK;
}

// H C and the density of the same block: per chunk one z pass in, then the
// fused plane kernel where it exists (else density, then the H plane pass, on
// the same column buffer), one z pass out; the nonlocal term after.
template <typename T>
static size_t apply_H_density_bytes(const jdft_basis_s* b, int ik, int nb, jdft_prec prec, bool split_c) {
    const ChainGeom g = make_geom(b, ik);
    const KSphere& sp = b->ks[ik];
    const int nc = chunk_bands(g, sizeof(c_t<T>), nb, chunk_budget(b));
    const size_t colbytes = ((size_t)nc * g.S2 * g.ncols * sizeof(c_t<T>) + 255) / 256 * 256;
    return colbytes + nonlocal_workspace_bytes(sp.nproj, nb, sizeof(c_t<T>), sp.npw, prec, split_c, true);
}

// Csplit: the BF16 planes of C (tcx_split) when the caller has them, so the
// projection reads them instead of splitting C again.
template <typename T>
static jdft_status run_apply_H_density(jdft_basis_s* b, int ik, const void* C, int ldc, void* HC, int ldhc, int nb,
                                       const double* f, double* n_r, jdft_prec prec, cudaStream_t st,
                                       const void* Csplit = nullptr) {
    const ChainGeom g = make_geom(b, ik);
    const KSphere& sp = b->ks[ik];
    const int nc = chunk_bands(g, sizeof(c_t<T>), nb, chunk_budget(b));
    const size_t colbytes = ((size_t)nc * g.S2 * g.ncols * sizeof(c_t<T>) + 255) / 256 * 256;
    const size_t nlbytes = nonlocal_workspace_bytes(sp.nproj, nb, sizeof(c_t<T>), sp.npw, prec, !Csplit, true);
    jdft_status s = ensure_workspace(b, colbytes + nlbytes);
    if (s != JDFT_OK) return s;
    c_t<T>* colbuf = (c_t<T>*)b->work.ptr;
    const T omega = (T)b->omega, invN = (T)(1.0 / (double)b->N);
    const double wk = b->kweight[ik];
    for (int b0 = 0; b0 < nb; b0 += nc) {
        const int n = std::min(nc, nb - b0);
        const c_t<T>* Cc = (const c_t<T>*)C + (size_t)b0 * ldc;
        c_t<T>* Hc = (c_t<T>*)HC + (size_t)b0 * ldhc;
        if ((s = launch_zpass_inverse<T>(g, Cc, ldc, colbuf, n, twiddles<T>(b), st))) return s;
        jdft_status fs = JDFT_ERR_UNSUPPORTED;
        if constexpr (std::is_same<T, float>::value) {
            fs = launch_plane_apply_density_pair(g, colbuf, potential<float>(b), n, f + b0, wk, n_r, twiddles<float>(b),
                                                 st);
            if (fs == JDFT_ERR_UNSUPPORTED)
                fs = launch_plane_apply_density_fast(g, colbuf, potential<float>(b), n, f + b0, wk, n_r,
                                                     twiddles<float>(b), st);
        }
        if (fs == JDFT_ERR_UNSUPPORTED) {
            if ((s = launch_plane_density<T>(g, colbuf, f + b0, wk, n_r, n, twiddles<T>(b), st))) return s;
            if ((s = launch_plane_apply<T>(g, colbuf, potential<T>(b), n, twiddles<T>(b), st))) return s;
        } else if (fs != JDFT_OK) {
            return fs;
        }
        if ((s = launch_zpass_forward<T, 0>(g, colbuf, Cc, ldc, Hc, ldhc, n, kinetic<T>(sp), omega, invN,
                                            twiddles<T>(b), st)))
            return s;
    }
    if (sp.nproj > 0)
        return nonlocal_accumulate<T>(sp, C, ldc, HC, ldhc, nb, prec, (char*)b->work.ptr + colbytes, st, !Csplit,
                                      Csplit, true);
    return JDFT_OK;
}

size_t apply_H_density_workspace(const jdft_basis_s* b, int ik, int nb, jdft_prec prec, bool split_c) {
    return is_fp64(prec) ? apply_H_density_bytes<double>(b, ik, nb, prec, split_c)
                         : apply_H_density_bytes<float>(b, ik, nb, prec, split_c);
}

jdft_status apply_H_density_with_split(jdft_basis_s* b, int ik, const void* C, int ldc, void* HC, int ldhc, int nb,
                                       const double* f, double* n_r, jdft_prec prec, cudaStream_t st,
                                       const void* Csplit) {
    return is_fp64(prec) ? run_apply_H_density<double>(b, ik, C, ldc, HC, ldhc, nb, f, n_r, prec, st, Csplit)
                         : run_apply_H_density<float>(b, ik, C, ldc, HC, ldhc, nb, f, n_r, prec, st, Csplit);
}

template <typename T>
static jdft_status run_density(jdft_basis_s* b, int ik, const void* C, int ldc, const double* f, int nb,
                               double* n_r, cudaStream_t st) {
    const ChainGeom g = make_geom(b, ik);
    const int nc = chunk_bands(g, sizeof(c_t<T>), nb, chunk_budget(b));
    jdft_status s = ensure_workspace(b, (size_t)nc * g.S2 * g.ncols * sizeof(c_t<T>));
    if (s != JDFT_OK) return s;
    c_t<T>* colbuf = (c_t<T>*)b->work.ptr;
    for (int b0 = 0; b0 < nb; b0 += nc) {
        const int n = std::min(nc, nb - b0);
        if ((s = launch_zpass_inverse<T>(g, (const c_t<T>*)C + (size_t)b0 * ldc, ldc, colbuf, n, twiddles<T>(b), st)))
            return s;
        if ((s = launch_plane_density<T>(g, colbuf, f + b0, b->kweight[ik], n_r, n, twiddles<T>(b), st))) return s;
    }
    return JDFT_OK;
}

template <typename T>
__global__ void scale_block_kernel(const c_t<T>* __restrict__ C, int ldc, c_t<T>* __restrict__ out, int ldo, int npw,
                                   int nb, T s) {
    const int64_t total = (int64_t)npw * nb;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t bb = i / npw, q = i - bb * npw;
        out[bb * ldo + q] = cscale(C[bb * ldc + q], s);
    }
}

}  // namespace jdft

using namespace jdft;

#define JDFT_DISPATCH(prec, CALL_D, CALL_F) (is_fp64(prec) ? (CALL_D) : (CALL_F))

extern "C" {

jdft_status jdft_op_I(jdft_basis_t b, int ik, const void* C, int ldc, void* psi, int nb, jdft_prec prec,
                      void* stream) {
    clear_error();
    jdft_status s;
    if ((s = check_common(b, ik, nb)) || (s = check_prec(prec))) return s;
    if ((s = check_block(C, ldc, b->ks[ik].npw, nb, prec, "C"))) return s;
    JDFT_CHECK_ARG(nb == 0 || psi, "psi is null");
    if (nb == 0) return JDFT_OK;
    cudaStream_t st = (cudaStream_t)stream;
    return JDFT_DISPATCH(prec, run_inverse_full<double>(b, ik, C, ldc, psi, nb, 1.0, st),
                         run_inverse_full<float>(b, ik, C, ldc, psi, nb, 1.0f, st));
}

jdft_status jdft_op_Jdag(jdft_basis_t b, int ik, const void* C, int ldc, void* psi, int nb, jdft_prec prec,
                         void* stream) {
    clear_error();
    jdft_status s;
    if ((s = check_common(b, ik, nb)) || (s = check_prec(prec))) return s;
    if ((s = check_block(C, ldc, b->ks[ik].npw, nb, prec, "C"))) return s;
    JDFT_CHECK_ARG(nb == 0 || psi, "psi is null");
    if (nb == 0) return JDFT_OK;
    cudaStream_t st = (cudaStream_t)stream;
    const double inv = 1.0 / (double)b->N;
    return JDFT_DISPATCH(prec, run_inverse_full<double>(b, ik, C, ldc, psi, nb, inv, st),
                         run_inverse_full<float>(b, ik, C, ldc, psi, nb, (float)inv, st));
}

jdft_status jdft_op_J(jdft_basis_t b, int ik, const void* psi, void* C, int ldc, int nb, jdft_prec prec,
                      void* stream) {
    clear_error();
    jdft_status s;
    if ((s = check_common(b, ik, nb)) || (s = check_prec(prec))) return s;
    if ((s = check_block(C, ldc, b->ks[ik].npw, nb, prec, "C"))) return s;
    JDFT_CHECK_ARG(nb == 0 || psi, "psi is null");
    if (nb == 0) return JDFT_OK;
    cudaStream_t st = (cudaStream_t)stream;
    const double inv = 1.0 / (double)b->N;
    return JDFT_DISPATCH(prec, run_forward_full<double>(b, ik, psi, C, ldc, nb, inv, st),
                         run_forward_full<float>(b, ik, psi, C, ldc, nb, (float)inv, st));
}

jdft_status jdft_op_Idag(jdft_basis_t b, int ik, const void* psi, void* C, int ldc, int nb, jdft_prec prec,
                         void* stream) {
    clear_error();
    jdft_status s;
    if ((s = check_common(b, ik, nb)) || (s = check_prec(prec))) return s;
    if ((s = check_block(C, ldc, b->ks[ik].npw, nb, prec, "C"))) return s;
    JDFT_CHECK_ARG(nb == 0 || psi, "psi is null");
    if (nb == 0) return JDFT_OK;
    cudaStream_t st = (cudaStream_t)stream;
    return JDFT_DISPATCH(prec, run_forward_full<double>(b, ik, psi, C, ldc, nb, 1.0, st),
                         run_forward_full<float>(b, ik, psi, C, ldc, nb, 1.0f, st));
}

jdft_status jdft_op_O(jdft_basis_t b, int ik, const void* C, int ldc, void* OC, int ldoc, int nb, jdft_prec prec,
                      void* stream) {
    clear_error();
    jdft_status s;
    if ((s = check_common(b, ik, nb)) || (s = check_prec(prec))) return s;
    const int npw = b->ks[ik].npw;
    if ((s = check_block(C, ldc, npw, nb, prec, "C")) || (s = check_block(OC, ldoc, npw, nb, prec, "OC"))) return s;
    if (nb == 0) return JDFT_OK;
    cudaStream_t st = (cudaStream_t)stream;
    const int grid = 152 * 8;
    if (is_fp64(prec))
        {
            Trace tr_("scale_block", st);
            scale_block_kernel<double><<<grid, 256, 0, st>>>((const double2*)C, ldc, (double2*)OC, ldoc, npw, nb, b->omega);
        }
    else
        {
            Trace tr_("scale_block", st);
            scale_block_kernel<float><<<grid, 256, 0, st>>>((const float2*)C, ldc, (float2*)OC, ldoc, npw, nb,
                                                             (float)b->omega);
        }
    return check_launch("scale_block");
}

jdft_status jdft_apply_H(jdft_basis_t b, int ik, const void* C, int ldc, void* HC, int ldhc, int nb, jdft_prec prec,
                         void* stream) {
    clear_error();
    jdft_status s;
    if ((s = check_common(b, ik, nb)) || (s = check_prec(prec))) return s;
    const int npw = b->ks[ik].npw;
    if ((s = check_block(C, ldc, npw, nb, prec, "C")) || (s = check_block(HC, ldhc, npw, nb, prec, "HC"))) return s;
    if (!b->have_V) return set_error(JDFT_ERR_ARG, "no potential set (call jdft_set_potential first)");
    if (nb == 0) return JDFT_OK;
    cudaStream_t st = (cudaStream_t)stream;
    return JDFT_DISPATCH(prec, run_apply_H<double>(b, ik, C, ldc, HC, ldhc, nb, prec, st),
                         run_apply_H<float>(b, ik, C, ldc, HC, ldhc, nb, prec, st));
}

jdft_status jdft_apply_H_density(jdft_basis_t b, int ik, const void* C, int ldc, void* HC, int ldhc, int nb,
                                 const double* f, double* n_r, jdft_prec prec, void* stream) {
    clear_error();
    jdft_status s;
    if ((s = check_common(b, ik, nb)) || (s = check_prec(prec))) return s;
    const int npw = b->ks[ik].npw;
    if ((s = check_block(C, ldc, npw, nb, prec, "C")) || (s = check_block(HC, ldhc, npw, nb, prec, "HC"))) return s;
    JDFT_CHECK_ARG(nb == 0 || (f && n_r), "f or n_r is null");
    if (!b->have_V) return set_error(JDFT_ERR_ARG, "no potential set (call jdft_set_potential first)");
    if (nb == 0) return JDFT_OK;
    cudaStream_t st = (cudaStream_t)stream;
    return JDFT_DISPATCH(prec, run_apply_H_density<double>(b, ik, C, ldc, HC, ldhc, nb, f, n_r, prec, st),
                         run_apply_H_density<float>(b, ik, C, ldc, HC, ldhc, nb, f, n_r, prec, st));
}

jdft_status jdft_density(jdft_basis_t b, int ik, const void* C, int ldc, const double* f, int nb, double* n_r,
                         jdft_prec prec, void* stream) {
    clear_error();
    jdft_status s;
    if ((s = check_common(b, ik, nb)) || (s = check_prec(prec))) return s;
    if ((s = check_block(C, ldc, b->ks[ik].npw, nb, prec, "C"))) return s;
    JDFT_CHECK_ARG(nb == 0 || (f && n_r), "f or n_r is null");
    if (nb == 0) return JDFT_OK;
    cudaStream_t st = (cudaStream_t)stream;
    return JDFT_DISPATCH(prec, run_density<double>(b, ik, C, ldc, f, nb, n_r, st),
                         run_density<float>(b, ik, C, ldc, f, nb, n_r, st));
}

}  // extern "C"

extern "C" jdft_status jdft_autotune_chunk(jdft_basis_t b, int ik, const void* C, int ldc, void* HC, int ldhc, int nb,
                                           jdft_prec prec, int* chunk_mb, void* stream) {
    clear_error();
    JDFT_CHECK_ARG(b && C && HC && nb >= 1, "bad arguments");
    JDFT_CHECK_ARG(ik >= 0 && ik < b->nk, "k-point index out of range");
    if (!b->have_V) return set_error(JDFT_ERR_ARG, "no potential set");
    cudaStream_t st = (cudaStream_t)stream;
    const int cand[] = {32, 64, 128, 256, 512, 1024};
    cudaEvent_t e0, e1;
    JDFT_CUDA_TRY(cudaEventCreate(&e0));
    JDFT_CUDA_TRY(cudaEventCreate(&e1));
    float best = 1e30f;
    int best_mb = 64;
    const int saved = b->chunk_mb;
    jdft_status s = JDFT_OK;
    for (int mb : cand) {
        b->chunk_mb = mb;
        // one untimed call grows the workspace and warms the kernels, then two timed calls
        if ((s = jdft_apply_H(b, ik, C, ldc, HC, ldhc, nb, prec, stream))) break;
        cudaEventRecord(e0, st);
        for (int r = 0; r < 2 && s == JDFT_OK; ++r) s = jdft_apply_H(b, ik, C, ldc, HC, ldhc, nb, prec, stream);
        cudaEventRecord(e1, st);
        if (s) break;
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) { best = ms; best_mb = mb; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (s != JDFT_OK) { b->chunk_mb = saved; return s; }
    b->chunk_mb = best_mb;
    if (chunk_mb) *chunk_mb = best_mb;
    return JDFT_OK;
}

extern "C" jdft_status jdft_autotune(jdft_basis_t b, int ik, const void* C, int ldc, void* HC, int ldhc, int nb,
                                     jdft_prec prec, jdft_tune_report* report, void* stream) {
    clear_error();
    JDFT_CHECK_ARG(b && C && HC && report && nb >= 1, "bad arguments");
    JDFT_CHECK_ARG(ik >= 0 && ik < b->nk, "k-point index out of range");
    *report = jdft_tune_report{0, 0, 0, 0};
    int mb = 0;
    jdft_status s = jdft_autotune_chunk(b, ik, C, ldc, HC, ldhc, nb, prec, &mb, stream);
    if (s != JDFT_OK) return s;
    report->chunk_mb = mb;
    b->plane_bands = 0;
    if (!is_fp64(prec) && plane_pair_batch_supported(make_geom(b, ik))) {
        // plane-pass work items of one band or of a band pair: time H C with each
        cudaStream_t st = (cudaStream_t)stream;
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        float best = 1e30f;
        int best_n = 0;
        for (int bands : {2, 1}) {
            b->plane_bands = bands == 1 ? 1 : 0;
            if ((s = jdft_apply_H(b, ik, C, ldc, HC, ldhc, nb, prec, stream))) break;
            cudaEventRecord(e0, st);
            for (int r = 0; r < 2 && s == JDFT_OK; ++r) s = jdft_apply_H(b, ik, C, ldc, HC, ldhc, nb, prec, stream);
            cudaEventRecord(e1, st);
            if (s != JDFT_OK) break;
            cudaEventSynchronize(e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < best) {
                best = ms;
                best_n = bands;
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        b->plane_bands = best_n == 1 ? 1 : 0;
        if (s != JDFT_OK) return s;
        report->plane_bands = best_n;
    }
    if (prec != JDFT_TF32X3 && prec != JDFT_BF16X3) return JDFT_OK;
    const KSphere& sp = b->ks[ik];
    if ((s = jdft_autotune_gemm(nb, nb, sp.npw, C, ldc, C, ldc, prec, &report->splits_subspace, stream))) return s;
    if (sp.nproj > 0)
        s = jdft_autotune_gemm(sp.nproj, nb, sp.npw, sp.P32, sp.npw, C, ldc, prec, &report->splits_projector, stream);
    return s;
}
