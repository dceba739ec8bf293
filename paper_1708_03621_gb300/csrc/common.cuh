// Shared definitions of the libjdft CUDA sources: complex arithmetic on
// double2/float2, status plumbing, and the device-resident basis.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/jdft.h"

namespace jdft {

// ---------------------------------------------------------------------------
// Error reporting: every entry point returns a jdft_status and records a
// message in a thread-local string.
// ---------------------------------------------------------------------------
jdft_status set_error(jdft_status s, const std::string& msg);
void clear_error();

#define JDFT_CHECK_ARG(cond, msg)                                  \
    do {                                                           \
        if (!(cond)) return ::jdft::set_error(JDFT_ERR_ARG, (msg)); \
    } while (0)

#define JDFT_CUDA_TRY(call)                                                          \
    do {                                                                             \
        cudaError_t e_ = (call);                                                     \
        if (e_ != cudaSuccess)                                                       \
            return ::jdft::set_error(e_ == cudaErrorMemoryAllocation ? JDFT_ERR_OOM  \
                                                                     : JDFT_ERR_CUDA, \
                                     std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

// Reports a kernel launch failure (the launch itself, not later execution).
jdft_status check_launch(const char* what);

// cudaFuncSetAttribute(MaxDynamicSharedMemorySize) once per (device, kernel,
// size): later launches, including those recorded into a CUDA graph, make no
// attribute calls.
cudaError_t set_smem_attr(const void* func, size_t smem);

// ---------------------------------------------------------------------------
// Complex arithmetic on the CUDA vector types.  T is double or float.
// ---------------------------------------------------------------------------
template <typename T> struct cplx;
template <> struct cplx<double> { using type = double2; };
template <> struct cplx<float> { using type = float2; };
template <typename T> using c_t = typename cplx<T>::type;

template <typename T> __host__ __device__ __forceinline__ c_t<T> mk(T re, T im) {
    c_t<T> z; z.x = re; z.y = im; return z;
}
template <typename V> __host__ __device__ __forceinline__ V cadd(V a, V b) { a.x += b.x; a.y += b.y; return a; }
template <typename V> __host__ __device__ __forceinline__ V csub(V a, V b) { a.x -= b.x; a.y -= b.y; return a; }
template <typename V> __host__ __device__ __forceinline__ V cmul(V a, V b) {
    V z; z.x = a.x * b.x - a.y * b.y; z.y = a.x * b.y + a.y * b.x; return z;
}
// a * conj(b)
template <typename V> __host__ __device__ __forceinline__ V cmulc(V a, V b) {
    V z; z.x = a.x * b.x + a.y * b.y; z.y = a.y * b.x - a.x * b.y; return z;
}
template <typename V, typename S> __host__ __device__ __forceinline__ V cscale(V a, S s) {
    a.x *= s; a.y *= s; return a;
}
// multiply by sign*i : (x + iy) * (s i) = -s y + i s x
template <int SIGN, typename V> __host__ __device__ __forceinline__ V cmul_i(V a) {
    V z; z.x = -SIGN * a.y; z.y = SIGN * a.x; return z;
}

// ---------------------------------------------------------------------------
// Transform plans: one per distinct box edge length.  Radices (passes of the
// Stockham autosort FFT) and a table W[e] = exp(+2 pi i e / n), e in [0, n).
// ---------------------------------------------------------------------------
constexpr int kMaxPasses = 12;
constexpr int kMaxEdge = 512;

struct FftPlan {
    int n;
    int npass;
    int radix[kMaxPasses];
    int tw_offset;  // offset of this length's table in the basis twiddle arrays
};

// Per k-point sphere maps on the device.
struct KSphere {
    int npw = 0;
    int ncols = 0;          // number of distinct (i0, i1) columns
    int nrows = 0;          // i0 range covered by the columns: i0min .. i0min + nrows - 1
    int i0min = 0;
    int i1min = 0, i1max = 0;   // range of i1 over the sphere
    // device arrays
    int* col_start = nullptr;   // ncols + 1: first sphere index of each column (prefix sums)
    int* col_slot01 = nullptr;  // ncols: packed (row r = i0 - i0min) << 16 | (i1 mod S1)
    int* row_col_start = nullptr; // nrows + 1: first column of each row r
    int* row_i1lo = nullptr;    // nrows: signed i1 of each row's first column (rows are i1 intervals)
    int* pw_col = nullptr;      // npw: column of each plane wave
    int* pw_z = nullptr;        // npw: i2 mod S2 of each plane wave
    double* kin = nullptr;      // npw: (1/2)|k+G|^2
    double* kvec = nullptr;     // npw x 3: Cartesian k+G
    float* kin32 = nullptr;     // npw: FP32 copy of kin
    // host copies
    std::vector<int32_t> iG;    // npw x 3
    // nonlocal term
    int nproj = 0;
    void* P = nullptr;          // complex128 npw x nproj column-major
    void* P32 = nullptr;        // complex64 copy
    void* Psplit = nullptr;     // BF16 planes of P32 for the BF16x3 products (Re hi, Re lo, Im hi, Im lo)
    void* Psplit_t = nullptr;   // the same of P32's transpose (rows = plane waves), for P X
    double* D = nullptr;        // nproj x nproj
    // D as ELL rows: Dw entries per row (the widest row's nonzero count),
    // columns and values, padded with column 0 and value 0
    int Dw = 0;
    int* Dcol = nullptr;        // nproj x Dw
    double* Dval = nullptr;     // nproj x Dw
    // augmentation of the overlap (S = Omega + P Q P^dag), dense and as ELL
    // rows like D; Q == nullptr when the overlap is the plain Omega
    double* Q = nullptr;        // nproj x nproj
    int Qw = 0;
    int* Qcol = nullptr;
    double* Qval = nullptr;
};

// Library-owned scratch buffer that only grows.
struct Workspace {
    void* ptr = nullptr;
    size_t bytes = 0;
};

}  // namespace jdft

struct jdft_basis_s {
    double R[9];
    double B[9];            // 2 pi R^{-T}, row-major, column d = b_d
    double omega;
    int S[3];
    int64_t N;
    double ecut;
    int nk;
    std::vector<double> kfrac;
    std::vector<double> kweight;
    std::vector<jdft::KSphere> ks;
    // transforms
    jdft::FftPlan plan[3];
    double2* tw64 = nullptr;  // twiddle tables, all lengths back to back
    float2* tw32 = nullptr;
    // local potential, permuted for the plane pass: Vp[(j2 * S1 + j1) * S0 + j0]
    double* V = nullptr;
    float* V32 = nullptr;
    bool have_V = false;
    int device = 0;
    int chunk_mb = 0;         // band-chunk budget chosen by jdft_autotune_chunk (0 = default)
    int reserve_sms = 0;      // SMs the persistent plane kernels leave free (work on a side stream)
    int plane_bands = 0;      // bands per plane-pass item of FP32 blocks: 0 = 2 where compiled (autotuned), 1
    jdft::Workspace work;
    // jdft_hamiltonian_step: the overlap factorisation's own scratch (it runs
    // on a side stream while the chain uses `work`), the side stream and its
    // fork / join events (created on first use)
    jdft::Workspace fwork;
    // full-box field transforms (Hartree, Kohn-Sham potential): a complex FP64
    // box and per-block partial sums (grown on first use)
    jdft::Workspace fieldwork;
    // spinor calls: real-space boxes and sphere blocks of a band chunk
    jdft::Workspace spinwork;
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
};

namespace jdft {
// Grows the basis workspace to at least `bytes` (synchronous cudaMalloc).
jdft_status ensure_workspace(jdft_basis_s* b, size_t bytes);
// The same for any library-owned workspace of the basis.
jdft_status ensure_ws(Workspace& w, size_t bytes);
}  // namespace jdft
