// Basis construction and set-up calls of libjdft: plane-wave spheres per
// k-point, the (i0, i1) column maps the FFT chain is organised around,
// transform plans and twiddle tables, the potential and projector stores,
// and the synthetic Gaussian potential/projector generators.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <map>
#include <mutex>

#include "common.cuh"
#include "gemm.cuh"
#include "profile.cuh"

namespace jdft {

static thread_local std::string g_last_error;

jdft_status set_error(jdft_status s, const std::string& msg) {
    g_last_error = msg;
    return s;
}
void clear_error() { g_last_error.clear(); }

jdft_status check_launch(const char* what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return set_error(JDFT_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
    return JDFT_OK;
}

cudaError_t set_smem_attr(const void* func, size_t smem) {
    static std::mutex mu;
    static std::map<std::pair<int, const void*>, size_t> done;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(mu);
    auto key = std::make_pair(dev, func);
    auto it = done.find(key);
    if (it != done.end() && it->second >= smem) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) done[key] = smem;
    return e;
}

jdft_status ensure_ws(Workspace& w, size_t bytes) {
    if (w.bytes >= bytes) return JDFT_OK;
    if (w.ptr) {
        JDFT_CUDA_TRY(cudaDeviceSynchronize());
        JDFT_CUDA_TRY(cudaFree(w.ptr));
        w.ptr = nullptr;
        w.bytes = 0;
    }
    size_t want = std::max(bytes, (size_t)1 << 20);
    JDFT_CUDA_TRY(cudaMalloc(&w.ptr, want));
    w.bytes = want;
    return JDFT_OK;
}

jdft_status ensure_workspace(jdft_basis_s* b, size_t bytes) { return ensure_ws(b->work, bytes); }

// Radices for a length n = 2^a 3^b 5^c: eights first, then a four or two,
// then threes and fives (fewest passes for the lengths in use).
static bool make_plan(int n, FftPlan* p) {
    p->n = n;
    p->npass = 0;
    int m = n;
    while (m % 8 == 0) { p->radix[p->npass++] = 8; m /= 8; }
    if (m % 4 == 0) { p->radix[p->npass++] = 4; m /= 4; }
    if (m % 2 == 0) { p->radix[p->npass++] = 2; m /= 2; }
    while (m % 3 == 0) { p->radix[p->npass++] = 3; m /= 3; }
    while (m % 5 == 0) { p->radix[p->npass++] = 5; m /= 5; }
    if (m != 1 || p->npass > kMaxPasses) return false;
    return true;
}

static void inv3(const double* A, double* X) {
    // X = A^{-1}, row-major 3x3 by cofactors
    double c00 = A[4] * A[8] - A[5] * A[7];
    double c01 = A[5] * A[6] - A[3] * A[8];
    double c02 = A[3] * A[7] - A[4] * A[6];
    double det = A[0] * c00 + A[1] * c01 + A[2] * c02;
    X[0] = c00 / det; X[1] = (A[2] * A[7] - A[1] * A[8]) / det; X[2] = (A[1] * A[5] - A[2] * A[4]) / det;
    X[3] = c01 / det; X[4] = (A[0] * A[8] - A[2] * A[6]) / det; X[5] = (A[2] * A[3] - A[0] * A[5]) / det;
    X[6] = c02 / det; X[7] = (A[1] * A[6] - A[0] * A[7]) / det; X[8] = (A[0] * A[4] - A[1] * A[3]) / det;
}

template <typename T> static jdft_status upload(T** dst, const std::vector<T>& src) {
    JDFT_CUDA_TRY(cudaMalloc((void**)dst, std::max<size_t>(1, src.size()) * sizeof(T)));
    if (!src.empty())
        JDFT_CUDA_TRY(cudaMemcpy(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice));
    return JDFT_OK;
}

static void free_sphere(KSphere& s) {
    cudaFree(s.col_start); cudaFree(s.col_slot01); cudaFree(s.row_col_start); cudaFree(s.row_i1lo);
    cudaFree(s.pw_col); cudaFree(s.pw_z); cudaFree(s.kin); cudaFree(s.kvec); cudaFree(s.kin32);
    cudaFree(s.P); cudaFree(s.P32); cudaFree(s.Psplit); cudaFree(s.Psplit_t); cudaFree(s.D); cudaFree(s.Dcol);
    cudaFree(s.Dval);
    cudaFree(s.Q); cudaFree(s.Qcol); cudaFree(s.Qval);
    s = KSphere();
}

// Sphere at k: iG with (1/2)|B (iG + k)|^2 <= ecut, lexicographic (i0, i1, i2).
static jdft_status build_sphere(jdft_basis_s* b, int ik) {
    KSphere& s = b->ks[ik];
    const double* k = &b->kfrac[3 * ik];
    const double qmax = std::sqrt(2.0 * b->ecut);
    int lo[3], hi[3];
    for (int d = 0; d < 3; ++d) {
        double len = std::sqrt(b->R[0 + d] * b->R[0 + d] + b->R[3 + d] * b->R[3 + d] + b->R[6 + d] * b->R[6 + d]);
        double reach = len * qmax / (2.0 * M_PI);
        lo[d] = (int)std::floor(-reach - k[d]) - 1;
        hi[d] = (int)std::ceil(reach - k[d]) + 1;
    }
    std::vector<int32_t>& iG = s.iG;
    iG.clear();
    std::vector<double> kin, kvec;
    for (int i0 = lo[0]; i0 <= hi[0]; ++i0)
        for (int i1 = lo[1]; i1 <= hi[1]; ++i1)
            for (int i2 = lo[2]; i2 <= hi[2]; ++i2) {
                double f[3] = {i0 + k[0], i1 + k[1], i2 + k[2]};
                double q[3];
                for (int c = 0; c < 3; ++c) q[c] = b->B[3 * c + 0] * f[0] + b->B[3 * c + 1] * f[1] + b->B[3 * c + 2] * f[2];
                double t = 0.5 * (q[0] * q[0] + q[1] * q[1] + q[2] * q[2]);
                if (t <= b->ecut) {
                    iG.push_back(i0); iG.push_back(i1); iG.push_back(i2);
                    kin.push_back(t);
                    kvec.push_back(q[0]); kvec.push_back(q[1]); kvec.push_back(q[2]);
                }
            }
    s.npw = (int)kin.size();
    if (s.npw == 0) return set_error(JDFT_ERR_ARG, "empty plane-wave sphere (ecut too small)");
    int mn[3] = {1 << 30, 1 << 30, 1 << 30}, mx[3] = {-(1 << 30), -(1 << 30), -(1 << 30)};
    for (int g = 0; g < s.npw; ++g)
        for (int d = 0; d < 3; ++d) {
            mn[d] = std::min(mn[d], iG[3 * g + d]);
            mx[d] = std::max(mx[d], iG[3 * g + d]);
        }
    for (int d = 0; d < 3; ++d)
        if (mx[d] - mn[d] + 1 > b->S[d]) {
            char buf[160];
            snprintf(buf, sizeof buf, "FFT box S%d=%d smaller than the sphere extent %d..%d at k-point %d",
                     d, b->S[d], mn[d], mx[d], ik);
            return set_error(JDFT_ERR_ARG, buf);
        }
    // Columns: runs of equal (i0, i1).
    std::vector<int> col_start, col_slot01, pw_col(s.npw), pw_z(s.npw), col_i0;
    for (int g = 0; g < s.npw; ++g) {
        bool newcol = g == 0 || iG[3 * g] != iG[3 * (g - 1)] || iG[3 * g + 1] != iG[3 * (g - 1) + 1];
        if (newcol) {
            col_start.push_back(g);
            int i1slot = ((iG[3 * g + 1] % b->S[1]) + b->S[1]) % b->S[1];
            col_slot01.push_back(((iG[3 * g] - mn[0]) << 16) | i1slot);
            col_i0.push_back(iG[3 * g]);
        }
        pw_col[g] = (int)col_start.size() - 1;
        pw_z[g] = ((iG[3 * g + 2] % b->S[2]) + b->S[2]) % b->S[2];
    }
    s.ncols = (int)col_start.size();
    col_start.push_back(s.npw);
    s.i0min = mn[0];
    s.nrows = mx[0] - mn[0] + 1;
    s.i1min = mn[1];
    s.i1max = mx[1];
    // First column of each row r (i0 = i0min + r): columns are sorted by i0.
    std::vector<int> row_col_start(s.nrows + 1);
    for (int r = 0; r <= s.nrows; ++r)
        row_col_start[r] = (int)(std::lower_bound(col_i0.begin(), col_i0.end(), mn[0] + r) - col_i0.begin());
    // Each row's columns are consecutive i1 values (a sphere meets a line in an interval).
    std::vector<int> row_i1lo(s.nrows, 0);
    for (int r = 0; r < s.nrows; ++r)
        if (row_col_start[r] < row_col_start[r + 1]) row_i1lo[r] = iG[3 * col_start[row_col_start[r]] + 1];
    std::vector<float> kin32(kin.begin(), kin.end());
    jdft_status st;
    if ((st = upload(&s.col_start, col_start)) != JDFT_OK) return st;
    if ((st = upload(&s.col_slot01, col_slot01)) != JDFT_OK) return st;
    if ((st = upload(&s.row_col_start, row_col_start)) != JDFT_OK) return st;
    if ((st = upload(&s.row_i1lo, row_i1lo)) != JDFT_OK) return st;
    if ((st = upload(&s.pw_col, pw_col)) != JDFT_OK) return st;
    if ((st = upload(&s.pw_z, pw_z)) != JDFT_OK) return st;
    if ((st = upload(&s.kin, kin)) != JDFT_OK) return st;
    if ((st = upload(&s.kvec, kvec)) != JDFT_OK) return st;
    if ((st = upload(&s.kin32, kin32)) != JDFT_OK) return st;
    return JDFT_OK;
}

static jdft_status build_twiddles(jdft_basis_s* b) {
    std::vector<double2> t64;
    std::vector<float2> t32;
    for (int d = 0; d < 3; ++d) {
        int n = b->S[d];
        int found = -1;
        for (int e = 0; e < d; ++e)
            if (b->S[e] == n) found = e;
        if (found >= 0) { b->plan[d].tw_offset = b->plan[found].tw_offset; continue; }
        b->plan[d].tw_offset = (int)t64.size();
        for (int e = 0; e < n; ++e) {
            // exp(+2 pi i e / n) in FP64 (float table rounded from it)
            double a = 2.0 * M_PI * (double)e / (double)n;
            double2 w = make_double2(std::cos(a), std::sin(a));
            t64.push_back(w);
            t32.push_back(make_float2((float)w.x, (float)w.y));
        }
    }
    jdft_status st;
    if ((st = upload(&b->tw64, t64)) != JDFT_OK) return st;
    if ((st = upload(&b->tw32, t32)) != JDFT_OK) return st;
    return JDFT_OK;
}

// ------------------------------------------------------------------------
// Potential store: permute V (j2 fastest) into the plane-pass order
// Vp[(j2 * S1 + j1) * S0 + j0], in FP64 and FP32.
// ------------------------------------------------------------------------
__global__ void permute_potential(const double* __restrict__ V, double* __restrict__ Vp, float* __restrict__ V32,
                                  int S0, int S1, int S2) {
    int64_t N = (int64_t)S0 * S1 * S2;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        int64_t j0 = i % S0;
        int64_t t = i / S0;
        int64_t j1 = t % S1;
        int64_t j2 = t / S1;
        double v = V[(j0 * S1 + j1) * S2 + j2];
        Vp[i] = v;
        V32[i] = (float)v;
    }
}

__global__ void to_complex64(const double2* __restrict__ a, float2* __restrict__ b, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        b[i] = make_float2((float)a[i].x, (float)a[i].y);
}

// ------------------------------------------------------------------------
// Synthetic Gaussian potential: point-by-point sum over atoms and images.
// ------------------------------------------------------------------------
struct Cell { double R[9]; int S[3]; int nmax[3]; };

__global__ void gaussian_potential_kernel(Cell cell, const double* __restrict__ atoms, int natoms,
                                          double depth, double inv2w2, double cut2, double* __restrict__ V) {
    int64_t N = (int64_t)cell.S[0] * cell.S[1] * cell.S[2];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        int j2 = (int)(i % cell.S[2]);
        int j1 = (int)((i / cell.S[2]) % cell.S[1]);
        int j0 = (int)(i / ((int64_t)cell.S[2] * cell.S[1]));
        double f[3] = {(double)j0 / cell.S[0], (double)j1 / cell.S[1], (double)j2 / cell.S[2]};
        double r[3];
        for (int c = 0; c < 3; ++c) r[c] = cell.R[3 * c] * f[0] + cell.R[3 * c + 1] * f[1] + cell.R[3 * c + 2] * f[2];
        double acc = 0.0;
        for (int a = 0; a < natoms; ++a)
            for (int n0 = -cell.nmax[0]; n0 <= cell.nmax[0]; ++n0)
                for (int n1 = -cell.nmax[1]; n1 <= cell.nmax[1]; ++n1)
                    for (int n2 = -cell.nmax[2]; n2 <= cell.nmax[2]; ++n2) {
                        double d2 = 0.0;
                        for (int c = 0; c < 3; ++c) {
                            double dc = r[c] - atoms[3 * a + c] -
                                        (cell.R[3 * c] * n0 + cell.R[3 * c + 1] * n1 + cell.R[3 * c + 2] * n2);
                            d2 += dc * dc;
                        }
                        if (d2 < cut2) acc += exp(-d2 * inv2w2);
                    }
        V[i] = -depth * acc;
    }
}

// Synthetic projectors: closed-form Fourier transforms of unit-norm Gaussian s and p functions.
__global__ void gaussian_projectors_kernel(const double* __restrict__ kvec, int npw, const double* __restrict__ atoms,
                                           int natoms, double sigma, double2* __restrict__ P) {
    const double pi = 3.14159265358979323846;
    double Ns = pow(pi * sigma * sigma, -0.75);
    double pref = Ns * pow(2.0 * pi * sigma * sigma, 1.5);
    double pscale = sigma * sigma * sqrt(2.0) / sigma;  // sigma^2 * (N_p / N_s)
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < npw; g += gridDim.x * blockDim.x) {
        double q0 = kvec[3 * g], q1 = kvec[3 * g + 1], q2 = kvec[3 * g + 2];
        double Fs = pref * exp(-0.5 * sigma * sigma * (q0 * q0 + q1 * q1 + q2 * q2));
        // F_s real; F_p_l = -i sigma^2 q_l (N_p/N_s) F_s, purely imaginary
        double Fp[3] = {-pscale * q0 * Fs, -pscale * q1 * Fs, -pscale * q2 * Fs};
        for (int a = 0; a < natoms; ++a) {
            double s, c;
            sincos(-(q0 * atoms[3 * a] + q1 * atoms[3 * a + 1] + q2 * atoms[3 * a + 2]), &s, &c);
            // phase e^{-i q.R} = c + i s
            P[(int64_t)(4 * a) * npw + g] = make_double2(Fs * c, Fs * s);
            for (int l = 0; l < 3; ++l)  // (i Fp) * (c + i s) = -Fp s + i Fp c
                P[(int64_t)(4 * a + 1 + l) * npw + g] = make_double2(-Fp[l] * s, Fp[l] * c);
        }
    }
}

static int grid_for(int64_t n, int threads) {
    int64_t g = (n + threads - 1) / threads;
    return (int)std::min<int64_t>(std::max<int64_t>(g, 1), 152 * 32);
}

}  // namespace jdft

using namespace jdft;

extern "C" {

jdft_status jdft_basis_create(const jdft_cell_desc* desc, jdft_basis_t* out) {
    clear_error();
    JDFT_CHECK_ARG(desc && out, "null argument");
    JDFT_CHECK_ARG(desc->nk >= 1 && desc->kfrac, "need nk >= 1 and kfrac");
    JDFT_CHECK_ARG(desc->ecut > 0, "ecut must be positive");
    *out = nullptr;
    jdft_basis_s* b = new jdft_basis_s();
    memcpy(b->R, desc->R, sizeof b->R);
    double Rinv[9];
    double det = b->R[0] * (b->R[4] * b->R[8] - b->R[5] * b->R[7]) - b->R[1] * (b->R[3] * b->R[8] - b->R[5] * b->R[6]) +
                 b->R[2] * (b->R[3] * b->R[7] - b->R[4] * b->R[6]);
    if (!(std::fabs(det) > 0)) { delete b; return set_error(JDFT_ERR_ARG, "singular lattice matrix"); }
    inv3(b->R, Rinv);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) b->B[3 * i + j] = 2.0 * M_PI * Rinv[3 * j + i];  // 2 pi R^{-T}
    b->omega = std::fabs(det);
    for (int d = 0; d < 3; ++d) {
        b->S[d] = desc->S[d];
        if (b->S[d] < 1 || b->S[d] > kMaxEdge || !make_plan(b->S[d], &b->plan[d])) {
            delete b;
            return set_error(JDFT_ERR_UNSUPPORTED, "box edges must be products of 2, 3, 5 and at most 512");
        }
    }
    b->N = (int64_t)b->S[0] * b->S[1] * b->S[2];
    b->ecut = desc->ecut;
    b->nk = desc->nk;
    b->kfrac.assign(desc->kfrac, desc->kfrac + 3 * desc->nk);
    if (desc->kweight) b->kweight.assign(desc->kweight, desc->kweight + desc->nk);
    else b->kweight.assign(desc->nk, 1.0 / desc->nk);
    cudaGetDevice(&b->device);
    b->ks.resize(b->nk);
    jdft_status st = JDFT_OK;
    for (int ik = 0; ik < b->nk && st == JDFT_OK; ++ik) st = build_sphere(b, ik);
    if (st == JDFT_OK) st = build_twiddles(b);
    if (st != JDFT_OK) {
        std::string msg = jdft_last_error();
        jdft_basis_destroy(b);
        return set_error(st, msg);
    }
    *out = b;
    return JDFT_OK;
}

jdft_status jdft_basis_destroy(jdft_basis_t b) {
    if (!b) return JDFT_OK;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(b->device);
    for (auto& s : b->ks) free_sphere(s);
    cudaFree(b->tw64); cudaFree(b->tw32); cudaFree(b->V); cudaFree(b->V32); cudaFree(b->work.ptr);
    if (b->side) {
        cudaStreamSynchronize(b->side);
        cudaStreamDestroy(b->side);
    }
    if (b->ev_fork) cudaEventDestroy(b->ev_fork);
    if (b->ev_join) cudaEventDestroy(b->ev_join);
    cudaFree(b->fwork.ptr);
    cudaFree(b->fieldwork.ptr);
    cudaFree(b->spinwork.ptr);
    cudaSetDevice(prev);
    delete b;
    return JDFT_OK;
}

jdft_status jdft_basis_npw(jdft_basis_t b, int ik, int* npw) {
    clear_error();
    JDFT_CHECK_ARG(b && npw, "null argument");
    JDFT_CHECK_ARG(ik >= 0 && ik < b->nk, "k-point index out of range");
    *npw = b->ks[ik].npw;
    return JDFT_OK;
}

jdft_status jdft_basis_gvectors(jdft_basis_t b, int ik, int32_t* iG) {
    clear_error();
    JDFT_CHECK_ARG(b && iG, "null argument");
    JDFT_CHECK_ARG(ik >= 0 && ik < b->nk, "k-point index out of range");
    memcpy(iG, b->ks[ik].iG.data(), b->ks[ik].iG.size() * sizeof(int32_t));
    return JDFT_OK;
}

jdft_status jdft_basis_info(jdft_basis_t b, int ik, double* omega, int64_t* nbox, int* ncols) {
    clear_error();
    JDFT_CHECK_ARG(b, "null basis");
    JDFT_CHECK_ARG(ik >= 0 && ik < b->nk, "k-point index out of range");
    if (omega) *omega = b->omega;
    if (nbox) *nbox = b->N;
    if (ncols) *ncols = b->ks[ik].ncols;
    return JDFT_OK;
}

jdft_status jdft_set_potential(jdft_basis_t b, const double* V, void* stream) {
    clear_error();
    JDFT_CHECK_ARG(b && V, "null argument");
    if (!b->V) {
        JDFT_CUDA_TRY(cudaMalloc(&b->V, b->N * sizeof(double)));
        JDFT_CUDA_TRY(cudaMalloc(&b->V32, b->N * sizeof(float)));
    }
    {
        Trace tr_("permute_potential", (cudaStream_t)stream);
        permute_potential<<<grid_for(b->N, 256), 256, 0, (cudaStream_t)stream>>>(V, b->V, b->V32, b->S[0], b->S[1],
                                                                                 b->S[2]);
    }
    b->have_V = true;
    return check_launch("permute_potential");
}

jdft_status jdft_set_projectors(jdft_basis_t b, int ik, const void* P, int nproj, const double* D, void* stream) {
    clear_error();
    JDFT_CHECK_ARG(b, "null basis");
    JDFT_CHECK_ARG(ik >= 0 && ik < b->nk, "k-point index out of range");
    JDFT_CHECK_ARG(nproj >= 0, "nproj must be >= 0");
    KSphere& s = b->ks[ik];
    if (s.P) {
        JDFT_CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
        cudaFree(s.P); cudaFree(s.P32); cudaFree(s.Psplit); cudaFree(s.Psplit_t); cudaFree(s.D); cudaFree(s.Dcol);
        cudaFree(s.Dval);
        s.P = s.P32 = s.Psplit = s.Psplit_t = nullptr; s.D = nullptr; s.Dcol = nullptr; s.Dval = nullptr; s.Dw = 0;
    }
    if (s.Q) {
        // the augmentation belongs to the projectors it was set for
        JDFT_CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
        cudaFree(s.Q); cudaFree(s.Qcol); cudaFree(s.Qval);
        s.Q = nullptr; s.Qcol = nullptr; s.Qval = nullptr; s.Qw = 0;
    }
    s.nproj = nproj;
    if (nproj == 0) return JDFT_OK;
    JDFT_CHECK_ARG(P && D, "null projector or D pointer");
    size_t n = (size_t)s.npw * nproj;
    JDFT_CUDA_TRY(cudaMalloc(&s.P, n * sizeof(double2)));
    JDFT_CUDA_TRY(cudaMalloc(&s.P32, n * sizeof(float2)));
    JDFT_CUDA_TRY(cudaMalloc(&s.D, (size_t)nproj * nproj * sizeof(double)));
    cudaStream_t st = (cudaStream_t)stream;
    JDFT_CUDA_TRY(cudaMemcpyAsync(s.P, P, n * sizeof(double2), cudaMemcpyDeviceToDevice, st));
    JDFT_CUDA_TRY(cudaMemcpyAsync(s.D, D, (size_t)nproj * nproj * sizeof(double), cudaMemcpyDeviceToDevice, st));
    {
        // ELL copy of D for the products D (P^dag C): nonlocal D matrices couple
        // only the projectors of one atom, so rows hold a few nonzeros
        std::vector<double> h((size_t)nproj * nproj);
        JDFT_CUDA_TRY(cudaMemcpyAsync(h.data(), D, h.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
        JDFT_CUDA_TRY(cudaStreamSynchronize(st));
        int w = 1;
        for (int i = 0; i < nproj; ++i) {
            int c = 0;
            for (int j = 0; j < nproj; ++j) c += h[(size_t)i * nproj + j] != 0.0;
            w = std::max(w, c);
        }
        std::vector<int> col((size_t)nproj * w, 0);
        std::vector<double> val((size_t)nproj * w, 0.0);
        for (int i = 0; i < nproj; ++i) {
            int c = 0;
            for (int j = 0; j < nproj; ++j)
                if (h[(size_t)i * nproj + j] != 0.0) {
                    col[(size_t)i * w + c] = j;
                    val[(size_t)i * w + c] = h[(size_t)i * nproj + j];
                    ++c;
                }
        }
        s.Dw = w;
        JDFT_CUDA_TRY(cudaMalloc(&s.Dcol, col.size() * sizeof(int)));
        JDFT_CUDA_TRY(cudaMalloc(&s.Dval, val.size() * sizeof(double)));
        JDFT_CUDA_TRY(cudaMemcpy(s.Dcol, col.data(), col.size() * sizeof(int), cudaMemcpyHostToDevice));
        JDFT_CUDA_TRY(cudaMemcpy(s.Dval, val.data(), val.size() * sizeof(double), cudaMemcpyHostToDevice));
    }
    {
        Trace tr_("to_complex64", st);
        to_complex64<<<grid_for((int64_t)n, 256), 256, 0, st>>>((const double2*)s.P, (float2*)s.P32, (int64_t)n);
    }
    jdft_status r = check_launch("to_complex64");
    if (r != JDFT_OK) return r;
    // BF16 planes of the projectors for the split-operand products
    JDFT_CUDA_TRY(cudaMalloc(&s.Psplit, tcx_split_bytes(nproj, s.npw)));
    if ((r = tcx_split((const float2*)s.P32, s.npw, nproj, s.npw, s.Psplit, st)) != JDFT_OK) return r;
    JDFT_CUDA_TRY(cudaMalloc(&s.Psplit_t, tcx_split_bytes(s.npw, nproj)));
    return tcx_split_t((const float2*)s.P32, s.npw, s.npw, nproj, s.Psplit_t, st);
}

jdft_status jdft_gaussian_potential(jdft_basis_t b, int natoms, const double* atoms, double depth, double width,
                                    double* V_out, void* stream) {
    clear_error();
    JDFT_CHECK_ARG(b && V_out, "null argument");
    JDFT_CHECK_ARG(natoms >= 0 && (natoms == 0 || atoms), "bad atom list");
    JDFT_CHECK_ARG(width > 0, "width must be positive");
    Cell cell;
    memcpy(cell.R, b->R, sizeof cell.R);
    const double cut = 10.0;
    for (int d = 0; d < 3; ++d) {
        cell.S[d] = b->S[d];
        double blen = std::sqrt(b->B[d] * b->B[d] + b->B[3 + d] * b->B[3 + d] + b->B[6 + d] * b->B[6 + d]);
        cell.nmax[d] = 1 + (int)std::ceil(cut * blen / (2.0 * M_PI));
    }
    double* d_atoms = nullptr;
    cudaStream_t st = (cudaStream_t)stream;
    JDFT_CUDA_TRY(cudaMalloc(&d_atoms, std::max(1, natoms) * 3 * sizeof(double)));
    if (natoms) JDFT_CUDA_TRY(cudaMemcpyAsync(d_atoms, atoms, natoms * 3 * sizeof(double), cudaMemcpyHostToDevice, st));
    {
        Trace tr_("gaussian_potential", st);
        gaussian_potential_kernel<<<grid_for(b->N, 128), 128, 0, st>>>(cell, d_atoms, natoms, depth,
                                                                        1.0 / (2 * width * width), cut * cut, V_out);
    }
    jdft_status s = check_launch("gaussian_potential_kernel");
    JDFT_CUDA_TRY(cudaStreamSynchronize(st));
    cudaFree(d_atoms);
    return s;
}

jdft_status jdft_gaussian_projectors(jdft_basis_t b, int ik, int natoms, const double* atoms, double sigma,
                                     void* P_out, void* stream) {
    clear_error();
    JDFT_CHECK_ARG(b && P_out, "null argument");
    JDFT_CHECK_ARG(ik >= 0 && ik < b->nk, "k-point index out of range");
    JDFT_CHECK_ARG(natoms >= 1 && atoms, "need at least one atom");
    JDFT_CHECK_ARG(sigma > 0, "sigma must be positive");
    double* d_atoms = nullptr;
    cudaStream_t st = (cudaStream_t)stream;
    JDFT_CUDA_TRY(cudaMalloc(&d_atoms, natoms * 3 * sizeof(double)));
    JDFT_CUDA_TRY(cudaMemcpyAsync(d_atoms, atoms, natoms * 3 * sizeof(double), cudaMemcpyHostToDevice, st));
    const KSphere& s = b->ks[ik];
    {
        Trace tr_("gaussian_projectors", st);
        gaussian_projectors_kernel<<<grid_for(s.npw, 128), 128, 0, st>>>(s.kvec, s.npw, d_atoms, natoms, sigma,
                                                                          (double2*)P_out);
    }
    jdft_status r = check_launch("gaussian_projectors_kernel");
    JDFT_CUDA_TRY(cudaStreamSynchronize(st));
    cudaFree(d_atoms);
    return r;
}

const char* jdft_last_error(void) { return g_last_error.c_str(); }

const char* jdft_version(void) { return "jdft-gb300 0.1 (sm_103a)"; }

}  // extern "C"
