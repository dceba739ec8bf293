// Two-component (spinor) bands in a noncollinear potential: the Hamiltonian
// and the density/magnetisation of spinor ColumnBundles.  The JDFTx paper
// lists noncollinear magnetism among its electronic features (Sec. 2.2) and
// holds wavefunctions in ColumnBundles (Sec. 2.1); it prints no formula.
//
// Readings (shared with the test oracle only through the paper):
//   * a spinor block of nb bands is 2 nb coefficient rows, row 2b the up and
//     row 2b + 1 the down component of band b, on the same sphere;
//   * the local potential is V 1 + M . sigma (Pauli matrices): the scalar V is
//     the basis potential, M a real 3-vector field, so
//       phi_up = (V + M_z) psi_up + (M_x - i M_y) psi_dn,
//       phi_dn = (M_x + i M_y) psi_up + (V - M_z) psi_dn;
//   * kinetic and projector terms act on each component alike;
//   * n = sum_b f_b (|psi_up|^2 + |psi_dn|^2), m = sum_b f_b psi^dag sigma psi.
//
// Design.  FP32 blocks on boxes the band-pair plane kernel serves (128 x 128
// planes): the chain of jdft_apply_H with the band-pair plane pass made spinor
// -- a pair of rows (2b, 2b + 1) is band b's (up, down) components, so the
// 2 x 2 product V 1 + M . sigma replaces the multiply by V inside the fused
// pass (z pass in, plane pass, z pass out with the kinetic term), then the
// nonlocal term on all rows.  Elsewhere (FP64, other boxes): the scalar
// Hamiltonian on all 2 nb rows plus the coupling formed in chunks of bands:
// psi = I C for the chunk's rows (jdft_op_I), the 2 x 2 product in place,
// J of the result (jdft_op_J), and HC += Omega * that.  The density and
// magnetisation come from the inverse transforms, summed per point over the
// chunk's bands.
#include <cmath>

#include "chain.cuh"
#include "common.cuh"
#include "gemm.cuh"
#include "profile.cuh"

namespace jdft {
namespace {

constexpr int kThreads = 256;
constexpr size_t kSpinChunkBytes = (size_t)256 << 20;   // budget of the real-space boxes per chunk

int grid_of(int64_t n) {
    int64_t g = (n + kThreads - 1) / kThreads;
    return (int)std::max<int64_t>(1, std::min<int64_t>(g, 152 * 16));
}

// In place on psi (2 nb rows of N): (up, dn) <- (M . sigma) (up, dn).
template <typename T>
__global__ void __launch_bounds__(kThreads)
spinor_couple_kernel(c_t<T>* __restrict__ psi, const double* __restrict__ M, int nb, int64_t N) {
    const int64_t total = (int64_t)nb * N;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = i / N, j = i - b * N;
        c_t<T>* up = psi + (2 * b) * N + j;
        c_t<T>* dn = psi + (2 * b + 1) * N + j;
        const T mx = (T)M[j], my = (T)M[N + j], mz = (T)M[2 * N + j];
        const c_t<T> u = *up, d = *dn;
        // (M_x - i M_y) d and (M_x + i M_y) u
        const T a_re = mx * d.x + my * d.y, a_im = mx * d.y - my * d.x;
        const T b_re = mx * u.x - my * u.y, b_im = mx * u.y + my * u.x;
        *up = mk<T>(mz * u.x + a_re, mz * u.y + a_im);
        *dn = mk<T>(b_re - mz * d.x, b_im - mz * d.y);
    }
}

// HC[r * ldhc + g] += s * D[r * npw + g] for rows r < rows.
template <typename T>
__global__ void __launch_bounds__(kThreads)
add_scaled_rows_kernel(c_t<T>* __restrict__ HC, int ldhc, const c_t<T>* __restrict__ D, int npw, int rows, T s) {
    const int64_t total = (int64_t)rows * npw;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = i / npw, g = i - r * npw;
        c_t<T> h = HC[r * ldhc + g];
        const c_t<T> d = D[i];
        h.x += s * d.x;
        h.y += s * d.y;
        HC[r * ldhc + g] = h;
    }
}

// n[j] += w sum_b f_b (|up|^2 + |dn|^2), m[c N + j] += w sum_b f_b (psi^dag sigma_c psi)
// over the chunk's nb bands (FP64 sums).
template <typename T>
__global__ void __launch_bounds__(kThreads)
spinor_density_kernel(const c_t<T>* __restrict__ psi, const double* __restrict__ f, int nb, int64_t N, double w,
                      double* __restrict__ n, double* __restrict__ m) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < N; j += (int64_t)gridDim.x * blockDim.x) {
        double sn = 0.0, sx = 0.0, sy = 0.0, sz = 0.0;
        for (int b = 0; b < nb; ++b) {
            const c_t<T> u = psi[(int64_t)(2 * b) * N + j], d = psi[(int64_t)(2 * b + 1) * N + j];
            const double uu = (double)u.x * u.x + (double)u.y * u.y;
            const double dd = (double)d.x * d.x + (double)d.y * d.y;
            // conj(u) d
            const double cr = (double)u.x * d.x + (double)u.y * d.y;
            const double ci = (double)u.x * d.y - (double)u.y * d.x;
            const double fb = f[b];
            sn += fb * (uu + dd);
            sx += fb * 2.0 * cr;
            sy += fb * 2.0 * ci;
            sz += fb * (uu - dd);
        }
        n[j] += w * sn;
        m[j] += w * sx;
        m[N + j] += w * sy;
        m[2 * N + j] += w * sz;
    }
}

bool fp64(jdft_prec p) { return p == JDFT_FP64; }

jdft_status spin_ws(jdft_basis_s* b, size_t bytes, void** p) {
    jdft_status s = ensure_ws(b->spinwork, bytes);
    if (s) return s;
    *p = b->spinwork.ptr;
    return JDFT_OK;
}

// Bands per chunk so that the chunk's 2 x nbc real-space boxes fit the budget.
int chunk_bands(const jdft_basis_s* b, int nb, size_t elem) {
    const size_t per_band = 2 * (size_t)b->N * elem;
    const int c = (int)std::max<size_t>(1, kSpinChunkBytes / per_band);
    return std::min(nb, c);
}

template <typename T>
jdft_status couple(jdft_basis_s* b, int ik, const double* M, const void* C, int ldc, void* HC, int ldhc, int nb,
                   jdft_prec prec, cudaStream_t st) {
    const int npw = b->ks[ik].npw;
    const size_t e = sizeof(c_t<T>);
    const int nbc = chunk_bands(b, nb, e);
    void* ws = nullptr;
    const size_t box_bytes = 2 * (size_t)nbc * b->N * e;
    jdft_status s = spin_ws(b, box_bytes + 2 * (size_t)nbc * npw * e, &ws);
    if (s) return s;
    c_t<T>* psi = reinterpret_cast<c_t<T>*>(ws);
    c_t<T>* D = reinterpret_cast<c_t<T>*>(reinterpret_cast<char*>(ws) + box_bytes);
    for (int b0 = 0; b0 < nb; b0 += nbc) {
        const int n = std::min(nbc, nb - b0);
        const c_t<T>* Cb = reinterpret_cast<const c_t<T>*>(C) + (size_t)2 * b0 * ldc;
        c_t<T>* Hb = reinterpret_cast<c_t<T>*>(HC) + (size_t)2 * b0 * ldhc;
        if ((s = jdft_op_I(b, ik, Cb, ldc, psi, 2 * n, prec, st))) return s;
        {
            Trace tr_("spinor_couple", st);
            spinor_couple_kernel<T><<<grid_of((int64_t)n * b->N), kThreads, 0, st>>>(psi, M, n, b->N);
        }
        if ((s = check_launch("spinor_couple"))) return s;
        if ((s = jdft_op_J(b, ik, psi, D, npw, 2 * n, prec, st))) return s;
        {
            Trace tr_("spinor_add", st);
            add_scaled_rows_kernel<T><<<grid_of((int64_t)2 * n * npw), kThreads, 0, st>>>(Hb, ldhc, D, npw, 2 * n,
                                                                                          (T)b->omega);
        }
        if ((s = check_launch("spinor_add"))) return s;
    }
    return JDFT_OK;
}

template <typename T>
jdft_status spin_density(jdft_basis_s* b, int ik, const void* C, int ldc, const double* f, int nb, double* n_r,
                         double* m_r, jdft_prec prec, cudaStream_t st) {
    const size_t e = sizeof(c_t<T>);
    const int nbc = chunk_bands(b, nb, e);
    void* ws = nullptr;
    jdft_status s = spin_ws(b, 2 * (size_t)nbc * b->N * e, &ws);
    if (s) return s;
    c_t<T>* psi = reinterpret_cast<c_t<T>*>(ws);
    for (int b0 = 0; b0 < nb; b0 += nbc) {
        const int n = std::min(nbc, nb - b0);
        const c_t<T>* Cb = reinterpret_cast<const c_t<T>*>(C) + (size_t)2 * b0 * ldc;
        if ((s = jdft_op_I(b, ik, Cb, ldc, psi, 2 * n, prec, st))) return s;
        {
            Trace tr_("spinor_density", st);
            spinor_density_kernel<T><<<grid_of(b->N), kThreads, 0, st>>>(psi, f + b0, n, b->N, b->kweight[ik], n_r,
                                                                         m_r);
        }
        if ((s = check_launch("spinor_density"))) return s;
    }
    return JDFT_OK;
}

// Mp[c N + (j2 S1 + j1) S0 + j0] = M[c N + (j0 S1 + j1) S2 + j2] in FP32 (the plane pass's layout).
__global__ void __launch_bounds__(kThreads)
permute_field3_kernel(const double* __restrict__ M, float* __restrict__ Mp, int S0, int S1, int S2) {
    const int64_t N = (int64_t)S0 * S1 * S2;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < 3 * N; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = i / N, j = i - c * N;
        const int j2 = (int)(j % S2);
        const int64_t r = j / S2;
        const int j1 = (int)(r % S1), j0 = (int)(r / S1);
        Mp[c * N + ((int64_t)j2 * S1 + j1) * S0 + j0] = (float)M[i];
    }
}

// The fused FP32 path; JDFT_ERR_UNSUPPORTED (nothing launched) when the box has
// no band-pair plane kernel.
jdft_status spinor_fused(jdft_basis_s* b, int ik, const double* M, const void* C, int ldc, void* HC, int ldhc, int nb,
                         jdft_prec prec, cudaStream_t st) {
    const ChainGeom g = make_geom(b, ik);
    if (!((g.S0 == 128 && g.S1 == 128) || (g.S0 == 16 && g.S1 == 12))) return JDFT_ERR_UNSUPPORTED;
    if (!b->V32) return set_error(JDFT_ERR_ARG, "no potential set");
    const KSphere& sp = b->ks[ik];
    const int rows = 2 * nb;
    const size_t rowbytes = (size_t)g.S2 * g.ncols * sizeof(float2);
    int nc = (int)std::min<size_t>((size_t)rows, std::max<size_t>(2, ((size_t)512 << 20) / rowbytes));
    nc &= ~1;
    const size_t colbytes = ((size_t)nc * rowbytes + 255) / 256 * 256;
    const size_t mbytes = 3 * (size_t)b->N * sizeof(float);
    void* ws = nullptr;
    jdft_status s = spin_ws(b, colbytes + mbytes, &ws);
    if (s) return s;
    float2* colbuf = reinterpret_cast<float2*>(ws);
    float* Mp = reinterpret_cast<float*>(reinterpret_cast<char*>(ws) + colbytes);
    {
        Trace tr_("permute_field3", st);
        permute_field3_kernel<<<grid_of(3 * b->N), kThreads, 0, st>>>(M, Mp, b->S[0], b->S[1], b->S[2]);
    }
    if ((s = check_launch("permute_field3"))) return s;
    const float2* tw = b->tw32;
    const float omega = (float)b->omega, invN = (float)(1.0 / (double)b->N);
    for (int r0 = 0; r0 < rows; r0 += nc) {
        const int n = std::min(nc, rows - r0);
        const float2* Cc = reinterpret_cast<const float2*>(C) + (size_t)r0 * ldc;
        float2* Hc = reinterpret_cast<float2*>(HC) + (size_t)r0 * ldhc;
        if ((s = launch_zpass_inverse<float>(g, Cc, ldc, colbuf, n, tw, st))) return s;
        if ((s = launch_plane_apply_pair_spinor(g, colbuf, b->V32, Mp, n, tw, st))) return s;
        if ((s = launch_zpass_forward<float, 0>(g, colbuf, Cc, ldc, Hc, ldhc, n, sp.kin32, omega, invN, tw, st)))
            return s;
    }
    if (sp.nproj == 0) return JDFT_OK;
    if ((s = ensure_workspace(b, nonlocal_workspace_bytes(sp.nproj, rows, sizeof(float2), sp.npw, prec, true, true))))
        return s;
    return nonlocal_accumulate<float>(sp, C, ldc, HC, ldhc, rows, prec, b->work.ptr, st, true, nullptr, true);
}

jdft_status check_spinor_args(jdft_basis_s* b, int ik, const void* C, int ldc, int nb, jdft_prec prec) {
    JDFT_CHECK_ARG(b && C, "null argument");
    JDFT_CHECK_ARG(ik >= 0 && ik < b->nk, "k-point index out of range");
    JDFT_CHECK_ARG(nb >= 1, "nb must be >= 1");
    JDFT_CHECK_ARG(prec >= JDFT_FP64 && prec <= JDFT_BF16X3, "unknown precision");
    JDFT_CHECK_ARG(ldc >= b->ks[ik].npw, "leading dimension below npw");
    return JDFT_OK;
}

}  // namespace
}  // namespace jdft

using namespace jdft;

extern "C" {

jdft_status jdft_apply_H_spinor(jdft_basis_t b, int ik, const double* M, const void* C, int ldc, void* HC, int ldhc,
                                int nb, jdft_prec prec, void* stream) {
    clear_error();
    jdft_status s = check_spinor_args(b, ik, C, ldc, nb, prec);
    if (s) return s;
    JDFT_CHECK_ARG(M && HC, "null argument");
    JDFT_CHECK_ARG(ldhc >= b->ks[ik].npw, "leading dimension below npw");
    JDFT_CHECK_ARG(C != HC, "C and HC must not overlap");
    cudaStream_t st = (cudaStream_t)stream;
    if (!fp64(prec)) {
        s = spinor_fused(b, ik, M, C, ldc, HC, ldhc, nb, prec, st);
        if (s != JDFT_ERR_UNSUPPORTED) return s;
        clear_error();
    }
    // scalar part on every component row: Omega [T C + J(V I C)] + P D P^dag C
    if ((s = jdft_apply_H(b, ik, C, ldc, HC, ldhc, 2 * nb, prec, stream))) return s;
    return fp64(prec) ? couple<double>(b, ik, M, C, ldc, HC, ldhc, nb, prec, st)
                      : couple<float>(b, ik, M, C, ldc, HC, ldhc, nb, prec, st);
}

jdft_status jdft_density_spinor(jdft_basis_t b, int ik, const void* C, int ldc, const double* f, int nb,
                                double* n_r, double* m_r, jdft_prec prec, void* stream) {
    clear_error();
    jdft_status s = check_spinor_args(b, ik, C, ldc, nb, prec);
    if (s) return s;
    JDFT_CHECK_ARG(f && n_r && m_r, "null argument");
    cudaStream_t st = (cudaStream_t)stream;
    return fp64(prec) ? spin_density<double>(b, ik, C, ldc, f, nb, n_r, m_r, prec, st)
                      : spin_density<float>(b, ik, C, ldc, f, nb, n_r, m_r, prec, st);
}

}  // extern "C"
