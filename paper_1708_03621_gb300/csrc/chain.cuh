// Kernels of the scatter -> FFT -> V -> FFT -> gather chain, shared by the
// operator, Hamiltonian and density entry points.
#pragma once

#include "common.cuh"
#include "fft.cuh"

#include <vector>

namespace jdft {

// Everything a chain kernel needs to know about one sphere on one box.
struct ChainGeom {
    int S0, S1, S2;
    int npw, ncols, nrows, i0min;
    int i1min, i1max;          // range of i1 over the sphere
    const int* col_start;      // ncols + 1
    const int* col_slot01;     // ncols: (row << 16) | (i1 mod S1)
    const int* row_col_start;  // nrows + 1
    const int* row_i1lo;       // nrows
    const int* pw_col;         // npw
    const int* pw_z;           // npw
    FftPlan p0, p1, p2;
    int reserve_sms;           // SMs the persistent plane kernels leave free
    int one_band;              // 1: the one-band plane kernels even where band-pair ones exist
};

inline ChainGeom make_geom(const jdft_basis_s* b, int ik) {
    const KSphere& s = b->ks[ik];
    ChainGeom g;
    g.S0 = b->S[0]; g.S1 = b->S[1]; g.S2 = b->S[2];
    g.npw = s.npw; g.ncols = s.ncols; g.nrows = s.nrows; g.i0min = s.i0min;
    g.i1min = s.i1min; g.i1max = s.i1max;
    g.col_start = s.col_start; g.col_slot01 = s.col_slot01; g.row_col_start = s.row_col_start;
    g.row_i1lo = s.row_i1lo;
    g.pw_col = s.pw_col; g.pw_z = s.pw_z;
    g.p0 = b->plan[0]; g.p1 = b->plan[1]; g.p2 = b->plan[2];
    g.reserve_sms = b->reserve_sms;
    g.one_band = b->plane_bands == 1 ? 1 : 0;
    return g;
}

// Column buffer layout: value of column c, z-slot j2, band b (within the
// current chunk) at colbuf[(b * S2 + j2) * ncols + c].
__host__ __device__ inline size_t colbuf_index(const ChainGeom& g, int b, int j2, int c) {
    return ((size_t)b * g.S2 + j2) * g.ncols + c;
}

// Launch helpers (defined in chain.cu), all on `stream`, bands [0, nb) of the chunk.
template <typename T>
jdft_status launch_zpass_inverse(const ChainGeom& g, const c_t<T>* C, int ldc, c_t<T>* colbuf, int nb,
                                 const c_t<T>* tw_base, cudaStream_t st);
// MODE 0: out = omega (kin C + scale y); MODE 1: out = scale y.
template <typename T, int MODE>
jdft_status launch_zpass_forward(const ChainGeom& g, const c_t<T>* colbuf, const c_t<T>* C, int ldc, c_t<T>* out,
                                 int ldo, int nb, const T* kin, T omega, T scale, const c_t<T>* tw_base,
                                 cudaStream_t st);
template <typename T>
jdft_status launch_plane_apply(const ChainGeom& g, c_t<T>* colbuf, const T* Vp, int nb, const c_t<T>* tw_base,
                               cudaStream_t st);
template <typename T>
jdft_status launch_plane_inverse_full(const ChainGeom& g, const c_t<T>* colbuf, c_t<T>* psi, T scale, int nb,
                                      const c_t<T>* tw_base, cudaStream_t st);
template <typename T>
jdft_status launch_plane_forward_full(const ChainGeom& g, const c_t<T>* psi, c_t<T>* colbuf, int nb,
                                      const c_t<T>* tw_base, cudaStream_t st);
// Register-FFT plane passes for the box shapes they are compiled for; they
// return JDFT_ERR_UNSUPPORTED (without launching) for other shapes.
template <typename T>
jdft_status launch_plane_apply_fast(const ChainGeom& g, c_t<T>* colbuf, const T* Vp, int nb, const c_t<T>* tw_base,
                                    cudaStream_t st);
jdft_status launch_plane_density_fast(const ChainGeom& g, const float2* colbuf, const double* f, double w,
                                      double* n_r, int nb, const float2* tw_base, cudaStream_t st);
// H plane pass and density of the same FP32 column buffer in one kernel (for
// the box shapes it is compiled for; JDFT_ERR_UNSUPPORTED otherwise):
// colbuf becomes the plane-pass output as in launch_plane_apply, and
// n_r += w sum_b f_b |psi_b|^2.
jdft_status launch_plane_apply_density_fast(const ChainGeom& g, float2* colbuf, const float* Vp, int nb,
                                            const double* f, double w, double* n_r, const float2* tw_base,
                                            cudaStream_t st);
// The same for two bands at a time with packed FP32 arithmetic (plane_pair.cu;
// JDFT_ERR_UNSUPPORTED, without launching, for shapes it is not compiled for).
jdft_status launch_plane_apply_density_pair(const ChainGeom& g, float2* colbuf, const float* Vp, int nb,
                                            const double* f, double w, double* n_r, const float2* tw_base,
                                            cudaStream_t st);
// The plane pass alone, two bands at a time (same contract as launch_plane_apply).
jdft_status launch_plane_apply_pair(const ChainGeom& g, float2* colbuf, const float* Vp, int nb,
                                    const float2* tw_base, cudaStream_t st);
// The plane pass of spinor rows: each pair (2p, 2p + 1) is one band's (up, down)
// components, multiplied by V 1 + M . sigma between the transforms; Mp holds
// M_x, M_y, M_z in Vp's permuted layout, one box after another (FP32).
// JDFT_ERR_UNSUPPORTED, without launching, for shapes it is not compiled for.
jdft_status launch_plane_apply_pair_spinor(const ChainGeom& g, float2* colbuf, const float* Vp, const float* Mp,
                                           int nb, const float2* tw_base, cudaStream_t st);
// One k-point (or cell on the same box) of a k-batched chain: its sphere
// maps, blocks, column buffer and first plane-pass item (kbatch.cu).
struct KJob {
    ChainGeom g;
    const float2* C;
    int ldc;
    float2* HC;
    int ldhc;
    float2* colbuf;    // nb x S2 x ncols
    const float* kin;  // (1/2)|k+G|^2, FP32
    int nb;
    int64_t item0;     // first (plane, band pair) item of this job in the batch
};
// The band-pair plane pass (no density) over all jobs in one launch, for the
// shapes the band-pair kernels are compiled for (JDFT_ERR_UNSUPPORTED
// otherwise).  gs: the jobs' geometries on the host (the launch checks the
// window on all of them); jobs: the same jobs on the device.
bool plane_pair_batch_supported(const ChainGeom& g);
jdft_status launch_plane_apply_pair_batch(const std::vector<ChainGeom>& gs, const KJob* jobs, int64_t items,
                                          const float* Vp, const float2* tw_base, cudaStream_t st);
// The z passes over all jobs (blockIdx.z = job), for the lengths the register
// line FFTs are compiled for (JDFT_ERR_UNSUPPORTED otherwise).  max_ncols,
// max_nb: the largest column and band counts over the jobs.
jdft_status launch_zpass_inverse_batch(const ChainGeom& g, const KJob* jobs, int njobs, int max_ncols, int max_nb,
                                       const float2* tw2, cudaStream_t st);
jdft_status launch_zpass_forward_batch(const ChainGeom& g, const KJob* jobs, int njobs, int max_ncols, int max_nb,
                                       float omega, float scale, const float2* tw2, cudaStream_t st);
// Workspace bytes of apply_H_density_with_split, and H C plus the density
// with an optional caller-made BF16 split of C for the projection (chain.cu).
size_t apply_H_density_workspace(const jdft_basis_s* b, int ik, int nb, jdft_prec prec, bool split_c);
jdft_status apply_H_density_with_split(jdft_basis_s* b, int ik, const void* C, int ldc, void* HC, int ldhc, int nb,
                                       const double* f, double* n_r, jdft_prec prec, cudaStream_t st,
                                       const void* Csplit);
// Register-FFT z passes for the lengths S2 they are compiled for (same
// contract as launch_zpass_*, tw2 = the length-S2 twiddle table); they return
// JDFT_ERR_UNSUPPORTED (without launching) for other lengths.
template <typename T>
jdft_status launch_zpass_inverse_fast(const ChainGeom& g, const c_t<T>* C, int ldc, c_t<T>* colbuf, int nb,
                                      const c_t<T>* tw2, cudaStream_t st);
template <typename T, int MODE>
jdft_status launch_zpass_forward_fast(const ChainGeom& g, const c_t<T>* colbuf, const c_t<T>* C, int ldc, c_t<T>* out,
                                      int ldo, int nb, const T* kin, T omega, T scale, const c_t<T>* tw2,
                                      cudaStream_t st);

template <typename T>
jdft_status launch_plane_density(const ChainGeom& g, const c_t<T>* colbuf, const double* f, double w, double* n_r,
                                 int nb, const c_t<T>* tw_base, cudaStream_t st);

}  // namespace jdft
