// Internal interfaces between the minimiser and the learned preconditioner.
#pragma once

#include "common.cuh"

namespace jdft {

// KG = K_theta(features) G for every coefficient (see jdft_mlp_t in jdft.h):
// features from kin (FP64 per plane wave), Tb (band kinetic energies) and the
// diagonal of Hs (complex128 nb x nb); bf is scratch for 3 nb floats.
template <typename T>
jdft_status mlp_precondition(jdft_mlp_t mlp, int npw, int nb, const c_t<T>* G, int ldg, c_t<T>* KG, int ldk,
                             const double* kin, const double* Tb, const double2* Hs, float* bf, cudaStream_t st);

// JDFT_ERR_TIMEOUT (and clears the record) if a bounded wait of the network's
// tensor-core kernels gave up since the last call; else JDFT_OK (mlp.cu).
jdft_status mlp_device_status();

}  // namespace jdft
