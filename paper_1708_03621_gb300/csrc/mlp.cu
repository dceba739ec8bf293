// Learned per-coefficient preconditioner (placeholder until the network kernels land).
#include "minimize.cuh"

namespace jdft {

template <typename T>
jdft_status mlp_precondition(jdft_mlp_t, int, int, const c_t<T>*, int, c_t<T>*, int, const double*, const double*,
                             const double2*, cudaStream_t) {
    return set_error(JDFT_ERR_UNSUPPORTED, "learned preconditioner not built yet");
}
template jdft_status mlp_precondition<double>(jdft_mlp_t, int, int, const double2*, int, double2*, int, const double*,
                                              const double*, const double2*, cudaStream_t);
template jdft_status mlp_precondition<float>(jdft_mlp_t, int, int, const float2*, int, float2*, int, const double*,
                                             const double*, const double2*, cudaStream_t);

}  // namespace jdft
