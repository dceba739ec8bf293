// Launch counting and optional per-kernel event timing (see profile.cu).
#pragma once

#include <cuda_runtime.h>

namespace jdft {

// Construct immediately before a kernel launch on `st`, destroy right after
// it: counts the launch and, while profiling is on, brackets it with events.
class Trace {
  public:
    Trace(const char* name, cudaStream_t st);
    ~Trace();
    Trace(const Trace&) = delete;
    Trace& operator=(const Trace&) = delete;

  private:
    cudaStream_t st_;
    int slot_;
};

}  // namespace jdft
