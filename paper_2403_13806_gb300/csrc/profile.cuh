// Per-launch timing of the library's own kernels (the tracing subsystem).
//
// While enabled with rs_profile_enable(1), every kernel launch of the library is bracketed
// by two CUDA events recorded on the launch's stream; rs_profile_read() then reports each
// launch's name and device time.  Launches on a stream that is being captured into a CUDA
// graph are not recorded.  Disabled (the default), a scope costs one branch.
#pragma once

#include <cuda_runtime.h>

namespace rs {
namespace prof {

bool enabled();
void begin(const char* name, cudaStream_t s);
void end(cudaStream_t s);

// Brackets the launches made in its lifetime.
struct Scope {
  bool on;
  cudaStream_t s;
  Scope(const char* name, cudaStream_t stream) : on(enabled()), s(stream) {
    if (on) begin(name, s);
  }
  ~Scope() {
    if (on) end(s);
  }
};

}  // namespace prof
}  // namespace rs
