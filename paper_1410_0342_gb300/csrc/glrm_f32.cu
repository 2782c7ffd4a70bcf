// FP32 instantiation of the sweep, objective, gradient, imputation and ALS
// engines (compiled as its own translation unit so the precisions build in
// parallel).
#include "glrm_als.cuh"
#include "glrm_tiled.cuh"

template struct glrm::Engine<float>;

namespace glrm {
cudaError_t launch_build_runptr(const Orient &o, cudaStream_t st) { return launch_build_runptr_impl(o, st); }
}  // namespace glrm
