// FP32 staged (fused / blocked) half-step, and the blocked path's run table.
#include "glrm_tiled.cuh"

template cudaError_t glrm::Engine<float>::tiled_half_step(glrm_s *h, bool xstep);

namespace glrm {
cudaError_t launch_build_runptr(const Orient &o, cudaStream_t st) { return launch_build_runptr_impl(o, st); }
}  // namespace glrm
