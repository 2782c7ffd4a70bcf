// FP32 instantiation of the sweep, objective, gradient, imputation and ALS
// engines (compiled as its own translation unit so the precisions build in
// parallel).
#include "glrm_als.cuh"
#include "glrm_tiled.cuh"
#include "glrm_masked.cuh"

template struct glrm::Engine<float>;

namespace glrm {
cudaError_t launch_build_runptr(const Orient &o, cudaStream_t st) { return launch_build_runptr_impl(o, st); }
cudaError_t launch_mt_count(const Orient &o, int32_t *cnt, cudaStream_t st) { return mt_count(o, cnt, st); }
cudaError_t launch_mt_build(const Orient &o, int prec, cudaStream_t st)
{
    return prec == GLRM_FP64 ? mt_build<double>(o, st) : mt_build<float>(o, st);
}
}  // namespace glrm
