// FP32 instantiation of the sweep, objective, gradient, imputation and ALS
// engines (compiled as its own translation unit so the precisions build in
// parallel).
#include "glrm_als.cuh"
#include "glrm_tiled.cuh"
#include "glrm_masked.cuh"
#include "glrm_bf16.cuh"

template struct glrm::Engine<float>;

namespace glrm {
cudaError_t launch_build_runptr(const Orient &o, cudaStream_t st) { return launch_build_runptr_impl(o, st); }
cudaError_t launch_mt_count(const Orient &o, int32_t *cnt, cudaStream_t st) { return mt_count(o, cnt, st); }
cudaError_t launch_mt_build(const Orient &o, int prec, cudaStream_t st)
{
    return prec == GLRM_FP64 ? mt_build<double>(o, st) : mt_build<float>(o, st);
}
}  // namespace glrm

namespace glrm {
cudaError_t bf16_half_step_entry(glrm_s *h, bool xstep) { return bf16_half_step(h, xstep); }
cudaError_t launch_perm(const Orient &o, const Orient &other, cudaStream_t st)
{
    perm_kernel<<<blocks_for(o.nseg, 8), 256, 0, st>>>(o.nseg, o.ptr, o.idx, other.ptr, other.idx, o.perm);
    return cudaGetLastError();
}
}  // namespace glrm
