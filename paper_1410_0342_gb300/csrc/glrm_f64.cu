// FP64 instantiation of the sweep, objective, gradient, imputation and ALS
// engines (compiled as its own translation unit so the precisions build in
// parallel).
#include "glrm_als.cuh"
#include "glrm_tiled.cuh"
#include "glrm_masked.cuh"

template struct glrm::Engine<double>;

namespace glrm {
// the BF16 form exists for FP32 models only (glrm_f32.cu)
}  // namespace glrm
