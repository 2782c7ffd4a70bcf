// Set-up helpers shared by the observed-set entry points (glrm_api.cu), the
// entry checks (glrm_validate.cu) and the CSC build (glrm_transpose.cu).
// Internal to libglrm.
#pragma once

#include "glrm_handle.h"

namespace glrm {

// Entry checks of the CSR rows ptr[0] .. ptr[nseg] (ptr may point into the
// middle of a pointer array: entry indices are absolute): index range
// [0, other), strict column order, finite values, loss domains; flags as
// launch_check_entries, no digests.
cudaError_t launch_check_rows(const int32_t *ptr, const int32_t *idx, const void *val, int64_t nseg,
                              int64_t nnz_part, int prec, int64_t other, const LossSpec *loss, int *flag,
                              cudaStream_t st);

// The CSC build of glrm_transpose.cu in three steps, so that the counting can
// follow the CSR arrays piece by piece as they arrive: begin (count table),
// count over row blocks [b0, b1) (entries outside the column range are
// skipped, so it is safe before the checks' verdict), finish (prefixes,
// column pointers into h->csc.ptr and colptr_host, the placement, release).
// With A (FP32 / BF16 models: the set's dense table, lda floats per row, NaN
// outside the set) the placement reads the entries from its tiles, after
// a_ready (if given) on st.  colptr_host must live until st has passed the
// upload of the column pointers from it.
struct CscBuild {
    int RB = 0;        // rows per block (a multiple of 32)
    int64_t nblk = 0;  // row blocks
    int32_t *cnt = nullptr, *tot = nullptr;
};
cudaError_t csc_build_begin(glrm_s *h, CscBuild &b, cudaStream_t st);
cudaError_t csc_build_count(glrm_s *h, const CscBuild &b, int64_t b0, int64_t b1, cudaStream_t st);
cudaError_t csc_build_finish(glrm_s *h, CscBuild &b, std::vector<int32_t> &colptr_host, cudaStream_t st,
                             const float *A = nullptr, int64_t lda = 0, cudaEvent_t a_ready = nullptr);

}  // namespace glrm
