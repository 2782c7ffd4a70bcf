// Device-side validation of an observed set handed to glrm_set_observed:
// pointer arrays, index ranges and ordering, finite values, and that CSR and
// CSC list the same entries with bit-identical values.  Each check ORs a bit
// into a device flag word; nothing traps.
#include "glrm_handle.h"

namespace glrm {
namespace {

__global__ void validate_ptr_kernel(const int32_t *__restrict__ ptr, int64_t nseg, int64_t nnz,
                                    int *flag)
{
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s > nseg) return;
    if (s == 0 && ptr[0] != 0) atomicOr(flag, 1);
    if (s == nseg) {
        if ((int64_t)ptr[nseg] != nnz) atomicOr(flag, 1);
        return;
    }
    if (ptr[s] > ptr[s + 1]) atomicOr(flag, 1);
}

__device__ __forceinline__ bool finite_val(float v) { return isfinite(v); }
__device__ __forceinline__ bool finite_val(double v) { return isfinite(v); }
__device__ __forceinline__ long long bits(float v) { return __float_as_int(v); }
__device__ __forceinline__ long long bits(double v) { return __double_as_longlong(v); }

// One warp per segment: indices in range, strictly ascending, values finite.
template <class T>
__global__ void validate_idx_kernel(const int32_t *__restrict__ ptr, const int32_t *__restrict__ idx,
                                    const T *__restrict__ val, int64_t nseg, int64_t other, int *flag)
{
    const int lane = threadIdx.x & 31;
    const int64_t s = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (s >= nseg) return;
    const int b = ptr[s], e = ptr[s + 1];
    int f = 0;
    for (int q = b + lane; q < e; q += 32) {
        const int v = idx[q];
        if (v < 0 || v >= other) f |= 2;
        if (q > b && idx[q - 1] >= v) f |= 4;
        if (!finite_val(val[q])) f |= 8;
    }
    for (int o = 16; o > 0; o >>= 1) f |= __shfl_xor_sync(0xffffffffu, f, o);
    if (lane == 0 && f) atomicOr(flag, f);
}

// One warp per column: every CSC entry (i, j) found in CSR row i by binary
// search with the same value bits.  With equal counts and no duplicates on
// either side this makes the two a bijection.
template <class T>
__global__ void validate_cross_kernel(const int32_t *__restrict__ colptr,
                                      const int32_t *__restrict__ rowidx, const T *__restrict__ cval,
                                      int64_t n, const int32_t *__restrict__ rowptr,
                                      const int32_t *__restrict__ colidx, const T *__restrict__ rval,
                                      int *flag)
{
    const int lane = threadIdx.x & 31;
    const int64_t j = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (j >= n) return;
    int f = 0;
    for (int q = colptr[j] + lane; q < colptr[j + 1]; q += 32) {
        const int i = rowidx[q];
        int lo = rowptr[i], hi = rowptr[i + 1];
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (colidx[mid] < j) lo = mid + 1;
            else hi = mid;
        }
        if (lo >= rowptr[i + 1] || colidx[lo] != j) f |= 16;
        else if (bits(rval[lo]) != bits(cval[q])) f |= 32;
    }
    for (int o = 16; o > 0; o >>= 1) f |= __shfl_xor_sync(0xffffffffu, f, o);
    if (lane == 0 && f) atomicOr(flag, f);
}

// One warp per column: values inside the column loss's domain (Boolean
// losses: -1 or +1; ordinal hinge: an integer in 1..d).
template <class T>
__global__ void validate_domain_kernel(const int32_t *__restrict__ colptr, const T *__restrict__ cval,
                                       int64_t n, const LossSpec *__restrict__ loss, int *flag)
{
    const int lane = threadIdx.x & 31;
    const int64_t j = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (j >= n) return;
    const LossSpec sp = loss[j];
    int f = 0;
    for (int q = colptr[j] + lane; q < colptr[j + 1]; q += 32) {
        const T a = cval[q];
        if ((sp.kind == kLossHinge || sp.kind == kLossLogistic) && !(a == T(1) || a == T(-1))) f |= 64;
        if (sp.kind == kLossOrdinal && !(a >= T(1) && a <= T(sp.levels) && a == (T)(int)a)) f |= 64;
    }
    for (int o = 16; o > 0; o >>= 1) f |= __shfl_xor_sync(0xffffffffu, f, o);
    if (lane == 0 && f) atomicOr(flag, f);
}

}  // namespace

cudaError_t launch_validate_domain(const Orient &csc, int prec, const LossSpec *loss, int *flag,
                                   cudaStream_t st)
{
    const unsigned nb = (unsigned)((csc.nseg + 7) / 8);
    if (prec == GLRM_FP64)
        validate_domain_kernel<double><<<nb, 256, 0, st>>>(csc.ptr, (const double *)csc.val, csc.nseg,
                                                           loss, flag);
    else
        validate_domain_kernel<float><<<nb, 256, 0, st>>>(csc.ptr, (const float *)csc.val, csc.nseg,
                                                          loss, flag);
    return cudaGetLastError();
}

cudaError_t launch_validate_ptr(const int32_t *ptr, int64_t nseg, int64_t nnz, int *flag,
                                cudaStream_t st)
{
    validate_ptr_kernel<<<(unsigned)((nseg + 1 + 255) / 256), 256, 0, st>>>(ptr, nseg, nnz, flag);
    return cudaGetLastError();
}

cudaError_t launch_validate_idx(const int32_t *ptr, const int32_t *idx, const void *val, int prec,
                                int64_t nseg, int64_t other, int *flag, cudaStream_t st)
{
    const unsigned nb = (unsigned)((nseg + 7) / 8);
    if (prec == GLRM_FP64)
        validate_idx_kernel<double><<<nb, 256, 0, st>>>(ptr, idx, (const double *)val, nseg, other, flag);
    else
        validate_idx_kernel<float><<<nb, 256, 0, st>>>(ptr, idx, (const float *)val, nseg, other, flag);
    return cudaGetLastError();
}

cudaError_t launch_validate_cross(const Orient &csr, const Orient &csc, int prec, int *flag,
                                  cudaStream_t st)
{
    const unsigned nb = (unsigned)((csc.nseg + 7) / 8);
    if (prec == GLRM_FP64)
        validate_cross_kernel<double><<<nb, 256, 0, st>>>(csc.ptr, csc.idx, (const double *)csc.val,
                                                          csc.nseg, csr.ptr, csr.idx,
                                                          (const double *)csr.val, flag);
    else
        validate_cross_kernel<float><<<nb, 256, 0, st>>>(csc.ptr, csc.idx, (const float *)csc.val,
                                                         csc.nseg, csr.ptr, csr.idx,
                                                         (const float *)csr.val, flag);
    return cudaGetLastError();
}

}  // namespace glrm
