// An objective evaluation that allocates nothing on the device.
//
// It is for callers that cannot call cudaMalloc at the point where they need
// the objective: code running while a CUDA graph is being captured into
// (allocation calls are not allowed inside a capture), a host that hands all
// device memory to its own pool allocator up front, or a tight loop that must
// not touch the allocator at all.  Such a caller passes its own Omega (CSR),
// factors and loss table, and the library uses only the scratch array below,
// which lives in the library's device image: every GPU that loads the library
// holds it until the process exits.
//
// The work matches glrm_objective_at (a per-row loss sum plus the
// regularisers, reduced in FP64) but without a handle.  The per-row and
// per-column terms are written to the scratch array, one slot each, and a
// single block then adds the slots in a fixed order, so the result does not
// depend on scheduling.  Every call overwrites the slots it uses, so nothing
// needs clearing between calls; calls that overlap on the GPU (two streams, or
// no ordering between them) share the array and race.
#include <cuda_runtime.h>

#include <cmath>
#include <cstddef>
#include <mutex>

#include "glrm.h"
#include "glrm_device.cuh"

namespace {

using glrm::LossSpec;

// The caller's glrm_loss array is read in place as the kernels' LossSpec.
static_assert(sizeof(glrm_loss) == sizeof(LossSpec), "glrm_loss and LossSpec differ in size");
static_assert(offsetof(glrm_loss, kind) == offsetof(LossSpec, kind), "kind offset differs");
static_assert(offsetof(glrm_loss, levels) == offsetof(LossSpec, levels), "levels offset differs");
static_assert(offsetof(glrm_loss, param) == offsetof(LossSpec, param), "param offset differs");

// Rows plus columns the scratch array can hold (8 MiB of doubles).
constexpr int64_t kNoAllocMaxTerms = GLRM_NOALLOC_MAX_TERMS;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_noalloc_terms[kNoAllocMaxTerms];

std::mutex g_setup_mutex;
double *g_terms_ptr[kMaxDevices] = {};

// A loss descriptor the sweep accepts: a known kind, a positive finite Huber
// threshold, a quantile alpha in (0, 1), at least two ordinal levels.
__device__ __forceinline__ bool loss_ok(const LossSpec &L)
{
    switch (L.kind) {
    case glrm::kLossQuad:
    case glrm::kLossHinge:
    case glrm::kLossLogistic:
        return true;
    case glrm::kLossL1:
        return true;
    case glrm::kLossHuber:
        return L.param > 0.0 && L.param <= 1e300;
    case glrm::kLossQuantile:
        return L.param > 0.0 && L.param < 1.0;
    case glrm::kLossOrdinal:
        return L.levels >= 2;
    default:
        return false;
    }
}

// Warp per row: sum of the row's losses plus r(x_i); then one thread per
// column: rt(y_j).  A row whose entry range leaves [0, nnz] or runs
// backwards, a column index outside [0, n), or a malformed loss descriptor
// makes the row's term NaN (so the result is NaN); nothing is read out of
// range.
__global__ void noalloc_terms_kernel(int64_t m, int64_t n, int k, int64_t nnz,
                                     const int32_t *__restrict__ rowptr,
                                     const int32_t *__restrict__ colidx, const float *__restrict__ val,
                                     const LossSpec *__restrict__ loss, int rxk, float rxw, int ryk,
                                     float ryw, const float *__restrict__ X,
                                     const float *__restrict__ Yt, double *__restrict__ terms)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = warp; i < m; i += nwarps) {
        const float *x = X + i * k;
        double s = 0.0;
        const int64_t eb = rowptr[i], ee = rowptr[i + 1];
        bool bad = eb < 0 || ee < eb || ee > nnz;
        const int64_t lo = bad ? 0 : eb, hi = bad ? 0 : ee;
        for (int64_t e = lo + lane; e < hi; e += 32) {
            const int j = colidx[e];
            if (j < 0 || j >= n || !loss_ok(loss[j])) {
                bad = true;
                continue;
            }
            const float *y = Yt + (int64_t)j * k;
            float u = 0.f;
            for (int c = 0; c < k; ++c) u = fmaf(x[c], y[c], u);
            float L;
            glrm::loss_deriv<float>(loss[j], u, val[e], L);
            s += (double)L;
        }
        if (lane < k)
            for (int c = lane; c < k; c += 32) s += glrm::reg1<float>(rxk, rxw, x[c]);
        s = glrm::warp_sum(s);
        bad = __any_sync(0xffffffffu, bad);
        if (lane == 0) terms[i] = bad ? (double)NAN : s;
    }
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
    for (int64_t j = tid; j < n; j += nthreads) {
        double r = 0.0;
        for (int c = 0; c < k; ++c) r += glrm::reg1<float>(ryk, ryw, Yt[j * k + c]);
        terms[m + j] = r;
    }
}

// One block: thread t adds slots t, t + 256, ... in order, then a fixed tree.
__global__ void __launch_bounds__(256) noalloc_sum_kernel(const double *__restrict__ terms,
                                                          int64_t count, double *__restrict__ out)
{
    __shared__ double sh[256];
    double v = 0.0;
    for (int64_t q = threadIdx.x; q < count; q += 256) v += terms[q];
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sh[0];
}

// Device address of the scratch array on the current device, looked up once
// per device (cudaGetSymbolAddress must run with that device current).
cudaError_t terms_ptr(double **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_terms_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_terms);
        if (e != cudaSuccess) return e;
        g_terms_ptr[dev] = static_cast<double *>(p);
    }
    *out = g_terms_ptr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" int glrm_objective_noalloc(int64_t m, int64_t n, int32_t k, int64_t nnz,
                                      const int32_t *csr_rowptr_dev, const int32_t *csr_colidx_dev,
                                      const float *csr_val_dev, const glrm_loss *col_loss_dev,
                                      int32_t rx_kind, double rx_weight, int32_t ry_kind,
                                      double ry_weight, const float *X_dev, const float *Yt_dev,
                                      double *out_dev, void *stream)
{
    if (m < 1 || n < 1 || k < 1 || k > 64) return GLRM_ERR_RANGE;
    if (m + n > kNoAllocMaxTerms) return GLRM_ERR_RANGE;
    if (nnz < 0 || nnz >= (int64_t(1) << 31)) return GLRM_ERR_RANGE;
    if (!csr_rowptr_dev || !col_loss_dev || !X_dev || !Yt_dev || !out_dev) return GLRM_ERR_ARG;
    if (nnz > 0 && (!csr_colidx_dev || !csr_val_dev)) return GLRM_ERR_ARG;
    if (reinterpret_cast<uintptr_t>(col_loss_dev) % 16 != 0) return GLRM_ERR_ARG;
    for (int r : {rx_kind, ry_kind})
        if (r < GLRM_REG_ZERO || r > GLRM_REG_NONNEG) return GLRM_ERR_ARG;
    for (double w : {rx_weight, ry_weight})
        if (!std::isfinite(w) || w < 0.0) return GLRM_ERR_ARG;
    double *terms = nullptr;
    if (terms_ptr(&terms) != cudaSuccess) return GLRM_ERR_CUDA;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int sms = 0;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return GLRM_ERR_CUDA;
    noalloc_terms_kernel<<<sms * 4, 256, 0, st>>>(
        m, n, k, nnz, csr_rowptr_dev, csr_colidx_dev, csr_val_dev,
        reinterpret_cast<const LossSpec *>(col_loss_dev), rx_kind, (float)rx_weight, ry_kind,
        (float)ry_weight, X_dev, Yt_dev, terms);
    if (cudaGetLastError() != cudaSuccess) return GLRM_ERR_CUDA;
    noalloc_sum_kernel<<<1, 256, 0, st>>>(terms, m + n, out_dev);
    if (cudaGetLastError() != cudaSuccess) return GLRM_ERR_CUDA;
    return GLRM_OK;
}
