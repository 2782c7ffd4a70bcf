// Column statistics of the automatic loss scaling (Section 4.3, "Offsets and
// scaling"): for every column j with observed entries a_1 .. a_c,
//   mu_j     = the smallest minimiser of S_j(mu) = sum_e L_j(mu, a_e),
//   sigma2_j = S_j(mu_j) / (c - 1).
// S_j is convex for every loss kind here, so its smallest minimiser is the
// infimum of the points u with S_j'(u+) >= 0.  The kernels find it by
// bisection on the sign of the FP64 derivative sum g(u) = sum_e L_j'(u, a_e):
// a point with g(u) < 0 lies at or below every minimiser and one with
// g(u) >= 0 at or above the smallest one (the subgradient taken at a kink
// lies between the one-sided derivatives), so the bracket keeps the smallest
// minimiser (a sum within 1e-12 of the sum of its terms' magnitudes counts
// as zero, so that rounding does not decide the side on an interval of
// minimisers).  It starts at [min a - 32, max a + 32]; where S_j has no
// minimiser (a hinge or logistic column with one label) the result is the
// bracket end the derivative pushes towards.
#include "glrm_handle.h"

namespace glrm {
namespace {

constexpr double kStatBracket = 32.0;
constexpr int kStatMaxIters = 80;   // the bracket shrinks to 2^-62 of its width well before
constexpr int kDenseStatWarps = 32;  // warps per CTA of the dense-table kernel (32 columns per CTA)
// A derivative sum within this fraction of the sum of its terms' magnitudes
// counts as zero: on an interval of minimisers (a flat bottom) the rounding
// of the sum must not decide the side, so the bracket closes on its smallest
// point.
constexpr double kStatTieRel = 1e-12;

__device__ __forceinline__ double warp_min(double v)
{
#pragma unroll
    for (int o = 16; o; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

__device__ __forceinline__ double warp_max(double v)
{
#pragma unroll
    for (int o = 16; o; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

__device__ __forceinline__ double nan64() { return __longlong_as_double(0x7ff8000000000000LL); }

// One warp per column of the CSC arrays (grid-stride over columns).  Every
// lane ends each reduction with the same value (xor butterfly), so the
// bisection's branches are uniform over the warp.
template <class T>
__global__ void __launch_bounds__(256)
colstats_csc_kernel(int64_t n, const int32_t *__restrict__ ptr, const T *__restrict__ val,
                    const LossSpec *__restrict__ loss, double *__restrict__ mu, double *__restrict__ s2)
{
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t j = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; j < n; j += nw) {
        const int b = ptr[j], e = ptr[j + 1];
        if (b == e) {
            if (lane == 0) mu[j] = s2[j] = nan64();
            continue;
        }
        const LossSpec sp = loss[j];
        double lo = __longlong_as_double(0x7ff0000000000000LL), hi = -lo;
        for (int q = b + lane; q < e; q += 32) {
            const double a = (double)val[q];
            lo = fmin(lo, a);
            hi = fmax(hi, a);
        }
        lo = warp_min(lo) - kStatBracket;
        hi = warp_max(hi) + kStatBracket;
        const double tol = (hi - lo) * 0x1p-62;
        for (int it = 0; it < kStatMaxIters && hi - lo > tol; ++it) {
            const double mid = lo + 0.5 * (hi - lo);
            if (!(mid > lo && mid < hi)) break;
            double g = 0.0, ga = 0.0;
            for (int q = b + lane; q < e; q += 32) {
                double L;
                const double d = loss_deriv<double>(sp, mid, (double)val[q], L);
                g += d;
                ga += fabs(d);
            }
            g = warp_sum(g);
            ga = warp_sum(ga);
            if (g < -kStatTieRel * ga) lo = mid;
            else hi = mid;
        }
        double ls = 0.0;
        for (int q = b + lane; q < e; q += 32) {
            double L;
            loss_deriv<double>(sp, hi, (double)val[q], L);
            ls += L;
        }
        ls = warp_sum(ls);
        if (lane == 0) {
            mu[j] = hi;
            s2[j] = e - b > 1 ? ls / (double)(e - b - 1) : nan64();
        }
    }
}

// Block-wide sums / extrema (256 threads), the result on every thread in a
// fixed order (warp butterflies, then the 8 warp results in warp order).
__device__ __forceinline__ void block_sum2(double &a, double &b, double (*sh)[2])
{
    a = warp_sum(a);
    b = warp_sum(b);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();  // the previous use of sh is over
    if (lane == 0) {
        sh[w][0] = a;
        sh[w][1] = b;
    }
    __syncthreads();
    double x = 0.0, y = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) {
        x += sh[q][0];
        y += sh[q][1];
    }
    a = x;
    b = y;
}

__device__ __forceinline__ void block_minmax(double &lo, double &hi, double (*sh)[2])
{
    lo = warp_min(lo);
    hi = warp_max(hi);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) {
        sh[w][0] = lo;
        sh[w][1] = hi;
    }
    __syncthreads();
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) {
        lo = fmin(lo, sh[q][0]);
        hi = fmax(hi, sh[q][1]);
    }
}

// The same bisection with one CTA (256 threads) per column, for long columns
// (a tall table has few columns: a warp each would leave most of the GPU idle).
template <class T>
__global__ void __launch_bounds__(256)
colstats_csc_block_kernel(int64_t n, const int32_t *__restrict__ ptr, const T *__restrict__ val,
                          const LossSpec *__restrict__ loss, double *__restrict__ mu, double *__restrict__ s2)
{
    __shared__ double sh[8][2];
    for (int64_t j = blockIdx.x; j < n; j += gridDim.x) {
        const int b = ptr[j], e = ptr[j + 1];
        if (b == e) {
            if (threadIdx.x == 0) mu[j] = s2[j] = nan64();
            continue;
        }
        const LossSpec sp = loss[j];
        double lo = __longlong_as_double(0x7ff0000000000000LL), hi = -lo;
        for (int q = b + threadIdx.x; q < e; q += blockDim.x) {
            const double a = (double)val[q];
            lo = fmin(lo, a);
            hi = fmax(hi, a);
        }
        block_minmax(lo, hi, sh);
        lo -= kStatBracket;
        hi += kStatBracket;
        const double tol = (hi - lo) * 0x1p-62;
        for (int it = 0; it < kStatMaxIters && hi - lo > tol; ++it) {
            const double mid = lo + 0.5 * (hi - lo);
            if (!(mid > lo && mid < hi)) break;
            double g = 0.0, ga = 0.0;
            for (int q = b + threadIdx.x; q < e; q += blockDim.x) {
                double L;
                const double d = loss_deriv<double>(sp, mid, (double)val[q], L);
                g += d;
                ga += fabs(d);
            }
            block_sum2(g, ga, sh);
            if (g < -kStatTieRel * ga) lo = mid;
            else hi = mid;
        }
        double ls = 0.0, unused = 0.0;
        for (int q = b + threadIdx.x; q < e; q += blockDim.x) {
            double L;
            loss_deriv<double>(sp, hi, (double)val[q], L);
            ls += L;
        }
        block_sum2(ls, unused, sh);
        if (threadIdx.x == 0) {
            mu[j] = hi;
            s2[j] = e - b > 1 ? ls / (double)(e - b - 1) : nan64();
        }
    }
}

// Dense, fully observed table (m x lda FP32): one CTA per 32 consecutive
// columns, lane = column, the warps striding over rows (every load a
// coalesced 128-byte row segment).  The CTA's columns bisect in lockstep;
// a column whose bracket has closed keeps it.
__global__ void __launch_bounds__(kDenseStatWarps * 32)
colstats_dense_kernel(int64_t m, int64_t n, const float *__restrict__ A, int64_t lda,
                      const LossSpec *__restrict__ loss, double *__restrict__ mu, double *__restrict__ s2)
{
    __shared__ double red[kDenseStatWarps][33], red2[kDenseStatWarps][33];
    __shared__ double lo_s[32], hi_s[32], tol_s[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t j = (int64_t)blockIdx.x * 32 + lane;
    const bool col = j < n;
    const LossSpec sp = col ? loss[j] : LossSpec{kLossQuad, 0, 0.0};
    const float *Aj = A + (col ? j : 0);
    double lo = __longlong_as_double(0x7ff0000000000000LL), hi = -lo;
    if (col)
        for (int64_t r = w; r < m; r += kDenseStatWarps) {
            const double a = (double)Aj[r * lda];
            lo = fmin(lo, a);
            hi = fmax(hi, a);
        }
    red[w][lane] = lo;
    __syncthreads();
    if (w == 0) {
        double v = red[0][lane];
        for (int q = 1; q < kDenseStatWarps; ++q) v = fmin(v, red[q][lane]);
        lo_s[lane] = v - kStatBracket;
    }
    __syncthreads();
    red[w][lane] = hi;
    __syncthreads();
    if (w == 0) {
        double v = red[0][lane];
        for (int q = 1; q < kDenseStatWarps; ++q) v = fmax(v, red[q][lane]);
        hi_s[lane] = v + kStatBracket;
        tol_s[lane] = (hi_s[lane] - lo_s[lane]) * 0x1p-62;
    }
    __syncthreads();
    for (int it = 0; it < kStatMaxIters; ++it) {
        const double l = lo_s[lane], hh = hi_s[lane];
        const double mid = l + 0.5 * (hh - l);
        const bool live = col && hh - l > tol_s[lane] && mid > l && mid < hh;
        double g = 0.0, ga = 0.0;
        if (live)
            for (int64_t r = w; r < m; r += kDenseStatWarps) {
                double L;
                const double d = loss_deriv<double>(sp, mid, (double)Aj[r * lda], L);
                g += d;
                ga += fabs(d);
            }
        red[w][lane] = g;
        red2[w][lane] = ga;
        // every thread reads its column's bracket above; the barrier orders
        // those reads before warp 0 moves it
        if (!__syncthreads_or(live)) break;
        if (w == 0 && live) {
            double v = 0.0, va = 0.0;
            for (int q = 0; q < kDenseStatWarps; ++q) {
                v += red[q][lane];
                va += red2[q][lane];
            }
            if (v < -kStatTieRel * va) lo_s[lane] = mid;
            else hi_s[lane] = mid;
        }
        __syncthreads();
    }
    const double muj = hi_s[lane];
    double ls = 0.0;
    if (col)
        for (int64_t r = w; r < m; r += kDenseStatWarps) {
            double L;
            loss_deriv<double>(sp, muj, (double)Aj[r * lda], L);
            ls += L;
        }
    __syncthreads();
    red[w][lane] = ls;
    __syncthreads();
    if (w == 0 && col) {
        double v = 0.0;
        for (int q = 0; q < kDenseStatWarps; ++q) v += red[q][lane];
        mu[j] = muj;
        s2[j] = m > 1 ? v / (double)(m - 1) : nan64();
    }
}

}  // namespace

cudaError_t launch_column_stats(glrm_s *h, double *mu, double *s2)
{
    if (h->n == 0) return cudaSuccess;
    if (h->dn.on && !h->dn.missing) {
        colstats_dense_kernel<<<(unsigned)((h->n + 31) / 32), kDenseStatWarps * 32, 0, h->stream>>>(
            h->m, h->n, h->dn.A, h->dn.lda, h->loss_dev, mu, s2);
    } else {
        int sms = 0;
        cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device);
        if (e != cudaSuccess) return e;
        if (h->nnz >= 2048 * h->n) {  // long columns: a CTA per column
            const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(h->n, (int64_t)sms * 8));
            if (h->prec == GLRM_FP64)
                colstats_csc_block_kernel<double><<<grid, 256, 0, h->stream>>>(
                    h->n, h->csc.ptr, (const double *)h->csc.val, h->loss_dev, mu, s2);
            else
                colstats_csc_block_kernel<float><<<grid, 256, 0, h->stream>>>(
                    h->n, h->csc.ptr, (const float *)h->csc.val, h->loss_dev, mu, s2);
            ++h->launches;
            return cudaGetLastError();
        }
        const int64_t want = (h->n + 7) / 8;  // 8 warps (columns) per CTA
        const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)sms * 8));
        if (h->prec == GLRM_FP64)
            colstats_csc_kernel<double><<<grid, 256, 0, h->stream>>>(h->n, h->csc.ptr, (const double *)h->csc.val,
                                                                     h->loss_dev, mu, s2);
        else
            colstats_csc_kernel<float><<<grid, 256, 0, h->stream>>>(h->n, h->csc.ptr, (const float *)h->csc.val,
                                                                    h->loss_dev, mu, s2);
    }
    ++h->launches;
    return cudaGetLastError();
}

}  // namespace glrm
