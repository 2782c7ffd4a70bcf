// Tables of multi-dimensional features (Section 6, eq. mpca): the embedding
// of categorical (one-vs-all) and ordinal (eq. ord-mpca) features into the
// Boolean columns of their blocks of Y, and their imputation.
//
// Both losses are sums of one hinge term per column of the feature's block:
//   categorical, labels 1..d:  L(u, a) = sum_l (1 - b_l u_l)_+,  b_l = +1 if l = a else -1;
//   ordinal, levels 1..d:      L(u, a) = sum_{l<d} (1 - b_l u_l)_+, b_l = +1 if a > l else -1.
// So the model of a feature table is exactly the scalar model of the table
// whose entry (i, j) is replaced by the d_j entries (i, first_j + l, b_l)
// with hinge loss, and every sweep kernel of the library fits it unchanged:
// the Y-step's segments are the block's columns, the X-step's row objective
// sums every column's term.  The kernels here build that table (CSR and
// CSC, both orders in one pass each) and decode labels from x_i Y_j.
#include "glrm_handle.h"

namespace glrm {
namespace {

__device__ __forceinline__ bool label_ok(double a, int levels)
{
    return a == floor(a) && a >= 1.0 && a <= (double)levels;
}

// The value of column l (0-based) of a block feature's embedding.
__device__ __forceinline__ double embed_value(const FeatDev &f, double a, int l)
{
    if (f.kind == kFeatCategorical) return (double)(l + 1) == a ? 1.0 : -1.0;
    return a > (double)(l + 1) ? 1.0 : -1.0;
}

// Per row: the number of embedded entries (sum of the widths of its features).
__global__ void embed_rowcount_kernel(int64_t m, const int32_t *__restrict__ rowptr,
                                      const int32_t *__restrict__ featidx, const FeatDev *__restrict__ F,
                                      int64_t *__restrict__ cnt)
{
    const int lane = threadIdx.x & 31;
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (i >= m) return;
    int64_t c = 0;
    for (int e = rowptr[i] + lane; e < rowptr[i + 1]; e += 32) c += F[featidx[e]].width;
#pragma unroll
    for (int o = 16; o; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if (lane == 0) cnt[i] = c;
}

// CSR of the embedded table: one warp per row, the row's entries 32 at a
// time; a lane's output offset is the warp's exclusive prefix of widths.
template <class T>
__global__ void embed_csr_kernel(int64_t m, const int32_t *__restrict__ rowptr, const int32_t *__restrict__ featidx,
                                 const T *__restrict__ val, const FeatDev *__restrict__ F,
                                 const int32_t *__restrict__ e_rowptr, int32_t *__restrict__ e_colidx,
                                 T *__restrict__ e_val, int *__restrict__ flag)
{
    const int lane = threadIdx.x & 31;
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (i >= m) return;
    int64_t base = e_rowptr[i];
    for (int e0 = rowptr[i]; e0 < rowptr[i + 1]; e0 += 32) {
        const int e = e0 + lane;
        const bool ok = e < rowptr[i + 1];
        FeatDev f{0, 0, 0, 0};
        double a = 0.0;
        if (ok) {
            f = F[featidx[e]];
            a = (double)val[e];
        }
        int w = ok ? f.width : 0;
        int incl = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        const int64_t out = base + incl - w;
        if (ok) {
            if (f.kind == kFeatScalar) {
                e_colidx[out] = f.first;
                e_val[out] = val[e];
            } else {
                if (!label_ok(a, f.levels)) atomicOr(flag, 1);
                for (int l = 0; l < w; ++l) {
                    e_colidx[out + l] = f.first + l;
                    e_val[out + l] = (T)embed_value(f, a, l);
                }
            }
        }
        base += __shfl_sync(0xffffffffu, incl, 31);
    }
}

// CSC of the embedded table: column first_j + l of a block holds the rows of
// feature j's column in the same order; thread = one entry of feature
// blockIdx.y (striding by gridDim.y over the features), writing its value
// into every column of the block.
template <class T>
__global__ void embed_csc_kernel(int64_t nf, const int32_t *__restrict__ colptr, const int32_t *__restrict__ rowidx,
                                 const T *__restrict__ cval, const FeatDev *__restrict__ F,
                                 const int32_t *__restrict__ e_colptr, int32_t *__restrict__ e_rowidx,
                                 T *__restrict__ e_cval)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    for (int64_t j = blockIdx.y; j < nf; j += gridDim.y) {
        const int b = colptr[j];
        if (q >= colptr[j + 1] - b) continue;
        const FeatDev f = F[j];
        const int32_t r = rowidx[b + q];
        if (f.kind == kFeatScalar) {
            const int64_t out = (int64_t)e_colptr[f.first] + q;
            e_rowidx[out] = r;
            e_cval[out] = cval[b + q];
            continue;
        }
        const double a = (double)cval[b + q];
        for (int l = 0; l < f.width; ++l) {
            const int64_t out = (int64_t)e_colptr[f.first + l] + q;
            e_rowidx[out] = r;
            e_cval[out] = (T)embed_value(f, a, l);
        }
    }
}

// Imputation of requested (row, feature) pairs: u_l = x_i . y_{first + l} in
// the model's precision; a scalar feature decodes as glrm_predict does, a
// categorical one to argmax_l u_l (the first of equal maxima; Section 6,
// "Categorical PCA"), an ordinal one to argmin_a L(u, a): with
// delta(u) = (1 - u)_+ - (1 + u)_+, L(u, a + 1) = L(u, a) + delta(u_a), so
// L(u, a) - L(u, 1) is the prefix sum S_a of delta (FP64) and the level is
// the first a with the smallest S_a.  Out-of-range pairs give NaN.
template <class T>
__global__ void decode_features_kernel(int64_t cnt, const int32_t *__restrict__ rows,
                                       const int32_t *__restrict__ feats, int64_t m, int32_t nf,
                                       const FeatDev *__restrict__ F, const LossSpec *__restrict__ loss,
                                       const T *__restrict__ X, const T *__restrict__ Yt, int k,
                                       T *__restrict__ out)
{
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= cnt) return;
    const int32_t i = rows[r], j = feats[r];
    if (i < 0 || i >= m || j < 0 || j >= nf) {
        out[r] = (T)nan("");
        return;
    }
    const FeatDev f = F[j];
    const T *x = X + (int64_t)i * k;
    auto dotu = [&](int c) {
        const T *y = Yt + (int64_t)c * k;
        T u = T(0);
        for (int q = 0; q < k; ++q) u = fma(x[q], y[q], u);
        return u;
    };
    if (f.kind == kFeatScalar) {
        out[r] = decode_value<T>(loss[f.first], dotu(f.first));
        return;
    }
    int best = 1;
    if (f.kind == kFeatCategorical) {
        T bu = dotu(f.first);
        for (int l = 1; l < f.width; ++l) {
            const T ul = dotu(f.first + l);
            if (ul > bu) {
                bu = ul;
                best = l + 1;
            }
        }
    } else {
        double S = 0.0, bestS = 0.0;
        for (int l = 0; l < f.width; ++l) {
            const double ul = (double)dotu(f.first + l);
            S += fmax(1.0 - ul, 0.0) - fmax(1.0 + ul, 0.0);
            if (S < bestS) {
                bestS = S;
                best = l + 2;
            }
        }
    }
    out[r] = (T)best;
}

__global__ void check_index_kernel(const int32_t *__restrict__ idx, int64_t n, int64_t bound, int *flag)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n && (idx[e] < 0 || idx[e] >= bound)) atomicOr(flag, 1);
}

}  // namespace

cudaError_t launch_check_index(const int32_t *idx, int64_t n, int64_t bound, int *flag, cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    check_index_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(idx, n, bound, flag);
    return cudaGetLastError();
}

cudaError_t launch_embed_rowcount(int64_t m, const int32_t *rowptr, const int32_t *featidx, const FeatDev *F,
                                  int64_t *cnt, cudaStream_t st)
{
    if (m == 0) return cudaSuccess;
    embed_rowcount_kernel<<<(unsigned)((m + 7) / 8), 256, 0, st>>>(m, rowptr, featidx, F, cnt);
    return cudaGetLastError();
}

cudaError_t launch_embed(int prec, int64_t m, int64_t nf, int64_t maxcnt, const int32_t *rowptr,
                         const int32_t *featidx, const void *val, const int32_t *colptr, const int32_t *rowidx,
                         const void *cval, const FeatDev *F, const int32_t *e_rowptr, int32_t *e_colidx, void *e_val,
                         const int32_t *e_colptr, int32_t *e_rowidx, void *e_cval, int *flag, cudaStream_t st)
{
    const unsigned gr = (unsigned)((m + 7) / 8);
    const dim3 gc((unsigned)std::max<int64_t>(1, (maxcnt + 255) / 256), (unsigned)std::min<int64_t>(nf, 65535));
    if (prec == GLRM_FP64) {
        if (m) embed_csr_kernel<double><<<gr, 256, 0, st>>>(m, rowptr, featidx, (const double *)val, F, e_rowptr,
                                                           e_colidx, (double *)e_val, flag);
        if (nf && maxcnt) embed_csc_kernel<double><<<gc, 256, 0, st>>>(nf, colptr, rowidx, (const double *)cval, F,
                                                                       e_colptr, e_rowidx, (double *)e_cval);
    } else {
        if (m) embed_csr_kernel<float><<<gr, 256, 0, st>>>(m, rowptr, featidx, (const float *)val, F, e_rowptr,
                                                          e_colidx, (float *)e_val, flag);
        if (nf && maxcnt) embed_csc_kernel<float><<<gc, 256, 0, st>>>(nf, colptr, rowidx, (const float *)cval, F,
                                                                      e_colptr, e_rowidx, (float *)e_cval);
    }
    return cudaGetLastError();
}

cudaError_t launch_decode_features(glrm_s *h, const FeatDev *F, int32_t nf, int64_t cnt, const int32_t *rows,
                                   const int32_t *feats, void *out)
{
    if (cnt == 0) return cudaSuccess;
    const unsigned g = (unsigned)((cnt + 255) / 256);
    if (h->prec == GLRM_FP64)
        decode_features_kernel<double><<<g, 256, 0, h->stream>>>(cnt, rows, feats, h->m, nf, F, h->loss_dev,
                                                                 (const double *)h->X, (const double *)h->Yt,
                                                                 h->k, (double *)out);
    else
        decode_features_kernel<float><<<g, 256, 0, h->stream>>>(cnt, rows, feats, h->m, nf, F, h->loss_dev,
                                                                (const float *)h->X, (const float *)h->Yt,
                                                                h->k, (float *)out);
    ++h->launches;
    return cudaGetLastError();
}

}  // namespace glrm
