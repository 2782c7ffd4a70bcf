// The CSC orientation of an observed set built on the device from its CSR
// orientation (glrm_set_observed_csr): a stable counting sort of the entries
// by column, so the rows of every column come out ascending and the result
// does not depend on scheduling.
//
// Rows are cut into nblk blocks of RB consecutive rows (at most about 4,096
// blocks, and n x nblk <= 2^26 counters).  Pass 1: per row block, the count
// of its entries in every column (the block's n counters are contiguous; one
// CTA per row block with the counters in shared memory where n of them fit,
// else one warp per row block on global counters).  Pass 2: per column, the
// exclusive prefix of its counts over the row blocks (two levels over
// segments of row blocks) and the column's total.  The column pointers are
// the exclusive prefix of the totals (host).  Pass 3: per row block, its rows
// in order, every entry placed at colptr[j] + the running count of column j
// in the block: read from the set's dense table tile by tile when the dense
// form holds one, else 32 rows merged at a time; either way the stores for
// one column are coalesced.
#include <algorithm>
#include <climits>

#include "glrm_setup.h"

namespace glrm {
namespace {

__global__ void tr_count_kernel(int64_t m, int64_t n, int RB, int64_t b0, int64_t b1,
                                const int32_t *__restrict__ rowptr, const int32_t *__restrict__ colidx,
                                int32_t *__restrict__ cnt)
{
    const int lane = threadIdx.x & 31;
    const int64_t b = b0 + (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (b >= b1) return;
    int32_t *c = cnt + b * n;
    const int64_t r1 = std::min<int64_t>(m, (b + 1) * RB);
    for (int64_t i = b * RB; i < r1; ++i) {
        for (int e = rowptr[i] + lane; e < rowptr[i + 1]; e += 32) {
            const int32_t j = colidx[e];
            if (j >= 0 && j < n) c[j] += 1;  // unchecked input: never out of the table
        }
        __syncwarp();  // the next row may share a column with this one
    }
}

// Pass 1 with the counters in shared memory: one CTA per row block, its
// entries (contiguous in the CSR arrays) taken in any order, since a count
// does not depend on it; the n counts are written out whole, zeros included.
__global__ void tr_count_smem_kernel(int64_t m, int64_t n, int RB, int64_t b0, int64_t b1,
                                     const int32_t *__restrict__ rowptr, const int32_t *__restrict__ colidx,
                                     int32_t *__restrict__ cnt)
{
    extern __shared__ int32_t sc[];
    const int64_t b = b0 + blockIdx.x;
    if (b >= b1) return;  // the same on every thread of the CTA
    for (int64_t j = threadIdx.x; j < n; j += blockDim.x) sc[j] = 0;
    __syncthreads();
    const int64_t r0 = b * RB, r1 = std::min<int64_t>(m, (b + 1) * RB);
    const int64_t e0 = rowptr[r0], e1 = rowptr[r1];
    for (int64_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
        const int32_t j = __ldg(colidx + e);
        if (j >= 0 && j < n) atomicAdd(&sc[j], 1);  // unchecked input: never out of the table
    }
    __syncthreads();
    int32_t *c = cnt + b * n;
    for (int64_t j = threadIdx.x; j < n; j += blockDim.x) c[j] = sc[j];
}

// Pass 2 in two levels over S segments of L consecutive row blocks, one
// thread per (segment, column), so consecutive threads read consecutive
// counters: first each segment's sum per column; then each segment's start
// (the sum of the segments before it) carried through its blocks, the counts
// replaced in place by their exclusive prefix; the last segment's thread
// writes the column's total.
__global__ void tr_segsum_kernel(int64_t n, int64_t nblk, int64_t S, int64_t L, const int32_t *__restrict__ cnt,
                                 int32_t *__restrict__ seg)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= S * n) return;
    const int64_t s = t / n, j = t - s * n;
    const int64_t b0 = s * L, b1 = std::min<int64_t>(nblk, b0 + L);
    int32_t acc = 0;
#pragma unroll 4
    for (int64_t b = b0; b < b1; ++b) acc += cnt[b * n + j];
    seg[t] = acc;
}

__global__ void tr_segscan_kernel(int64_t n, int64_t nblk, int64_t S, int64_t L, int32_t *__restrict__ cnt,
                                  const int32_t *__restrict__ seg, int32_t *__restrict__ tot)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= S * n) return;
    const int64_t s = t / n, j = t - s * n;
    int32_t carry = 0;
    for (int64_t q = 0; q < s; ++q) carry += seg[q * n + j];
    if (s == S - 1) tot[j] = carry + seg[t];
    const int64_t b0 = s * L, b1 = std::min<int64_t>(nblk, b0 + L);
    // a batch of counts is loaded before any of it is overwritten, so the
    // loads are in flight together instead of each waiting for the last store
    constexpr int kBatch = 16;
    for (int64_t b = b0; b < b1; b += kBatch) {
        int32_t v[kBatch];
#pragma unroll
        for (int u = 0; u < kBatch; ++u) v[u] = b + u < b1 ? cnt[(b + u) * n + j] : 0;
#pragma unroll
        for (int u = 0; u < kBatch; ++u)
            if (b + u < b1) {
                cnt[(b + u) * n + j] = carry;
                carry += v[u];
            }
    }
}

// Pass 3 walks 32 rows at a time (lane = row) and merges their sorted column
// lists: at each step the smallest current column j and the mask of lanes
// holding it; those lanes write to consecutive slots colptr[j] + off + rank
// (rank = position in the mask), so the stores of a step are coalesced.
template <class T>
__global__ void tr_scatter_kernel(int64_t m, int64_t n, int RB, int64_t nblk, const int32_t *__restrict__ rowptr,
                                  const int32_t *__restrict__ colidx, const T *__restrict__ val,
                                  const int32_t *__restrict__ colptr, int32_t *__restrict__ off,
                                  int32_t *__restrict__ rowidx, T *__restrict__ cval)
{
    const int lane = threadIdx.x & 31;
    const uint32_t lt = (1u << lane) - 1u;
    const int64_t b = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (b >= nblk) return;
    int32_t *o = off + b * n;
    const int64_t r1 = std::min<int64_t>(m, (b + 1) * RB);
    for (int64_t i0 = b * RB; i0 < r1; i0 += 32) {
        const int64_t i = i0 + lane;
        int e = 0, ee = 0;
        if (i < r1) {
            e = rowptr[i];
            ee = rowptr[i + 1];
        }
        int32_t cur = e < ee ? colidx[e] : INT32_MAX;
        for (;;) {
            const int32_t j = __reduce_min_sync(0xffffffffu, cur);
            if (j == INT32_MAX) break;
            const uint32_t mask = __ballot_sync(0xffffffffu, cur == j);
            const int32_t base = colptr[j] + o[j];  // the same address on every lane: one load
            if (cur == j) {
                const int32_t p = base + __popc(mask & lt);
                rowidx[p] = (int32_t)i;
                cval[p] = val[e];
                ++e;
                cur = e < ee ? colidx[e] : INT32_MAX;
            }
            __syncwarp();
            if (lane == __ffs(mask) - 1) o[j] = base - colptr[j] + __popc(mask);
            __syncwarp();
        }
    }
}

// Pass 3 from the dense table of the same set (NaN at the cells outside it),
// when the dense form holds one: one warp per tile of 32 rows x 32 columns,
// staged in shared memory; per column, the rows holding an entry (a ballot
// over the column's 32 cells) go to consecutive slots colptr[j] + off[b][j] +
// rank, so the stores of a column are coalesced and its rows ascend.  Every
// read is a whole 128-byte row segment, so the pass streams the table once.
constexpr int kFillWarps = 8;
__global__ void __launch_bounds__(kFillWarps * 32)
tr_fill_dense_kernel(int64_t m, int64_t n, int RB, int64_t nblk, const float *__restrict__ A, int64_t lda,
                     const int32_t *__restrict__ colptr, const int32_t *__restrict__ off,
                     int32_t *__restrict__ rowidx, float *__restrict__ cval)
{
    __shared__ float tile[kFillWarps][32][33];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const uint32_t lt = (1u << lane) - 1u;
    const int64_t nch = (n + 31) / 32;
    const int64_t gw = (int64_t)blockIdx.x * kFillWarps + w;
    if (gw >= nblk * nch) return;  // whole warps
    const int64_t b = gw / nch, c0 = (gw - b * nch) * 32, j = c0 + lane;
    const int cols = (int)std::min<int64_t>(32, n - c0);
    int32_t slot = j < n ? colptr[j] + off[b * n + j] : 0;  // lane: column j's next slot
    const int64_t r1 = std::min<int64_t>(m, (b + 1) * RB);
    for (int64_t i0 = b * RB; i0 < r1; i0 += 32) {
#pragma unroll 8
        for (int r = 0; r < 32; ++r) {
            const int64_t i = i0 + r;
            tile[w][r][lane] = (i < r1 && j < n) ? A[i * lda + j] : __int_as_float(0x7fffffff);
        }
        __syncwarp();
        for (int c = 0; c < cols; ++c) {  // lane: row i0 + lane
            const float v = tile[w][lane][c];
            const bool has = v == v;
            const uint32_t mask = __ballot_sync(0xffffffffu, has);
            const int32_t base = __shfl_sync(0xffffffffu, slot, c);
            if (has) {
                const int32_t p = base + __popc(mask & lt);
                rowidx[p] = (int32_t)(i0 + lane);
                cval[p] = v;
            }
            if (lane == c) slot += __popc(mask);
        }
        __syncwarp();
    }
}

// Shared memory for pass 1's n counters per CTA, at most; wider tables count
// on global counters.
constexpr size_t kTrSmemMax = 160 * 1024;

}  // namespace

cudaError_t csc_build_begin(glrm_s *h, CscBuild &b, cudaStream_t st)
{
    const int64_t m = h->m, n = h->n;
    const int64_t budget = (int64_t)1 << 26;
    const int64_t rb = std::max<int64_t>(std::max<int64_t>(1, (m + 4095) / 4096), (m * n + budget - 1) / budget);
    b.RB = (int)((rb + 31) / 32 * 32);  // whole 32-row groups for the merge walk
    b.nblk = (m + b.RB - 1) / b.RB;
    cudaError_t e = dalloc_on(h, &b.cnt, (size_t)std::max<int64_t>(1, n * b.nblk) * sizeof(int32_t), st);
    if (e == cudaSuccess) e = dalloc_on(h, &b.tot, (size_t)std::max<int64_t>(1, n) * sizeof(int32_t), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(b.cnt, 0, (size_t)n * b.nblk * sizeof(int32_t), st);
    return e;
}

cudaError_t csc_build_count(glrm_s *h, const CscBuild &b, int64_t b0, int64_t b1, cudaStream_t st)
{
    if (b1 <= b0 || h->nnz == 0) return cudaSuccess;
    const size_t sm = (size_t)h->n * sizeof(int32_t);
    if (sm <= kTrSmemMax) {
        if (sm > 48 * 1024) {
            const cudaError_t e =
                cudaFuncSetAttribute(tr_count_smem_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
            if (e != cudaSuccess) return e;
        }
        tr_count_smem_kernel<<<(unsigned)(b1 - b0), 256, sm, st>>>(h->m, h->n, b.RB, b0, b1, h->csr.ptr,
                                                                   h->csr.idx, b.cnt);
    } else {
        tr_count_kernel<<<(unsigned)((b1 - b0 + 7) / 8), 256, 0, st>>>(h->m, h->n, b.RB, b0, b1, h->csr.ptr,
                                                                        h->csr.idx, b.cnt);
    }
    ++h->launches;
    return cudaGetLastError();
}

cudaError_t csc_build_finish(glrm_s *h, CscBuild &b, std::vector<int32_t> &cp, cudaStream_t st, const float *A,
                             int64_t lda, cudaEvent_t a_ready)
{
    const int64_t m = h->m, n = h->n, nnz = h->nnz;
    Orient &R = h->csr, &C = h->csc;
    cudaError_t e = cudaSuccess;
    if (nnz > 0) {
        // segments: at most 64, at most 2^22 segment sums
        const int64_t S = std::max<int64_t>(1, std::min<int64_t>({64, b.nblk, ((int64_t)1 << 22) / std::max<int64_t>(1, n)}));
        const int64_t L = (b.nblk + S - 1) / S;
        int32_t *seg = nullptr;
        e = dalloc_on(h, &seg, (size_t)(S * n) * sizeof(int32_t), st);
        if (e == cudaSuccess) {
            const unsigned g = (unsigned)((S * n + 255) / 256);
            tr_segsum_kernel<<<g, 256, 0, st>>>(n, b.nblk, S, L, b.cnt, seg);
            tr_segscan_kernel<<<g, 256, 0, st>>>(n, b.nblk, S, L, b.cnt, seg, b.tot);
            e = cudaGetLastError();
            dfree(seg, st);
            h->launches += 1;
        }
    } else {
        e = cudaMemsetAsync(b.tot, 0, (size_t)std::max<int64_t>(1, n) * sizeof(int32_t), st);
    }
    std::vector<int32_t> ht((size_t)n);
    cp.assign((size_t)n + 1, 0);
    if (e == cudaSuccess && n > 0)
        e = cudaMemcpyAsync(ht.data(), b.tot, (size_t)n * sizeof(int32_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) {
        for (int64_t j = 0; j < n; ++j) cp[(size_t)j + 1] = cp[(size_t)j] + ht[(size_t)j];
        e = cudaMemcpyAsync(C.ptr, cp.data(), cp.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st);
    }
    if (e == cudaSuccess && nnz > 0 && A && h->prec != GLRM_FP64) {
        if (a_ready) e = cudaStreamWaitEvent(st, a_ready, 0);
        const int64_t warps = b.nblk * ((n + 31) / 32);
        tr_fill_dense_kernel<<<(unsigned)((warps + kFillWarps - 1) / kFillWarps), kFillWarps * 32, 0, st>>>(
            m, n, b.RB, b.nblk, A, lda, C.ptr, b.cnt, C.idx, (float *)C.val);
        e = cudaGetLastError();
    } else if (e == cudaSuccess && nnz > 0) {
        const unsigned g = (unsigned)((b.nblk + 7) / 8);
        if (h->prec == GLRM_FP64)
            tr_scatter_kernel<double><<<g, 256, 0, st>>>(m, n, b.RB, b.nblk, R.ptr, R.idx, (const double *)R.val,
                                                         C.ptr, b.cnt, C.idx, (double *)C.val);
        else
            tr_scatter_kernel<float><<<g, 256, 0, st>>>(m, n, b.RB, b.nblk, R.ptr, R.idx, (const float *)R.val,
                                                        C.ptr, b.cnt, C.idx, (float *)C.val);
        e = cudaGetLastError();
    }
    h->launches += 2;
    // the column pointers went out from cp (the caller's) before this
    // returns; the tables are released in stream order
    dfree(b.cnt, st);
    dfree(b.tot, st);
    return e;
}

cudaError_t build_csc_from_csr(glrm_s *h, cudaStream_t st, const float *A, int64_t lda, cudaEvent_t a_ready)
{
    CscBuild b;
    cudaError_t e = csc_build_begin(h, b, st);
    if (e == cudaSuccess) e = csc_build_count(h, b, 0, b.nblk, st);
    std::vector<int32_t> cp;
    if (e == cudaSuccess) {
        e = csc_build_finish(h, b, cp, st, A, lda, a_ready);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // cp goes out of scope
        return e;
    }
    dfree(b.cnt, st);
    dfree(b.tot, st);
    return e;
}

}  // namespace glrm
