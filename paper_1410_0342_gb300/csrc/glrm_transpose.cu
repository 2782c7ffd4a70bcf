// The CSC orientation of an observed set built on the device from its CSR
// orientation (glrm_set_observed_csr): a stable counting sort of the entries
// by column, so the rows of every column come out ascending and the result
// does not depend on scheduling.
//
// Rows are cut into nblk blocks of RB consecutive rows (at most about 4,096
// blocks, and n x nblk <= 2^26 counters).  Pass 1: per row block, the count
// of its entries in every column (one warp per row block, its rows in order;
// the columns of a row are distinct, so no two lanes touch the same counter;
// the block's n counters are contiguous).  Pass 2: per column, the exclusive
// prefix of its counts over the row blocks (one warp per column) and the
// column's total.  The column pointers are the exclusive prefix of the totals
// (host).  Pass 3: per row block, its rows in order, every entry placed at
// colptr[j] + the running count of column j in the block (32 rows merged at a
// time, so the stores for one column are coalesced).
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

// Exclusive prefix over the row blocks of one column's counts (in place), one
// warp per column, 32 blocks at a time with a carried total; tot[j] receives
// the column's count.
__global__ void tr_scan_kernel(int64_t n, int64_t nblk, int32_t *__restrict__ cnt, int32_t *__restrict__ tot)
{
    const int lane = threadIdx.x & 31;
    const int64_t j = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (j >= n) return;
    int32_t carry = 0;
    for (int64_t b0 = 0; b0 < nblk; b0 += 32) {
        const int64_t b = b0 + lane;
        const int32_t v = b < nblk ? cnt[b * n + j] : 0;
        int32_t incl = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        if (b < nblk) cnt[b * n + j] = carry + incl - v;
        carry += __shfl_sync(0xffffffffu, incl, 31);
    }
    if (lane == 0) tot[j] = carry;
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
    tr_count_kernel<<<(unsigned)((b1 - b0 + 7) / 8), 256, 0, st>>>(h->m, h->n, b.RB, b0, b1, h->csr.ptr, h->csr.idx,
                                                                    b.cnt);
    ++h->launches;
    return cudaGetLastError();
}

cudaError_t csc_build_finish(glrm_s *h, CscBuild &b, std::vector<int32_t> &cp, cudaStream_t st)
{
    const int64_t m = h->m, n = h->n, nnz = h->nnz;
    Orient &R = h->csr, &C = h->csc;
    cudaError_t e = cudaSuccess;
    if (nnz > 0) {
        tr_scan_kernel<<<(unsigned)((n + 7) / 8), 256, 0, st>>>(n, b.nblk, b.cnt, b.tot);
        e = cudaGetLastError();
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
    if (e == cudaSuccess && nnz > 0) {
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
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // the host table goes out of scope
    dfree(b.cnt, st);
    dfree(b.tot, st);
    return e;
}

cudaError_t build_csc_from_csr(glrm_s *h, cudaStream_t st)
{
    CscBuild b;
    cudaError_t e = csc_build_begin(h, b, st);
    if (e == cudaSuccess) e = csc_build_count(h, b, 0, b.nblk, st);
    std::vector<int32_t> cp;
    if (e == cudaSuccess) return csc_build_finish(h, b, cp, st);
    dfree(b.cnt, st);
    dfree(b.tot, st);
    return e;
}

}  // namespace glrm
