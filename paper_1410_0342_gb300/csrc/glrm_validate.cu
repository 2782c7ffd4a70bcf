// Device-side validation of an observed set handed to glrm_set_observed:
// pointer arrays, index ranges and ordering, finite values, and that CSR and
// CSC list the same entries with bit-identical values (64-bit digests).  Each
// check ORs a bit into a device flag word; nothing traps.
#include <algorithm>

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

// The entry checks below run one warp per piece of a segment: segment s is
// cut into `pieces` equal ranges of its entries (pieces is about the mean
// segment length / 1024, so a table with few long segments, such as the CSC
// of a tall table, still spreads over the whole GPU).  Returns false for a
// warp past the last piece; [b, e) is the warp's range, sb the segment start.
__device__ __forceinline__ bool piece_range(const int32_t *__restrict__ ptr, int64_t nseg, int pieces, int64_t &s,
                                            int &sb, int &b, int &e)
{
    const int64_t w = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    s = w / pieces;
    if (s >= nseg) return false;
    const int64_t pc = w - s * pieces;
    sb = ptr[s];
    const int se = ptr[s + 1];
    const int64_t len = se > sb ? se - sb : 0, per = (len + pieces - 1) / pieces;
    b = (int)(sb + std::min(len, pc * per));
    e = (int)(sb + std::min(len, (pc + 1) * per));
    return true;
}

// Indices in range, strictly ascending within the segment, values finite.
template <class T>
__global__ void validate_idx_kernel(const int32_t *__restrict__ ptr, const int32_t *__restrict__ idx,
                                    const T *__restrict__ val, int64_t nseg, int pieces, int64_t other, int *flag)
{
    const int lane = threadIdx.x & 31;
    int64_t s;
    int sb, b, e;
    if (!piece_range(ptr, nseg, pieces, s, sb, b, e)) return;
    int f = 0;
    for (int q = b + lane; q < e; q += 32) {
        const int v = idx[q];
        if (v < 0 || v >= other) f |= 2;
        if (q > sb && idx[q - 1] >= v) f |= 4;
        if (!finite_val(val[q])) f |= 8;
    }
    for (int o = 16; o > 0; o >>= 1) f |= __shfl_xor_sync(0xffffffffu, f, o);
    if (lane == 0 && f) atomicOr(flag, f);
}

// The CSR / CSC agreement check compares two order-free digests of each
// orientation's entries: the sum (mod 2^64) of H(i n + j) over its entries,
// and the sum of H(H(i n + j) ^ value bits), H being the splitmix64 finaliser
// (Steele, Lea and Flood, "Fast splittable pseudorandom number generators").
// Both orientations already passed the per-segment checks (counts, ranges,
// strict order, so no duplicates); equal index digests then mean the same
// entries and equal value digests the same values, except with probability
// about 2^-64 for a given mismatch.  One warp per segment, a grid-wide sum.
__device__ __forceinline__ unsigned long long mix64(unsigned long long z)
{
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// digest[0], digest[1]: index and value sums of this orientation (CSR: seg is
// the row; CSC: seg is the column).
template <class T>
__global__ void digest_kernel(const int32_t *__restrict__ ptr, const int32_t *__restrict__ idx,
                              const T *__restrict__ val, int64_t nseg, int pieces, int64_t n, bool rows,
                              unsigned long long *__restrict__ digest)
{
    const int lane = threadIdx.x & 31;
    int64_t s;
    int sb, qb, qe;
    if (!piece_range(ptr, nseg, pieces, s, sb, qb, qe)) return;
    unsigned long long a = 0, b = 0;
    for (int q = qb + lane; q < qe; q += 32) {
        const int64_t i = rows ? s : idx[q], j = rows ? idx[q] : s;
        const unsigned long long h = mix64((unsigned long long)(i * n + j));
        a += h;
        b += mix64(h ^ (unsigned long long)bits(val[q]));
    }
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    if (lane == 0) {
        atomicAdd(&digest[0], a);
        atomicAdd(&digest[1], b);
    }
}

__global__ void digest_compare_kernel(const unsigned long long *__restrict__ d, int *flag)
{
    if (d[0] != d[2]) atomicOr(flag, 16);
    else if (d[1] != d[3]) atomicOr(flag, 32);
}

// One warp per segment: values inside their column loss's domain (Boolean
// losses: -1 or +1; ordinal hinge: an integer in 1..d).  rows: the segments
// are rows and an entry's column is its index (entries with an index outside
// 0 .. n - 1 are skipped); else the segments are the n columns.  Non-finite
// values are skipped too: the index check reports them.
template <class T>
__global__ void validate_domain_kernel(const int32_t *__restrict__ ptr, const int32_t *__restrict__ idx,
                                       const T *__restrict__ val, int64_t nseg, int pieces, bool rows, int64_t n,
                                       const LossSpec *__restrict__ loss, int *flag)
{
    const int lane = threadIdx.x & 31;
    int64_t s;
    int sb, b, e;
    if (!piece_range(ptr, nseg, pieces, s, sb, b, e)) return;
    int f = 0;
    for (int q = b + lane; q < e; q += 32) {
        const int64_t j = rows ? (int64_t)idx[q] : s;
        const T a = val[q];
        if (j < 0 || j >= n || !finite_val(a)) continue;
        const LossSpec sp = loss[j];
        if ((sp.kind == kLossHinge || sp.kind == kLossLogistic) && !(a == T(1) || a == T(-1))) f |= 64;
        if (sp.kind == kLossOrdinal && !(a >= T(1) && a <= T(sp.levels) && a == (T)(int)a)) f |= 64;
    }
    for (int o = 16; o > 0; o >>= 1) f |= __shfl_xor_sync(0xffffffffu, f, o);
    if (lane == 0 && f) atomicOr(flag, f);
}

// Pieces per segment and blocks (eight warps each) for nnz entries over nseg segments.
int seg_pieces(int64_t nnz, int64_t nseg)
{
    const int64_t mean = nseg > 0 ? nnz / nseg : 0;
    return (int)std::max<int64_t>(1, std::min<int64_t>(1024, (mean + 1023) / 1024));
}
unsigned piece_blocks(int64_t nseg, int pieces) { return (unsigned)((nseg * pieces + 7) / 8); }

}  // namespace

cudaError_t launch_validate_domain(const Orient &o, bool rows, int64_t n, int64_t nnz, int prec,
                                   const LossSpec *loss, int *flag, cudaStream_t st)
{
    if (o.nseg == 0) return cudaSuccess;
    const int pc = seg_pieces(nnz, o.nseg);
    const unsigned nb = piece_blocks(o.nseg, pc);
    if (prec == GLRM_FP64)
        validate_domain_kernel<double><<<nb, 256, 0, st>>>(o.ptr, o.idx, (const double *)o.val, o.nseg, pc, rows,
                                                           n, loss, flag);
    else
        validate_domain_kernel<float><<<nb, 256, 0, st>>>(o.ptr, o.idx, (const float *)o.val, o.nseg, pc, rows,
                                                          n, loss, flag);
    return cudaGetLastError();
}

cudaError_t launch_validate_ptr(const int32_t *ptr, int64_t nseg, int64_t nnz, int *flag,
                                cudaStream_t st)
{
    validate_ptr_kernel<<<(unsigned)((nseg + 1 + 255) / 256), 256, 0, st>>>(ptr, nseg, nnz, flag);
    return cudaGetLastError();
}

cudaError_t launch_validate_idx(const int32_t *ptr, const int32_t *idx, const void *val, int prec,
                                int64_t nseg, int64_t other, int64_t nnz, int *flag, cudaStream_t st)
{
    if (nseg == 0) return cudaSuccess;
    const int pc = seg_pieces(nnz, nseg);
    const unsigned nb = piece_blocks(nseg, pc);
    if (prec == GLRM_FP64)
        validate_idx_kernel<double><<<nb, 256, 0, st>>>(ptr, idx, (const double *)val, nseg, pc, other, flag);
    else
        validate_idx_kernel<float><<<nb, 256, 0, st>>>(ptr, idx, (const float *)val, nseg, pc, other, flag);
    return cudaGetLastError();
}

// Digest of one orientation into d[0] (index sum) and d[1] (value sum); d
// zeroed by the caller.  n: the table's column count.
cudaError_t launch_digest(const Orient &o, bool rows, int64_t n, int64_t nnz, int prec, unsigned long long *d,
                          cudaStream_t st)
{
    if (o.nseg == 0) return cudaSuccess;
    const int pc = seg_pieces(nnz, o.nseg);
    const unsigned nb = piece_blocks(o.nseg, pc);
    if (prec == GLRM_FP64)
        digest_kernel<double><<<nb, 256, 0, st>>>(o.ptr, o.idx, (const double *)o.val, o.nseg, pc, n, rows, d);
    else
        digest_kernel<float><<<nb, 256, 0, st>>>(o.ptr, o.idx, (const float *)o.val, o.nseg, pc, n, rows, d);
    return cudaGetLastError();
}

// Flag 16 when the CSR and CSC index digests (d[0], d[2]) differ, else 32
// when the value digests (d[1], d[3]) do.
cudaError_t launch_digest_compare(const unsigned long long *d, int *flag, cudaStream_t st)
{
    digest_compare_kernel<<<1, 1, 0, st>>>(d, flag);
    return cudaGetLastError();
}

}  // namespace glrm
