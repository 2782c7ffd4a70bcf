// Device-side validation of an observed set handed to glrm_set_observed:
// pointer arrays, index ranges and ordering, finite values, and that CSR and
// CSC list the same entries with bit-identical values (64-bit digests).  Each
// check ORs a bit into a device flag word; nothing traps.
#include <algorithm>

#include "glrm_setup.h"

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

// The CSR / CSC agreement check compares two order-free digests of each
// orientation's entries: the sum (mod 2^64) of H(i n + j) over its entries,
// and the sum of H(H(i n + j) ^ value bits), H being the splitmix64 finaliser
// (Steele, Lea and Flood, "Fast splittable pseudorandom number generators").
// Both orientations already passed the per-segment checks (counts, ranges,
// strict order, so no duplicates); equal index digests then mean the same
// entries and equal value digests the same values, except with probability
// about 2^-64 for a given mismatch.  One warp per segment piece, a grid-wide sum.
__device__ __forceinline__ unsigned long long mix64(unsigned long long z)
{
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__global__ void digest_compare_kernel(const unsigned long long *__restrict__ d, int *flag)
{
    if (d[0] != d[2]) atomicOr(flag, 16);
    else if (d[1] != d[3]) atomicOr(flag, 32);
}

// One pass over the entries of a segment piece: indices in range and
// strictly ascending within the segment, values finite (flags 2, 4, 8); with
// `loss`, each value inside its column loss's domain (Boolean losses: -1 or
// +1; ordinal hinge: an integer in 1..d; flag 64; entries whose index or
// value already failed are skipped); with `digest`, the orientation's two
// digests added into digest[0], digest[1].  rows: the segments are rows and
// an entry's index its column; else the segments are columns.  n: the
// table's column count; other: the index bound.
template <class T>
__global__ void check_entries_kernel(const int32_t *__restrict__ ptr, const int32_t *__restrict__ idx,
                                     const T *__restrict__ val, int64_t nseg, int pieces, int64_t other, bool rows,
                                     int64_t n, const LossSpec *__restrict__ loss, int *flag,
                                     unsigned long long *__restrict__ digest)
{
    const int lane = threadIdx.x & 31;
    int64_t s;
    int sb, qb, qe;
    if (!piece_range(ptr, nseg, pieces, s, sb, qb, qe)) return;
    int f = 0;
    unsigned long long da = 0, dv = 0;
    for (int q = qb + lane; q < qe; q += 32) {
        const int v = idx[q];
        const T a = val[q];
        const bool in_range = v >= 0 && v < other, fin = finite_val(a);
        if (!in_range) f |= 2;
        if (q > sb && idx[q - 1] >= v) f |= 4;
        if (!fin) f |= 8;
        if (loss && in_range && fin) {
            const LossSpec sp = loss[rows ? (int64_t)v : s];
            if ((sp.kind == kLossHinge || sp.kind == kLossLogistic) && !(a == T(1) || a == T(-1))) f |= 64;
            if (sp.kind == kLossOrdinal && !(a >= T(1) && a <= T(sp.levels) && a == (T)(int)a)) f |= 64;
        }
        if (digest) {
            const int64_t i = rows ? s : (int64_t)v, j = rows ? (int64_t)v : s;
            const unsigned long long h = mix64((unsigned long long)(i * n + j));
            da += h;
            dv += mix64(h ^ (unsigned long long)bits(a));
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        f |= __shfl_xor_sync(0xffffffffu, f, o);
        da += __shfl_xor_sync(0xffffffffu, da, o);
        dv += __shfl_xor_sync(0xffffffffu, dv, o);
    }
    if (lane == 0) {
        if (f) atomicOr(flag, f);
        if (digest) {
            atomicAdd(&digest[0], da);
            atomicAdd(&digest[1], dv);
        }
    }
}

// Pieces per segment and blocks (eight warps each) for nnz entries over nseg segments.
int seg_pieces(int64_t nnz, int64_t nseg)
{
    const int64_t mean = nseg > 0 ? nnz / nseg : 0;
    return (int)std::max<int64_t>(1, std::min<int64_t>(1024, (mean + 1023) / 1024));
}
unsigned piece_blocks(int64_t nseg, int pieces) { return (unsigned)((nseg * pieces + 7) / 8); }

}  // namespace

cudaError_t launch_validate_ptr(const int32_t *ptr, int64_t nseg, int64_t nnz, int *flag,
                                cudaStream_t st)
{
    validate_ptr_kernel<<<(unsigned)((nseg + 1 + 255) / 256), 256, 0, st>>>(ptr, nseg, nnz, flag);
    return cudaGetLastError();
}

cudaError_t launch_check_entries(const Orient &o, bool rows, int64_t other, int64_t n, int64_t nnz, int prec,
                                 const LossSpec *loss, int *flag, unsigned long long *digest, cudaStream_t st)
{
    if (o.nseg == 0) return cudaSuccess;
    const int pc = seg_pieces(nnz, o.nseg);
    const unsigned nb = piece_blocks(o.nseg, pc);
    if (prec == GLRM_FP64)
        check_entries_kernel<double><<<nb, 256, 0, st>>>(o.ptr, o.idx, (const double *)o.val, o.nseg, pc, other,
                                                         rows, n, loss, flag, digest);
    else
        check_entries_kernel<float><<<nb, 256, 0, st>>>(o.ptr, o.idx, (const float *)o.val, o.nseg, pc, other,
                                                        rows, n, loss, flag, digest);
    return cudaGetLastError();
}

cudaError_t launch_check_rows(const int32_t *ptr, const int32_t *idx, const void *val, int64_t nseg,
                              int64_t nnz_part, int prec, int64_t other, const LossSpec *loss, int *flag,
                              cudaStream_t st)
{
    if (nseg == 0) return cudaSuccess;
    const int pc = seg_pieces(nnz_part, nseg);
    const unsigned nb = piece_blocks(nseg, pc);
    if (prec == GLRM_FP64)
        check_entries_kernel<double><<<nb, 256, 0, st>>>(ptr, idx, (const double *)val, nseg, pc, other, true,
                                                         other, loss, flag, nullptr);
    else
        check_entries_kernel<float><<<nb, 256, 0, st>>>(ptr, idx, (const float *)val, nseg, pc, other, true, other,
                                                        loss, flag, nullptr);
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
