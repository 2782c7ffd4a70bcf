// Masked-tile form of the proximal-gradient half-step (Section 7.2 of Udell
// et al., "Generalized Low Rank Models") for tables whose observed set is
// dense enough that 32 consecutive segments (rows in the X-step, columns in
// the Y-step) share most of their other-indices.
//
// Layout (built once from CSR / CSC at set-up): segments are grouped in tiles
// of 32; for each tile, the union of its segments' other-indices in ascending
// order is stored as pairs (index j, 32-bit mask of the lanes whose segment
// holds j), and the tile's values are stored in (j, lane) order.  A segment's
// entries, hence its values, are exactly those of the CSR/CSC list: only
// their order changes.
//
// Kernels: a warp owns a tile, lane l owns segment 32t + l and keeps its
// factor, gradient and objective in registers.  The warp walks the pairs; for
// each j it loads the other factor's row j once from shared memory as a
// broadcast (no bank conflicts), and every lane in the mask applies the entry
// to its own segment.  The loss branch is warp-uniform in the X-step (one
// column per pair).  Values stream through a per-warp ring of shared-memory
// chunks filled by TMA bulk copies; pair lists are read in coalesced batches
// of 32.
#pragma once

#include "glrm_tiled.cuh"

namespace glrm {

constexpr int kRingSlots = kRingSlotsHost;

// ------------------------------------------------------------ construction

// Pairs per tile: a 32-way merge of the tile's sorted index lists.
static __global__ void mt_count_kernel(int64_t nseg, const int32_t *__restrict__ ptr,
                                const int32_t *__restrict__ idx, int32_t *__restrict__ cnt)
{
    const int lane = threadIdx.x & 31;
    const int64_t t = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int64_t ntiles = (nseg + 31) / 32;
    if (t >= ntiles) return;
    const int64_t s = t * 32 + lane;
    int p = 0, e = 0;
    if (s < nseg) {
        p = ptr[s];
        e = ptr[s + 1];
    }
    int nxt = p < e ? idx[p] : INT_MAX;
    int c = 0;
    for (;;) {
        const int j = __reduce_min_sync(0xffffffffu, nxt);
        if (j == INT_MAX) break;
        ++c;
        if (nxt == j) {
            ++p;
            nxt = p < e ? idx[p] : INT_MAX;
        }
    }
    if (lane == 0) cnt[t] = c;
}

// The same count from a bitmap of the other dimension in shared memory (one
// CTA per tile, nother bits): every entry of the tile's 32 segments (one
// contiguous range) sets its index's bit, the count is the number of bits
// set.  Its cost is the tile's entries plus nother / 32 words, where the
// merge above takes one dependent step per distinct index.  Indices were
// validated to lie in [0, nother); any other is skipped so the bitmap is never
// left.
static __global__ void mt_count_bitmap_kernel(int64_t nseg, int64_t nother, const int32_t *__restrict__ ptr,
                                              const int32_t *__restrict__ idx, int32_t *__restrict__ cnt)
{
    extern __shared__ uint32_t bits[];
    const int64_t t = blockIdx.x;
    const int64_t words = (nother + 31) / 32;
    for (int64_t w = threadIdx.x; w < words; w += blockDim.x) bits[w] = 0u;
    __syncthreads();
    const int64_t s0 = t * 32, s1 = std::min<int64_t>(nseg, s0 + 32);
    const int64_t e0 = ptr[s0], e1 = ptr[s1];
    for (int64_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
        const int32_t j = __ldg(idx + e);
        if (j >= 0 && j < nother) atomicOr(&bits[j >> 5], 1u << (j & 31));
    }
    __syncthreads();
    int c = 0;
    for (int64_t w = threadIdx.x; w < words; w += blockDim.x) c += __popc(bits[w]);
    c = __reduce_add_sync(0xffffffffu, c);
    __shared__ int part[32];
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        int tot = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += part[w];
        cnt[t] = tot;
    }
}

// Emit pairs and tile-ordered values.  A tile's pair list is cut into units
// of at most P pairs (unit q of tile t starts at pair tptr[t] + q P); the
// value offset where each unit starts goes to uvoff[ubeg[t] + q].
template <class T>
__global__ void mt_emit_kernel(int64_t nseg, const int32_t *__restrict__ ptr,
                               const int32_t *__restrict__ idx, const T *__restrict__ val,
                               const int32_t *__restrict__ tptr, const int32_t *__restrict__ ubeg,
                               int P, int32_t *__restrict__ tidx, uint32_t *__restrict__ tmask,
                               T *__restrict__ tval, int32_t *__restrict__ uvoff)
{
    const int lane = threadIdx.x & 31;
    const int64_t t = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int64_t ntiles = (nseg + 31) / 32;
    if (t >= ntiles) return;
    const int64_t s = t * 32 + lane;
    int p = 0, e = 0;
    if (s < nseg) {
        p = ptr[s];
        e = ptr[s + 1];
    }
    int nxt = p < e ? idx[p] : INT_MAX;
    const int pair0 = tptr[t];
    int pair = pair0;
    int voff = ptr[t * 32];
    const uint32_t lt = (1u << lane) - 1u;
    for (;;) {
        const int j = __reduce_min_sync(0xffffffffu, nxt);
        if (j == INT_MAX) break;
        if (lane == 0 && (pair - pair0) % P == 0) uvoff[ubeg[t] + (pair - pair0) / P] = voff;
        const uint32_t m = __ballot_sync(0xffffffffu, nxt == j);
        if (lane == 0) {
            tidx[pair] = j;
            tmask[pair] = m;
        }
        if (nxt == j) {
            tval[voff + __popc(m & lt)] = val[p];
            ++p;
            nxt = p < e ? idx[p] : INT_MAX;
        }
        voff += __popc(m);
        ++pair;
    }
}

// ------------------------------------------------------------ value stream

// Sequential reader of a contiguous range of values through a ring of
// kRingSlots chunks of C values in shared memory (one mbarrier per slot),
// filled by TMA bulk copies.  Offsets are relative to the 16-byte aligned
// start of the range; since the ring holds a power-of-two number of values and
// chunk q lives in slot q mod kRingSlots, offset o sits at ring[o mod size].
template <class T>
struct Ring {
    static constexpr int C = kRingBytes / (int)sizeof(T);  // values per chunk
    static constexpr int N = C * kRingSlots;                // values in the ring
    static_assert((N & (N - 1)) == 0, "ring size must be a power of two");
    T *buf;
    uint64_t *bars;
    const T *src;
    uint32_t hi;       // aligned end of the range (offset)
    uint32_t issued;   // offsets < issued have been requested
    uint32_t ready;    // offsets < ready have landed
    uint32_t freed;    // offsets < freed may be overwritten
    unsigned phases;   // parity bit per slot
    bool ok;

    __device__ __forceinline__ void init(T *b, uint64_t *br)
    {
        buf = b;
        bars = br;
        phases = 0;
        issued = ready = freed = hi = 0;
        ok = true;
    }

    __device__ __forceinline__ void issue_one()
    {
        const int slot = (int)((issued / C) % kRingSlots);
        const uint32_t n = min((uint32_t)C, hi - issued);
        __syncwarp();
        if ((threadIdx.x & 31) == 0) {
            fence_proxy_async();
            mbar_expect_tx(bars + slot, n * (unsigned)sizeof(T));
            bulk_g2s(buf + (size_t)slot * C, src + issued, n * (unsigned)sizeof(T), bars + slot);
        }
        issued += C;
    }

    // Start reading global values [start, end); returns the offset of start.
    __device__ __forceinline__ uint32_t begin(const T *s, int64_t start, int64_t end)
    {
        const int64_t base = start & ~(int64_t)3;
        src = s + base;
        hi = end > start ? (uint32_t)(((end + 3) & ~(int64_t)3) - base) : 0u;
        issued = ready = freed = 0;
        while (issued < hi && issued < (uint32_t)N) issue_one();
        return (uint32_t)(start - base);
    }

    // Make offsets < e readable (bounded waits).
    __device__ __forceinline__ void ensure(uint32_t e)
    {
        while (ready < e && ready < hi) {
            const int slot = (int)((ready / C) % kRingSlots);
            bool w = mbar_wait_bounded(bars + slot, (phases >> slot) & 1u);
            if (!w) w = mbar_wait_bounded(bars + slot, (phases >> slot) & 1u);
            ok = __all_sync(0xffffffffu, ok && w);  // warp-uniform verdict
            phases ^= 1u << slot;
            ready += C;
        }
    }

    // Offsets < c are consumed: recycle their chunks for the next requests.
    __device__ __forceinline__ void release(uint32_t c)
    {
        while (freed + C <= c && freed + C <= ready) {
            freed += C;
            if (issued < hi) issue_one();
        }
    }

    __device__ __forceinline__ T at(uint32_t o) const { return buf[o & (uint32_t)(N - 1)]; }

    // Wait for every requested chunk so that no copy targets the ring after
    // the range is left.
    __device__ __forceinline__ void drain()
    {
        while (ready < issued) {
            const int slot = (int)((ready / C) % kRingSlots);
            bool w = mbar_wait_bounded(bars + slot, (phases >> slot) & 1u);
            ok = __all_sync(0xffffffffu, ok && w);
            phases ^= 1u << slot;
            ready += C;
        }
        freed = ready;
    }
};

// Loss and derivative with the kind fixed at compile time when KIND >= 0.
template <class T, int KIND, class LS>
__device__ __forceinline__ T loss_k(const LS &s, T u, T a, T &L)
{
    if constexpr (KIND < 0) {
        return loss_deriv<T>(s, u, a, L);
    } else {
        LS q = s;
        q.kind = KIND;
        return loss_deriv<T>(q, u, a, L);
    }
}

// Process `cnt` pairs of a batch (indices / masks in lane q of myj / mym).
// Every lane runs the same instructions; lanes outside a pair's mask get zero
// weight, so nothing diverges.  FULL: row j of the resident factor; else row
// q of the batch buffer.
template <class T, int K, bool XSTEP, bool GRAD, int KIND, bool FULL>
__device__ __forceinline__ void mt_batch2(int cnt, int myj, uint32_t mym, uint32_t &voff,
                                          const Ring<T> &rg, const T *rows, const LossOf<T> *Ls,
                                          const LossOf<T> &segspec, const Vec<T, K> &f, Vec<T, K> &g,
                                          T &lsum)
{
    const int lane = threadIdx.x & 31;
    const uint32_t lt = (1u << lane) - 1u;
#pragma unroll 2
    for (int q = 0; q < cnt; ++q) {
        const int j = __shfl_sync(0xffffffffu, myj, q);
        const uint32_t m = __shfl_sync(0xffffffffu, mym, q);
        const bool act = (m >> lane) & 1u;
        // lanes outside the mask take a = 1 (inside every loss's domain)
        const T a = act ? rg.at(voff + __popc(m & lt)) : T(1);
        Vec<T, K> w;
        w.load(rows + (int64_t)(FULL ? j : q) * K);
        const T u = f.dot(w);
        T L;
        T d;
        if constexpr (XSTEP) d = loss_k<T, KIND>(Ls[j], u, a, L);
        else d = loss_k<T, KIND>(segspec, u, a, L);
        d = act ? d : T(0);
        lsum += act ? L : T(0);
        if constexpr (GRAD) g.axpy(d, w);
        voff += __popc(m);
    }
}

// Other-factor rows for one batch of 32 pairs, copied by each lane with
// cp.async (16-byte pieces) into the warp's batch buffer.
template <class T, int K>
__device__ __forceinline__ void gather_rows(T *dst, const T *__restrict__ W, int j, bool valid)
{
    constexpr int PIECES = K * (int)sizeof(T) / 16;
    if (valid) {
        const char *src = reinterpret_cast<const char *>(W + (int64_t)j * K);
        char *d = reinterpret_cast<char *>(dst);
#pragma unroll
        for (int q = 0; q < PIECES; ++q)
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(d + 16 * q)),
                         "l"(src + 16 * q)
                         : "memory");
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
}

__device__ __forceinline__ void gather_wait_all()
{
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    __syncwarp();
}

// One pass of a warp over pairs [pb, pe) of a tile whose values are global
// positions [vstart, vend).  FULL: the other factor is in shared memory (Ws,
// row j at j - jbase); else rows are gathered per batch into gbuf (two
// buffers of 32 rows).
template <class T, int K, bool XSTEP, bool GRAD, bool FULL>
__device__ __forceinline__ T mt_pass2(Ring<T> &rg, const Vec<T, K> &f, Vec<T, K> &g, int pb, int pe,
                                      int64_t vstart, int64_t vend, const int32_t *__restrict__ tidx,
                                      const uint32_t *__restrict__ tmask, const T *__restrict__ tval,
                                      const T *Ws, const T *__restrict__ W, T *gbuf,
                                      const LossOf<T> *__restrict__ Lsrc, const LossOf<T> &segspec)
{
    const int lane = threadIdx.x & 31;
    T lsum = T(0);
    uint32_t voff = rg.begin(tval, vstart, vend);
    int nj = 0;
    uint32_t nm = 0;
    if (pb + lane < pe) {
        nj = __ldg(tidx + pb + lane);
        nm = __ldg(tmask + pb + lane);
    }
    int cur = 0;
    if constexpr (!FULL) gather_rows<T, K>(gbuf + lane * K, W, nj, pb + lane < pe);
    int segkind = -1;
    if constexpr (!XSTEP) {
        const int k0 = __shfl_sync(0xffffffffu, segspec.kind, 0);
        if (__all_sync(0xffffffffu, segspec.kind == k0)) segkind = segspec.kind;
    }
    for (int c0 = pb; c0 < pe; c0 += 32) {
        const int myj = nj;
        const uint32_t mym = nm;
        const int cnt = min(32, pe - c0);
        const bool more = c0 + 32 + lane < pe;
        if (more) {  // next batch of pairs
            nj = __ldg(tidx + c0 + 32 + lane);
            nm = __ldg(tmask + c0 + 32 + lane);
        }
        const T *rows;
        if constexpr (FULL) {
            rows = Ws;
        } else {
            gather_wait_all();                       // this batch's rows have landed
            rows = gbuf + cur * 32 * K;
            if (c0 + 32 < pe)                          // request the next batch's rows
                gather_rows<T, K>(gbuf + (cur ^ 1) * 32 * K + lane * K, W, nj, more);
        }
        const uint32_t total = __reduce_add_sync(0xffffffffu, (unsigned)__popc(mym));
        rg.ensure(voff + total);
        int kind = segkind;
        const LossOf<T> *Ls = Lsrc;
        if constexpr (XSTEP) {
            const int j0 = __shfl_sync(0xffffffffu, myj, 0);
            const int kj = Lsrc[lane < cnt ? myj : j0].kind;
            const int k0 = __shfl_sync(0xffffffffu, kj, 0);
            kind = __all_sync(0xffffffffu, kj == k0) ? kj : -1;
        }
        // rows are addressed by pair position q in the batch when gathered,
        // by the other-index j when the whole factor is resident
        switch (kind) {
        case kLossQuad:
            mt_batch2<T, K, XSTEP, GRAD, kLossQuad, FULL>(cnt, myj, mym, voff, rg, rows, Ls, segspec, f, g, lsum);
            break;
        case kLossHuber:
            mt_batch2<T, K, XSTEP, GRAD, kLossHuber, FULL>(cnt, myj, mym, voff, rg, rows, Ls, segspec, f, g, lsum);
            break;
        case kLossHinge:
            mt_batch2<T, K, XSTEP, GRAD, kLossHinge, FULL>(cnt, myj, mym, voff, rg, rows, Ls, segspec, f, g, lsum);
            break;
        case kLossLogistic:
            mt_batch2<T, K, XSTEP, GRAD, kLossLogistic, FULL>(cnt, myj, mym, voff, rg, rows, Ls, segspec, f, g, lsum);
            break;
        case kLossOrdinal:
            mt_batch2<T, K, XSTEP, GRAD, kLossOrdinal, FULL>(cnt, myj, mym, voff, rg, rows, Ls, segspec, f, g, lsum);
            break;
        default:
            mt_batch2<T, K, XSTEP, GRAD, -1, FULL>(cnt, myj, mym, voff, rg, rows, Ls, segspec, f, g, lsum);
        }
        rg.release(voff);
        cur ^= 1;
    }
    if constexpr (!FULL) gather_wait_all();
    rg.drain();
    return lsum;
}

// Modes of the masked kernel.
constexpr int kMtFused = 0;  // unit = whole tile: gradient, prox, re-evaluation, decision
constexpr int kMtGrad = 1;   // unit = part of a tile: partial gradient and loss at F
constexpr int kMtLoss = 2;   // unit = part of a tile: partial loss at F (the candidate)

// Dynamic shared memory: FULL: the other factor (nother x K) and, for the
// X-step, its loss table; then per warp a value ring and (gather) two batch
// buffers of 32 rows.
template <class T, int K, bool XSTEP, bool FULL, int MODE>
__global__ void __launch_bounds__(kMaskedWarps * 32, 1)
mt_kernel(int64_t nseg, int64_t nunits, int P, const int32_t *__restrict__ utile,
          const int32_t *__restrict__ tptr, const int32_t *__restrict__ uvoff,
          const int32_t *__restrict__ ubeg, const int32_t *__restrict__ segptr,
          const int32_t *__restrict__ tidx, const uint32_t *__restrict__ tmask,
          const T *__restrict__ tval, T *__restrict__ F, const T *__restrict__ W, int64_t nother,
          int k, T *__restrict__ alpha, const LossOf<T> *__restrict__ loss, int rk, T rw,
          double *__restrict__ kept_obj, double *__restrict__ kept_reg,
          int32_t *__restrict__ accepted, T *__restrict__ part_grad, double *__restrict__ part_loss,
          int *__restrict__ err)
{
    extern __shared__ __align__(128) unsigned char dsm[];
    __shared__ uint64_t bar_panel;
    __shared__ uint64_t bar_ring[kMaskedWarps][kRingSlots];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    size_t off = 0;
    T *Ws = reinterpret_cast<T *>(dsm);
    LossOf<T> *Ls = nullptr;
    if constexpr (FULL) {
        off = align16((size_t)nother * K * sizeof(T));
        if constexpr (XSTEP) {
            Ls = reinterpret_cast<LossOf<T> *>(dsm + off);
            off += (size_t)nother * sizeof(LossOf<T>);
        }
    }
    constexpr size_t kWarpBytes = (size_t)kRingSlots * kRingBytes + (FULL ? 0 : 2 * 32 * K * sizeof(T));
    unsigned char *wbase = dsm + off + (size_t)wid * kWarpBytes;
    T *ring = reinterpret_cast<T *>(wbase);
    T *gbuf = reinterpret_cast<T *>(wbase + (size_t)kRingSlots * kRingBytes);
    if (threadIdx.x == 0) mbar_init(&bar_panel, 1);
    if (lane < kRingSlots) mbar_init(&bar_ring[wid][lane], 1);
    __syncthreads();
    if constexpr (FULL) {
        if constexpr (XSTEP) {
            for (int64_t q = threadIdx.x; q < nother; q += blockDim.x) Ls[q] = loss[q];
        }
        if (!stage_panel<T>(Ws, W, 0, (int)nother, k, K, &bar_panel, 0, err)) return;
    }
    const LossOf<T> *Lsrc = FULL ? Ls : loss;
    Ring<T> vs;
    vs.init(ring, &bar_ring[wid][0]);
    for (int64_t u = (int64_t)blockIdx.x * nwarps + wid; u < nunits; u += (int64_t)gridDim.x * nwarps) {
        const int64_t t = utile[u];
        const int q = (int)(u - ubeg[t]);
        const int pb = tptr[t] + q * P;
        const int pe = min(tptr[t + 1], pb + P);
        const int64_t vb = uvoff[u];
        const int64_t tend = t * 32 + 32 < nseg ? t * 32 + 32 : nseg;
        const int64_t ve = (u + 1 < ubeg[t + 1]) ? uvoff[u + 1] : segptr[tend];
        const int64_t s = t * 32 + lane;
        const bool live = s < nseg;
        Vec<T, K> f, g;
        if (live) f.load_masked(F + s * k, k);
        else f.zero();
        g.zero();
        LossOf<T> sp{};
        if constexpr (!XSTEP) {
            if (live) sp = loss[s];
        }
        if constexpr (MODE == kMtFused) {
            const T l1 = mt_pass2<T, K, XSTEP, true, FULL>(vs, f, g, pb, pe, vb, ve, tidx, tmask, tval,
                                                          Ws, W, gbuf, Lsrc, sp);
            const T al = live ? alpha[s] : T(0);
            Vec<T, K> fp;
            T rold = T(0), rnew = T(0);
            {
                T tmp[K];
#pragma unroll
                for (int c = 0; c < K; ++c) {
                    const T x = f.get(c);
                    const T xp = c < k ? prox1<T>(reg_kind_at(rk, c, k), rw, al, x - al * g.get(c)) : T(0);
                    tmp[c] = xp;
                    if (c < k) {
                        rold += reg1t<T>(reg_kind_at(rk, c, k), rw, x);
                        rnew += reg1t<T>(reg_kind_at(rk, c, k), rw, xp);
                    }
                }
                fp.load_masked(tmp, K);
            }
            Vec<T, K> unused;
            const T l2 = mt_pass2<T, K, XSTEP, false, FULL>(vs, fp, unused, pb, pe, vb, ve, tidx, tmask,
                                                            tval, Ws, W, gbuf, Lsrc, sp);
            if (!vs.ok) {
                if (lane == 0) atomicOr(err, 1);
                return;
            }
            if (live) {
                const double fold = (double)l1 + rold;
                const double fnew = (double)l2 + rnew;
                const bool acc = fnew <= fold;
                if (acc) {
#pragma unroll
                    for (int c = 0; c < K; ++c)
                        if (c < k) F[s * k + c] = fp.get(c);
                }
                alpha[s] = al * (acc ? T(1.05) : T(0.7));
                kept_obj[s] = acc ? fnew : fold;
                kept_reg[s] = acc ? rnew : rold;
                accepted[s] = acc ? 1 : 0;
            }
        } else {
            const T l = mt_pass2<T, K, XSTEP, MODE == kMtGrad, FULL>(vs, f, g, pb, pe, vb, ve, tidx, tmask,
                                                                    tval, Ws, W, gbuf, Lsrc, sp);
            if (!vs.ok) {
                if (lane == 0) atomicOr(err, 1);
                return;
            }
            const int64_t slot = u * 32 + lane;
            if constexpr (MODE == kMtGrad) {
#pragma unroll
                for (int c = 0; c < K; ++c) part_grad[slot * K + c] = g.get(c);
            }
            part_loss[slot] = (double)l;
        }
    }
}

// Per-segment prox / decide over unit partials: segment s of tile t has
// partials at (u * 32 + s % 32) for the units u of t, summed in order.
template <class T, int K>
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
unit_prox_kernel(int64_t nseg, const int32_t *__restrict__ ubeg, const T *__restrict__ part_grad,
                 const double *__restrict__ part_loss, const T *__restrict__ F,
                 const T *__restrict__ alpha, int k, int rkind, T rw, T *__restrict__ cand,
                 double *__restrict__ f_old, double *__restrict__ r_old, double *__restrict__ r_new)
{
    const int lane = threadIdx.x & 31;
    const int64_t s = (int64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
    if (s >= nseg) return;
    const int64_t t = s / 32, l = s % 32;
    const int u0 = ubeg[t], u1 = ubeg[t + 1];
    const T al = alpha[s];
    T ro = T(0), rn = T(0);
    for (int c = lane; c < k; c += 32) {
        T g = T(0);
        for (int u = u0; u < u1; ++u) g += part_grad[((int64_t)u * 32 + l) * K + c];
        const T x = F[s * k + c];
        const int rkc = reg_kind_at(rkind, c, k);
        const T xp = prox1<T>(rkc, rw, al, x - al * g);
        cand[s * k + c] = xp;
        ro += reg1t<T>(rkc, rw, x);
        rn += reg1t<T>(rkc, rw, xp);
    }
    ro = warp_sum(ro);
    rn = warp_sum(rn);
    double ls;
    if (u1 - u0 == 1) {
        ls = part_loss[(int64_t)u0 * 32 + l];
    } else {
        ls = 0.0;
        for (int u = u0 + lane; u < u1; u += 32) ls += part_loss[(int64_t)u * 32 + l];
        ls = warp_sum(ls);
    }
    if (lane == 0) {
        f_old[s] = ls + ro;
        r_old[s] = ro;
        r_new[s] = rn;
    }
}

template <class T>
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
unit_decide_kernel(int64_t nseg, const int32_t *__restrict__ ubeg,
                   const double *__restrict__ part_loss_new, const double *__restrict__ f_old,
                   const double *__restrict__ r_old, const double *__restrict__ r_new,
                   const T *__restrict__ cand, T *__restrict__ F, T *__restrict__ alpha, int k,
                   double *__restrict__ kept_obj, double *__restrict__ kept_reg,
                   int32_t *__restrict__ accepted)
{
    const int lane = threadIdx.x & 31;
    const int64_t s = (int64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
    if (s >= nseg) return;
    const int64_t t = s / 32, l = s % 32;
    double ls;
    if (ubeg[t + 1] - ubeg[t] == 1) {
        ls = part_loss_new[(int64_t)ubeg[t] * 32 + l];
    } else {
        ls = 0.0;
        for (int u = ubeg[t] + lane; u < ubeg[t + 1]; u += 32) ls += part_loss_new[(int64_t)u * 32 + l];
        ls = warp_sum(ls);
    }
    const double fn = ls + r_new[s];
    const double fo = f_old[s];
    const bool acc = fn <= fo;
    if (acc)
        for (int c = lane; c < k; c += 32) F[s * k + c] = cand[s * k + c];
    if (lane == 0) {
        alpha[s] = alpha[s] * (acc ? T(1.05) : T(0.7));
        kept_obj[s] = acc ? fn : fo;
        kept_reg[s] = acc ? r_new[s] : r_old[s];
        accepted[s] = acc ? 1 : 0;
    }
}

// ---------------------------------------------------------------- launchers

template <class T, int K, bool XSTEP, bool FULL, int MODE>
cudaError_t launch_mt(glrm_s *h, const Orient &o, T *F, const T *W, int64_t nother, T *alpha, int rk,
                      T rw, double *kobj, double *kreg, int32_t *acc, T *pg, double *pl)
{
    auto kern = mt_kernel<T, K, XSTEP, FULL, MODE>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)o.smem_bytes);
    if (e != cudaSuccess) return e;
    kern<<<o.grid, o.warps * 32, o.smem_bytes, h->stream>>>(
        o.nseg, o.nunits, o.P, o.utile, o.tptr, o.uvoff, o.ubeg, o.ptr, o.tidx, o.tmask,
        (const T *)o.tval, F, W, nother, h->k, alpha, loss_of<T>(h), rk, rw, kobj, kreg, acc, pg, pl,
        h->s.err);
    return cudaGetLastError();
}

template <class T, int K, bool XSTEP, bool FULL>
cudaError_t mt_half_src(glrm_s *h)
{
    const Orient &o = XSTEP ? h->csr : h->csc;
    T *F = (T *)(XSTEP ? h->X : h->Yt);
    const T *W = (const T *)(XSTEP ? h->Yt : h->X);
    const int64_t nother = XSTEP ? h->n : h->m;
    T *alpha = (T *)(XSTEP ? h->alpha_x : h->alpha_y);
    const int rk = reg_code(h, XSTEP);
    const T rw = (T)(XSTEP ? h->rx_w : h->ry_w);
    Scratch &s = h->s;
    double *kobj = XSTEP ? s.kept_obj_x : s.kept_obj_y;
    double *kreg = XSTEP ? s.kept_reg_x : s.kept_reg_y;
    int32_t *acc = XSTEP ? s.acc_x : s.acc_y;
    cudaError_t e;
    if (o.nunits == (o.nseg + 31) / 32) {  // one unit per tile: fused
        tmark(h, XSTEP ? "masked_fused_x" : "masked_fused_y");
        e = launch_mt<T, K, XSTEP, FULL, kMtFused>(h, o, F, W, nother, alpha, rk, rw, kobj, kreg, acc,
                                                   nullptr, nullptr);
        tmark(h, nullptr);
        h->launches += 1;
        return e;
    }
    tmark(h, XSTEP ? "masked_grad_x" : "masked_grad_y");
    e = launch_mt<T, K, XSTEP, FULL, kMtGrad>(h, o, F, W, nother, alpha, rk, rw, kobj, kreg, acc,
                                              (T *)s.part_grad, s.part_loss);
    if (e != cudaSuccess) return e;
    const unsigned nbs = blocks_for(o.nseg, kWarpsPerBlock);
    tmark(h, XSTEP ? "masked_prox_x" : "masked_prox_y");
    unit_prox_kernel<T, K><<<nbs, kWarpsPerBlock * 32, 0, h->stream>>>(
        o.nseg, o.ubeg, (const T *)s.part_grad, s.part_loss, F, alpha, h->k, rk, rw, (T *)s.cand,
        s.f_old, s.r_old, s.r_new);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    tmark(h, XSTEP ? "masked_loss_x" : "masked_loss_y");
    e = launch_mt<T, K, XSTEP, FULL, kMtLoss>(h, o, (T *)s.cand, W, nother, alpha, rk, rw, kobj, kreg,
                                              acc, nullptr, s.part_loss2);
    if (e != cudaSuccess) return e;
    tmark(h, XSTEP ? "masked_decide_x" : "masked_decide_y");
    unit_decide_kernel<T><<<nbs, kWarpsPerBlock * 32, 0, h->stream>>>(
        o.nseg, o.ubeg, s.part_loss2, s.f_old, s.r_old, s.r_new, (const T *)s.cand, F, alpha, h->k,
        kobj, kreg, acc);
    tmark(h, nullptr);
    h->launches += 4;
    return cudaGetLastError();
}

template <class T, int K, bool XSTEP>
cudaError_t mt_half_K(glrm_s *h)
{
    const Orient &o = XSTEP ? h->csr : h->csc;
    return o.full ? mt_half_src<T, K, XSTEP, true>(h) : mt_half_src<T, K, XSTEP, false>(h);
}

template <class T, bool XSTEP>
cudaError_t mt_half(glrm_s *h)
{
    const int k = h->k;
    if (k <= 4) return mt_half_K<T, 4, XSTEP>(h);
    if (k <= 8) return mt_half_K<T, 8, XSTEP>(h);
    if (k <= 12) return mt_half_K<T, 12, XSTEP>(h);
    if (k <= 16) return mt_half_K<T, 16, XSTEP>(h);
    if (k <= 20) return mt_half_K<T, 20, XSTEP>(h);
    if (k <= 24) return mt_half_K<T, 24, XSTEP>(h);
    if (k <= 32) return mt_half_K<T, 32, XSTEP>(h);
    return cudaErrorInvalidValue;
}

template <class T>
cudaError_t Engine<T>::masked_half_step(glrm_s *h, bool xstep)
{
    return xstep ? mt_half<T, true>(h) : mt_half<T, false>(h);
}

// Build the masked tiles of one orientation (tptr holds the exclusive scan of
// the pair counts, ubeg the first unit of each tile).
template <class T>
cudaError_t mt_build(const Orient &o, cudaStream_t st)
{
    const int64_t ntiles = (o.nseg + 31) / 32;
    mt_emit_kernel<T><<<blocks_for(ntiles, 8), 256, 0, st>>>(o.nseg, o.ptr, o.idx, (const T *)o.val,
                                                             o.tptr, o.ubeg, o.P, o.tidx, o.tmask,
                                                             (T *)o.tval, o.uvoff);
    return cudaGetLastError();
}

inline cudaError_t mt_count(const Orient &o, int64_t nother, int32_t *cnt, cudaStream_t st)
{
    const int64_t ntiles = (o.nseg + 31) / 32;
    const size_t bitmap = (size_t)((nother + 31) / 32) * sizeof(uint32_t);
    if (ntiles > 0 && bitmap <= 160 * 1024) {
        if (bitmap > 48 * 1024) {
            const cudaError_t e = cudaFuncSetAttribute(mt_count_bitmap_kernel,
                                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bitmap);
            if (e != cudaSuccess) return e;
        }
        mt_count_bitmap_kernel<<<(unsigned)ntiles, 256, bitmap, st>>>(o.nseg, nother, o.ptr, o.idx, cnt);
    } else {
        mt_count_kernel<<<blocks_for(ntiles, 8), 256, 0, st>>>(o.nseg, o.ptr, o.idx, cnt);
    }
    return cudaGetLastError();
}

}  // namespace glrm
