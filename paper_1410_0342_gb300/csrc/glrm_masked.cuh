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

// Emit pairs and tile-ordered values; record for every panel b (other-index
// in [b R, (b+1) R)) the first pair and the value offset of the panel.
template <class T>
__global__ void mt_emit_kernel(int64_t nseg, const int32_t *__restrict__ ptr,
                               const int32_t *__restrict__ idx, const T *__restrict__ val,
                               const int32_t *__restrict__ tptr, int nb, int R,
                               int32_t *__restrict__ tidx, uint32_t *__restrict__ tmask,
                               T *__restrict__ tval, int32_t *__restrict__ tpan,
                               int32_t *__restrict__ tvpan)
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
    int pair = tptr[t];
    int voff = ptr[t * 32];
    int curb = 0;
    const uint32_t lt = (1u << lane) - 1u;
    if (lane == 0) {
        tpan[t * (nb + 1)] = pair;
        tvpan[t * (nb + 1)] = voff;
    }
    for (;;) {
        const int j = __reduce_min_sync(0xffffffffu, nxt);
        if (j == INT_MAX) break;
        const int pb = j / R;
        while (curb < pb) {
            ++curb;
            if (lane == 0) {
                tpan[t * (nb + 1) + curb] = pair;
                tvpan[t * (nb + 1) + curb] = voff;
            }
        }
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
    while (curb < nb) {
        ++curb;
        if (lane == 0) {
            tpan[t * (nb + 1) + curb] = pair;
            tvpan[t * (nb + 1) + curb] = voff;
        }
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
template <class T, int KIND>
__device__ __forceinline__ T loss_k(const LossSpec &s, T u, T a, T &L)
{
    if constexpr (KIND < 0) {
        return loss_deriv<T>(s, u, a, L);
    } else {
        LossSpec q = s;
        q.kind = KIND;
        return loss_deriv<T>(q, u, a, L);
    }
}

// Process `cnt` pairs of a batch (indices / masks in lane q of myj / mym).
// Every lane runs the same instructions; lanes outside a pair's mask get zero
// weight, so nothing diverges.
template <class T, int K, bool XSTEP, bool GRAD, int KIND>
__device__ __forceinline__ void mt_batch(int cnt, int myj, uint32_t mym, uint32_t &voff,
                                         const Ring<T> &rg, const T *Ws, int jbase,
                                         const LossSpec *Ls, const LossSpec &segspec,
                                         const Vec<T, K> &f, Vec<T, K> &g, T &lsum)
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
        w.load(Ws + (int64_t)(j - jbase) * K);
        const T u = f.dot(w);
        T L;
        T d;
        if constexpr (XSTEP) d = loss_k<T, KIND>(Ls[j - jbase], u, a, L);
        else d = loss_k<T, KIND>(segspec, u, a, L);
        d = act ? d : T(0);
        lsum += act ? L : T(0);
        if constexpr (GRAD) g.axpy(d, w);
        voff += __popc(m);
    }
}

// One pass of a warp over pairs [pb, pe) of a tile whose values are global
// positions [vstart, vend); jbase: first other-index held in shared memory.
template <class T, int K, bool XSTEP, bool GRAD>
__device__ __forceinline__ T mt_pass(Ring<T> &rg, const Vec<T, K> &f, Vec<T, K> &g, int pb, int pe,
                                     int64_t vstart, int64_t vend, int jbase,
                                     const int32_t *__restrict__ tidx,
                                     const uint32_t *__restrict__ tmask, const T *__restrict__ tval,
                                     const T *Ws, const LossSpec *Ls, const LossSpec &segspec)
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
    // Y-step: the tile's loss kind is fixed when all its segments share it
    int segkind = -1;
    if constexpr (!XSTEP) {
        const int k0 = __shfl_sync(0xffffffffu, segspec.kind, 0);
        if (__all_sync(0xffffffffu, segspec.kind == k0)) segkind = segspec.kind;
    }
    for (int c0 = pb; c0 < pe; c0 += 32) {
        const int myj = nj;
        const uint32_t mym = nm;
        const int cnt = min(32, pe - c0);
        if (c0 + 32 + lane < pe) {  // next batch of pairs
            nj = __ldg(tidx + c0 + 32 + lane);
            nm = __ldg(tmask + c0 + 32 + lane);
        }
        const uint32_t total = __reduce_add_sync(0xffffffffu, (unsigned)__popc(mym));
        rg.ensure(voff + total);
        int kind = segkind;
        if constexpr (XSTEP) {
            // every lane shuffles (full mask), then lanes past the batch reuse pair 0
            const int j0 = __shfl_sync(0xffffffffu, myj, 0);
            const int kj = Ls[(lane < cnt ? myj : j0) - jbase].kind;
            const int k0 = __shfl_sync(0xffffffffu, kj, 0);
            kind = __all_sync(0xffffffffu, kj == k0) ? kj : -1;
        }
        switch (kind) {
        case kLossQuad:
            mt_batch<T, K, XSTEP, GRAD, kLossQuad>(cnt, myj, mym, voff, rg, Ws, jbase, Ls, segspec, f, g, lsum);
            break;
        case kLossHuber:
            mt_batch<T, K, XSTEP, GRAD, kLossHuber>(cnt, myj, mym, voff, rg, Ws, jbase, Ls, segspec, f, g, lsum);
            break;
        case kLossHinge:
            mt_batch<T, K, XSTEP, GRAD, kLossHinge>(cnt, myj, mym, voff, rg, Ws, jbase, Ls, segspec, f, g, lsum);
            break;
        case kLossLogistic:
            mt_batch<T, K, XSTEP, GRAD, kLossLogistic>(cnt, myj, mym, voff, rg, Ws, jbase, Ls, segspec, f, g, lsum);
            break;
        case kLossOrdinal:
            mt_batch<T, K, XSTEP, GRAD, kLossOrdinal>(cnt, myj, mym, voff, rg, Ws, jbase, Ls, segspec, f, g, lsum);
            break;
        default:
            mt_batch<T, K, XSTEP, GRAD, -1>(cnt, myj, mym, voff, rg, Ws, jbase, Ls, segspec, f, g, lsum);
        }
        rg.release(voff);
    }
    rg.drain();
    return lsum;
}

// Fused masked-tile half-step: the whole other factor (and for the X-step its
// loss table) in shared memory; one warp per tile runs gradient, prox,
// re-evaluation and decision for its 32 segments.
template <class T, int K, bool XSTEP>
__global__ void __launch_bounds__(kMaskedWarps * 32, 1)
mt_fused_kernel(int64_t nseg, const int32_t *__restrict__ tpan, const int32_t *__restrict__ tvpan,
                const int32_t *__restrict__ tidx, const uint32_t *__restrict__ tmask,
                const T *__restrict__ tval, T *__restrict__ F, const T *__restrict__ W,
                int64_t nother, int k, T *__restrict__ alpha, const LossSpec *__restrict__ loss,
                int rk, T rw, double *__restrict__ kept_obj, double *__restrict__ kept_reg,
                int32_t *__restrict__ accepted, int *__restrict__ err)
{
    extern __shared__ __align__(128) unsigned char dsm[];
    __shared__ uint64_t bar_panel;
    __shared__ uint64_t bar_ring[kMaskedWarps][kRingSlots];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    T *Ws = reinterpret_cast<T *>(dsm);
    size_t off = align16((size_t)nother * K * sizeof(T));
    LossSpec *Ls = reinterpret_cast<LossSpec *>(dsm + off);
    if constexpr (XSTEP) off += (size_t)nother * sizeof(LossSpec);
    T *ring = reinterpret_cast<T *>(dsm + off) + (size_t)wid * Ring<T>::N;
    if (threadIdx.x == 0) mbar_init(&bar_panel, 1);
    if (lane < kRingSlots) mbar_init(&bar_ring[wid][lane], 1);
    __syncthreads();
    if constexpr (XSTEP) {
        for (int64_t q = threadIdx.x; q < nother; q += blockDim.x) Ls[q] = loss[q];
    }
    if (!stage_panel<T>(Ws, W, 0, (int)nother, k, K, &bar_panel, 0, err)) return;
    Ring<T> vs;
    vs.init(ring, &bar_ring[wid][0]);
    const int64_t ntiles = (nseg + 31) / 32;
    for (int64_t t = (int64_t)blockIdx.x * kMaskedWarps + wid; t < ntiles;
         t += (int64_t)gridDim.x * kMaskedWarps) {
        const int64_t s = t * 32 + lane;
        const bool live = s < nseg;
        const int pb = tpan[2 * t], pe = tpan[2 * t + 1];
        const int64_t vb = tvpan[2 * t], ve = tvpan[2 * t + 1];
        Vec<T, K> f, g;
        if (live) f.load_masked(F + s * k, k);
        else f.zero();
        g.zero();
        LossSpec sp{};
        if constexpr (!XSTEP) {
            if (live) sp = loss[s];
        }
        const T l1 = mt_pass<T, K, XSTEP, true>(vs, f, g, pb, pe, vb, ve, 0, tidx, tmask, tval, Ws,
                                                Ls, sp);
        const T al = live ? alpha[s] : T(0);
        Vec<T, K> fp;
        double rold = 0.0, rnew = 0.0;
        {
            T tmp[K];
#pragma unroll
            for (int c = 0; c < K; ++c) {
                const T x = f.get(c);
                const T xp = c < k ? prox1<T>(rk, rw, al, x - al * g.get(c)) : T(0);
                tmp[c] = xp;
                if (c < k) {
                    rold += reg1<T>(rk, rw, x);
                    rnew += reg1<T>(rk, rw, xp);
                }
            }
            fp.load_masked(tmp, K);
        }
        Vec<T, K> unused;
        const T l2 = mt_pass<T, K, XSTEP, false>(vs, fp, unused, pb, pe, vb, ve, 0, tidx, tmask,
                                                 tval, Ws, Ls, sp);
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
    }
}

// Panel pass of the masked-tile form: unit = (panel b, group of tiles); the
// CTA stages the panel, each warp reduces its tiles' pairs in that panel into
// per-(panel, segment) partials (GRAD: gradient and loss at F; else loss).
template <class T, int K, bool XSTEP, bool GRAD>
__global__ void __launch_bounds__(kMaskedWarps * 32, 1)
mt_pass_kernel(int64_t nseg, int nb, int R, int ngroups, int64_t nother,
               const int32_t *__restrict__ tpan, const int32_t *__restrict__ tvpan,
               const int32_t *__restrict__ tidx, const uint32_t *__restrict__ tmask,
               const T *__restrict__ tval, const T *__restrict__ F, const T *__restrict__ W, int k,
               const LossSpec *__restrict__ loss, T *__restrict__ part_grad,
               double *__restrict__ part_loss, int *__restrict__ err)
{
    extern __shared__ __align__(128) unsigned char dsm[];
    __shared__ uint64_t bar_panel;
    __shared__ uint64_t bar_ring[kMaskedWarps][kRingSlots];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    T *Ws = reinterpret_cast<T *>(dsm);
    size_t off = align16((size_t)R * K * sizeof(T));
    LossSpec *Ls = reinterpret_cast<LossSpec *>(dsm + off);
    if constexpr (XSTEP) off += (size_t)R * sizeof(LossSpec);
    T *ring = reinterpret_cast<T *>(dsm + off) + (size_t)wid * Ring<T>::N;
    if (threadIdx.x == 0) mbar_init(&bar_panel, 1);
    if (lane < kRingSlots) mbar_init(&bar_ring[wid][lane], 1);
    __syncthreads();
    Ring<T> vs;
    vs.init(ring, &bar_ring[wid][0]);
    const int64_t ntiles = (nseg + 31) / 32;
    const int64_t tiles_per = (ntiles + ngroups - 1) / ngroups;
    const int64_t nunits = (int64_t)nb * ngroups;
    unsigned pphase = 0;
    for (int64_t u = blockIdx.x; u < nunits; u += gridDim.x) {
        const int b = (int)(u / ngroups);
        const int64_t grp = u % ngroups;
        const int64_t r0 = (int64_t)b * R;
        const int rows = (int)((r0 + R <= nother) ? R : nother - r0);
        __syncthreads();
        if constexpr (XSTEP) {
            for (int q = threadIdx.x; q < rows; q += blockDim.x) Ls[q] = loss[r0 + q];
        }
        if (!stage_panel<T>(Ws, W, r0, rows, k, K, &bar_panel, pphase, err)) return;
        pphase ^= 1u;
        const int64_t t0 = grp * tiles_per;
        const int64_t t1 = t0 + tiles_per < ntiles ? t0 + tiles_per : ntiles;
        for (int64_t t = t0 + wid; t < t1; t += kMaskedWarps) {
            const int64_t s = t * 32 + lane;
            const bool live = s < nseg;
            const int64_t pi = t * (nb + 1) + b;
            const int pb = tpan[pi], pe = tpan[pi + 1];
            const int64_t vb = tvpan[pi], ve = tvpan[pi + 1];
            Vec<T, K> f, g;
            if (live) f.load_masked(F + s * k, k);
            else f.zero();
            g.zero();
            LossSpec sp{};
            if constexpr (!XSTEP) {
                if (live) sp = loss[s];
            }
            const T l = mt_pass<T, K, XSTEP, GRAD>(vs, f, g, pb, pe, vb, ve, (int)r0, tidx, tmask,
                                                   tval, Ws, Ls, sp);
            if (live) {
                const int64_t slot = (int64_t)b * nseg + s;
                if constexpr (GRAD) {
#pragma unroll
                    for (int c = 0; c < K; ++c) part_grad[slot * K + c] = g.get(c);
                }
                part_loss[slot] = (double)l;
            }
        }
        if (__syncthreads_or(!vs.ok)) {
            if (threadIdx.x == 0) atomicOr(err, 1);
            return;
        }
    }
}

// ---------------------------------------------------------------- launchers

template <class T, int K, bool XSTEP>
cudaError_t mt_half_K(glrm_s *h)
{
    const Orient &o = XSTEP ? h->csr : h->csc;
    T *F = (T *)(XSTEP ? h->X : h->Yt);
    const T *W = (const T *)(XSTEP ? h->Yt : h->X);
    const int64_t nother = XSTEP ? h->n : h->m;
    T *alpha = (T *)(XSTEP ? h->alpha_x : h->alpha_y);
    const int rk = XSTEP ? h->rx_kind : h->ry_kind;
    const T rw = (T)(XSTEP ? h->rx_w : h->ry_w);
    Scratch &s = h->s;
    double *kobj = XSTEP ? s.kept_obj_x : s.kept_obj_y;
    double *kreg = XSTEP ? s.kept_reg_x : s.kept_reg_y;
    int32_t *acc = XSTEP ? s.acc_x : s.acc_y;
    cudaError_t e;
    if (o.nb == 1) {
        auto kern = mt_fused_kernel<T, K, XSTEP>;
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)o.smem_bytes);
        if (e != cudaSuccess) return e;
        tmark(h, XSTEP ? "masked_fused_x" : "masked_fused_y");
        kern<<<o.grid, kMaskedWarps * 32, o.smem_bytes, h->stream>>>(
            o.nseg, o.tpan, o.tvpan, o.tidx, o.tmask, (const T *)o.tval, F, W, nother, h->k, alpha,
            h->loss_dev, rk, rw, kobj, kreg, acc, h->s.err);
        tmark(h, nullptr);
        h->launches += 1;
        return cudaGetLastError();
    }
    auto pass_g = mt_pass_kernel<T, K, XSTEP, true>;
    auto pass_l = mt_pass_kernel<T, K, XSTEP, false>;
    if ((e = cudaFuncSetAttribute(pass_g, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)o.smem_bytes)) != cudaSuccess)
        return e;
    if ((e = cudaFuncSetAttribute(pass_l, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)o.smem_bytes)) != cudaSuccess)
        return e;
    tmark(h, XSTEP ? "masked_grad_x" : "masked_grad_y");
    pass_g<<<o.grid, kMaskedWarps * 32, o.smem_bytes, h->stream>>>(
        o.nseg, o.nb, o.R, o.ngroups, nother, o.tpan, o.tvpan, o.tidx, o.tmask, (const T *)o.tval,
        F, W, h->k, h->loss_dev, (T *)s.part_grad, s.part_loss, h->s.err);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const unsigned nbs = blocks_for(o.nseg, kWarpsPerBlock);
    tmark(h, XSTEP ? "masked_prox_x" : "masked_prox_y");
    blocked_prox_kernel<T, K><<<nbs, kWarpsPerBlock * 32, 0, h->stream>>>(
        o.nseg, o.nb, (const T *)s.part_grad, s.part_loss, F, alpha, h->k, rk, rw, (T *)s.cand,
        s.f_old, s.r_old, s.r_new);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    tmark(h, XSTEP ? "masked_loss_x" : "masked_loss_y");
    pass_l<<<o.grid, kMaskedWarps * 32, o.smem_bytes, h->stream>>>(
        o.nseg, o.nb, o.R, o.ngroups, nother, o.tpan, o.tvpan, o.tidx, o.tmask, (const T *)o.tval,
        (const T *)s.cand, W, h->k, h->loss_dev, nullptr, s.part_loss2, h->s.err);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    tmark(h, XSTEP ? "masked_decide_x" : "masked_decide_y");
    blocked_decide_kernel<T><<<nbs, kWarpsPerBlock * 32, 0, h->stream>>>(
        o.nseg, o.nb, s.part_loss2, s.f_old, s.r_old, s.r_new, (const T *)s.cand, F, alpha, h->k,
        kobj, kreg, acc);
    tmark(h, nullptr);
    h->launches += 4;
    return cudaGetLastError();
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

// Build the masked tiles of one orientation (the pair counts are already in
// o.tptr as an exclusive scan).
template <class T>
cudaError_t mt_build(const Orient &o, cudaStream_t st)
{
    const int64_t ntiles = (o.nseg + 31) / 32;
    mt_emit_kernel<T><<<blocks_for(ntiles, 8), 256, 0, st>>>(o.nseg, o.ptr, o.idx, (const T *)o.val,
                                                             o.tptr, o.nb, o.R, o.tidx, o.tmask,
                                                             (T *)o.tval, o.tpan, o.tvpan);
    return cudaGetLastError();
}

inline cudaError_t mt_count(const Orient &o, int32_t *cnt, cudaStream_t st)
{
    const int64_t ntiles = (o.nseg + 31) / 32;
    mt_count_kernel<<<blocks_for(ntiles, 8), 256, 0, st>>>(o.nseg, o.ptr, o.idx, cnt);
    return cudaGetLastError();
}

}  // namespace glrm
