// Shared-memory staged forms of the proximal-gradient half-step (Section 7.2
// of Udell et al., "Generalized Low Rank Models": gradient over a row's
// (column's) observed entries, prox, re-evaluation of the row objective,
// accept / reject with the step-size rule).
//
// fused:   the whole other factor fits in shared memory.  Each CTA stages it
//          once with a TMA bulk copy, then every warp owns one segment at a
//          time and runs gradient, prox, re-evaluation and decision without
//          leaving the SM.  One launch per half-step, no scratch.
// blocked: the other factor is cut into panels of R rows that fit in shared
//          memory.  A segment's entries with other-index in panel b form one
//          contiguous run of its CSR/CSC list (indices are sorted), found by
//          binary search once at set-up, so no data moves.  Work unit =
//          (panel, group of segments): the CTA stages the panel with TMA and
//          its warps reduce the runs of their segments into per-(panel,
//          segment) partials; prox / decide kernels then sum the partials of
//          a segment over panels in a fixed order.
// Every wait on a TMA copy is bounded; on expiry the kernel raises a flag in
// device memory, waits once more (bounded) for its copy and leaves.
#pragma once

#include <type_traits>

#include "glrm_engine.cuh"

namespace glrm {

constexpr long kWaitLimit = 1L << 22;

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

// 1-D TMA bulk copy global -> shared, completion counted on the mbarrier.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned phase)
{
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(phase)
        : "memory");
    return ok != 0;
}

// Wait for phase `phase` of the mbarrier to complete, giving up after `limit`
// try_wait attempts (each may suspend the thread for a while).  Returns false
// on expiry; the caller then raises the error flag and leaves.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, unsigned phase, long limit = kWaitLimit)
{
    for (long it = 0; it < limit; ++it)
        if (mbar_try_wait(bar, phase)) return true;
    return false;
}

// Stage rows [r0, r0 + rows) of a row-major (ld = k) factor into shared memory
// with row stride K.  TMA bulk copies when k == K and the source is 16-byte
// aligned (the caller guarantees k % 4 == 0 then); otherwise plain loads with
// zero padding.  Every thread of the CTA must call it.  `phase` is the
// mbarrier phase this staging completes.  Returns false (after raising *err)
// if the copy did not complete in time.
template <class T>
__device__ bool stage_panel(T *dst, const T *__restrict__ src, int64_t r0, int rows, int k, int K,
                            uint64_t *bar, unsigned phase, int *err)
{
    const size_t bytes = (size_t)rows * K * sizeof(T);
    const T *s = src + r0 * k;
    if (k == K && ((uintptr_t)s % 16) == 0 && bytes % 16 == 0) {
        if (threadIdx.x == 0 && bytes > 0) {
            mbar_expect_tx(bar, (unsigned)bytes);
            for (size_t off = 0; off < bytes; off += 32768) {
                const size_t len = bytes - off < 32768 ? bytes - off : 32768;
                bulk_g2s((char *)dst + off, (const char *)s + off, (unsigned)len, bar);
            }
        } else if (threadIdx.x == 0) {
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
        }
        bool ok = mbar_wait_bounded(bar, phase);
        if (!ok) ok = mbar_wait_bounded(bar, phase);  // second bounded wait for the copy
        const int fail = __syncthreads_or(!ok);
        if (fail && threadIdx.x == 0) atomicOr(err, 1);
        return !fail;
    }
    for (int64_t q = threadIdx.x; q < (int64_t)rows * K; q += blockDim.x) {
        const int64_t r = q / K;
        const int c = (int)(q % K);
        dst[q] = c < k ? s[r * k + c] : T(0);
    }
    __syncthreads();
    if (threadIdx.x == 0)
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
    const bool ok = mbar_wait_bounded(bar, phase);
    const int fail = __syncthreads_or(!ok);
    if (fail && threadIdx.x == 0) atomicOr(err, 1);
    return !fail;
}

// ------------------------------------------------------------ small vectors

__device__ __forceinline__ unsigned long long pk2(float lo, float hi)
{
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}

__device__ __forceinline__ void upk2(unsigned long long v, float &lo, float &hi)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}

// Two independent FP32 fused multiply-adds in one instruction (sm_100+).
__device__ __forceinline__ unsigned long long ffma2(unsigned long long a, unsigned long long b,
                                                    unsigned long long c)
{
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

// A K-vector held by one lane: float pairs for FP32 (packed FMA), plain
// doubles for FP64.
template <class T, int K>
struct Vec;

template <int K>
struct Vec<float, K> {
    static_assert(K % 4 == 0, "K must be a multiple of 4");
    unsigned long long p[K / 2];

    __device__ __forceinline__ void zero()
    {
#pragma unroll
        for (int q = 0; q < K / 2; ++q) p[q] = 0ull;
    }
    // 16-byte aligned row (shared or global)
    __device__ __forceinline__ void load(const float *row)
    {
        const float4 *r = reinterpret_cast<const float4 *>(row);
#pragma unroll
        for (int q = 0; q < K / 4; ++q) {
            const float4 t = r[q];
            p[2 * q] = pk2(t.x, t.y);
            p[2 * q + 1] = pk2(t.z, t.w);
        }
    }
    __device__ __forceinline__ void load_masked(const float *row, int k)
    {
#pragma unroll
        for (int q = 0; q < K / 2; ++q)
            p[q] = pk2(2 * q < k ? row[2 * q] : 0.f, 2 * q + 1 < k ? row[2 * q + 1] : 0.f);
    }
    __device__ __forceinline__ float get(int c) const
    {
        float lo, hi;
        upk2(p[c >> 1], lo, hi);
        return (c & 1) ? hi : lo;
    }
    __device__ __forceinline__ float dot(const Vec &o) const
    {
        unsigned long long a = 0ull;
#pragma unroll
        for (int q = 0; q < K / 2; ++q) a = ffma2(p[q], o.p[q], a);
        float lo, hi;
        upk2(a, lo, hi);
        return lo + hi;
    }
    __device__ __forceinline__ void axpy(float s, const Vec &o)
    {
        const unsigned long long ss = pk2(s, s);
#pragma unroll
        for (int q = 0; q < K / 2; ++q) p[q] = ffma2(ss, o.p[q], p[q]);
    }
    __device__ __forceinline__ void warp_allsum()
    {
#pragma unroll
        for (int q = 0; q < K / 2; ++q) {
            float lo, hi;
            upk2(p[q], lo, hi);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                lo += __shfl_xor_sync(0xffffffffu, lo, o);
                hi += __shfl_xor_sync(0xffffffffu, hi, o);
            }
            p[q] = pk2(lo, hi);
        }
    }
};

template <int K>
struct Vec<double, K> {
    double p[K];

    __device__ __forceinline__ void zero()
    {
#pragma unroll
        for (int q = 0; q < K; ++q) p[q] = 0.0;
    }
    __device__ __forceinline__ void load(const double *row)
    {
        const double2 *r = reinterpret_cast<const double2 *>(row);
#pragma unroll
        for (int q = 0; q < K / 2; ++q) {
            const double2 t = r[q];
            p[2 * q] = t.x;
            p[2 * q + 1] = t.y;
        }
    }
    __device__ __forceinline__ void load_masked(const double *row, int k)
    {
#pragma unroll
        for (int q = 0; q < K; ++q) p[q] = q < k ? row[q] : 0.0;
    }
    __device__ __forceinline__ double get(int c) const { return p[c]; }
    __device__ __forceinline__ double dot(const Vec &o) const
    {
        double a = 0.0;
#pragma unroll
        for (int q = 0; q < K; ++q) a = fma(p[q], o.p[q], a);
        return a;
    }
    __device__ __forceinline__ void axpy(double s, const Vec &o)
    {
#pragma unroll
        for (int q = 0; q < K; ++q) p[q] = fma(s, o.p[q], p[q]);
    }
    __device__ __forceinline__ void warp_allsum()
    {
#pragma unroll
        for (int q = 0; q < K; ++q) p[q] = warp_sum(p[q]);
    }
};

// Per-segment objective pieces after a pass: every lane holds the totals.
template <class T, int K>
__device__ __forceinline__ double reg_of(const Vec<T, K> &v, int k, int rk, T rw)
{
    T r = T(0);
#pragma unroll
    for (int c = 0; c < K; ++c)
        if (c < k) r += reg1t<T>(reg_kind_at(rk, c, k), rw, v.get(c));
    return (double)r;
}

// ------------------------------------------------- per-warp entry streams

__device__ __forceinline__ void fence_proxy_async()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// One warp's two staging buffers for the (index, value) lists of its
// segments: while it works on one segment from buffer `cur`, a TMA bulk copy
// fills buffer cur^1 with the next segment's entries.  A range is copied as
// its 16-byte aligned superset [lo, hi) (the library pads its copies of Omega
// with kPad zero entries), so entry q sits at position q - lo.  Ranges longer
// than `cap` are not staged and are read from global memory instead.
template <class T>
struct EntryStream {
    // two buffers, kept in scalar members so that runtime selection stays in
    // registers
    int32_t *ib0, *ib1;
    T *vb0, *vb1;
    uint64_t *bar0, *bar1;
    unsigned ph0, ph1;
    int lo0, lo1;
    bool st0, st1;
    int cap;

    __device__ __forceinline__ void init(unsigned char *base, uint64_t *bars, int cap_)
    {
        cap = cap_;
        const size_t one = (size_t)cap * (sizeof(int32_t) + sizeof(T));
        ib0 = reinterpret_cast<int32_t *>(base);
        vb0 = reinterpret_cast<T *>(base + (size_t)cap * sizeof(int32_t));
        ib1 = reinterpret_cast<int32_t *>(base + one);
        vb1 = reinterpret_cast<T *>(base + one + (size_t)cap * sizeof(int32_t));
        bar0 = bars;
        bar1 = bars + 1;
        ph0 = ph1 = 0;
        lo0 = lo1 = 0;
        st0 = st1 = false;
    }
    __device__ __forceinline__ bool staged(int q) const { return q ? st1 : st0; }
    __device__ __forceinline__ const int32_t *ibase(int q) const { return q ? ib1 - lo1 : ib0 - lo0; }
    __device__ __forceinline__ const T *vbase(int q) const { return q ? vb1 - lo1 : vb0 - lo0; }

    // Whole warp calls; lane 0 issues.  Every issue completes one phase of
    // the buffer's barrier (with the copy, or at once when not staged).
    __device__ __forceinline__ void issue(int q, int b, int e, const int32_t *__restrict__ idx,
                                          const T *__restrict__ val)
    {
        const int l = b & ~3, hi = (e + 3) & ~3, n = hi - l;
        const bool stg = n > 0 && n <= cap;
        if (q) { lo1 = l; st1 = stg; } else { lo0 = l; st0 = stg; }
        int32_t *ib = q ? ib1 : ib0;
        T *vb = q ? vb1 : vb0;
        uint64_t *bar = q ? bar1 : bar0;
        __syncwarp();
        if ((threadIdx.x & 31) == 0) {
            fence_proxy_async();
            if (stg) {
                mbar_expect_tx(bar, (unsigned)(n * (sizeof(int32_t) + sizeof(T))));
                bulk_g2s(ib, idx + l, (unsigned)(n * sizeof(int32_t)), bar);
                bulk_g2s(vb, val + l, (unsigned)(n * sizeof(T)), bar);
            } else {
                asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
            }
        }
    }

    // Wait for buffer q (bounded); false if the copy did not land in time.
    __device__ __forceinline__ bool wait(int q)
    {
        uint64_t *bar = q ? bar1 : bar0;
        const unsigned ph = q ? ph1 : ph0;
        bool ok = mbar_wait_bounded(bar, ph);
        if (!ok) ok = mbar_wait_bounded(bar, ph);
        if (q) ph1 ^= 1u; else ph0 ^= 1u;
        return __all_sync(0xffffffffu, ok);  // warp-uniform verdict
    }
};

// Pass over one segment's entries [b, e): u = f . w_j for the other-factor row
// j (panel-local, from shared memory), loss and derivative; with GRAD the
// gradient sum L' w_j accumulates in g.  Entries come from the staging buffer
// (SM) or from global memory.
template <class T, int K, bool XSTEP, bool GRAD, bool SM>
__device__ __forceinline__ T seg_pass(const Vec<T, K> &f, Vec<T, K> &g, int b, int e, int jbase,
                                      const int32_t *__restrict__ ip, const T *__restrict__ vp,
                                      const T *__restrict__ Ws, const LossOf<T> *__restrict__ Ls,
                                      const LossOf<T> &segspec)
{
    const int lane = threadIdx.x & 31;
    T lsum = T(0);
    LossOf<T> sp = segspec;
    for (int q = b + lane; q < e; q += 32) {
        int j;
        T a;
        if constexpr (SM) {
            j = ip[q];
            a = vp[q];
        } else {
            j = __ldg(ip + q);
            a = __ldg(vp + q);
        }
        j -= jbase;
        Vec<T, K> w;
        w.load(Ws + (int64_t)j * K);
        const T u = f.dot(w);
        if constexpr (XSTEP) sp = Ls[j];
        T L;
        const T d = loss_deriv<T>(sp, u, a, L);
        if constexpr (GRAD) g.axpy(d, w);
        lsum += L;
    }
    return lsum;
}

template <class T, int K, bool XSTEP, bool GRAD>
__device__ __forceinline__ T seg_pass_any(const EntryStream<T> &st, int q, const Vec<T, K> &f,
                                          Vec<T, K> &g, int b, int e, int jbase,
                                          const int32_t *__restrict__ idx, const T *__restrict__ val,
                                          const T *Ws, const LossOf<T> *Ls, const LossOf<T> &segspec)
{
    if (st.staged(q))
        return seg_pass<T, K, XSTEP, GRAD, true>(f, g, b, e, jbase, st.ibase(q), st.vbase(q), Ws,
                                                 Ls, segspec);
    return seg_pass<T, K, XSTEP, GRAD, false>(f, g, b, e, jbase, idx, val, Ws, Ls, segspec);
}

__host__ __device__ __forceinline__ size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

// Bytes of one warp's pair of staging buffers.
template <class T>
__host__ __device__ __forceinline__ size_t stream_bytes(int cap)
{
    return 2 * (size_t)cap * (sizeof(int32_t) + sizeof(T));
}

// ----------------------------------------------------------- fused kernel

// Dynamic shared memory: the other factor (nother x K), for the X-step its
// loss table (nother LossSpecs), then kStreamWarps pairs of staging buffers.
template <class T, int K, bool XSTEP>
__global__ void __launch_bounds__(kStreamWarps * 32, 1)
fused_half_kernel(int64_t nseg, const int32_t *__restrict__ ptr, const int32_t *__restrict__ idx,
                  const T *__restrict__ val, T *__restrict__ F, const T *__restrict__ W,
                  int64_t nother, int k, T *__restrict__ alpha, const LossOf<T> *__restrict__ loss,
                  int rk, T rw, double *__restrict__ kept_obj, double *__restrict__ kept_reg,
                  int32_t *__restrict__ accepted, int *__restrict__ err, int cap)
{
    extern __shared__ __align__(128) unsigned char dsm[];
    __shared__ uint64_t bar_panel;
    __shared__ uint64_t bar_seg[kStreamWarps][2];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    T *Ws = reinterpret_cast<T *>(dsm);
    size_t off = align16((size_t)nother * K * sizeof(T));
    LossOf<T> *Ls = reinterpret_cast<LossOf<T> *>(dsm + off);
    if constexpr (XSTEP) off += (size_t)nother * sizeof(LossOf<T>);
    EntryStream<T> st;
    st.init(dsm + off + (size_t)wid * stream_bytes<T>(cap), &bar_seg[wid][0], cap);
    if (threadIdx.x == 0) mbar_init(&bar_panel, 1);
    if (lane == 0) {
        mbar_init(&bar_seg[wid][0], 1);
        mbar_init(&bar_seg[wid][1], 1);
    }
    __syncthreads();
    if constexpr (XSTEP) {
        for (int64_t q = threadIdx.x; q < nother; q += blockDim.x) Ls[q] = loss[q];
    }
    if (!stage_panel<T>(Ws, W, 0, (int)nother, k, K, &bar_panel, 0, err)) return;

    const int64_t wstride = (int64_t)gridDim.x * kStreamWarps;
    int64_t s = (int64_t)blockIdx.x * kStreamWarps + wid;
    int cur = 0;
    if (s < nseg) st.issue(0, ptr[s], ptr[s + 1], idx, val);
    for (; s < nseg; s += wstride) {
        const int64_t nx = s + wstride;
        if (nx < nseg) st.issue(cur ^ 1, ptr[nx], ptr[nx + 1], idx, val);
        if (!st.wait(cur)) {
            if (lane == 0) atomicOr(err, 1);
            if (nx < nseg) st.wait(cur ^ 1);
            return;
        }
        const int b = ptr[s], e = ptr[s + 1];
        Vec<T, K> f, g;
        f.load_masked(F + s * k, k);
        g.zero();
        LossOf<T> sp;
        if constexpr (!XSTEP) sp = loss[s];
        // pass 1: gradient and loss at the current factor
        const T lsum = seg_pass_any<T, K, XSTEP, true>(st, cur, f, g, b, e, 0, idx, val, Ws, Ls, sp);
        g.warp_allsum();
        const double lold = warp_sum((double)lsum);
        const T al = alpha[s];
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
        // pass 2: loss at the candidate
        Vec<T, K> unused;
        const T lsum2 = seg_pass_any<T, K, XSTEP, false>(st, cur, fp, unused, b, e, 0, idx, val, Ws, Ls, sp);
        const double fnew = warp_sum((double)lsum2) + rnew;
        const double fold = lold + rold;
        const bool acc = fnew <= fold;
        if (acc) {
#pragma unroll
            for (int c = 0; c < K; ++c)
                if (c < k && lane == (c & 31)) F[s * k + c] = fp.get(c);
        }
        if (lane == 0) {
            alpha[s] = al * (acc ? T(1.05) : T(0.7));
            kept_obj[s] = acc ? fnew : fold;
            kept_reg[s] = acc ? rnew : rold;
            accepted[s] = acc ? 1 : 0;
        }
        cur ^= 1;
    }
}

// ---------------------------------------------------------- blocked kernels

// runptr[b * nseg + s] = first entry of segment s whose other-index is >= b*R
// (b = 0 .. nb); run (b, s) = [runptr[b*nseg+s], runptr[(b+1)*nseg+s]).
static __global__ void build_runptr_kernel(int64_t nseg, int nb, int R, const int32_t *__restrict__ ptr,
                                    const int32_t *__restrict__ idx, int32_t *__restrict__ runptr)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)(nb + 1) * nseg) return;
    const int b = (int)(t / nseg);
    const int64_t s = t % nseg;
    const int64_t key = (int64_t)b * R;
    int lo = ptr[s], hi = ptr[s + 1];
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if ((int64_t)idx[mid] < key) lo = mid + 1;
        else hi = mid;
    }
    runptr[t] = lo;
}

// One work unit = (panel b, segments [s0, s1)).  GRAD: partial gradient and
// loss at F; else loss only at F (the candidate).  Partials at (b*nseg + s).
// Each warp streams its runs through its staging buffers.
template <class T, int K, bool XSTEP, bool GRAD>
__global__ void __launch_bounds__(kStreamWarps * 32, 1)
blocked_pass_kernel(int64_t nseg, int nb, int R, int ngroups, int64_t nother,
                    const int32_t *__restrict__ runptr, const int32_t *__restrict__ idx,
                    const T *__restrict__ val, const T *__restrict__ F, const T *__restrict__ W,
                    int k, const LossOf<T> *__restrict__ loss, T *__restrict__ part_grad,
                    double *__restrict__ part_loss, int *__restrict__ err, int cap)
{
    extern __shared__ __align__(128) unsigned char dsm[];
    __shared__ uint64_t bar_panel;
    __shared__ uint64_t bar_seg[kStreamWarps][2];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    T *Ws = reinterpret_cast<T *>(dsm);
    size_t off = align16((size_t)R * K * sizeof(T));
    LossOf<T> *Ls = reinterpret_cast<LossOf<T> *>(dsm + off);
    if constexpr (XSTEP) off += (size_t)R * sizeof(LossOf<T>);
    EntryStream<T> st;
    st.init(dsm + off + (size_t)wid * stream_bytes<T>(cap), &bar_seg[wid][0], cap);
    if (threadIdx.x == 0) mbar_init(&bar_panel, 1);
    if (lane == 0) {
        mbar_init(&bar_seg[wid][0], 1);
        mbar_init(&bar_seg[wid][1], 1);
    }
    __syncthreads();
    const int64_t seg_per = (nseg + ngroups - 1) / ngroups;
    const int64_t nunits = (int64_t)nb * ngroups;
    unsigned pphase = 0;
    for (int64_t u = blockIdx.x; u < nunits; u += gridDim.x) {
        const int b = (int)(u / ngroups);
        const int64_t grp = u % ngroups;
        const int64_t r0 = (int64_t)b * R;
        const int rows = (int)((r0 + R <= nother) ? R : nother - r0);
        __syncthreads();  // previous panel no longer in use
        if constexpr (XSTEP) {
            for (int q = threadIdx.x; q < rows; q += blockDim.x) Ls[q] = loss[r0 + q];
        }
        if (!stage_panel<T>(Ws, W, r0, rows, k, K, &bar_panel, pphase, err)) return;
        pphase ^= 1u;
        const int64_t s0 = grp * seg_per;
        const int64_t s1 = s0 + seg_per < nseg ? s0 + seg_per : nseg;
        int64_t s = s0 + wid;
        int cur = 0;
        bool bad = false;
        if (s < s1) {
            const int64_t slot = (int64_t)b * nseg + s;
            st.issue(0, runptr[slot], runptr[slot + nseg], idx, val);
        }
        for (; s < s1; s += kStreamWarps) {
            const int64_t nx = s + kStreamWarps;
            if (nx < s1) {
                const int64_t ns = (int64_t)b * nseg + nx;
                st.issue(cur ^ 1, runptr[ns], runptr[ns + nseg], idx, val);
            }
            if (!st.wait(cur)) {
                if (nx < s1) st.wait(cur ^ 1);
                bad = true;
                break;
            }
            const int64_t slot = (int64_t)b * nseg + s;
            const int qb = runptr[slot], qe = runptr[slot + nseg];
            Vec<T, K> f, g;
            f.load_masked(F + s * k, k);
            g.zero();
            LossOf<T> sp;
            if constexpr (!XSTEP) sp = loss[s];
            const T lsum = seg_pass_any<T, K, XSTEP, GRAD>(st, cur, f, g, qb, qe, (int)r0, idx, val,
                                                          Ws, Ls, sp);
            const double ls = warp_sum((double)lsum);
            if constexpr (GRAD) {
                g.warp_allsum();
#pragma unroll
                for (int c = 0; c < K; ++c)
                    if (lane == (c & 31)) part_grad[slot * K + c] = g.get(c);
            }
            if (lane == 0) part_loss[slot] = ls;
            cur ^= 1;
        }
        if (__syncthreads_or(bad)) {
            if (threadIdx.x == 0) atomicOr(err, 1);
            return;
        }
    }
}

inline cudaError_t launch_build_runptr_impl(const Orient &o, cudaStream_t st)
{
    const int64_t items = (int64_t)(o.nb + 1) * o.nseg;
    build_runptr_kernel<<<blocks_for(items, 256), 256, 0, st>>>(o.nseg, o.nb, o.R, o.ptr, o.idx,
                                                                o.runptr);
    return cudaGetLastError();
}

// prox over segments with partials strided by nseg over nb panels.
template <class T, int K>
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
blocked_prox_kernel(int64_t nseg, int nb, const T *__restrict__ part_grad,
                    const double *__restrict__ part_loss, const T *__restrict__ F,
                    const T *__restrict__ alpha, int k, int rkind, T rw, T *__restrict__ cand,
                    double *__restrict__ f_old, double *__restrict__ r_old, double *__restrict__ r_new)
{
    const int lane = threadIdx.x & 31;
    const int64_t s = (int64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
    if (s >= nseg) return;
    const T al = alpha[s];
    T ro = T(0), rn = T(0);
    for (int c = lane; c < k; c += 32) {
        T g = T(0);
        for (int b = 0; b < nb; ++b) g += part_grad[((int64_t)b * nseg + s) * K + c];
        const T x = F[s * k + c];
        const int rkc = reg_kind_at(rkind, c, k);
        const T xp = prox1<T>(rkc, rw, al, x - al * g);
        cand[s * k + c] = xp;
        ro += reg1t<T>(rkc, rw, x);
        rn += reg1t<T>(rkc, rw, xp);
    }
    ro = warp_sum(ro);
    rn = warp_sum(rn);
    double ls = 0.0;
    for (int b = lane; b < nb; b += 32) ls += part_loss[(int64_t)b * nseg + s];
    ls = warp_sum(ls);
    if (lane == 0) {
        f_old[s] = ls + ro;
        r_old[s] = ro;
        r_new[s] = rn;
    }
}

template <class T>
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
blocked_decide_kernel(int64_t nseg, int nb, const double *__restrict__ part_loss_new,
                      const double *__restrict__ f_old, const double *__restrict__ r_old,
                      const double *__restrict__ r_new, const T *__restrict__ cand,
                      T *__restrict__ F, T *__restrict__ alpha, int k,
                      double *__restrict__ kept_obj, double *__restrict__ kept_reg,
                      int32_t *__restrict__ accepted)
{
    const int lane = threadIdx.x & 31;
    const int64_t s = (int64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
    if (s >= nseg) return;
    double ls = 0.0;
    for (int b = lane; b < nb; b += 32) ls += part_loss_new[(int64_t)b * nseg + s];
    const double fn = warp_sum(ls) + r_new[s];
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

template <class T, int K, bool XSTEP>
cudaError_t launch_fused(glrm_s *h, const Orient &o, T *F, const T *W, int64_t nother, T *alpha,
                         int rk, T rw, double *kept_obj, double *kept_reg, int32_t *acc)
{
    auto kern = fused_half_kernel<T, K, XSTEP>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)o.smem_bytes);
    if (e != cudaSuccess) return e;
    kern<<<o.grid, kStreamWarps * 32, o.smem_bytes, h->stream>>>(
        o.nseg, o.ptr, o.idx, (const T *)o.val, F, W, nother, h->k, alpha, loss_of<T>(h), rk, rw,
        kept_obj, kept_reg, acc, h->s.err, o.cap);
    return cudaGetLastError();
}

template <class T, int K, bool XSTEP, bool GRAD>
cudaError_t launch_blocked_pass(glrm_s *h, const Orient &o, const T *F, const T *W, int64_t nother,
                                T *part_grad, double *part_loss)
{
    auto kern = blocked_pass_kernel<T, K, XSTEP, GRAD>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)o.smem_bytes);
    if (e != cudaSuccess) return e;
    kern<<<o.grid, kStreamWarps * 32, o.smem_bytes, h->stream>>>(
        o.nseg, o.nb, o.R, o.ngroups, nother, o.runptr, o.idx, (const T *)o.val, F, W, h->k,
        loss_of<T>(h), part_grad, part_loss, h->s.err, o.cap);
    return cudaGetLastError();
}

template <class T, int K, bool XSTEP>
cudaError_t tiled_half_K(glrm_s *h, bool xstep_unused)
{
    (void)xstep_unused;
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
    if (o.mode == kModeFused) {
        tmark(h, XSTEP ? "fused_x" : "fused_y");
        e = launch_fused<T, K, XSTEP>(h, o, F, W, nother, alpha, rk, rw, kobj, kreg, acc);
        tmark(h, nullptr);
        h->launches += 1;
        return e;
    }
    // blocked
    tmark(h, XSTEP ? "blocked_grad_x" : "blocked_grad_y");
    e = launch_blocked_pass<T, K, XSTEP, true>(h, o, F, W, nother, (T *)s.part_grad, s.part_loss);
    if (e != cudaSuccess) return e;
    const unsigned nbs = blocks_for(o.nseg, kWarpsPerBlock);
    tmark(h, XSTEP ? "blocked_prox_x" : "blocked_prox_y");
    blocked_prox_kernel<T, K><<<nbs, kWarpsPerBlock * 32, 0, h->stream>>>(
        o.nseg, o.nb, (const T *)s.part_grad, s.part_loss, F, alpha, h->k, rk, rw, (T *)s.cand,
        s.f_old, s.r_old, s.r_new);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    tmark(h, XSTEP ? "blocked_loss_x" : "blocked_loss_y");
    e = launch_blocked_pass<T, K, XSTEP, false>(h, o, (const T *)s.cand, W, nother, nullptr,
                                                s.part_loss2);
    if (e != cudaSuccess) return e;
    tmark(h, XSTEP ? "blocked_decide_x" : "blocked_decide_y");
    blocked_decide_kernel<T><<<nbs, kWarpsPerBlock * 32, 0, h->stream>>>(
        o.nseg, o.nb, s.part_loss2, s.f_old, s.r_old, s.r_new, (const T *)s.cand, F, alpha, h->k,
        kobj, kreg, acc);
    tmark(h, nullptr);
    h->launches += 4;
    return cudaGetLastError();
}

template <class T, bool XSTEP>
cudaError_t tiled_half(glrm_s *h)
{
    const int k = h->k;
    if (k <= 4) return tiled_half_K<T, 4, XSTEP>(h, XSTEP);
    if (k <= 8) return tiled_half_K<T, 8, XSTEP>(h, XSTEP);
    if (k <= 12) return tiled_half_K<T, 12, XSTEP>(h, XSTEP);
    if (k <= 16) return tiled_half_K<T, 16, XSTEP>(h, XSTEP);
    if (k <= 20) return tiled_half_K<T, 20, XSTEP>(h, XSTEP);
    if (k <= 24) return tiled_half_K<T, 24, XSTEP>(h, XSTEP);
    if (k <= 32) return tiled_half_K<T, 32, XSTEP>(h, XSTEP);
    return cudaErrorInvalidValue;
}

template <class T>
cudaError_t Engine<T>::tiled_half_step(glrm_s *h, bool xstep)
{
    return xstep ? tiled_half<T, true>(h) : tiled_half<T, false>(h);
}

}  // namespace glrm
