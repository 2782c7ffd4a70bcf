// Kernels of the alternating proximal-gradient sweep (Algorithm 2 with the
// proximal gradient update and the step-size rule of Section 7.2 of Udell et
// al., "Generalized Low Rank Models") and of the objective, gradient and
// imputation, templated on the element type T and the padded rank K.
//
// A half-step updates the factor F of every segment (row x_i of X in the
// X-step over CSR, column y_j of Y in the Y-step over CSC) against the other
// factor W, in four launches:
//   pass_kernel<GRAD=1>  per chunk: u = f . w_idx, L'(u, a), partial gradient
//                        sum L' w and partial loss sum L
//   prox_kernel          per segment: g = sum of partials, f+ = prox(f - alpha g),
//                        f_old = loss + r(f), r(f+)
//   pass_kernel<GRAD=0>  per chunk: partial loss at f+
//   decide_kernel        per segment: keep f+ (alpha *= 1.05) if
//                        f_new <= f_old, else keep f (alpha *= 0.7)
// Chunks hold at most kChunk entries, so long columns spread over many warps.
// All reductions run in a fixed order: results are bitwise reproducible.
#pragma once

#include <type_traits>

#include "glrm_handle.h"

namespace glrm {

constexpr int kWarpsPerBlock = 8;

template <int K>
struct Lanes {
    // G lanes share one entry, each holding S = K / G coordinates.
    static constexpr int G = K > 32 ? 4 : 1;
    static constexpr int S = K / G;
    static constexpr int PER = 32 / G;  // entries per warp iteration
};

// Lane layout of an entry's k coordinates over the G lanes that share it.
// The vector form cuts a row into 16-byte units of VW coordinates (VW = 4
// FP32, 2 FP64, 8 BF16 values) and gives lane gl units gl, G + gl, 2G + gl,
// ...: at every load instruction the G lanes of an entry read G adjacent
// units, whole 32-byte sectors of the row, so each sector is fetched once.
// Slot s of lane gl holds coordinate VW ((s / VW) G + gl) + s % VW.  The
// scalar form (any k) gives lane gl the contiguous coordinates gl S .. gl S + S - 1.
template <int S, int G, int VW, bool VEC>
__device__ __forceinline__ int slot_coord(int s, int gl)
{
    return VEC ? VW * ((s / VW) * G + gl) + s % VW : gl * S + s;
}

// A row's slots for lane gl in the layout above (T values, units of VW).
template <class T, int S, int G, int VW, bool VEC>
__device__ __forceinline__ void load_lane(T (&v)[S], const T *__restrict__ row, int gl, int k)
{
    if constexpr (VEC) {
        constexpr int VT = 16 / (int)sizeof(T);  // values per 16-byte load
        static_assert(S % VW == 0 && VW % VT == 0, "slots must be whole units");
#pragma unroll
        for (int q = 0; q < S / VW; ++q) {
#pragma unroll
            for (int h = 0; h < VW / VT; ++h) {
                const T *src = row + VW * (q * G + gl) + VT * h;
                if constexpr (sizeof(T) == 4) {
                    const float4 t = __ldg(reinterpret_cast<const float4 *>(src));
                    v[q * VW + VT * h + 0] = t.x;
                    v[q * VW + VT * h + 1] = t.y;
                    v[q * VW + VT * h + 2] = t.z;
                    v[q * VW + VT * h + 3] = t.w;
                } else {
                    const double2 t = __ldg(reinterpret_cast<const double2 *>(src));
                    v[q * VW + VT * h + 0] = t.x;
                    v[q * VW + VT * h + 1] = t.y;
                }
            }
        }
    } else {
#pragma unroll
        for (int s = 0; s < S; ++s) v[s] = (gl * S + s < k) ? __ldg(row + gl * S + s) : T(0);
    }
}

// The same for a BF16 row (units of 8 values), widened to FP32.
template <int S, int G, bool VEC>
__device__ __forceinline__ void load_lane_bf16(float (&v)[S], const __nv_bfloat16 *__restrict__ row, int gl,
                                               int k)
{
    if constexpr (VEC) {
        static_assert(S % 8 == 0, "bf16 slots must be whole units");
#pragma unroll
        for (int q = 0; q < S / 8; ++q) {
            const uint4 t = __ldg(reinterpret_cast<const uint4 *>(row + 8 * (q * G + gl)));
            const uint32_t w[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                v[8 * q + 2 * h] = __uint_as_float(w[h] << 16);
                v[8 * q + 2 * h + 1] = __uint_as_float(w[h] & 0xffff0000u);
            }
        }
    } else {
#pragma unroll
        for (int s = 0; s < S; ++s) v[s] = (gl * S + s < k) ? __bfloat162float(row[gl * S + s]) : 0.f;
    }
}

// Coordinates per 16-byte unit of a row of type WT.
template <class WT>
constexpr int unit_of() { return 16 / (int)sizeof(WT); }

template <class T, int S, int G, bool VEC, class WT>
__device__ __forceinline__ void load_lane_w(T (&v)[S], const WT *__restrict__ row, int gl, int k)
{
    if constexpr (std::is_same<WT, __nv_bfloat16>::value) load_lane_bf16<S, G, VEC>(v, row, gl, k);
    else load_lane<T, S, G, unit_of<WT>(), VEC>(v, row, gl, k);
}

// One warp per chunk: entries base + grp for base = begin, begin + PER, ...
// (G lanes per entry, PER = 32 / G entries per iteration), the rows of the
// other factor gathered in the lane layout above.  `order` (nullable) is the
// chunk launch order; with `sel` (nullable) the launch takes only the chunks
// of segments whose sel value is nonzero exactly when want is.  `lsc`
// (nullable) holds per-column loss weights: entry (i, j) contributes
// lsc[j] L_j and lsc[j] L_j' (the scaled losses of Section 4.3).
template <class T, int K, bool XSTEP, bool VEC, bool GRAD, class WT = T>
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
pass_kernel(int64_t nchunks, const int4 *__restrict__ chunks, const int32_t *__restrict__ order,
            const int32_t *__restrict__ idx, const T *__restrict__ val, const T *__restrict__ F,
            const WT *__restrict__ W, int k, const LossOf<T> *__restrict__ loss, T *__restrict__ part_grad,
            double *__restrict__ part_loss, const int32_t *__restrict__ sel, int want,
            const T *__restrict__ lsc)
{
    using LN = Lanes<K>;
    constexpr int G = LN::G, S = LN::S, PER = LN::PER;
    constexpr int VW = unit_of<WT>();  // f and the gathered rows share the layout of WT's units
    const int lane = threadIdx.x & 31;
    const int64_t lin = (int64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
    if (lin >= nchunks) return;  // the whole warp leaves together
    const int64_t c = order ? (int64_t)__ldg(order + lin) : lin;
    const int gl = lane % G, grp = lane / G;
    const int4 ch = chunks[c];
    if (sel && ((__ldg(sel + ch.x) != 0) != (want != 0))) return;  // another launch takes this segment
    T f[S], g[S];
    load_lane<T, S, G, VW, VEC>(f, F + (int64_t)ch.x * k, gl, k);
#pragma unroll
    for (int s = 0; s < S; ++s) g[s] = T(0);
    T lsum = T(0);
    LossOf<T> sp;
    T wsc = T(1);
    if constexpr (!XSTEP) {
        sp = loss[ch.x];
        if (lsc) wsc = __ldg(lsc + ch.x);
    }
    if constexpr (!GRAD) {
        // loss passes: a software pipeline, the next group of entries' index,
        // value, loss and gathered row loaded before the current group is
        // evaluated (two gathers per lane in flight).  The gradient passes
        // keep one: their gradient registers would cut the occupancy more
        // than the second gather gains (94 against 73 registers, measured
        // slower on the k = 64 completion table).
        int jn = 0;
        T an = T(0);
        T wn[S];
        LossOf<T> spn = sp;
        T wscn = wsc;
        auto fetch = [&](int e) {
            if (e < ch.z) {
                jn = __ldg(idx + e);
                an = __ldg(val + e);
                load_lane_w<T, S, G, VEC, WT>(wn, W + (int64_t)jn * k, gl, k);
                if constexpr (XSTEP) {
                    spn = loss[jn];
                    if (lsc) wscn = __ldg(lsc + jn);
                }
            } else {
#pragma unroll
                for (int s = 0; s < S; ++s) wn[s] = T(0);
            }
        };
        fetch(ch.y + grp);
        for (int base = ch.y; base < ch.z; base += PER) {
            const bool ok = base + grp < ch.z;
            const T a = an;
            T w[S];
#pragma unroll
            for (int s = 0; s < S; ++s) w[s] = wn[s];
            if constexpr (XSTEP) {
                sp = spn;
                wsc = wscn;
            }
            fetch(base + PER + grp);
            T u = T(0);
#pragma unroll
            for (int s = 0; s < S; ++s) u = fma(f[s], w[s], u);
#pragma unroll
            for (int o = 1; o < G; o <<= 1) u += shfl_xor(u, o);
            if (ok) {
                T L;
                loss_deriv<T>(sp, u, a, L);
                if (lsc) L *= wsc;
                if (gl == 0) lsum += L;
            }
        }
    } else {
        for (int base = ch.y; base < ch.z; base += PER) {
            const int e = base + grp;
            const bool ok = e < ch.z;
            int j = 0;
            T a = T(0);
            T w[S];
            if (ok) {
                j = __ldg(idx + e);
                a = __ldg(val + e);
                load_lane_w<T, S, G, VEC, WT>(w, W + (int64_t)j * k, gl, k);
            } else {
#pragma unroll
                for (int s = 0; s < S; ++s) w[s] = T(0);
            }
            T u = T(0);
#pragma unroll
            for (int s = 0; s < S; ++s) u = fma(f[s], w[s], u);
#pragma unroll
            for (int o = 1; o < G; o <<= 1) u += shfl_xor(u, o);
            if (ok) {
                if constexpr (XSTEP) {
                    sp = loss[j];
                    if (lsc) wsc = __ldg(lsc + j);
                }
                T L;
                T d = loss_deriv<T>(sp, u, a, L);
                if (lsc) {
                    d *= wsc;
                    L *= wsc;
                }
#pragma unroll
                for (int s = 0; s < S; ++s) g[s] = fma(d, w[s], g[s]);
                if (gl == 0) lsum += L;
            }
        }
    }
    if constexpr (GRAD) {
#pragma unroll
        for (int s = 0; s < S; ++s) {
#pragma unroll
            for (int o = G; o < 32; o <<= 1) g[s] += shfl_xor(g[s], o);
        }
        if (grp == 0) {
#pragma unroll
            for (int s = 0; s < S; ++s) {
                const int cc = slot_coord<S, G, VW, VEC>(s, gl);
                if (cc < k) part_grad[c * k + cc] = g[s];
            }
        }
    }
    const double ls = warp_sum((double)lsum);
    if (lane == 0) part_loss[c] = ls;
}

// Round FP32 values to BF16 (round to nearest even).
static __global__ void to_bf16_kernel(const float *__restrict__ src, int64_t n, __nv_bfloat16 *__restrict__ dst)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = __float2bfloat16_rn(src[i]);
}

// Sum of a segment's chunk partials, lanes strided then a butterfly: fixed order.
__device__ __forceinline__ double seg_loss_sum(const double *__restrict__ part, int c_beg, int c_end,
                                               int lane)
{
    if (c_end - c_beg == 1) return part[c_beg];  // one partial: no FP64 reduction (slow on GB300)
    double v = 0.0;
    for (int c = c_beg + lane; c < c_end; c += 32) v += part[c];
    return warp_sum(v);
}

template <class T>
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
prox_kernel(int64_t nseg, const int32_t *__restrict__ segchunk, const T *__restrict__ part_grad,
            const double *__restrict__ part_loss, const T *__restrict__ F,
            const T *__restrict__ alpha, int k, int rkind, T rw, T *__restrict__ cand,
            double *__restrict__ f_old, double *__restrict__ r_old, double *__restrict__ r_new)
{
    const int lane = threadIdx.x & 31;
    const int64_t s = (int64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
    if (s >= nseg) return;
    const int cb = segchunk[s], ce = segchunk[s + 1];
    const T al = alpha[s];
    T ro = T(0), rn = T(0);
    for (int c = lane; c < k; c += 32) {
        // in slot order; unrolled so the loads of a segment with many slots overlap
        T g = ce > cb ? part_grad[(int64_t)cb * k + c] : T(0);
        if (ce - cb > 1) {
#pragma unroll 8
            for (int q = cb + 1; q < ce; ++q) g += part_grad[(int64_t)q * k + c];
        }
        const T x = F[s * k + c];
        const int rkc = reg_kind_at(rkind, c, k);
        const T xp = prox1<T>(rkc, rw, al, x - al * g);
        cand[s * k + c] = xp;
        ro += reg1t<T>(rkc, rw, x);
        rn += reg1t<T>(rkc, rw, xp);
    }
    ro = warp_sum(ro);
    rn = warp_sum(rn);
    const double ls = seg_loss_sum(part_loss, cb, ce, lane);
    if (lane == 0) {
        f_old[s] = ls + ro;
        r_old[s] = ro;
        r_new[s] = rn;
    }
}

template <class T>
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
decide_kernel(int64_t nseg, const int32_t *__restrict__ segchunk,
              const double *__restrict__ part_loss_new, const double *__restrict__ f_old,
              const double *__restrict__ r_old, const double *__restrict__ r_new,
              const T *__restrict__ cand, T *__restrict__ F, T *__restrict__ alpha, int k,
              double *__restrict__ kept_obj, double *__restrict__ kept_reg,
              int32_t *__restrict__ accepted, const double *__restrict__ part_loss_old = nullptr)
{
    const int lane = threadIdx.x & 31;
    const int64_t s = (int64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
    if (s >= nseg) return;
    const double fn = seg_loss_sum(part_loss_new, segchunk[s], segchunk[s + 1], lane) + r_new[s];
    // f_old from the prox step, or (part_loss_old given) from the chunk partials of a later pass
    const double fo = part_loss_old ? seg_loss_sum(part_loss_old, segchunk[s], segchunk[s + 1], lane) + r_old[s]
                                    : f_old[s];
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

// The same two steps with LG lanes per segment (32 / LG segments per warp),
// for half-steps with many segments: a warp per segment leaves most lanes
// idle at small k and runs as many warps as segments.  Partial gradients are
// summed per coordinate in slot order as above; the segment's FP64 loss
// partials in slot order by each lane of the group.
template <class T, int LG>
__global__ void __launch_bounds__(256)
prox_narrow_kernel(int64_t nseg, const int32_t *__restrict__ segchunk, const T *__restrict__ part_grad,
                   const double *__restrict__ part_loss, const T *__restrict__ F, const T *__restrict__ alpha,
                   int k, int rkind, T rw, T *__restrict__ cand, double *__restrict__ f_old,
                   double *__restrict__ r_old, double *__restrict__ r_new)
{
    const int gl = threadIdx.x % LG;
    const int64_t s = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / LG;
    const bool live = s < nseg;  // whole groups: the shuffles below run on every lane
    int cb = 0, ce = 0;
    T al = T(0);
    if (live) {
        cb = segchunk[s];
        ce = segchunk[s + 1];
        al = alpha[s];
    }
    T ro = T(0), rn = T(0);
    if (live)
        for (int c = gl; c < k; c += LG) {
            T g = T(0);
            for (int q = cb; q < ce; ++q) g += part_grad[(int64_t)q * k + c];
            const T x = F[s * k + c];
            const int rkc = reg_kind_at(rkind, c, k);
            const T xp = prox1<T>(rkc, rw, al, x - al * g);
            cand[s * k + c] = xp;
            ro += reg1t<T>(rkc, rw, x);
            rn += reg1t<T>(rkc, rw, xp);
        }
#pragma unroll
    for (int o = 1; o < LG; o <<= 1) {
        ro += shfl_xor(ro, o);
        rn += shfl_xor(rn, o);
    }
    if (live && gl == 0) {
        double ls = 0.0;
        for (int q = cb; q < ce; ++q) ls += part_loss[q];
        f_old[s] = ls + ro;
        r_old[s] = ro;
        r_new[s] = rn;
    }
}

template <class T, int LG>
__global__ void __launch_bounds__(256)
decide_narrow_kernel(int64_t nseg, const int32_t *__restrict__ segchunk, const double *__restrict__ part_loss_new,
                     const double *__restrict__ f_old, const double *__restrict__ r_old,
                     const double *__restrict__ r_new, const T *__restrict__ cand, T *__restrict__ F,
                     T *__restrict__ alpha, int k, double *__restrict__ kept_obj, double *__restrict__ kept_reg,
                     int32_t *__restrict__ accepted, const double *__restrict__ part_loss_old)
{
    const int gl = threadIdx.x % LG;
    const int64_t s = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / LG;
    if (s >= nseg) return;  // no shuffles here
    const int cb = segchunk[s], ce = segchunk[s + 1];
    double fn = 0.0;
    for (int q = cb; q < ce; ++q) fn += part_loss_new[q];
    fn += r_new[s];
    double fo;
    if (part_loss_old) {
        fo = 0.0;
        for (int q = cb; q < ce; ++q) fo += part_loss_old[q];
        fo += r_old[s];
    } else {
        fo = f_old[s];
    }
    const bool acc = fn <= fo;
    if (acc)
        for (int c = gl; c < k; c += LG) F[s * k + c] = cand[s * k + c];
    if (gl == 0) {
        alpha[s] = alpha[s] * (acc ? T(1.05) : T(0.7));
        kept_obj[s] = acc ? fn : fo;
        kept_reg[s] = acc ? r_new[s] : r_old[s];
        accepted[s] = acc ? 1 : 0;
    }
}

inline unsigned blocks_for(int64_t items, int per_block)
{
    return (unsigned)((items + per_block - 1) / per_block);
}

// Segments above which the prox / decide steps run LG lanes per segment.
constexpr int64_t kNarrowSegments = 32768;

template <class T>
cudaError_t launch_prox(int64_t nseg, const int32_t *segchunk, const T *part_grad, const double *part_loss,
                        const T *F, const T *alpha, int k, int rk, T rw, T *cand, double *f_old, double *r_old,
                        double *r_new, cudaStream_t st)
{
    if (nseg >= kNarrowSegments && k <= 64) {
        if (k <= 16)
            prox_narrow_kernel<T, 4><<<(unsigned)((nseg * 4 + 255) / 256), 256, 0, st>>>(
                nseg, segchunk, part_grad, part_loss, F, alpha, k, rk, rw, cand, f_old, r_old, r_new);
        else
            prox_narrow_kernel<T, 8><<<(unsigned)((nseg * 8 + 255) / 256), 256, 0, st>>>(
                nseg, segchunk, part_grad, part_loss, F, alpha, k, rk, rw, cand, f_old, r_old, r_new);
    } else {
        prox_kernel<T><<<blocks_for(nseg, kWarpsPerBlock), kWarpsPerBlock * 32, 0, st>>>(
            nseg, segchunk, part_grad, part_loss, F, alpha, k, rk, rw, cand, f_old, r_old, r_new);
    }
    return cudaGetLastError();
}

template <class T>
cudaError_t launch_decide(int64_t nseg, const int32_t *segchunk, const double *part_loss_new, const double *f_old,
                          const double *r_old, const double *r_new, const T *cand, T *F, T *alpha, int k,
                          double *kept_obj, double *kept_reg, int32_t *accepted, cudaStream_t st,
                          const double *part_loss_old = nullptr)
{
    if (nseg >= kNarrowSegments && k <= 64) {
        if (k <= 16)
            decide_narrow_kernel<T, 4><<<(unsigned)((nseg * 4 + 255) / 256), 256, 0, st>>>(
                nseg, segchunk, part_loss_new, f_old, r_old, r_new, cand, F, alpha, k, kept_obj, kept_reg, accepted,
                part_loss_old);
        else
            decide_narrow_kernel<T, 8><<<(unsigned)((nseg * 8 + 255) / 256), 256, 0, st>>>(
                nseg, segchunk, part_loss_new, f_old, r_old, r_new, cand, F, alpha, k, kept_obj, kept_reg, accepted,
                part_loss_old);
    } else {
        decide_kernel<T><<<blocks_for(nseg, kWarpsPerBlock), kWarpsPerBlock * 32, 0, st>>>(
            nseg, segchunk, part_loss_new, f_old, r_old, r_new, cand, F, alpha, k, kept_obj, kept_reg, accepted,
            part_loss_old);
    }
    return cudaGetLastError();
}

// Deterministic two-level sums.  Stage 1: block b sums a fixed contiguous
// range of each source; stage 2: one block sums the kRedBlocks partials.
template <class T>
__global__ void __launch_bounds__(256)
reduce_stage1(const double *__restrict__ a, int64_t na, const double *__restrict__ b, int64_t nb,
              const T *__restrict__ X, int64_t m, int rxk, T rxw, const T *__restrict__ Yt,
              int64_t n, int ryk, T ryw, int k, const int32_t *__restrict__ ca, int64_t nca,
              const int32_t *__restrict__ cb, int64_t ncb, double *__restrict__ part,
              long long *__restrict__ cnt)
{
    __shared__ double sh[256];
    __shared__ long long shc[2][256];
    double v = 0.0;
    long long c1 = 0, c2 = 0;
    auto range = [&](int64_t len, int64_t &lo, int64_t &hi) {
        const int64_t per = (len + gridDim.x - 1) / gridDim.x;
        lo = per * blockIdx.x;
        hi = lo + per < len ? lo + per : len;
    };
    int64_t lo, hi;
    if (a) { range(na, lo, hi); for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) v += a[i]; }
    if (b) { range(nb, lo, hi); for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) v += b[i]; }
    if (X) {
        range(m * k, lo, hi);
        for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x)
            v += reg1<T>(reg_kind_at(rxk, (int)(i % k), k), rxw, X[i]);
    }
    if (Yt) {
        range(n * k, lo, hi);
        for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x)
            v += reg1<T>(reg_kind_at(ryk, (int)(i % k), k), ryw, Yt[i]);
    }
    if (ca) { range(nca, lo, hi); for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) c1 += ca[i]; }
    if (cb) { range(ncb, lo, hi); for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) c2 += cb[i]; }
    sh[threadIdx.x] = v;
    shc[0][threadIdx.x] = c1;
    shc[1][threadIdx.x] = c2;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            sh[threadIdx.x] += sh[threadIdx.x + o];
            shc[0][threadIdx.x] += shc[0][threadIdx.x + o];
            shc[1][threadIdx.x] += shc[1][threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[blockIdx.x] = sh[0];
        cnt[2 * blockIdx.x] = shc[0][0];
        cnt[2 * blockIdx.x + 1] = shc[1][0];
    }
}

static __global__ void __launch_bounds__(256)
reduce_stage2(const double *__restrict__ part, const long long *__restrict__ cnt, int nparts,
              double *__restrict__ out, long long *__restrict__ cnt_out)
{
    __shared__ double sh[256];
    __shared__ long long shc[2][256];
    double v = 0.0;
    long long c1 = 0, c2 = 0;
    for (int i = threadIdx.x; i < nparts; i += blockDim.x) {
        v += part[i];
        c1 += cnt[2 * i];
        c2 += cnt[2 * i + 1];
    }
    sh[threadIdx.x] = v;
    shc[0][threadIdx.x] = c1;
    shc[1][threadIdx.x] = c2;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            sh[threadIdx.x] += sh[threadIdx.x + o];
            shc[0][threadIdx.x] += shc[0][threadIdx.x + o];
            shc[1][threadIdx.x] += shc[1][threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        if (out) *out = sh[0];
        if (cnt_out) {
            cnt_out[0] = shc[0][0];
            cnt_out[1] = shc[1][0];
        }
    }
}

// Gradient of each segment: sum of its chunk partials (+ the regulariser's
// gradient), one warp per segment, lanes over coordinates.
template <class T>
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
seg_grad_kernel(int64_t nseg, const int32_t *__restrict__ segchunk, const T *__restrict__ part_grad,
                const T *__restrict__ F, int k, int rkind, T rw, bool reg,
                const double *__restrict__ scale, T *__restrict__ G)
{
    const int lane = threadIdx.x & 31;
    const int64_t s = (int64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
    if (s >= nseg) return;
    const int cb = segchunk[s], ce = segchunk[s + 1];
    const T sc = scale ? (T)*scale : T(1);
    for (int c = lane; c < k; c += 32) {
        // in slot order; unrolled so the loads of a segment with many slots overlap
        T g = ce > cb ? part_grad[(int64_t)cb * k + c] : T(0);
        if (ce - cb > 1) {
#pragma unroll 8
            for (int q = cb + 1; q < ce; ++q) g += part_grad[(int64_t)q * k + c];
        }
        if (reg) g += reg_grad1<T>(reg_kind_at(rkind, c, k), rw, F[s * k + c]);
        G[s * k + c] = sc * g;
    }
}

template <class T>
__global__ void predict_kernel(int64_t cnt, const int32_t *__restrict__ rows,
                               const int32_t *__restrict__ cols, const T *__restrict__ X,
                               const T *__restrict__ Yt, int64_t m, int64_t n, int k,
                               const LossSpec *__restrict__ loss, bool decode, T *__restrict__ out)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= cnt) return;
    const int32_t i = rows[e], j = cols[e];
    if (i < 0 || i >= m || j < 0 || j >= n) {
        out[e] = T(NAN);
        return;
    }
    T u = T(0);
    for (int c = 0; c < k; ++c) u = fma(X[(int64_t)i * k + c], Yt[(int64_t)j * k + c], u);
    out[e] = decode ? decode_value<T>(loss[j], u) : u;
}

template <class T>
__global__ void reset_alpha_kernel(const int32_t *__restrict__ ptr, int64_t nseg, T *__restrict__ alpha)
{
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nseg) return;
    const int len = ptr[s + 1] - ptr[s];
    alpha[s] = T(1) / T(len > 1 ? len : 1);
}

// ------------------------------------------------------------------ launchers


template <class T, int K, bool XSTEP, bool GRAD, class WT>
cudaError_t launch_pass(const Orient &o, const T *F, const WT *W, int k, const LossOf<T> *loss,
                        T *part_grad, double *part_loss, cudaStream_t st, const int32_t *sel, int want,
                        const T *lsc)
{
    if (o.nchunks == 0) return cudaSuccess;
    // the BF16 copy is read 8 values at a time, so its vector path needs k % 8 == 0
    constexpr int kVecMult = std::is_same<WT, __nv_bfloat16>::value ? 8 : 1;
    const bool vec = (k == K) && (Lanes<K>::S % kVecMult == 0) &&
                     ((reinterpret_cast<uintptr_t>(F) | reinterpret_cast<uintptr_t>(W)) % 16 == 0);
    const unsigned nb = blocks_for(o.nchunks, kWarpsPerBlock);
    if constexpr (std::is_same<WT, __nv_bfloat16>::value && Lanes<K>::S % 8 != 0) {
        pass_kernel<T, K, XSTEP, false, GRAD, WT><<<nb, kWarpsPerBlock * 32, 0, st>>>(
            o.nchunks, o.chunks, o.order, o.idx, (const T *)o.val, F, W, k, loss, part_grad, part_loss, sel, want, lsc);
    } else {
        if (vec)
            pass_kernel<T, K, XSTEP, true, GRAD, WT><<<nb, kWarpsPerBlock * 32, 0, st>>>(
                o.nchunks, o.chunks, o.order, o.idx, (const T *)o.val, F, W, k, loss, part_grad, part_loss, sel, want, lsc);
        else
            pass_kernel<T, K, XSTEP, false, GRAD, WT><<<nb, kWarpsPerBlock * 32, 0, st>>>(
                o.nchunks, o.chunks, o.order, o.idx, (const T *)o.val, F, W, k, loss, part_grad, part_loss, sel, want, lsc);
    }
    return cudaGetLastError();
}

// Dispatch a runtime k to the smallest padded width K >= k.
template <class T, bool XSTEP, bool GRAD, class WT = T>
cudaError_t dispatch_pass(const Orient &o, const T *F, const WT *W, int k, const LossOf<T> *loss,
                          T *part_grad, double *part_loss, cudaStream_t st, const int32_t *sel = nullptr,
                          int want = 0, const T *lsc = nullptr)
{
#define GLRM_PASS_CASE(KK) \
    if (k <= KK) return launch_pass<T, KK, XSTEP, GRAD, WT>(o, F, W, k, loss, part_grad, part_loss, st, sel, want, lsc);
    GLRM_PASS_CASE(4)
    GLRM_PASS_CASE(8)
    GLRM_PASS_CASE(12)
    GLRM_PASS_CASE(16)
    GLRM_PASS_CASE(20)
    GLRM_PASS_CASE(24)
    GLRM_PASS_CASE(32)
    GLRM_PASS_CASE(48)
    GLRM_PASS_CASE(64)
#undef GLRM_PASS_CASE
    return cudaErrorInvalidValue;
}

template <class T>
cudaError_t Engine<T>::half_step(glrm_s *h, bool xstep)
{
    const Orient &o = xstep ? h->csr : h->csc;
    T *F = (T *)(xstep ? h->X : h->Yt);
    const T *W = (const T *)(xstep ? h->Yt : h->X);
    T *alpha = (T *)(xstep ? h->alpha_x : h->alpha_y);
    const int rk = reg_code(h, xstep);
    const T rw = (T)(xstep ? h->rx_w : h->ry_w);
    Scratch &s = h->s;
    cudaStream_t st = h->stream;
    const int k = h->k;
    const int pass_launches = o.nchunks ? 1 : 0;
    cudaError_t e;
    if constexpr (std::is_same<T, float>::value) {
        if (h->prec == GLRM_BF16) return bf16_half_step_entry(h, xstep);
    }
    tmark(h, xstep ? "pass_grad_x" : "pass_grad_y");
    const T *lsc = (const T *)h->lscale;
    e = xstep ? dispatch_pass<T, true, true>(o, F, W, k, loss_of<T>(h), (T *)s.part_grad, s.part_loss, st, nullptr, 0, lsc)
              : dispatch_pass<T, false, true>(o, F, W, k, loss_of<T>(h), (T *)s.part_grad, s.part_loss, st, nullptr, 0, lsc);
    if (e != cudaSuccess) return e;
    tmark(h, xstep ? "prox_x" : "prox_y");
    e = launch_prox<T>(o.nseg, o.segchunk, (const T *)s.part_grad, s.part_loss, F, alpha, k, rk, rw, (T *)s.cand,
                       s.f_old, s.r_old, s.r_new, st);
    if (e != cudaSuccess) return e;
    tmark(h, xstep ? "pass_loss_x" : "pass_loss_y");
    e = xstep ? dispatch_pass<T, true, false>(o, (const T *)s.cand, W, k, loss_of<T>(h), nullptr, s.part_loss2, st,
                                              nullptr, 0, lsc)
              : dispatch_pass<T, false, false>(o, (const T *)s.cand, W, k, loss_of<T>(h), nullptr, s.part_loss2, st,
                                               nullptr, 0, lsc);
    if (e != cudaSuccess) return e;
    tmark(h, xstep ? "decide_x" : "decide_y");
    e = launch_decide<T>(o.nseg, o.segchunk, s.part_loss2, s.f_old, s.r_old, s.r_new, (const T *)s.cand, F, alpha, k,
                         xstep ? s.kept_obj_x : s.kept_obj_y, xstep ? s.kept_reg_x : s.kept_reg_y,
                         xstep ? s.acc_x : s.acc_y, st);
    tmark(h, nullptr);
    h->launches += 2 + 2 * pass_launches;
    return e;
}

// Objective after a sweep: the Y-step's kept column objectives hold every
// loss term plus rt(y_j); add the X-step's kept r(x_i).
template <class T>
cudaError_t Engine<T>::reduce_sweep(glrm_s *h, double *hist_slot)
{
    Scratch &s = h->s;
    tmark(h, "reduce_stage1");
    reduce_stage1<T><<<kRedBlocks, 256, 0, h->stream>>>(
        s.kept_obj_y, h->n, s.kept_reg_x, h->m, nullptr, 0, 0, T(0), nullptr, 0, 0, T(0), h->k,
        s.acc_x, h->m, s.acc_y, h->n, s.red_part, s.red_cnt);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    tmark(h, "reduce_stage2");
    reduce_stage2<<<1, 256, 0, h->stream>>>(s.red_part, s.red_cnt, kRedBlocks, hist_slot, s.accepts);
    tmark(h, nullptr);
    h->launches += 2;
    return cudaGetLastError();
}

template <class T>
cudaError_t Engine<T>::objective_at(glrm_s *h, const T *X, const T *Yt, double *out)
{
    Scratch &s = h->s;
    tmark(h, "objective_pass");
    cudaError_t e = dispatch_pass<T, true, false>(h->csr, X, Yt, h->k, loss_of<T>(h), nullptr,
                                                  s.part_loss, h->stream, nullptr, 0, (const T *)h->lscale);
    if (e != cudaSuccess) return e;
    tmark(h, "reduce_stage1");
    reduce_stage1<T><<<kRedBlocks, 256, 0, h->stream>>>(
        s.part_loss, h->csr.nchunks, nullptr, 0, X, h->m, reg_code(h, true), (T)h->rx_w, Yt, h->n,
        reg_code(h, false), (T)h->ry_w, h->k, nullptr, 0, nullptr, 0, s.red_part, s.red_cnt);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    tmark(h, "reduce_stage2");
    reduce_stage2<<<1, 256, 0, h->stream>>>(s.red_part, s.red_cnt, kRedBlocks, out, nullptr);
    tmark(h, nullptr);
    h->launches += 2 + (h->csr.nchunks ? 1 : 0);
    return cudaGetLastError();
}

template <class T>
cudaError_t Engine<T>::grad_at(glrm_s *h, const T *X, const T *Yt, T *GX, T *GYt, bool reg,
                               const double *scale)
{
    Scratch &s = h->s;
    cudaError_t e;
    bool bf16 = false;
    if constexpr (std::is_same<T, float>::value) bf16 = h->prec == GLRM_BF16;
    if (bf16) {
        // BF16 form: both gradient passes read BF16 copies of the factors
        to_bf16_kernel<<<blocks_for(h->n * h->k, 256), 256, 0, h->stream>>>((const float *)Yt, h->n * h->k,
                                                                           s.yt_bf16);
        to_bf16_kernel<<<blocks_for(h->m * h->k, 256), 256, 0, h->stream>>>((const float *)X, h->m * h->k,
                                                                           s.x_bf16);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        h->launches += 2;
    }
    tmark(h, "grad_pass_x");
    if constexpr (std::is_same<T, float>::value) {
        if (bf16)
            e = dispatch_pass<T, true, true, __nv_bfloat16>(h->csr, X, s.yt_bf16, h->k, loss_of<T>(h),
                                                            (T *)s.part_grad, s.part_loss, h->stream);
        else
            e = dispatch_pass<T, true, true>(h->csr, X, Yt, h->k, loss_of<T>(h), (T *)s.part_grad,
                                             s.part_loss, h->stream, nullptr, 0, (const T *)h->lscale);
    } else {
        e = dispatch_pass<T, true, true>(h->csr, X, Yt, h->k, loss_of<T>(h), (T *)s.part_grad, s.part_loss,
                                         h->stream, nullptr, 0, (const T *)h->lscale);
    }
    if (e != cudaSuccess) return e;
    tmark(h, "grad_seg_x");
    seg_grad_kernel<T><<<blocks_for(h->m, kWarpsPerBlock), kWarpsPerBlock * 32, 0, h->stream>>>(
        h->m, h->csr.segchunk, (const T *)s.part_grad, X, h->k, reg_code(h, true), (T)h->rx_w, reg, scale, GX);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    tmark(h, "grad_pass_y");
    if constexpr (std::is_same<T, float>::value) {
        if (bf16)
            e = dispatch_pass<T, false, true, __nv_bfloat16>(h->csc, Yt, s.x_bf16, h->k, loss_of<T>(h),
                                                             (T *)s.part_grad, s.part_loss, h->stream);
        else
            e = dispatch_pass<T, false, true>(h->csc, Yt, X, h->k, loss_of<T>(h), (T *)s.part_grad,
                                              s.part_loss, h->stream, nullptr, 0, (const T *)h->lscale);
    } else {
        e = dispatch_pass<T, false, true>(h->csc, Yt, X, h->k, loss_of<T>(h), (T *)s.part_grad,
                                          s.part_loss, h->stream, nullptr, 0, (const T *)h->lscale);
    }
    if (e != cudaSuccess) return e;
    tmark(h, "grad_seg_y");
    seg_grad_kernel<T><<<blocks_for(h->n, kWarpsPerBlock), kWarpsPerBlock * 32, 0, h->stream>>>(
        h->n, h->csc.segchunk, (const T *)s.part_grad, Yt, h->k, reg_code(h, false), (T)h->ry_w, reg, scale, GYt);
    tmark(h, nullptr);
    h->launches += 2 + (h->csr.nchunks ? 1 : 0) + (h->csc.nchunks ? 1 : 0);
    return cudaGetLastError();
}

template <class T>
cudaError_t Engine<T>::predict(glrm_s *h, int64_t cnt, const int32_t *rows, const int32_t *cols,
                               T *out, bool decode)
{
    if (cnt == 0) return cudaSuccess;
    h->launches += 1;
    predict_kernel<T><<<blocks_for(cnt, 256), 256, 0, h->stream>>>(
        cnt, rows, cols, (const T *)h->X, (const T *)h->Yt, h->m, h->n, h->k, h->loss_dev, decode,
        out);
    return cudaGetLastError();
}

template <class T>
cudaError_t Engine<T>::reset_steps(glrm_s *h)
{
    h->launches += 2;
    reset_alpha_kernel<T><<<blocks_for(h->m, 256), 256, 0, h->stream>>>(h->csr.ptr, h->m,
                                                                       (T *)h->alpha_x);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    reset_alpha_kernel<T><<<blocks_for(h->n, 256), 256, 0, h->stream>>>(h->csc.ptr, h->n,
                                                                       (T *)h->alpha_y);
    return cudaGetLastError();
}

}  // namespace glrm
