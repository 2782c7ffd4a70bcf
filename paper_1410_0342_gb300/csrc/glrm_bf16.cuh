// BF16 form of the proximal-gradient half-step (Section 7.2 of Udell et al.,
// "Generalized Low Rank Models").  The rows of the other factor are gathered
// from a BF16 copy; accuracy is kept by an exact FP32 product carried for
// every observed entry:
//
//   u_e = x_i . y_j  (FP32), stored in CSR order and in CSC order, refreshed
//                    exactly (FP32 gathers) every kBf16Refresh sweeps.
//   gradient pass:   r_e = L'(u_e, a_e) from the stored exact u (FP32 residual),
//                    g = sum r_e w^_j with w^ the BF16 row (FP32 accumulation),
//                    f_old from L(u_e).
//   prox:            f+ = prox(f - alpha g) in FP32.
//   re-evaluation:   u+_e = u_e + (f+ - f) . w^_j: the BF16 rounding only touches
//                    the step's contribution, which is small near convergence,
//                    so the accept / reject test sees nearly FP32-exact losses.
//   update:          for accepted segments u_e <- u+_e in both orders (the
//                    other order through a precomputed entry permutation).
//
// The gathered bytes per entry are those of BF16 rows (2k) in both passes
// instead of FP32 rows (4k), plus 12 bytes of u traffic.
#pragma once

#include "glrm_engine.cuh"

namespace glrm {

constexpr int kBf16Refresh = 8;

constexpr int kBfGrad = 0, kBfLoss = 1, kBfExact = 2, kBfUpdate = 3;

// CSR position -> CSC position (or back): entry (i, j) of segment i in the
// source order is found in segment j of the other order by binary search.
static __global__ void perm_kernel(int64_t nseg, const int32_t *__restrict__ ptr,
                                   const int32_t *__restrict__ idx, const int32_t *__restrict__ optr,
                                   const int32_t *__restrict__ oidx, int32_t *__restrict__ perm)
{
    const int lane = threadIdx.x & 31;
    const int64_t s = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (s >= nseg) return;
    for (int q = ptr[s] + lane; q < ptr[s + 1]; q += 32) {
        const int j = idx[q];
        int lo = optr[j], hi = optr[j + 1];
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (oidx[mid] < s) lo = mid + 1;
            else hi = mid;
        }
        perm[q] = lo;
    }
}

// One warp per chunk (lane groups as in the FP32 passes).  MODE:
//   kBfGrad:   partial gradient sum L'(u) w^ and loss sum L(u), u from useg
//   kBfLoss:   u+ = useg + (cand - F) . w^ -> unew, partial loss sum L(u+)
//   kBfExact:  u = F . W exactly (FP32 rows) -> useg and uoth[perm]
//   kBfUpdate: accepted segments copy unew -> useg and uoth[perm]
template <int K, bool XSTEP, bool VEC, int MODE>
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
bf16_pass_kernel(int64_t nchunks, const int4 *__restrict__ chunks, const int32_t *__restrict__ idx,
                 const float *__restrict__ val, const float *__restrict__ F,
                 const float *__restrict__ cand, const __nv_bfloat16 *__restrict__ Wb,
                 const float *__restrict__ W, int k, const LossSpec *__restrict__ loss,
                 float *__restrict__ useg, float *__restrict__ uoth, float *__restrict__ unew,
                 const int32_t *__restrict__ perm, const int32_t *__restrict__ accepted,
                 float *__restrict__ part_grad, double *__restrict__ part_loss)
{
    using LN = Lanes<K>;
    constexpr int G = LN::G, S = LN::S, PER = LN::PER;
    const int lane = threadIdx.x & 31;
    const int64_t c = (int64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
    if (c >= nchunks) return;
    // f and the gathered rows share one lane layout: FP32 units (4 values)
    // for the exact refresh, BF16 units (8 values) otherwise
    constexpr int VW = MODE == kBfExact ? 4 : 8;
    const int gl = lane % G, grp = lane / G;
    const int4 ch = chunks[c];
    if constexpr (MODE == kBfUpdate) {
        if (!accepted[ch.x]) return;
        for (int e = ch.y + lane; e < ch.z; e += 32) {
            const float v = unew[e];
            useg[e] = v;
            uoth[perm[e]] = v;
        }
        return;
    }
    float f[S], g[S];
    if constexpr (MODE == kBfLoss) {
        float fp[S];
        load_lane<float, S, G, VW, VEC>(f, F + (int64_t)ch.x * k, gl, k);
        load_lane<float, S, G, VW, VEC>(fp, cand + (int64_t)ch.x * k, gl, k);
#pragma unroll
        for (int s = 0; s < S; ++s) f[s] = fp[s] - f[s];  // the step
    } else {
        load_lane<float, S, G, VW, VEC>(f, F + (int64_t)ch.x * k, gl, k);
    }
#pragma unroll
    for (int s = 0; s < S; ++s) g[s] = 0.f;
    float lsum = 0.f;
    LossSpec sp;
    if constexpr (!XSTEP) sp = loss[ch.x];
    for (int base = ch.y; base < ch.z; base += PER) {
        const int e = base + grp;
        const bool ok = e < ch.z;
        int j = 0;
        float a = 0.f;
        float w[S];
        if (ok) {
            j = __ldg(idx + e);
            a = __ldg(val + e);
            if constexpr (MODE == kBfExact) load_lane<float, S, G, VW, VEC>(w, W + (int64_t)j * k, gl, k);
            else load_lane_bf16<S, G, VEC>(w, Wb + (int64_t)j * k, gl, k);
        } else {
#pragma unroll
            for (int s = 0; s < S; ++s) w[s] = 0.f;
        }
        float u = 0.f;
        if constexpr (MODE != kBfGrad) {
#pragma unroll
            for (int s = 0; s < S; ++s) u = fmaf(f[s], w[s], u);
#pragma unroll
            for (int o = 1; o < G; o <<= 1) u += shfl_xor(u, o);
        }
        if (ok) {
            if constexpr (MODE == kBfExact) {
                if (gl == 0) {
                    useg[e] = u;
                    uoth[perm[e]] = u;
                }
                continue;
            }
            if constexpr (MODE == kBfGrad) u = useg[e];
            else u += useg[e];
            if constexpr (XSTEP) sp = loss[j];
            float L;
            const float d = loss_deriv<float>(sp, u, a, L);
            if constexpr (MODE == kBfGrad) {
#pragma unroll
                for (int s = 0; s < S; ++s) g[s] = fmaf(d, w[s], g[s]);
            } else {
                if (gl == 0) unew[e] = u;
            }
            if (gl == 0) lsum += L;
        }
    }
    if constexpr (MODE == kBfExact) return;
    if constexpr (MODE == kBfGrad) {
#pragma unroll
        for (int s = 0; s < S; ++s) {
#pragma unroll
            for (int o = G; o < 32; o <<= 1) g[s] += shfl_xor(g[s], o);
        }
        if (grp == 0) {
#pragma unroll
            for (int s = 0; s < S; ++s)
                if (slot_coord<S, G, VW, VEC>(s, gl) < k) part_grad[c * k + slot_coord<S, G, VW, VEC>(s, gl)] = g[s];
        }
    }
    const double ls = warp_sum((double)lsum);
    if (lane == 0) part_loss[c] = ls;
}

template <int K, bool XSTEP, int MODE>
cudaError_t launch_bf16(glrm_s *h, const Orient &o, const float *F, const float *cand,
                        const __nv_bfloat16 *Wb, const float *W, float *useg, float *uoth,
                        const int32_t *perm, const int32_t *accepted)
{
    if (o.nchunks == 0) return cudaSuccess;
    Scratch &s = h->s;
    const int k = h->k;
    const bool vec = (k == K) && (Lanes<K>::S % 8 == 0);
    const unsigned nb = blocks_for(o.nchunks, kWarpsPerBlock);
    auto go = [&](auto kern) {
        kern<<<nb, kWarpsPerBlock * 32, 0, h->stream>>>(o.nchunks, o.chunks, o.idx, (const float *)o.val, F,
                                                        cand, Wb, W, k, h->loss_dev, useg, uoth, s.u_new,
                                                        perm, accepted, (float *)s.part_grad,
                                                        MODE == kBfLoss ? s.part_loss2 : s.part_loss);
    };
    if constexpr (Lanes<K>::S % 8 == 0) {
        if (vec) go(bf16_pass_kernel<K, XSTEP, true, MODE>);
        else go(bf16_pass_kernel<K, XSTEP, false, MODE>);
    } else {
        go(bf16_pass_kernel<K, XSTEP, false, MODE>);
    }
    h->launches += 1;
    return cudaGetLastError();
}

template <int K, bool XSTEP, int MODE>
cudaError_t run_bf16_pass(glrm_s *h, const float *cand, const int32_t *accepted)
{
    const Orient &o = XSTEP ? h->csr : h->csc;
    Scratch &s = h->s;
    const float *F = (const float *)(XSTEP ? h->X : h->Yt);
    const float *W = (const float *)(XSTEP ? h->Yt : h->X);
    const __nv_bfloat16 *Wb = XSTEP ? s.yt_bf16 : s.x_bf16;
    float *useg = XSTEP ? s.u_csr : s.u_csc;
    float *uoth = XSTEP ? s.u_csc : s.u_csr;
    return launch_bf16<K, XSTEP, MODE>(h, o, F, cand, Wb, W, useg, uoth, o.perm, accepted);
}

template <bool XSTEP, int MODE>
cudaError_t bf16_pass(glrm_s *h, const float *cand = nullptr, const int32_t *accepted = nullptr)
{
    const int k = h->k;
#define GLRM_BF_CASE(KK) \
    if (k <= KK) return run_bf16_pass<KK, XSTEP, MODE>(h, cand, accepted);
    GLRM_BF_CASE(8)
    GLRM_BF_CASE(16)
    GLRM_BF_CASE(24)
    GLRM_BF_CASE(32)
    GLRM_BF_CASE(64)
#undef GLRM_BF_CASE
    return cudaErrorInvalidValue;
}

// Exact FP32 products u for every entry, in both orders.
inline cudaError_t bf16_refresh(glrm_s *h)
{
    tmark(h, "bf16_exact_u");
    cudaError_t e = bf16_pass<true, kBfExact>(h);
    tmark(h, nullptr);
    if (e == cudaSuccess) h->s.u_sweeps = 0;
    return e;
}

// One half-step of the BF16 form.
inline cudaError_t bf16_half_step(glrm_s *h, bool xstep)
{
    const Orient &o = xstep ? h->csr : h->csc;
    Scratch &s = h->s;
    cudaStream_t st = h->stream;
    const int k = h->k;
    float *F = (float *)(xstep ? h->X : h->Yt);
    const float *W = (const float *)(xstep ? h->Yt : h->X);
    float *alpha = (float *)(xstep ? h->alpha_x : h->alpha_y);
    const int rk = xstep ? h->rx_kind : h->ry_kind;
    const float rw = (float)(xstep ? h->rx_w : h->ry_w);
    const int64_t nother = xstep ? h->n : h->m;
    cudaError_t e;
    if (xstep && (s.u_sweeps < 0 || s.u_sweeps >= kBf16Refresh)) {
        if ((e = bf16_refresh(h)) != cudaSuccess) return e;
    }
    __nv_bfloat16 *Wb = xstep ? s.yt_bf16 : s.x_bf16;
    tmark(h, xstep ? "to_bf16_y" : "to_bf16_x");
    to_bf16_kernel<<<blocks_for(nother * k, 256), 256, 0, st>>>(W, nother * k, Wb);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    h->launches += 1;
    tmark(h, xstep ? "bf16_grad_x" : "bf16_grad_y");
    e = xstep ? bf16_pass<true, kBfGrad>(h) : bf16_pass<false, kBfGrad>(h);
    if (e != cudaSuccess) return e;
    const unsigned nbs = blocks_for(o.nseg, kWarpsPerBlock);
    tmark(h, xstep ? "prox_x" : "prox_y");
    prox_kernel<float><<<nbs, kWarpsPerBlock * 32, 0, st>>>(o.nseg, o.segchunk, (const float *)s.part_grad,
                                                            s.part_loss, F, alpha, k, rk, rw, (float *)s.cand,
                                                            s.f_old, s.r_old, s.r_new);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    tmark(h, xstep ? "bf16_loss_x" : "bf16_loss_y");
    e = xstep ? bf16_pass<true, kBfLoss>(h, (const float *)s.cand) : bf16_pass<false, kBfLoss>(h, (const float *)s.cand);
    if (e != cudaSuccess) return e;
    int32_t *acc = xstep ? s.acc_x : s.acc_y;
    tmark(h, xstep ? "decide_x" : "decide_y");
    decide_kernel<float><<<nbs, kWarpsPerBlock * 32, 0, st>>>(
        o.nseg, o.segchunk, s.part_loss2, s.f_old, s.r_old, s.r_new, (const float *)s.cand, F, alpha, k,
        xstep ? s.kept_obj_x : s.kept_obj_y, xstep ? s.kept_reg_x : s.kept_reg_y, acc);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    tmark(h, xstep ? "bf16_update_x" : "bf16_update_y");
    e = xstep ? bf16_pass<true, kBfUpdate>(h, nullptr, acc) : bf16_pass<false, kBfUpdate>(h, nullptr, acc);
    tmark(h, nullptr);
    h->launches += 2;
    if (!xstep) s.u_sweeps++;
    return e;
}

}  // namespace glrm
