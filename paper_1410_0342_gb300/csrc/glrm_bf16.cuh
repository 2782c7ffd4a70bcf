// BF16 form of the proximal-gradient half-step (Section 7.2 of Udell et al.,
// "Generalized Low Rank Models"): factor products in BF16 where they only
// steer the step, FP32 where they decide it.
//
//   gradient pass:  a segment whose previous step was accepted gathers the
//                   rows of the other factor from its BF16 copy: u = f . w^
//                   (BF16 rows, FP32 accumulation), r = L'(u) in FP32,
//                   g = sum r w^ in FP32.  A segment whose previous step was
//                   rejected takes its retry's gradient from the FP32 rows, so
//                   near convergence, where the BF16 rounding of g would stall
//                   the fit, the step-size rule itself switches segments to
//                   FP32 gradients.
//   prox:           f+ = prox(f - alpha g) in FP32.
//   candidate pass: the FP32 rows, gathered once per entry: u_old = f . w and
//                   u_new = f+ . w, the losses at both; the accept / reject
//                   test and the reported objective are exactly those of the
//                   FP32 form.
//   decide:         as in the FP32 form, with f_old from the candidate pass.
//
// Gathered bytes per entry and half-step: 2k (BF16 rows) + 4k (FP32 rows)
// for a segment on BF16 gradients, against 4k + 4k in the FP32 form.
#pragma once

#include "glrm_engine.cuh"

namespace glrm {

// The candidate pass: per chunk, the losses at the segment's current factor
// f and at its candidate f+ from one gather of each other-factor row (FP32).
template <int K, bool XSTEP, bool VEC>
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
cand_pass_kernel(int64_t nchunks, const int4 *__restrict__ chunks, const int32_t *__restrict__ order,
                 const int32_t *__restrict__ idx, const float *__restrict__ val, const float *__restrict__ F,
                 const float *__restrict__ C, const float *__restrict__ W, int k,
                 const LossSpecF *__restrict__ loss, double *__restrict__ part_old, double *__restrict__ part_new)
{
    using LN = Lanes<K>;
    constexpr int G = LN::G, S = LN::S, PER = LN::PER, VW = 4;
    const int lane = threadIdx.x & 31;
    const int64_t lin = (int64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
    if (lin >= nchunks) return;
    const int64_t c = order ? (int64_t)__ldg(order + lin) : lin;
    const int gl = lane % G, grp = lane / G;
    const int4 ch = chunks[c];
    float f[S], fp[S];
    load_lane<float, S, G, VW, VEC>(f, F + (int64_t)ch.x * k, gl, k);
    load_lane<float, S, G, VW, VEC>(fp, C + (int64_t)ch.x * k, gl, k);
    float lo = 0.f, ln = 0.f;
    LossSpecF sp;
    if constexpr (!XSTEP) sp = loss[ch.x];
    // software pipeline as in the loss passes: the next group's index,
    // value, loss and row are loaded before the current group is evaluated
    float an = 0.f, wn[S];
    LossSpecF spn = sp;
    auto fetch = [&](int e) {
        if (e < ch.z) {
            const int jn = __ldg(idx + e);
            an = __ldg(val + e);
            load_lane<float, S, G, VW, VEC>(wn, W + (int64_t)jn * k, gl, k);
            if constexpr (XSTEP) spn = loss[jn];
        } else {
#pragma unroll
            for (int s = 0; s < S; ++s) wn[s] = 0.f;
        }
    };
    fetch(ch.y + grp);
    for (int base = ch.y; base < ch.z; base += PER) {
        const bool ok = base + grp < ch.z;
        const float a = an;
        float w[S];
#pragma unroll
        for (int s = 0; s < S; ++s) w[s] = wn[s];
        if constexpr (XSTEP) sp = spn;
        fetch(base + PER + grp);
        float u0 = 0.f, u1 = 0.f;
#pragma unroll
        for (int s = 0; s < S; ++s) {
            u0 = fmaf(f[s], w[s], u0);
            u1 = fmaf(fp[s], w[s], u1);
        }
#pragma unroll
        for (int o = 1; o < G; o <<= 1) {
            u0 += shfl_xor(u0, o);
            u1 += shfl_xor(u1, o);
        }
        if (ok && gl == 0) {
            float L0, L1;
            loss_deriv<float>(sp, u0, a, L0);
            loss_deriv<float>(sp, u1, a, L1);
            lo += L0;
            ln += L1;
        }
    }
    const double so = warp_sum((double)lo), sn = warp_sum((double)ln);
    if (lane == 0) {
        part_old[c] = so;
        part_new[c] = sn;
    }
}

template <int K, bool XSTEP>
cudaError_t launch_cand(glrm_s *h, const Orient &o, const float *F, const float *C, const float *W)
{
    if (o.nchunks == 0) return cudaSuccess;
    const int k = h->k;
    const bool vec = (k == K) && ((reinterpret_cast<uintptr_t>(F) | reinterpret_cast<uintptr_t>(C) |
                                   reinterpret_cast<uintptr_t>(W)) % 16 == 0);
    const unsigned nb = blocks_for(o.nchunks, kWarpsPerBlock);
    auto go = [&](auto kern) {
        kern<<<nb, kWarpsPerBlock * 32, 0, h->stream>>>(o.nchunks, o.chunks, o.order, o.idx, (const float *)o.val, F, C,
                                                        W, k, h->loss_f, h->s.part_loss, h->s.part_loss2);
    };
    if (vec) go(cand_pass_kernel<K, XSTEP, true>);
    else go(cand_pass_kernel<K, XSTEP, false>);
    h->launches += 1;
    return cudaGetLastError();
}

template <bool XSTEP>
cudaError_t cand_pass(glrm_s *h, const Orient &o, const float *F, const float *C, const float *W)
{
    const int k = h->k;
#define GLRM_CAND_CASE(KK) \
    if (k <= KK) return launch_cand<KK, XSTEP>(h, o, F, C, W);
    GLRM_CAND_CASE(4)
    GLRM_CAND_CASE(8)
    GLRM_CAND_CASE(12)
    GLRM_CAND_CASE(16)
    GLRM_CAND_CASE(20)
    GLRM_CAND_CASE(24)
    GLRM_CAND_CASE(32)
    GLRM_CAND_CASE(48)
    GLRM_CAND_CASE(64)
#undef GLRM_CAND_CASE
    return cudaErrorInvalidValue;
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
    const int rk = reg_code(h, xstep);
    const float rw = (float)(xstep ? h->rx_w : h->ry_w);
    const int64_t nother = xstep ? h->n : h->m;
    int32_t *acc = xstep ? s.acc_x : s.acc_y;  // previous decision per segment (1: accepted)
    cudaError_t e;
    __nv_bfloat16 *Wb = xstep ? s.yt_bf16 : s.x_bf16;
    tmark(h, xstep ? "to_bf16_y" : "to_bf16_x");
    to_bf16_kernel<<<blocks_for(nother * k, 256), 256, 0, st>>>(W, nother * k, Wb);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    h->launches += 1;
    // gradient: BF16 rows for segments whose last step was accepted, FP32 rows for the others
    tmark(h, xstep ? "bf16_grad_x" : "bf16_grad_y");
    e = xstep ? dispatch_pass<float, true, true, __nv_bfloat16>(o, F, Wb, k, h->loss_f, (float *)s.part_grad,
                                                                  s.part_loss, st, acc, 1)
              : dispatch_pass<float, false, true, __nv_bfloat16>(o, F, Wb, k, h->loss_f, (float *)s.part_grad,
                                                                   s.part_loss, st, acc, 1);
    if (e != cudaSuccess) return e;
    tmark(h, xstep ? "fp32_grad_x" : "fp32_grad_y");
    e = xstep ? dispatch_pass<float, true, true>(o, F, W, k, h->loss_f, (float *)s.part_grad, s.part_loss, st, acc, 0)
              : dispatch_pass<float, false, true>(o, F, W, k, h->loss_f, (float *)s.part_grad, s.part_loss, st, acc, 0);
    if (e != cudaSuccess) return e;
    h->launches += 2 * (o.nchunks ? 1 : 0);
    tmark(h, xstep ? "prox_x" : "prox_y");
    e = launch_prox<float>(o.nseg, o.segchunk, (const float *)s.part_grad, s.part_loss, F, alpha, k, rk, rw,
                           (float *)s.cand, s.f_old, s.r_old, s.r_new, st);
    if (e != cudaSuccess) return e;
    tmark(h, xstep ? "cand_x" : "cand_y");
    e = xstep ? cand_pass<true>(h, o, F, (const float *)s.cand, W) : cand_pass<false>(h, o, F, (const float *)s.cand, W);
    if (e != cudaSuccess) return e;
    tmark(h, xstep ? "decide_x" : "decide_y");
    e = launch_decide<float>(o.nseg, o.segchunk, s.part_loss2, s.f_old, s.r_old, s.r_new, (const float *)s.cand, F,
                             alpha, k, xstep ? s.kept_obj_x : s.kept_obj_y, xstep ? s.kept_reg_x : s.kept_reg_y, acc,
                             st, s.part_loss);
    tmark(h, nullptr);
    h->launches += 2;
    return e;
}

}  // namespace glrm
