// Alternating minimisation for quadratic loss with gamma ||.||^2 on both
// factors (Algorithm 1 of Udell et al., with the row and column problems of
// Section 2.4 solved exactly, the Gram matrices restricted to each row's or
// column's observed entries as in Section 2.5).  A half-step solves, for
// every segment s (row in the X-step, column in the Y-step),
//     (sum_{e in s} w_e w_e^T + gamma I) f_s = sum_{e in s} a_e w_e.
// Launch 1 (per chunk): partial Gram lower triangle and right-hand side in
// the element type.  Launch 2 (per segment, one warp): sum of the partials in
// a fixed order, then an FP64 Cholesky factorisation and two triangular
// solves in shared memory.
#pragma once

#include "glrm_engine.cuh"

namespace glrm {

constexpr int kAlsWarps = 4;

template <int K>
struct Tri {
    static constexpr int N = K * (K + 1) / 2;  // lower-triangle entries
    static constexpr int P = N + K;            // + right-hand side
    static constexpr int NP = (N + 31) / 32;   // per lane
};

// Row r and column c (c <= r) of lower-triangle entry p (row-major order).
__device__ __forceinline__ void tri_rc(int p, int &r, int &c)
{
    r = (int)((sqrtf(8.f * (float)p + 1.f) - 1.f) * 0.5f);
    while ((r + 1) * (r + 2) / 2 <= p) ++r;
    while (r * (r + 1) / 2 > p) --r;
    c = p - r * (r + 1) / 2;
}

template <class T, int K>
__global__ void __launch_bounds__(kAlsWarps * 32)
als_gram_kernel(int64_t nchunks, const int4 *__restrict__ chunks, const int32_t *__restrict__ idx,
                const T *__restrict__ val, const T *__restrict__ W, int k, T *__restrict__ part)
{
    using TR = Tri<K>;
    __shared__ T wsh[kAlsWarps][32][K + 1];
    __shared__ T ash[kAlsWarps][32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t c = (int64_t)blockIdx.x * kAlsWarps + wid;
    if (c >= nchunks) return;
    const int4 ch = chunks[c];
    int rq[TR::NP], cq[TR::NP];
    T acc[TR::NP];
#pragma unroll
    for (int q = 0; q < TR::NP; ++q) {
        const int p = lane + 32 * q;
        tri_rc(p < TR::N ? p : 0, rq[q], cq[q]);
        acc[q] = T(0);
    }
    T bacc = T(0);
    for (int base = ch.y; base < ch.z; base += 32) {
        const int e = base + lane;
        if (e < ch.z) {
            const int64_t j = __ldg(idx + e);
            ash[wid][lane] = __ldg(val + e);
#pragma unroll
            for (int q = 0; q < K; ++q) wsh[wid][lane][q] = q < k ? __ldg(W + j * k + q) : T(0);
        }
        __syncwarp();
        const int cnt = min(32, ch.z - base);
        for (int t = 0; t < cnt; ++t) {
#pragma unroll
            for (int q = 0; q < TR::NP; ++q)
                acc[q] = fma(wsh[wid][t][rq[q]], wsh[wid][t][cq[q]], acc[q]);
            if (lane < K) bacc = fma(ash[wid][t], wsh[wid][t][lane], bacc);
        }
        __syncwarp();
    }
    T *out = part + c * TR::P;
#pragma unroll
    for (int q = 0; q < TR::NP; ++q)
        if (lane + 32 * q < TR::N) out[lane + 32 * q] = acc[q];
    if (lane < K) out[TR::N + lane] = bacc;
}

template <class T, int K>
__global__ void __launch_bounds__(kAlsWarps * 32)
als_solve_kernel(int64_t nseg, const int32_t *__restrict__ segchunk, const T *__restrict__ part,
                 int k, double gamma, T *__restrict__ F, int *__restrict__ err)
{
    using TR = Tri<K>;
    __shared__ double G[kAlsWarps][K][K + 1];
    __shared__ double b[kAlsWarps][K];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t s = (int64_t)blockIdx.x * kAlsWarps + wid;
    if (s >= nseg) return;
    const int cb = segchunk[s], ce = segchunk[s + 1];
    for (int p = lane; p < TR::N; p += 32) {
        int r, c;
        tri_rc(p, r, c);
        double v = 0.0;
        for (int q = cb; q < ce; ++q) v += (double)part[(int64_t)q * TR::P + p];
        if (r == c) v += gamma;
        G[wid][r][c] = v;
    }
    if (lane < K) {
        double v = 0.0;
        for (int q = cb; q < ce; ++q) v += (double)part[(int64_t)q * TR::P + TR::N + lane];
        b[wid][lane] = v;
    }
    __syncwarp();
    // unused rows / columns beyond k become identity rows of a K x K system
    for (int c = k + lane; c < K; c += 32) {
        for (int q = 0; q < c; ++q) G[wid][c][q] = 0.0;
        G[wid][c][c] = 1.0;
        b[wid][c] = 0.0;
    }
    __syncwarp();
    // a failed factorisation keeps the segment's factor and raises the flag
    if (!warp_cholesky_solve<K, K + 1>(G[wid], b[wid])) {
        if (lane == 0) atomicOr(err, kErrPivot);
        return;
    }
    if (lane < k) F[s * k + lane] = (T)b[wid][lane];
}

// Prox-prox update for quadratic loss (Section 7.2, "Prox-prox method"; the
// cached factorisation of Section 7.3), one warp per segment: with the
// segment's Gram matrix G and right-hand side b (the ALS partials), factor
// M = 2 alpha G + I once in FP64, then `inner` times
//     f <- prox_{alpha r}(M^{-1} (2 alpha b + f)),
// prox_{alpha f}(f) = argmin alpha sum_e (f . w_e - a_e)^2 + ||f' - f||^2 / 2
// being M^{-1}(2 alpha b + f).  A failed factorisation keeps the factor and
// raises the status flag.
template <class T, int K>
__global__ void __launch_bounds__(kAlsWarps * 32)
proxprox_solve_kernel(int64_t nseg, const int32_t *__restrict__ segchunk, const T *__restrict__ part,
                      int k, double alpha, int inner, int rkind, double rw, T *__restrict__ F,
                      int *__restrict__ err)
{
    using TR = Tri<K>;
    __shared__ double G[kAlsWarps][K][K + 1];
    __shared__ double b[kAlsWarps][K];
    __shared__ double x[kAlsWarps][K];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t s = (int64_t)blockIdx.x * kAlsWarps + wid;
    if (s >= nseg) return;
    const int cb = segchunk[s], ce = segchunk[s + 1];
    for (int p = lane; p < TR::N; p += 32) {
        int r, c;
        tri_rc(p, r, c);
        double v = 0.0;
        for (int q = cb; q < ce; ++q) v += (double)part[(int64_t)q * TR::P + p];
        G[wid][r][c] = 2.0 * alpha * v + (r == c ? 1.0 : 0.0);
    }
    if (lane < K) {
        double v = 0.0;
        for (int q = cb; q < ce; ++q) v += (double)part[(int64_t)q * TR::P + TR::N + lane];
        b[wid][lane] = 2.0 * alpha * v;
    }
    __syncwarp();
    // unused rows / columns beyond k become identity rows of a K x K system
    for (int c = k + lane; c < K; c += 32) {
        for (int q = 0; q < c; ++q) G[wid][c][q] = 0.0;
        G[wid][c][c] = 1.0;
        b[wid][c] = 0.0;
    }
    __syncwarp();
    if (!warp_cholesky_factor<K, K + 1>(G[wid])) {
        if (lane == 0) atomicOr(err, kErrPivot);
        return;
    }
    double f = lane < k ? (double)F[s * k + lane] : 0.0;
    for (int it = 0; it < inner; ++it) {
        if (lane < K) x[wid][lane] = b[wid][lane] + f;
        __syncwarp();
        warp_cholesky_subst<K, K + 1>(G[wid], x[wid]);
        if (lane < K) f = lane < k ? prox1<double>(reg_kind_at(rkind, lane, k), rw, alpha, x[wid][lane]) : 0.0;
        __syncwarp();
    }
    if (lane < k) F[s * k + lane] = (T)f;
}

template <class T, int K>
cudaError_t launch_als_half(glrm_s *h, bool xstep, double gamma)
{
    const Orient &o = xstep ? h->csr : h->csc;
    T *F = (T *)(xstep ? h->X : h->Yt);
    const T *W = (const T *)(xstep ? h->Yt : h->X);
    const size_t need = (size_t)std::max<int64_t>(1, std::max(h->csr.nchunks, h->csc.nchunks)) *
                        Tri<K>::P * sizeof(T);
    if (h->s.als_bytes < need) {
        dfree(h->s.als_part, h->stream);
        h->s.als_part = nullptr;
        h->s.als_bytes = 0;
        cudaError_t e = dalloc(h, &h->s.als_part, need);
        if (e != cudaSuccess) return e;
        h->s.als_bytes = need;
    }
    T *part = (T *)h->s.als_part;
    h->launches += 1 + (o.nchunks ? 1 : 0);
    tmark(h, xstep ? "als_gram_x" : "als_gram_y");
    if (o.nchunks)
        als_gram_kernel<T, K><<<blocks_for(o.nchunks, kAlsWarps), kAlsWarps * 32, 0, h->stream>>>(
            o.nchunks, o.chunks, o.idx, (const T *)o.val, W, h->k, part);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    tmark(h, xstep ? "als_solve_x" : "als_solve_y");
    als_solve_kernel<T, K><<<blocks_for(o.nseg, kAlsWarps), kAlsWarps * 32, 0, h->stream>>>(
        o.nseg, o.segchunk, part, h->k, gamma, F, h->s.err);
    tmark(h, nullptr);
    return cudaGetLastError();
}

template <class T, int K>
cudaError_t launch_proxprox_half(glrm_s *h, bool xstep, double alpha, int inner)
{
    // the Gram partials of the ALS half-step (no solve), then the prox-prox solves
    const Orient &o = xstep ? h->csr : h->csc;
    T *F = (T *)(xstep ? h->X : h->Yt);
    const T *W = (const T *)(xstep ? h->Yt : h->X);
    const size_t need = (size_t)std::max<int64_t>(1, std::max(h->csr.nchunks, h->csc.nchunks)) *
                        Tri<K>::P * sizeof(T);
    if (h->s.als_bytes < need) {
        dfree(h->s.als_part, h->stream);
        h->s.als_part = nullptr;
        h->s.als_bytes = 0;
        cudaError_t e = dalloc(h, &h->s.als_part, need);
        if (e != cudaSuccess) return e;
        h->s.als_bytes = need;
    }
    T *part = (T *)h->s.als_part;
    h->launches += 1 + (o.nchunks ? 1 : 0);
    tmark(h, xstep ? "als_gram_x" : "als_gram_y");
    if (o.nchunks)
        als_gram_kernel<T, K><<<blocks_for(o.nchunks, kAlsWarps), kAlsWarps * 32, 0, h->stream>>>(
            o.nchunks, o.chunks, o.idx, (const T *)o.val, W, h->k, part);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    tmark(h, xstep ? "proxprox_x" : "proxprox_y");
    proxprox_solve_kernel<T, K><<<blocks_for(o.nseg, kAlsWarps), kAlsWarps * 32, 0, h->stream>>>(
        o.nseg, o.segchunk, part, h->k, alpha, inner, reg_code(h, xstep),
        xstep ? h->rx_w : h->ry_w, F, h->s.err);
    tmark(h, nullptr);
    return cudaGetLastError();
}

template <class T>
cudaError_t Engine<T>::proxprox_half(glrm_s *h, bool xstep, double alpha, int inner)
{
    const int k = h->k;
    if (k <= 4) return launch_proxprox_half<T, 4>(h, xstep, alpha, inner);
    if (k <= 8) return launch_proxprox_half<T, 8>(h, xstep, alpha, inner);
    if (k <= 16) return launch_proxprox_half<T, 16>(h, xstep, alpha, inner);
    if (k <= 32) return launch_proxprox_half<T, 32>(h, xstep, alpha, inner);
    return cudaErrorInvalidValue;
}

template <class T>
cudaError_t Engine<T>::als_half(glrm_s *h, bool xstep, double gamma)
{
    const int k = h->k;
    if (k <= 4) return launch_als_half<T, 4>(h, xstep, gamma);
    if (k <= 8) return launch_als_half<T, 8>(h, xstep, gamma);
    if (k <= 16) return launch_als_half<T, 16>(h, xstep, gamma);
    if (k <= 32) return launch_als_half<T, 32>(h, xstep, gamma);
    return cudaErrorInvalidValue;
}

}  // namespace glrm
