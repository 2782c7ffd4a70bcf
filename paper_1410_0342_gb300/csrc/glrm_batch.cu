// Batched form: many independent GLRMs of uneven size fitted together.
//
// Every instance is a GLRM of its own (eq. gpca) with one loss for all its
// columns and quadratic / l1 / nonnegativity / zero regularisers, fitted
// either by the alternating proximal-gradient sweep with the step-size rule
// (Algorithm 2, Section 7.2 of Udell et al., "Generalized Low Rank Models") or,
// for quadratic loss with gamma ||.||^2 on both factors, by alternating
// minimisation (Algorithm 1, rows and columns solved exactly as in Section 2.4
// with the Gram matrix of each row's / column's observed entries, Section 2.5).
//
// All the sweeps of a call run in ONE persistent launch.  Its warps take work
// items from a device queue (an atomic counter): for every sweep t, the
// X-step items (instance, range of rows), then the Y-step items (instance,
// range of columns), then one objective item per instance.  A warp runs each
// row (column) of its item to completion (gradient, prox, re-evaluation,
// decision; or Gram, FP64 Cholesky, solve).  Per-instance completion counters
// order the work: a Y-step item waits until every X-step item of its
// instance in that sweep is done, an objective item until every Y-step item
// is, and the next sweep's X-step items until the objective is.  An item is
// only ever waiting for items handed out before it, which are held by warps
// that are already running and never wait for a later item, so every wait
// ends; each wait is bounded all the same (a host-set number of polls), and
// on expiry the warp raises the error flag and carries on without the work.
// Items are as many rows / columns as the autotuned table says for the
// instance's (k, method, segment-length) bucket, ordered by decreasing work
// or grouped by instance.  The launch is captured once into a CUDA graph.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "glrm.h"
#include "glrm_device.cuh"

namespace {

using namespace glrm;

struct __align__(16) BInst {
    int64_t m, n;
    int64_t rp_off, cp_off;      // offsets of the instance's rowptr / colptr
    int64_t e_off;               // first entry (CSR and CSC)
    int64_t x_off, y_off;        // first element of X (m x k) and Yt (n x k)
    int64_t row_base, col_base;  // global ids of row 0 and column 0
    int32_t k, method, kind, levels;
    double param;
    int32_t rxk, ryk;
    double rxw, ryw;
};

constexpr int kBWarps = 8;
constexpr int kBK = 16;  // largest rank of a batched instance
constexpr long kBucketCount = 32;

}  // namespace

struct glrm_batch_s {
    int count = 0;
    int device = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t capture = nullptr;
    std::vector<BInst> inst_host;
    BInst *inst = nullptr;
    int64_t nnz = 0, rows = 0, cols = 0, xlen = 0, ylen = 0;
    int32_t *rowptr = nullptr, *colidx = nullptr, *colptr = nullptr, *rowidx = nullptr;
    float *val = nullptr, *cval = nullptr;
    float *X = nullptr, *Yt = nullptr, *ax = nullptr, *ay = nullptr;
    double *kept_obj_y = nullptr, *kept_reg_x = nullptr, *kept_obj_x = nullptr, *kept_reg_y = nullptr;
    int32_t *acc_x = nullptr, *acc_y = nullptr;
    double *hist = nullptr;
    int hist_cap = 0;
    int4 *items_x = nullptr, *items_y = nullptr;
    int64_t nitems_x = 0, nitems_y = 0;
    int32_t *need_x = nullptr, *need_y = nullptr;  // per instance: its items in items_x / items_y
    int32_t *obj_inst = nullptr;                   // 0 .. count - 1
    unsigned long long *qhead = nullptr;           // the queue's next item
    int32_t *done = nullptr;                       // 3 x count completion counters (X, Y, objective)
    int *status = nullptr;                         // device status word (kErrWait, kErrPivot bits)
    long long wait_limit = 1LL << 24;              // polls a dependency wait may take
    int qgrid = 0;                                 // CTAs of a full queue launch (all resident)
    std::vector<int64_t> inst_items_x, inst_items_y;  // first item of each instance (unbatched mode)
    int32_t tile_x[kBucketCount], tile_y[kBucketCount];
    int order_x = 0, order_y = 0;  // 0: items by decreasing work; 1: grouped by instance
    int grid = 0;
    cudaGraphExec_t graph = nullptr;
    int graph_sweeps = 0;
    std::string err;
};

namespace {

thread_local std::string g_berr;

int bfail(glrm_batch_s *b, int code, const std::string &msg)
{
    if (b) b->err = msg;
    else g_berr = msg;
    return code;
}

#define BCK(call)                                                                        \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess) return bfail(b, GLRM_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

template <class P>
void bfree(P *&p)
{
    if (p) cudaFree((void *)p);
    p = nullptr;
}

// ----------------------------------------------------------------- kernels

template <int K>
struct BVec {
    float v[K];
};

template <int K>
__device__ __forceinline__ void bload(float (&v)[K], const float *__restrict__ row)
{
    const float4 *p = reinterpret_cast<const float4 *>(row);
#pragma unroll
    for (int q = 0; q < K / 4; ++q) {
        const float4 t = __ldg(p + q);
        v[4 * q] = t.x;
        v[4 * q + 1] = t.y;
        v[4 * q + 2] = t.z;
        v[4 * q + 3] = t.w;
    }
}

template <int K>
__device__ __forceinline__ float bdot(const float (&a)[K], const float (&b)[K])
{
    float s0 = 0.f, s1 = 0.f;
#pragma unroll
    for (int c = 0; c < K; c += 2) {
        s0 = fmaf(a[c], b[c], s0);
        s1 = fmaf(a[c + 1], b[c + 1], s1);
    }
    return s0 + s1;
}

struct Seg {
    const int32_t *ptr, *idx;
    const float *val;
    float *F;
    const float *W;
    float *alpha;
    double *kobj, *kreg;
    int32_t *acc;
    int rk;
    float rw;
};

// One row (column) of a prox-grad instance, whole warp: gradient pass,
// prox, re-evaluation pass, accept / reject with the step-size rule.
template <int K>
__device__ void pg_segment(const Seg &g, const LossSpec &sp, int64_t s)
{
    const int lane = threadIdx.x & 31;
    const int b = g.ptr[s], e = g.ptr[s + 1];
    float f[K], gr[K];
    bload<K>(f, g.F + s * K);
#pragma unroll
    for (int c = 0; c < K; ++c) gr[c] = 0.f;
    float lsum = 0.f;
    for (int q = b + lane; q < e; q += 32) {
        float w[K];
        bload<K>(w, g.W + (int64_t)__ldg(g.idx + q) * K);
        float L;
        const float d = loss_deriv<float>(sp, bdot<K>(f, w), __ldg(g.val + q), L);
#pragma unroll
        for (int c = 0; c < K; ++c) gr[c] = fmaf(d, w[c], gr[c]);
        lsum += L;
    }
#pragma unroll
    for (int c = 0; c < K; ++c) gr[c] = warp_sum(gr[c]);
    const double lold = warp_sum((double)lsum);
    const float al = g.alpha[s];
    float fp[K];
    float rof = 0.f, rnf = 0.f;  // regulariser terms in FP32, combined with the losses in FP64
#pragma unroll
    for (int c = 0; c < K; ++c) {
        fp[c] = prox1<float>(g.rk, g.rw, al, f[c] - al * gr[c]);
        rof += reg1<float>(g.rk, g.rw, f[c]);
        rnf += reg1<float>(g.rk, g.rw, fp[c]);
    }
    const double rold = (double)rof, rnew = (double)rnf;
    float lsum2 = 0.f;
    for (int q = b + lane; q < e; q += 32) {
        float w[K];
        bload<K>(w, g.W + (int64_t)__ldg(g.idx + q) * K);
        float L;
        loss_deriv<float>(sp, bdot<K>(fp, w), __ldg(g.val + q), L);
        lsum2 += L;
    }
    const double fnew = warp_sum((double)lsum2) + rnew;
    const double fold = lold + rold;
    const bool acc = fnew <= fold;
    if (acc) {
#pragma unroll
        for (int c = 0; c < K; ++c)
            if (lane == (c & 31)) g.F[s * K + c] = fp[c];
    }
    if (lane == 0) {
        g.alpha[s] = al * (acc ? 1.05f : 0.7f);
        g.kobj[s] = acc ? fnew : fold;
        g.kreg[s] = acc ? rnew : rold;
        g.acc[s] = acc ? 1 : 0;
    }
}

struct AlsSmem {
    float w[32][kBK + 1];   // staged rows of the other factor, one per lane
    float a[32];            // their values
    double G[2 * kBK * (kBK + 1)];  // per lane group: its k x (k + 1) system (32 / k groups)
    double rhs[32];                 // per lane group: its k right-hand side values
};

// Sum over the K lanes of a lane group (K a power of two, groups aligned).
template <int K, class T>
__device__ __forceinline__ T group_sum(T v)
{
#pragma unroll
    for (int o = K / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// (C C^T) x = b for the k x k system of every lane group at once: G (row
// stride K + 1) and b in shared memory, lane lr of the group owns row lr.
// The same column-by-column scheme as warp_cholesky_solve (FP64 throughout,
// reciprocal square roots by rsqrt_fp64, the trailing update's pairs spread
// over the group's lanes), but each FP64 instruction serves 32 / K systems.
// Returns (to every lane of the group) false when a pivot was not positive,
// finite and normal.
template <int K>
__device__ bool group_cholesky_solve(double *G, double *b)
{
    constexpr int LD = K + 1;
    const int lane = threadIdx.x & 31, lr = lane % K;
    bool ok = true;
    for (int c = 0; c < K; ++c) {
        if (lr == 0) {
            double r;
            ok = rsqrt_fp64(G[c * LD + c], r) && ok;
            G[c * LD + c] = r;  // the pivot slot keeps 1/C[c][c] from here on
        }
        __syncwarp();
        const double r = G[c * LD + c];
        if (lr > c) G[lr * LD + c] *= r;
        __syncwarp();
        const int n = K - 1 - c;
        for (int p = lr; p < n * (n + 1) / 2; p += K) {
            int i = (int)((sqrtf(8.f * (float)p + 1.f) - 1.f) * 0.5f);
            while ((i + 1) * (i + 2) / 2 <= p) ++i;
            while (i * (i + 1) / 2 > p) --i;
            const int row = c + 1 + i, col = c + 1 + p - i * (i + 1) / 2;
            G[row * LD + col] -= G[row * LD + c] * G[col * LD + c];
        }
        __syncwarp();
    }
    for (int c = 0; c < K; ++c) {
        if (lr == 0) b[c] *= G[c * LD + c];
        __syncwarp();
        if (lr > c) b[lr] -= G[lr * LD + c] * b[c];
        __syncwarp();
    }
    for (int c = K - 1; c >= 0; --c) {
        if (lr == 0) b[c] *= G[c * LD + c];
        __syncwarp();
        if (lr < c) b[lr] -= G[c * LD + lr] * b[c];
        __syncwarp();
    }
    return __shfl_sync(0xffffffffu, ok ? 1 : 0, lane - lr) != 0;
}

// Up to 32 / K rows (columns) s_begin + grp of an ALS instance at once, one
// lane group of K lanes each: (sum_e w_e w_e^T + gamma I) f = sum_e a_e w_e,
// Gram in FP32 (lane lr accumulates entries lr, lr + K, ... of the lower
// triangle), factor and solves in FP64.  With `objective` the segment's loss
// sum at the solution is computed (Y-step: the column's share of the
// objective).  A system whose factorisation fails keeps its old factor and
// raises kErrPivot.
template <int K>
__device__ void als_group(const Seg &g, double gamma, int64_t s_begin, int64_t s_end, AlsSmem &sm,
                          bool objective, int *err)
{
    constexpr int N = K * (K + 1) / 2;
    constexpr int NQ = (N + K - 1) / K;
    constexpr int LD = K + 1;
    const int lane = threadIdx.x & 31, grp = lane / K, lr = lane % K;
    const int64_t s = s_begin + grp;
    const bool active = s < s_end;
    const int b = active ? g.ptr[s] : 0, e = active ? g.ptr[s + 1] : 0;
    const int len = e - b;
    int rq[NQ], cq[NQ];
    float acc[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        int p = lr + K * q;
        if (p >= N) p = 0;
        int r = 0;
        while ((r + 1) * (r + 2) / 2 <= p) ++r;
        rq[q] = r;
        cq[q] = p - r * (r + 1) / 2;
        acc[q] = 0.f;
    }
    float bacc = 0.f;
    int maxlen = len;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) maxlen = max(maxlen, __shfl_xor_sync(0xffffffffu, maxlen, o));
    for (int base = 0; base < maxlen; base += K) {
        if (base + lr < len) {
            const int q0 = b + base + lr;
            float w[K];
            bload<K>(w, g.W + (int64_t)__ldg(g.idx + q0) * K);
#pragma unroll
            for (int c = 0; c < K; ++c) sm.w[lane][c] = w[c];
            sm.a[lane] = __ldg(g.val + q0);
        }
        __syncwarp();
        const int cnt = min(K, len - base);
        for (int t = 0; t < cnt; ++t) {
            const float *wr = sm.w[grp * K + t];
#pragma unroll
            for (int q = 0; q < NQ; ++q) acc[q] = fmaf(wr[rq[q]], wr[cq[q]], acc[q]);
            bacc = fmaf(sm.a[grp * K + t], wr[lr], bacc);
        }
        __syncwarp();
    }
    double *G = sm.G + grp * K * LD;
    double *rhs = sm.rhs + grp * K;
#pragma unroll
    for (int q = 0; q < NQ; ++q)
        if (lr + K * q < N) G[rq[q] * LD + cq[q]] = (double)acc[q] + (rq[q] == cq[q] ? gamma : 0.0);
    rhs[lr] = (double)bacc;
    __syncwarp();
    const bool solved = group_cholesky_solve<K>(G, rhs);
    // lane lr holds coordinate lr of the solution (of the old factor when the
    // factorisation failed); the regulariser's terms once per coordinate
    const float fl = active ? (solved ? (float)rhs[lr] : g.F[s * K + lr]) : 0.f;
    const double reg = group_sum<K>(gamma * (double)fl * (double)fl);
    if (active && !solved && lr == 0) atomicOr(err, kErrPivot);
    float f[K];
#pragma unroll
    for (int c = 0; c < K; ++c) f[c] = __shfl_sync(0xffffffffu, fl, grp * K + c);
    if (active && solved) g.F[s * K + lr] = fl;
    double lsum = 0.0;
    if (objective) {
        float ls = 0.f;
        for (int q = b + lr; q < e; q += K) {
            float w[K];
            bload<K>(w, g.W + (int64_t)__ldg(g.idx + q) * K);
            const float r = bdot<K>(f, w) - __ldg(g.val + q);
            ls = fmaf(r, r, ls);
        }
        lsum = group_sum<K>((double)ls);
    }
    __syncwarp();
    if (active && lr == 0) {
        g.kobj[s] = lsum + reg;
        g.kreg[s] = reg;
        g.acc[s] = 1;
    }
}

// Everything one launch of the queue kernel needs.  The queue holds, for
// each sweep t = t0 .. t0 + sweeps - 1, nx X-step items, ny Y-step items and
// no objective items (instance numbers); item q of the launch is sweep
// t0 + q / (nx + ny + no), position q % (nx + ny + no).  With wait == 0 the
// dependency waits are skipped (a launch that times one phase on its own).
struct BQueue {
    const BInst *inst;
    const int4 *items_x, *items_y;
    const int32_t *obj_inst;
    int64_t nx, ny, no;
    const int32_t *need_x, *need_y;  // per instance: its X- / Y-step items in a full sweep
    int t0, sweeps, count, wait;
    unsigned long long *head;        // the queue's next item
    int32_t *done_x, *done_y, *done_o;  // per instance, counted over all sweeps of the call
    int *err;
    long long limit;                 // polls a wait may take
    double *hist;                    // objectives, sweep-major (sweep t at t * count)
    const int32_t *rowptr, *colidx, *colptr, *rowidx;
    const float *val, *cval;
    float *X, *Yt, *ax, *ay;
    double *kobj_x, *kreg_x, *kobj_y, *kreg_y;
    int32_t *acc_x, *acc_y;
};

__device__ __forceinline__ int load_acquire(const int32_t *p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Whole warp: wait until *ctr >= target (lane 0 polls, at most `limit`
// times, and gives up at once when the error flag is up).  True when the
// condition holds; the writes counted by *ctr are then visible to every lane.
__device__ bool warp_wait_count(const int32_t *ctr, int target, long long limit, int *err)
{
    const int lane = threadIdx.x & 31;
    int ok = 1;
    if (lane == 0) {
        long long it = 0;
        while (load_acquire(ctr) < target) {
            if (it++ >= limit || *(volatile int *)err) {
                ok = 0;
                break;
            }
            __nanosleep(64);
        }
    }
    ok = __shfl_sync(0xffffffffu, ok, 0);
    __threadfence();
    __syncwarp();
    return ok != 0;
}

// Whole warp: publish the warp's writes, then count one finished item.
__device__ __forceinline__ void warp_done(int32_t *ctr)
{
    __threadfence();
    __syncwarp();
    if ((threadIdx.x & 31) == 0) atomicAdd(ctr, 1);
}

template <bool XSTEP>
__device__ void run_item(const BQueue &Q, const int4 &it, AlsSmem &als)
{
    const BInst &I = Q.inst[it.x];
    Seg g;
    if (XSTEP) {
        g = Seg{Q.rowptr + I.rp_off, Q.colidx + I.e_off, Q.val + I.e_off, Q.X + I.x_off, Q.Yt + I.y_off,
                Q.ax + I.row_base, Q.kobj_x + I.row_base, Q.kreg_x + I.row_base, Q.acc_x + I.row_base,
                I.rxk, (float)I.rxw};
    } else {
        g = Seg{Q.colptr + I.cp_off, Q.rowidx + I.e_off, Q.cval + I.e_off, Q.Yt + I.y_off, Q.X + I.x_off,
                Q.ay + I.col_base, Q.kobj_y + I.col_base, Q.kreg_y + I.col_base, Q.acc_y + I.col_base,
                I.ryk, (float)I.ryw};
    }
    const LossSpec sp{I.kind, I.levels, I.param};
    if (I.method == GLRM_BATCH_ALS) {
        // 32 / k rows (columns) at a time, one lane group each
        const int spw = 32 / I.k;
        for (int64_t s = it.y; s < it.z; s += spw) {
            switch (I.k) {
            case 4: als_group<4>(g, I.rxw, s, it.z, als, !XSTEP, Q.err); break;
            case 8: als_group<8>(g, I.rxw, s, it.z, als, !XSTEP, Q.err); break;
            default: als_group<16>(g, I.rxw, s, it.z, als, !XSTEP, Q.err); break;
            }
        }
    } else {
        for (int64_t s = it.y; s < it.z; ++s) {
            switch (I.k) {
            case 4: pg_segment<4>(g, sp, s); break;
            case 8: pg_segment<8>(g, sp, s); break;
            default: pg_segment<16>(g, sp, s); break;
            }
        }
    }
}

// Objective of instance s after a sweep: the Y-step's kept column objectives
// (every loss term plus rt(y_j)) plus the X-step's kept r(x_i), one warp,
// lane-strided sums and a butterfly: a fixed order.
__device__ double instance_objective(const BQueue &Q, int s)
{
    const int lane = threadIdx.x & 31;
    const BInst &I = Q.inst[s];
    double v = 0.0;
    for (int64_t j = lane; j < I.n; j += 32) v += Q.kobj_y[I.col_base + j];
    for (int64_t i = lane; i < I.m; i += 32) v += Q.kreg_x[I.row_base + i];
    return warp_sum(v);
}

__global__ void __launch_bounds__(kBWarps * 32)
batch_queue_kernel(const BQueue Q)
{
    __shared__ AlsSmem als[kBWarps];
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t per = Q.nx + Q.ny + Q.no;
    const unsigned long long total = (unsigned long long)per * (unsigned long long)Q.sweeps;
    for (;;) {
        unsigned long long q = 0;
        if (lane == 0) q = atomicAdd(Q.head, 1ULL);
        q = __shfl_sync(0xffffffffu, q, 0);
        if (q >= total) break;  // warp-uniform
        const int t = Q.t0 + (int)(q / (unsigned long long)per);
        const int64_t r = (int64_t)(q % (unsigned long long)per);
        if (r < Q.nx) {
            const int4 it = Q.items_x[r];
            // the previous sweep's objective of the instance (which follows its Y-step) is in
            const bool ok = !Q.wait || warp_wait_count(Q.done_o + it.x, t, Q.limit, Q.err);
            if (ok) run_item<true>(Q, it, als[wid]);
            else if (lane == 0) atomicOr(Q.err, kErrWait);
            warp_done(Q.done_x + it.x);
        } else if (r < Q.nx + Q.ny) {
            const int4 it = Q.items_y[r - Q.nx];
            const bool ok = !Q.wait || warp_wait_count(Q.done_x + it.x, (t + 1) * Q.need_x[it.x], Q.limit, Q.err);
            if (ok) run_item<false>(Q, it, als[wid]);
            else if (lane == 0) atomicOr(Q.err, kErrWait);
            warp_done(Q.done_y + it.x);
        } else {
            const int s = Q.obj_inst[r - Q.nx - Q.ny];
            const bool ok = !Q.wait || warp_wait_count(Q.done_y + s, (t + 1) * Q.need_y[s], Q.limit, Q.err);
            const double v = ok ? instance_objective(Q, s) : (double)NAN;
            if (!ok && lane == 0) atomicOr(Q.err, kErrWait);
            if (lane == 0) Q.hist[(int64_t)t * Q.count + s] = v;
            warp_done(Q.done_o + s);
        }
    }
}

__global__ void batch_reset_alpha_kernel(const BInst *__restrict__ inst, int count,
                                         const int32_t *__restrict__ rowptr,
                                         const int32_t *__restrict__ colptr, float *ax, float *ay)
{
    for (int s = blockIdx.x; s < count; s += gridDim.x) {
        const BInst &I = inst[s];
        for (int64_t i = threadIdx.x; i < I.m; i += blockDim.x) {
            const int len = rowptr[I.rp_off + i + 1] - rowptr[I.rp_off + i];
            ax[I.row_base + i] = 1.f / (float)(len > 1 ? len : 1);
        }
        for (int64_t j = threadIdx.x; j < I.n; j += blockDim.x) {
            const int len = colptr[I.cp_off + j + 1] - colptr[I.cp_off + j];
            ay[I.col_base + j] = 1.f / (float)(len > 1 ? len : 1);
        }
    }
}

// Validation of every instance: pointers monotone from 0 to nnz, indices in
// range and strictly ascending, finite values, CSC entries found in CSR with
// the same value bits.  Bit flags as in the single-model validation.
__global__ void batch_validate_kernel(const BInst *__restrict__ inst, int count,
                                      const int32_t *__restrict__ rowptr, const int32_t *__restrict__ colidx,
                                      const float *__restrict__ val, const int32_t *__restrict__ colptr,
                                      const int32_t *__restrict__ rowidx, const float *__restrict__ cval,
                                      int *flag)
{
    for (int s = blockIdx.x; s < count; s += gridDim.x) {
        const BInst &I = inst[s];
        const int32_t *rp = rowptr + I.rp_off, *cp = colptr + I.cp_off;
        const int32_t *ci = colidx + I.e_off, *ri = rowidx + I.e_off;
        const float *rv = val + I.e_off, *cv = cval + I.e_off;
        const int64_t nnz = rp[I.m];  // equals the declared nnz (checked before this kernel)
        int f = 0;
        if (threadIdx.x == 0 && (rp[0] != 0 || cp[0] != 0 || cp[I.n] != nnz)) f |= 1;
        for (int64_t i = threadIdx.x; i < I.m; i += blockDim.x)
            if (rp[i] > rp[i + 1]) f |= 1;
        for (int64_t j = threadIdx.x; j < I.n; j += blockDim.x)
            if (cp[j] > cp[j + 1]) f |= 1;
        f = __syncthreads_or(f) ? 1 : 0;
        if (!f) {
            for (int64_t i = threadIdx.x; i < I.m; i += blockDim.x)
                for (int q = rp[i]; q < rp[i + 1]; ++q) {
                    if (ci[q] < 0 || ci[q] >= I.n) f |= 2;
                    else if (q > rp[i] && ci[q - 1] >= ci[q]) f |= 4;
                    if (!isfinite(rv[q])) f |= 8;
                }
            for (int64_t j = threadIdx.x; j < I.n; j += blockDim.x)
                for (int q = cp[j]; q < cp[j + 1]; ++q) {
                    if (ri[q] < 0 || ri[q] >= I.m) f |= 2;
                    else if (q > cp[j] && ri[q - 1] >= ri[q]) f |= 4;
                }
        }
        const int g = __syncthreads_or(f & 7);
        if (!g) {
            for (int64_t j = threadIdx.x; j < I.n; j += blockDim.x)
                for (int q = cp[j]; q < cp[j + 1]; ++q) {
                    const int i = ri[q];
                    int lo = rp[i], hi = rp[i + 1];
                    while (lo < hi) {
                        const int mid = (lo + hi) >> 1;
                        if (ci[mid] < j) lo = mid + 1;
                        else hi = mid;
                    }
                    if (lo >= rp[i + 1] || ci[lo] != j) f |= 16;
                    else if (__float_as_int(rv[lo]) != __float_as_int(cv[q])) f |= 32;
                }
        }
        if (f) atomicOr(flag, f);
        __syncthreads();
    }
}

// rowptr[m] and colptr[n] of every instance (checked against the declared
// nnz on the host before any kernel reads entries through the pointers).
__global__ void batch_last_ptr_kernel(const BInst *__restrict__ inst, int count,
                                      const int32_t *__restrict__ rowptr,
                                      const int32_t *__restrict__ colptr, int32_t *__restrict__ out)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= count) return;
    out[2 * s] = rowptr[inst[s].rp_off + inst[s].m];
    out[2 * s + 1] = colptr[inst[s].cp_off + inst[s].n];
}

// ----------------------------------------------------------------- host side

// Average entries per segment picks the size class.
int size_class(double avg)
{
    return avg < 64 ? 0 : (avg < 256 ? 1 : (avg < 1024 ? 2 : 3));
}

int bucket(const BInst &I, int64_t nnz, bool xstep)
{
    const int kc = I.k == 4 ? 0 : (I.k == 8 ? 1 : 2);
    const double avg = (double)nnz / (double)std::max<int64_t>(1, xstep ? I.m : I.n);
    return kc * 8 + I.method * 4 + size_class(avg);
}

// Items of one orientation: each instance's segments in ranges of the tile
// size of its bucket, ordered by decreasing estimated work (order 0) or
// instance by instance (order 1: warps running at the same time then share an
// instance's factors in L2).
void build_items(const glrm_batch_s *b, bool xstep, const int32_t *tiles, const std::vector<int> *only,
                 std::vector<int4> &items, std::vector<int64_t> *first, int order = 0)
{
    struct W {
        int4 it;
        double cost;
    };
    std::vector<W> all;
    if (first) first->assign((size_t)b->count + 1, 0);
    for (int s = 0; s < b->count; ++s) {
        if (only && std::find(only->begin(), only->end(), s) == only->end()) continue;
        const BInst &I = b->inst_host[s];
        const int64_t segs = xstep ? I.m : I.n;
        const int64_t nnzs = (s + 1 < b->count ? b->inst_host[s + 1].e_off : b->nnz) - I.e_off;
        const int t = std::max(1, tiles[bucket(I, nnzs, xstep)]);
        const double per = (double)nnzs / (double)std::max<int64_t>(1, segs);
        for (int64_t a = 0; a < segs; a += t) {
            const int64_t z = std::min(segs, a + t);
            const double w = (double)(z - a) * (per * (I.method == GLRM_BATCH_ALS ? 0.5 * I.k : 2.0) + 64.0);
            all.push_back(W{make_int4(s, (int)a, (int)z, 0), w});
        }
    }
    if (order == 0)
        std::stable_sort(all.begin(), all.end(), [](const W &x, const W &y) { return x.cost > y.cost; });
    items.clear();
    for (const W &w : all) items.push_back(w.it);
    if (first) {
        // unbatched mode wants each instance's items together
        std::stable_sort(items.begin(), items.end(), [](const int4 &x, const int4 &y) { return x.x < y.x; });
        for (const int4 &it : items) (*first)[it.x + 1]++;
        for (int s = 0; s < b->count; ++s) (*first)[s + 1] += (*first)[s];
    }
}

int upload_items(glrm_batch_s *b)
{
    std::vector<int4> ix, iy;
    build_items(b, true, b->tile_x, nullptr, ix, nullptr, b->order_x);
    build_items(b, false, b->tile_y, nullptr, iy, nullptr, b->order_y);
    bfree(b->items_x);
    bfree(b->items_y);
    BCK(cudaMalloc(&b->items_x, std::max<size_t>(1, ix.size()) * sizeof(int4)));
    BCK(cudaMalloc(&b->items_y, std::max<size_t>(1, iy.size()) * sizeof(int4)));
    BCK(cudaMemcpy(b->items_x, ix.data(), ix.size() * sizeof(int4), cudaMemcpyHostToDevice));
    BCK(cudaMemcpy(b->items_y, iy.data(), iy.size() * sizeof(int4), cudaMemcpyHostToDevice));
    b->nitems_x = (int64_t)ix.size();
    b->nitems_y = (int64_t)iy.size();
    std::vector<int32_t> nx((size_t)b->count, 0), ny((size_t)b->count, 0);
    for (const int4 &it : ix) nx[it.x]++;
    for (const int4 &it : iy) ny[it.x]++;
    BCK(cudaMemcpy(b->need_x, nx.data(), nx.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
    BCK(cudaMemcpy(b->need_y, ny.data(), ny.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
    if (b->graph) {
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
        b->graph_sweeps = 0;
    }
    return GLRM_OK;
}

// One launch of the queue kernel over the given lists (sweeps t0 ..
// t0 + sweeps - 1); the queue head is reset first.  A full launch uses the
// persistent grid, a small one no more CTAs than it has items for.
cudaError_t launch_queue(glrm_batch_s *b, const int4 *ix, int64_t nx, const int4 *iy, int64_t ny, int64_t no,
                         int t0, int sweeps, int wait, cudaStream_t st)
{
    const int64_t total = (nx + ny + no) * sweeps;
    if (total == 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(b->qhead, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    BQueue Q;
    Q.inst = b->inst;
    Q.items_x = ix;
    Q.items_y = iy;
    Q.obj_inst = b->obj_inst;
    Q.nx = nx;
    Q.ny = ny;
    Q.no = no;
    Q.need_x = b->need_x;
    Q.need_y = b->need_y;
    Q.t0 = t0;
    Q.sweeps = sweeps;
    Q.count = b->count;
    Q.wait = wait;
    Q.head = b->qhead;
    Q.done_x = b->done;
    Q.done_y = b->done + b->count;
    Q.done_o = b->done + 2 * (size_t)b->count;
    Q.err = b->status;
    Q.limit = b->wait_limit;
    Q.hist = b->hist;
    Q.rowptr = b->rowptr;
    Q.colidx = b->colidx;
    Q.colptr = b->colptr;
    Q.rowidx = b->rowidx;
    Q.val = b->val;
    Q.cval = b->cval;
    Q.X = b->X;
    Q.Yt = b->Yt;
    Q.ax = b->ax;
    Q.ay = b->ay;
    Q.kobj_x = b->kept_obj_x;
    Q.kreg_x = b->kept_reg_x;
    Q.kobj_y = b->kept_obj_y;
    Q.kreg_y = b->kept_reg_y;
    Q.acc_x = b->acc_x;
    Q.acc_y = b->acc_y;
    const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(b->qgrid, (total + kBWarps - 1) / kBWarps));
    batch_queue_kernel<<<grid, kBWarps * 32, 0, st>>>(Q);
    return cudaGetLastError();
}

// A half-step on its own (autotuning): no dependency waits.
cudaError_t launch_half(glrm_batch_s *b, bool xstep, const int4 *items, int64_t n, cudaStream_t st)
{
    return xstep ? launch_queue(b, items, n, nullptr, 0, 0, 0, 1, 0, st)
                 : launch_queue(b, nullptr, 0, items, n, 0, 0, 1, 0, st);
}

// Every sweep of a call in one launch, after the completion counters are reset.
cudaError_t enqueue_sweeps(glrm_batch_s *b, int nsweeps, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(b->done, 0, 3 * sizeof(int32_t) * (size_t)b->count, st);
    if (e != cudaSuccess) return e;
    return launch_queue(b, b->items_x, b->nitems_x, b->items_y, b->nitems_y, b->count, 0, nsweeps, 1, st);
}

}  // namespace

extern "C" {

const char *glrm_batch_last_error(glrm_batch_t b) { return b ? b->err.c_str() : g_berr.c_str(); }

int glrm_batch_create(int32_t count, const glrm_batch_instance *ih, const int32_t *rowptr,
                      const int32_t *colidx, const float *val, const int32_t *colptr,
                      const int32_t *rowidx, const float *cval, void *stream, glrm_batch_t *out)
{
    g_berr.clear();
    glrm_batch_s *b = nullptr;
    if (!out) return bfail(nullptr, GLRM_ERR_ARG, "out is null");
    *out = nullptr;
    if (count < 1 || !ih) return bfail(nullptr, GLRM_ERR_ARG, "count < 1 or no instances");
    std::vector<BInst> in((size_t)count);
    int64_t rp = 0, cp = 0, e = 0, xo = 0, yo = 0, rb = 0, cb = 0;
    for (int s = 0; s < count; ++s) {
        const glrm_batch_instance &q = ih[s];
        const std::string where = " (instance " + std::to_string(s) + ")";
        if (q.m < 1 || q.n < 1 || q.m >= INT32_MAX || q.n >= INT32_MAX || q.nnz < 0 || q.nnz >= INT32_MAX)
            return bfail(nullptr, GLRM_ERR_RANGE, "bad m, n or nnz" + where);
        if (q.k != 4 && q.k != 8 && q.k != 16) return bfail(nullptr, GLRM_ERR_RANGE, "k must be 4, 8 or 16" + where);
        if (q.method != GLRM_BATCH_PROXGRAD && q.method != GLRM_BATCH_ALS)
            return bfail(nullptr, GLRM_ERR_ARG, "bad method" + where);
        if (q.loss.kind < kLossQuad || q.loss.kind > kLossOrdinal) return bfail(nullptr, GLRM_ERR_ARG, "bad loss" + where);
        if (q.loss.kind == kLossHuber && !(q.loss.param > 0.0)) return bfail(nullptr, GLRM_ERR_ARG, "Huber threshold" + where);
        if (q.loss.kind == kLossOrdinal && (q.loss.levels < 2 || q.loss.levels > 1024))
            return bfail(nullptr, GLRM_ERR_ARG, "ordinal levels" + where);
        for (int r : {q.rx_kind, q.ry_kind})
            if (r < kRegZero || r > kRegNonneg) return bfail(nullptr, GLRM_ERR_ARG, "bad regulariser" + where);
        if (q.method == GLRM_BATCH_ALS &&
            (q.loss.kind != kLossQuad || q.rx_kind != kRegQuad || q.ry_kind != kRegQuad ||
             q.rx_weight != q.ry_weight || !(q.rx_weight > 0.0)))
            return bfail(nullptr, GLRM_ERR_ARG, "ALS needs quadratic loss and gamma||.||^2 (gamma > 0) on both factors" + where);
        BInst &I = in[s];
        I.m = q.m;
        I.n = q.n;
        I.rp_off = rp;
        I.cp_off = cp;
        I.e_off = e;
        I.x_off = xo;
        I.y_off = yo;
        I.row_base = rb;
        I.col_base = cb;
        I.k = q.k;
        I.method = q.method;
        I.kind = q.loss.kind;
        I.levels = q.loss.kind == kLossOrdinal ? q.loss.levels : 0;
        I.param = q.loss.kind == kLossHuber ? q.loss.param : 0.0;
        I.rxk = q.rx_kind;
        I.ryk = q.ry_kind;
        I.rxw = q.rx_weight;
        I.ryw = q.ry_weight;
        rp += q.m + 1;
        cp += q.n + 1;
        e += q.nnz;
        xo += q.m * q.k;
        yo += q.n * q.k;
        rb += q.m;
        cb += q.n;
    }
    if (!rowptr || !colptr || (e > 0 && (!colidx || !val || !rowidx || !cval)))
        return bfail(nullptr, GLRM_ERR_ARG, "null data pointer");
    b = new (std::nothrow) glrm_batch_s;
    if (!b) return bfail(nullptr, GLRM_ERR_NOMEM, "host allocation");
    *out = b;  // from here on errors leave a handle the caller destroys
    b->count = count;
    b->stream = (cudaStream_t)stream;
    b->inst_host = in;
    b->nnz = e;
    b->rows = rb;
    b->cols = cb;
    b->xlen = xo;
    b->ylen = yo;
    for (int q = 0; q < kBucketCount; ++q) b->tile_x[q] = b->tile_y[q] = 1;
    BCK(cudaGetDevice(&b->device));
    int sms = 0;
    BCK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device));
    int per_sm = 0;
    BCK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_queue_kernel, kBWarps * 32, 0));
    b->qgrid = sms * std::max(per_sm, 1);
    BCK(cudaStreamCreateWithFlags(&b->capture, cudaStreamNonBlocking));
    cudaStream_t st = b->stream;
    const size_t nz = (size_t)std::max<int64_t>(e, 1);
    BCK(cudaMalloc(&b->inst, sizeof(BInst) * count));
    BCK(cudaMalloc(&b->rowptr, sizeof(int32_t) * rp));
    BCK(cudaMalloc(&b->colptr, sizeof(int32_t) * cp));
    BCK(cudaMalloc(&b->colidx, sizeof(int32_t) * nz));
    BCK(cudaMalloc(&b->rowidx, sizeof(int32_t) * nz));
    BCK(cudaMalloc(&b->val, sizeof(float) * nz));
    BCK(cudaMalloc(&b->cval, sizeof(float) * nz));
    BCK(cudaMalloc(&b->X, sizeof(float) * std::max<int64_t>(xo, 1)));
    BCK(cudaMalloc(&b->Yt, sizeof(float) * std::max<int64_t>(yo, 1)));
    BCK(cudaMalloc(&b->ax, sizeof(float) * rb));
    BCK(cudaMalloc(&b->ay, sizeof(float) * cb));
    BCK(cudaMalloc(&b->kept_obj_x, sizeof(double) * rb));
    BCK(cudaMalloc(&b->kept_reg_x, sizeof(double) * rb));
    BCK(cudaMalloc(&b->kept_obj_y, sizeof(double) * cb));
    BCK(cudaMalloc(&b->kept_reg_y, sizeof(double) * cb));
    BCK(cudaMalloc(&b->acc_x, sizeof(int32_t) * rb));
    BCK(cudaMalloc(&b->acc_y, sizeof(int32_t) * cb));
    BCK(cudaMalloc(&b->need_x, sizeof(int32_t) * count));
    BCK(cudaMalloc(&b->need_y, sizeof(int32_t) * count));
    BCK(cudaMalloc(&b->obj_inst, sizeof(int32_t) * count));
    BCK(cudaMalloc(&b->qhead, sizeof(unsigned long long)));
    BCK(cudaMalloc(&b->done, 3 * sizeof(int32_t) * count));
    BCK(cudaMalloc(&b->status, sizeof(int)));
    BCK(cudaMemsetAsync(b->status, 0, sizeof(int), st));
    {
        std::vector<int32_t> ids((size_t)count);
        for (int q = 0; q < count; ++q) ids[q] = q;
        BCK(cudaMemcpyAsync(b->obj_inst, ids.data(), sizeof(int32_t) * count, cudaMemcpyHostToDevice, st));
        BCK(cudaStreamSynchronize(st));
    }
    BCK(cudaMemcpyAsync(b->inst, in.data(), sizeof(BInst) * count, cudaMemcpyHostToDevice, st));
    BCK(cudaMemcpyAsync(b->rowptr, rowptr, sizeof(int32_t) * rp, cudaMemcpyDeviceToDevice, st));
    BCK(cudaMemcpyAsync(b->colptr, colptr, sizeof(int32_t) * cp, cudaMemcpyDeviceToDevice, st));
    if (e > 0) {
        BCK(cudaMemcpyAsync(b->colidx, colidx, sizeof(int32_t) * e, cudaMemcpyDeviceToDevice, st));
        BCK(cudaMemcpyAsync(b->rowidx, rowidx, sizeof(int32_t) * e, cudaMemcpyDeviceToDevice, st));
        BCK(cudaMemcpyAsync(b->val, val, sizeof(float) * e, cudaMemcpyDeviceToDevice, st));
        BCK(cudaMemcpyAsync(b->cval, cval, sizeof(float) * e, cudaMemcpyDeviceToDevice, st));
    }
    BCK(cudaMemsetAsync(b->X, 0, sizeof(float) * std::max<int64_t>(xo, 1), st));
    BCK(cudaMemsetAsync(b->Yt, 0, sizeof(float) * std::max<int64_t>(yo, 1), st));
    // each instance's pointers must end at its declared nnz before anything
    // reads entries through them
    {
        int32_t *last = nullptr;
        BCK(cudaMalloc(&last, sizeof(int32_t) * 2 * count));
        batch_last_ptr_kernel<<<(count + 255) / 256, 256, 0, st>>>(b->inst, count, b->rowptr, b->colptr, last);
        BCK(cudaGetLastError());
        std::vector<int32_t> h((size_t)2 * count);
        BCK(cudaMemcpyAsync(h.data(), last, sizeof(int32_t) * 2 * count, cudaMemcpyDeviceToHost, st));
        BCK(cudaStreamSynchronize(st));
        cudaFree(last);
        for (int s = 0; s < count; ++s)
            if ((int64_t)h[2 * s] != ih[s].nnz || (int64_t)h[2 * s + 1] != ih[s].nnz)
                return bfail(b, GLRM_ERR_OMEGA, "instance " + std::to_string(s) +
                                                    ": rowptr[m] or colptr[n] differs from nnz");
    }
    int *flag = nullptr;
    BCK(cudaMalloc(&flag, sizeof(int)));
    BCK(cudaMemsetAsync(flag, 0, sizeof(int), st));
    batch_validate_kernel<<<std::min(count, 4096), 256, 0, st>>>(b->inst, count, b->rowptr, b->colidx,
                                                                 b->val, b->colptr, b->rowidx, b->cval, flag);
    int hflag = 0;
    BCK(cudaGetLastError());
    BCK(cudaMemcpyAsync(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, st));
    BCK(cudaStreamSynchronize(st));
    cudaFree(flag);
    if (hflag)
        return bfail(b, (hflag & 8) && !(hflag & ~8) ? GLRM_ERR_NONFINITE : GLRM_ERR_OMEGA,
                     "batched observed sets failed validation (flags " + std::to_string(hflag) + ")");
    batch_reset_alpha_kernel<<<std::min(count, 4096), 256, 0, st>>>(b->inst, count, b->rowptr, b->colptr,
                                                                     b->ax, b->ay);
    BCK(cudaGetLastError());
    int rc = upload_items(b);
    if (rc != GLRM_OK) return rc;
    BCK(cudaStreamSynchronize(st));
    return GLRM_OK;
}

int glrm_batch_set_factors(glrm_batch_t b, const float *X, const float *Yt)
{
    if (!b) return bfail(nullptr, GLRM_ERR_ARG, "null handle");
    if (X) BCK(cudaMemcpyAsync(b->X, X, sizeof(float) * b->xlen, cudaMemcpyDeviceToDevice, b->stream));
    if (Yt) BCK(cudaMemcpyAsync(b->Yt, Yt, sizeof(float) * b->ylen, cudaMemcpyDeviceToDevice, b->stream));
    return GLRM_OK;
}

int glrm_batch_get_factors(glrm_batch_t b, float *X, float *Yt)
{
    if (!b) return bfail(nullptr, GLRM_ERR_ARG, "null handle");
    if (X) BCK(cudaMemcpyAsync(X, b->X, sizeof(float) * b->xlen, cudaMemcpyDeviceToDevice, b->stream));
    if (Yt) BCK(cudaMemcpyAsync(Yt, b->Yt, sizeof(float) * b->ylen, cudaMemcpyDeviceToDevice, b->stream));
    return GLRM_OK;
}

int glrm_batch_get_steps(glrm_batch_t b, float *ax, float *ay)
{
    if (!b) return bfail(nullptr, GLRM_ERR_ARG, "null handle");
    if (ax) BCK(cudaMemcpyAsync(ax, b->ax, sizeof(float) * b->rows, cudaMemcpyDeviceToDevice, b->stream));
    if (ay) BCK(cudaMemcpyAsync(ay, b->ay, sizeof(float) * b->cols, cudaMemcpyDeviceToDevice, b->stream));
    return GLRM_OK;
}

int glrm_batch_set_steps(glrm_batch_t b, const float *ax, const float *ay)
{
    if (!b) return bfail(nullptr, GLRM_ERR_ARG, "null handle");
    if (ax) BCK(cudaMemcpyAsync(b->ax, ax, sizeof(float) * b->rows, cudaMemcpyDeviceToDevice, b->stream));
    if (ay) BCK(cudaMemcpyAsync(b->ay, ay, sizeof(float) * b->cols, cudaMemcpyDeviceToDevice, b->stream));
    return GLRM_OK;
}

int glrm_batch_sweep(glrm_batch_t b, int32_t nsweeps, double *objectives, int32_t mode)
{
    if (!b) return bfail(nullptr, GLRM_ERR_ARG, "null handle");
    if (nsweeps < 0 || mode < GLRM_BATCH_GRAPH || mode > GLRM_BATCH_PER_INSTANCE)
        return bfail(b, GLRM_ERR_ARG, "bad nsweeps or mode");
    if (nsweeps == 0) return GLRM_OK;
    if (b->hist_cap < nsweeps) {
        bfree(b->hist);
        BCK(cudaMalloc(&b->hist, sizeof(double) * (size_t)nsweeps * b->count));
        b->hist_cap = nsweeps;
        if (b->graph) {
            cudaGraphExecDestroy(b->graph);
            b->graph = nullptr;
            b->graph_sweeps = 0;
        }
    }
    cudaStream_t st = b->stream;
    if (mode == GLRM_BATCH_GRAPH) {
        // the counter reset and the one queue launch, captured once per sweep count
        if (!b->graph || b->graph_sweeps != nsweeps) {
            if (b->graph) cudaGraphExecDestroy(b->graph);
            b->graph = nullptr;
            cudaGraph_t g = nullptr;
            BCK(cudaStreamBeginCapture(b->capture, cudaStreamCaptureModeThreadLocal));
            const cudaError_t e = enqueue_sweeps(b, nsweeps, b->capture);
            const cudaError_t e2 = cudaStreamEndCapture(b->capture, &g);
            if (e != cudaSuccess || e2 != cudaSuccess) {
                if (g) cudaGraphDestroy(g);
                return bfail(b, GLRM_ERR_CUDA, std::string("graph capture: ") +
                                                   cudaGetErrorString(e != cudaSuccess ? e : e2));
            }
            const cudaError_t e3 = cudaGraphInstantiate(&b->graph, g, 0);
            cudaGraphDestroy(g);
            if (e3 != cudaSuccess)
                return bfail(b, GLRM_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e3));
            b->graph_sweeps = nsweeps;
        }
        BCK(cudaGraphLaunch(b->graph, st));
    } else if (mode == GLRM_BATCH_STREAM) {
        const cudaError_t e = enqueue_sweeps(b, nsweeps, st);
        if (e != cudaSuccess) return bfail(b, GLRM_ERR_CUDA, cudaGetErrorString(e));
    } else {
        // for comparison: one launch per instance and half-step (the same
        // kernel over each instance's items alone) and one for the objectives
        std::vector<int4> ix, iy;
        std::vector<int64_t> fx, fy;
        build_items(b, true, b->tile_x, nullptr, ix, &fx);
        build_items(b, false, b->tile_y, nullptr, iy, &fy);
        int4 *dx = nullptr, *dy = nullptr;
        BCK(cudaMalloc(&dx, std::max<size_t>(1, ix.size()) * sizeof(int4)));
        BCK(cudaMalloc(&dy, std::max<size_t>(1, iy.size()) * sizeof(int4)));
        BCK(cudaMemcpy(dx, ix.data(), ix.size() * sizeof(int4), cudaMemcpyHostToDevice));
        BCK(cudaMemcpy(dy, iy.data(), iy.size() * sizeof(int4), cudaMemcpyHostToDevice));
        cudaError_t e = cudaMemsetAsync(b->done, 0, 3 * sizeof(int32_t) * (size_t)b->count, st);
        for (int t = 0; t < nsweeps && e == cudaSuccess; ++t) {
            for (int s = 0; s < b->count && e == cudaSuccess; ++s)
                e = launch_queue(b, dx + fx[s], fx[s + 1] - fx[s], nullptr, 0, 0, t, 1, 1, st);
            for (int s = 0; s < b->count && e == cudaSuccess; ++s)
                e = launch_queue(b, nullptr, 0, dy + fy[s], fy[s + 1] - fy[s], 0, t, 1, 1, st);
            if (e == cudaSuccess) e = launch_queue(b, nullptr, 0, nullptr, 0, b->count, t, 1, 1, st);
        }
        cudaStreamSynchronize(st);
        cudaFree(dx);
        cudaFree(dy);
        if (e != cudaSuccess) return bfail(b, GLRM_ERR_CUDA, cudaGetErrorString(e));
    }
    if (objectives) {
        BCK(cudaMemcpyAsync(objectives, b->hist, sizeof(double) * (size_t)nsweeps * b->count,
                            cudaMemcpyDeviceToHost, st));
        int flag = 0;
        BCK(cudaMemcpyAsync(&flag, b->status, sizeof(int), cudaMemcpyDeviceToHost, st));
        BCK(cudaStreamSynchronize(st));
        if (flag) {
            BCK(cudaMemsetAsync(b->status, 0, sizeof(int), st));
            if (flag & kErrWait)
                return bfail(b, GLRM_ERR_TIMEOUT, "a work item's wait for the items it depends on ran past "
                                                  "its limit; results of this call are invalid");
            return bfail(b, GLRM_ERR_NONFINITE, "an ALS row or column system was not numerically positive "
                                                "definite; those rows or columns kept their previous factor");
        }
    }
    return GLRM_OK;
}

int glrm_batch_set_wait_limit(glrm_batch_t b, int64_t polls)
{
    if (!b) return bfail(nullptr, GLRM_ERR_ARG, "null handle");
    if (polls < 0) return bfail(b, GLRM_ERR_ARG, "polls < 0");
    b->wait_limit = polls;
    if (b->graph) {  // the limit is a kernel argument: capture again
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
        b->graph_sweeps = 0;
    }
    return GLRM_OK;
}

int glrm_batch_autotune(glrm_batch_t b, int32_t reps, int32_t *tiles_x, int32_t *tiles_y)
{
    if (!b) return bfail(nullptr, GLRM_ERR_ARG, "null handle");
    if (reps < 1) reps = 1;
    cudaStream_t st = b->stream;
    // keep the fit state: timing runs update factors and steps
    float *sx = nullptr, *sy = nullptr, *sax = nullptr, *say = nullptr;
    BCK(cudaMalloc(&sx, sizeof(float) * std::max<int64_t>(1, b->xlen)));
    BCK(cudaMalloc(&sy, sizeof(float) * std::max<int64_t>(1, b->ylen)));
    BCK(cudaMalloc(&sax, sizeof(float) * b->rows));
    BCK(cudaMalloc(&say, sizeof(float) * b->cols));
    BCK(cudaMemcpyAsync(sx, b->X, sizeof(float) * b->xlen, cudaMemcpyDeviceToDevice, st));
    BCK(cudaMemcpyAsync(sy, b->Yt, sizeof(float) * b->ylen, cudaMemcpyDeviceToDevice, st));
    BCK(cudaMemcpyAsync(sax, b->ax, sizeof(float) * b->rows, cudaMemcpyDeviceToDevice, st));
    BCK(cudaMemcpyAsync(say, b->ay, sizeof(float) * b->cols, cudaMemcpyDeviceToDevice, st));
    const int cand[4] = {1, 2, 4, 8};
    cudaEvent_t e0, e1;
    BCK(cudaEventCreate(&e0));
    BCK(cudaEventCreate(&e1));
    int rc = GLRM_OK;
    for (int side = 0; side < 2 && rc == GLRM_OK; ++side) {
        const bool xstep = side == 0;
        int32_t *table = xstep ? b->tile_x : b->tile_y;
        std::map<int, std::vector<int>> members;
        for (int s = 0; s < b->count; ++s) {
            const BInst &I = b->inst_host[s];
            const int64_t nnzs = (s + 1 < b->count ? b->inst_host[s + 1].e_off : b->nnz) - I.e_off;
            members[bucket(I, nnzs, xstep)].push_back(s);
        }
        for (auto &kv : members) {
            float best_ms = 1e30f;
            int best = 1;
            for (int c : cand) {
                int32_t trial[kBucketCount];
                for (int q = 0; q < kBucketCount; ++q) trial[q] = c;
                std::vector<int4> items;
                build_items(b, xstep, trial, &kv.second, items, nullptr);
                int4 *d = nullptr;
                if (cudaMalloc(&d, std::max<size_t>(1, items.size()) * sizeof(int4)) != cudaSuccess) {
                    rc = bfail(b, GLRM_ERR_NOMEM, "autotune items");
                    break;
                }
                cudaMemcpy(d, items.data(), items.size() * sizeof(int4), cudaMemcpyHostToDevice);
                launch_half(b, xstep, d, (int64_t)items.size(), st);  // warm
                cudaEventRecord(e0, st);
                for (int r = 0; r < reps; ++r) launch_half(b, xstep, d, (int64_t)items.size(), st);
                cudaEventRecord(e1, st);
                cudaEventSynchronize(e1);
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                cudaFree(d);
                if (ms < best_ms) {
                    best_ms = ms;
                    best = c;
                }
            }
            table[kv.first] = best;
        }
        // item order over the whole half-step with the chosen tiles
        float best_ms = 1e30f;
        for (int order = 0; order < 2 && rc == GLRM_OK; ++order) {
            std::vector<int4> items;
            build_items(b, xstep, table, nullptr, items, nullptr, order);
            int4 *d = nullptr;
            if (cudaMalloc(&d, std::max<size_t>(1, items.size()) * sizeof(int4)) != cudaSuccess) {
                rc = bfail(b, GLRM_ERR_NOMEM, "autotune items");
                break;
            }
            cudaMemcpy(d, items.data(), items.size() * sizeof(int4), cudaMemcpyHostToDevice);
            launch_half(b, xstep, d, (int64_t)items.size(), st);
            cudaEventRecord(e0, st);
            for (int r = 0; r < reps; ++r) launch_half(b, xstep, d, (int64_t)items.size(), st);
            cudaEventRecord(e1, st);
            cudaEventSynchronize(e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            cudaFree(d);
            if (ms < best_ms) {
                best_ms = ms;
                (xstep ? b->order_x : b->order_y) = order;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaMemcpyAsync(b->X, sx, sizeof(float) * b->xlen, cudaMemcpyDeviceToDevice, st);
    cudaMemcpyAsync(b->Yt, sy, sizeof(float) * b->ylen, cudaMemcpyDeviceToDevice, st);
    cudaMemcpyAsync(b->ax, sax, sizeof(float) * b->rows, cudaMemcpyDeviceToDevice, st);
    cudaMemcpyAsync(b->ay, say, sizeof(float) * b->cols, cudaMemcpyDeviceToDevice, st);
    cudaStreamSynchronize(st);
    cudaFree(sx);
    cudaFree(sy);
    cudaFree(sax);
    cudaFree(say);
    if (rc != GLRM_OK) return rc;
    if (tiles_x) std::memcpy(tiles_x, b->tile_x, sizeof(b->tile_x));
    if (tiles_y) std::memcpy(tiles_y, b->tile_y, sizeof(b->tile_y));
    return upload_items(b);
}

void glrm_batch_destroy(glrm_batch_t b)
{
    if (!b) return;
    cudaStreamSynchronize(b->stream);
    if (b->graph) cudaGraphExecDestroy(b->graph);
    if (b->capture) cudaStreamDestroy(b->capture);
    bfree(b->inst);
    bfree(b->rowptr);
    bfree(b->colidx);
    bfree(b->val);
    bfree(b->colptr);
    bfree(b->rowidx);
    bfree(b->cval);
    bfree(b->X);
    bfree(b->Yt);
    bfree(b->ax);
    bfree(b->ay);
    bfree(b->kept_obj_x);
    bfree(b->kept_reg_x);
    bfree(b->kept_obj_y);
    bfree(b->kept_reg_y);
    bfree(b->acc_x);
    bfree(b->acc_y);
    bfree(b->hist);
    bfree(b->items_x);
    bfree(b->items_y);
    bfree(b->need_x);
    bfree(b->need_y);
    bfree(b->obj_inst);
    bfree(b->qhead);
    bfree(b->done);
    bfree(b->status);
    delete b;
}

}  // extern "C"
