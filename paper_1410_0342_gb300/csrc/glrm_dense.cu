// Dense, fully observed form of the alternating proximal-gradient sweep
// (Algorithm 2 of Udell et al., "Generalized Low Rank Models", with Omega =
// every (i, j)) on the fifth-generation tensor cores.
//
// Naming: in a half-step the "own" factor F is the one being updated (X in
// the X-step, Y in the Y-step) and the "other" factor W is held fixed.  Each
// half-step is five launches:
//   pack   W split into BF16 parts x = hi + mid + lo (+ at most 2^-26 |x|) in
//          the tensor core's swizzled K-major shared-memory layouts: with K = k
//          (B operand of GEMM1) and, per 64-row chunk, with K = the chunk rows
//          (B operand of GEMM2);
//   grad   per 128 own rows and a range of 64-wide chunks of the other
//          dimension: U = F W^T (GEMM1), L(U, A) and its derivative R against
//          the A tile (staged by tensor TMA; a NaN cell is a missing entry and
//          contributes nothing), R split in three into tensor memory, G += R W
//          (GEMM2);
//   prox   f+ = prox(f - alpha g) per row / column (shared with the sparse form);
//   loss   the candidate's losses (GEMM1 and L only);
//   decide accept when the objective did not increase (shared with the
//          sparse form).
// Both GEMMs sum the six BF16 products of the splits whose order is at least
// 2^-18 (hi.hi, hi.mid, mid.hi, mid.mid, hi.lo, lo.hi) in FP32 in tensor
// memory; the dropped terms (mid.lo, lo.mid, lo.lo) and the split remainders
// are about 2^-25 of sum |f_c w_c|, below FP32's own rounding of a k-term
// dot product, so losses, the accept / reject test and the gradients see FP32
// quality values.
//
// Pipeline of one CTA (one lane each of three producer warps issues the
// GEMM1 MMAs, the copies and the GEMM2 MMAs; 16 warps run the per-entry
// work): GEMM1 runs two chunks ahead into a double-buffered accumulator, so
// the tensor core computes U of chunk q + 1 while the warps evaluate the
// losses of chunk q; R is double-buffered in tensor memory, so the warps
// write R of chunk q while GEMM2 of chunk q - 1 still reads the other buffer;
// W's GEMM1 and GEMM2 parts are triple-buffered, the A tiles two to four
// times.
#include <cuda.h>

#include <string.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <functional>
#include <queue>
#include <vector>

#include "glrm_tc.cuh"

namespace glrm {

constexpr int kDnNT = 64;        // chunk of the other dimension (UMMA N of GEMM1, K of GEMM2)
constexpr int kDnRows = 128;     // own rows per CTA (UMMA M)
constexpr int kDnWarps = 16;     // evaluating warp w: TMEM lanes 32 (w % 4) .. + 31, chunk columns 16 (w / 4) .. + 15
constexpr int kDnThreads = (kDnWarps + 3) * 32;  // + the GEMM1 warp, the copy warp, the GEMM2 warp
// TMEM columns: U at [0, 64) and [64, 128), G at [128, 128 + KP), two buffers
// of R (hi, mid, lo; 32 columns each) at [192, 288) and [288, 384), the own
// rows (hi, mid, lo; KP / 2 columns each) from 384
constexpr int kDnTmem = 512;
constexpr int kDnColG = 128, kDnColR = 192, kDnColOwn = 384;
constexpr int kDnMaxStages = 4;

// Column loss with its parameters in FP32 (kind as int bits, Huber
// threshold, ordinal level count, unused).
using LossF = float4;

struct DenseArgs {
    int64_t nown, nother;
    int k;
    const float *F;           // own factor, nown x k
    const __nv_bfloat16 *pk;  // other factor, K-major over k: parts hi, mid, lo (each pack_part)
    const __nv_bfloat16 *pt;  // other factor per chunk, K-major over the chunk rows: parts hi, mid, lo
    int64_t pack_part;        // elements per part
    const LossF *lossf;       // n column losses; w: the kind of the column's 16-column group, else -1
    const float *wcol;        // WGT kernels: n per-column loss weights (the scaled losses of Section 4.3)
    const DnItem *items;      // one per CTA
    const int32_t *blocks;    // Y-step: per tile its four 32-column blocks (-1: none)
    const int32_t *segchunk;  // own index -> first partial slot
    int nA;
    float *part_grad;     // slots x k
    double *part_loss;    // slots
    int *err;
};

// Dynamic shared memory of one CTA: the A stages first (1024-byte aligned for
// the swizzled boxes; 1024 bytes of slack align the base), then three stages
// of W's three GEMM1 parts, three stages of W's three GEMM2 parts and three
// stages of the loss table (every operand buffer on a 1024-byte boundary).
template <bool XSTEP, bool GRAD, int KP>
struct DnSmem {
    static constexpr size_t pk = (size_t)kDnNT * KP * 2;
    static constexpr size_t pt = GRAD ? (size_t)KP * kDnNT * 2 : 0;
    static constexpr size_t ls = XSTEP ? (size_t)kDnNT * sizeof(LossF) : 0;
    static constexpr size_t a = (size_t)kDnNT * kDnRows * 4;  // 32 KB A tile
    static constexpr size_t fixed = 9 * pk + 9 * pt + 3 * ls;
    static size_t bytes(int nA) { return 1024 + fixed + (size_t)nA * a; }
};

__device__ __forceinline__ uint32_t bf2_bits(__nv_bfloat162 v)
{
    return *reinterpret_cast<uint32_t *>(&v);
}

// 2-D tiled TMA load of one box into shared memory, completion on the mbarrier.
__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
        "[%4];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

// x = hi + mid + lo in BF16 (each remainder exact in FP32).
__device__ __forceinline__ void split3(float v, __nv_bfloat16 &hi, __nv_bfloat16 &mid, __nv_bfloat16 &lo)
{
    hi = __float2bfloat16_rn(v);
    const float r1 = v - __bfloat162float(hi);
    mid = __float2bfloat16_rn(r1);
    lo = __float2bfloat16_rn(r1 - __bfloat162float(mid));
}

// One MMA with A read from tensor memory: D[taddr] (+)= A[a_taddr] B^T.
__device__ __forceinline__ void umma_bf16_ta(uint32_t taddr, uint32_t a_taddr, uint64_t bdesc, uint32_t idesc,
                                             bool accumulate)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}\n" ::"r"(taddr),
        "r"(a_taddr), "l"(bdesc), "r"(idesc), "r"((uint32_t)accumulate)
        : "memory");
}

// Eight 32-bit columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_st8(uint32_t taddr, const uint32_t (&v)[8])
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"r"(taddr),
                 "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7])
                 : "memory");
}

__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ unsigned long long fadd2(unsigned long long a, unsigned long long b)
{
    unsigned long long d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

// Losses and derivatives of 16 entries that all lie inside the table and
// share one loss kind with parameters prm (Huber threshold) and lev (ordinal
// level count).  Quadratic entries run two at a time in packed FP32.  MISS:
// a NaN value marks a missing entry, which contributes nothing.
template <int KIND, bool MISS>
__device__ __forceinline__ void dn_block(const float (&u)[16], const float (&a)[16], float prm, float lev,
                                         float (&rr)[16], float &lsum)
{
    if constexpr (MISS && KIND == kLossQuad) {
        // a missing cell's NaN propagates into r and is replaced by 0
        const unsigned long long m1 = pk2(-1.f, -1.f);
        unsigned long long acc = pk2(0.f, 0.f);
#pragma unroll
        for (int w = 0; w < 16; w += 2) {
            float r0, r1;
            upk2(ffma2(pk2(a[w], a[w + 1]), m1, pk2(u[w], u[w + 1])), r0, r1);  // u - a
            r0 = a[w] == a[w] ? r0 : 0.f;
            r1 = a[w + 1] == a[w + 1] ? r1 : 0.f;
            const unsigned long long r = pk2(r0, r1);
            acc = ffma2(r, r, acc);
            upk2(fadd2(r, r), rr[w], rr[w + 1]);
        }
        float l0, l1;
        upk2(acc, l0, l1);
        lsum += l0 + l1;
    } else if constexpr (MISS) {
        // the losses tolerate a NaN value (no traps, no loops); its results are replaced by 0
#pragma unroll
        for (int w = 0; w < 16; ++w) {
            const bool v = a[w] == a[w];
            float L;
            const float d = loss_deriv_k<KIND, float>(u[w], a[w], prm, lev, L);
            lsum += v ? L : 0.f;
            rr[w] = v ? d : 0.f;
        }
    } else if constexpr (KIND == kLossQuad) {
        const unsigned long long m1 = pk2(-1.f, -1.f);
        unsigned long long acc = pk2(0.f, 0.f);
#pragma unroll
        for (int w = 0; w < 16; w += 2) {
            const unsigned long long r = ffma2(pk2(a[w], a[w + 1]), m1, pk2(u[w], u[w + 1]));  // u - a
            acc = ffma2(r, r, acc);
            upk2(fadd2(r, r), rr[w], rr[w + 1]);
        }
        float l0, l1;
        upk2(acc, l0, l1);
        lsum += l0 + l1;
    } else {
#pragma unroll
        for (int w = 0; w < 16; ++w) {
            float L;
            rr[w] = loss_deriv_k<KIND, float>(u[w], a[w], prm, lev, L);
            lsum += L;
        }
    }
}

// Any mix of kinds; entries outside the table (bit clear in `valid`) and
// missing entries (NaN) give 0.
// X-step: the entries are 16 columns (losses in lf); Y-step: one column (own).
template <bool XSTEP>
__device__ __forceinline__ void dn_block_any(const float (&u)[16], const float (&a)[16], const LossF *lf,
                                             LossF own, uint32_t valid, float (&rr)[16], float &lsum)
{
#pragma unroll
    for (int w = 0; w < 16; ++w) {
        const LossF sp = XSTEP ? lf[w] : own;
        float L;
        const float d = loss_deriv_kind<float>(__float_as_int(sp.x), u[w], a[w], sp.y, sp.z, L);
        const bool v = ((valid >> w) & 1u) && a[w] == a[w];
        lsum += v ? L : 0.f;
        rr[w] = v ? d : 0.f;
    }
}

// The X-step with per-column loss weights: 16 entries of 16 columns, each
// loss and derivative times its column's weight (wt: the weights of these
// columns; read only for entries inside the table).
__device__ __forceinline__ void dn_block_w(const float (&u)[16], const float (&a)[16], const LossF *lf,
                                           const float *__restrict__ wt, uint32_t valid, float (&rr)[16],
                                           float &lsum)
{
#pragma unroll
    for (int w = 0; w < 16; ++w) {
        const LossF sp = lf[w];
        float L;
        const float d = loss_deriv_kind<float>(__float_as_int(sp.x), u[w], a[w], sp.y, sp.z, L);
        const bool v = ((valid >> w) & 1u) && a[w] == a[w];
        const float c = v ? __ldg(wt + w) : 0.f;
        lsum += v ? c * L : 0.f;
        rr[w] = v ? c * d : 0.f;
    }
}

// One pass over a (128 own rows) x (range of chunks) block.  GRAD: partial
// gradient rows and partial losses; otherwise partial losses only.
// A tiles: X-step, two boxes of 32 columns x 128 own rows with the 128-byte
// swizzle (16-byte unit u of row r at u ^ (r % 8): conflict-free row reads);
// Y-step, one box of 128 own columns x 64 rows, unswizzled.
// Warps 0 .. 15 evaluate the entries; lane 0 of warp 16 issues the MMAs (and
// the copies of W's GEMM1 parts), lane 0 of warp 17 the other copies.  The
// MMA warp learns from barU[c % 2] (one arrival per evaluating warp) that U of
// chunk c has been read out of tensor memory and issues GEMM1 of chunk c + 2
// into that buffer at once; both learn from barE[c % 4] that the entries of
// chunk c are done (A stage read, R written): the copy warp refills the
// stages, the MMA warp issues GEMM2.  The evaluating warps never wait for each
// other inside the loop.  A warp can start chunk c only after every warp has
// read U of chunk c - 2, so after every warp has finished chunk c - 3: four
// barE barriers keep the arrivals of different chunks apart, and neither
// producer warp can fall two phases behind a barrier it waits on (the copy
// warp issues the A tile every chunk c needs after the wait for chunk c - 4
// at the latest; the MMA warp issues GEMM1 of c after its wait for c - 2).
// B16 (gradient passes of the BF16 form): GEMM2 takes the single product of
// R's and W's BF16 high parts (FP32 accumulation) and only R's high part is
// written to tensor memory; GEMM1, the losses, derivatives and objectives
// keep the six-product FP32 quality.
template <bool XSTEP, bool GRAD, int KP, bool MISS, bool B16 = false, bool WGT = false>
__global__ void __launch_bounds__(kDnThreads, 1)
dense_pass_kernel(const DenseArgs p, const __grid_constant__ CUtensorMap amap)
{
    using SM = DnSmem<XSTEP, GRAD, KP>;
    extern __shared__ __align__(1024) unsigned char dsm_dense[];
    __shared__ uint64_t barA[kDnMaxStages], barP[3], barL[3], barT[3], barG1[2], barG2[2], barU[2], barE[4];
    __shared__ uint32_t tslot;
    __shared__ double red[4][kDnRows];
    unsigned char *base = dsm_dense + ((1024 - (smem_u32(dsm_dense) & 1023)) & 1023);
    unsigned char *ast = base;                                   // A stage s at ast + s * a
    unsigned char *fx = base + (size_t)p.nA * SM::a;             // fixed buffers
    unsigned char *pkst = fx;                                    // pk stage s at pkst + s * 3 pk
    unsigned char *ptst = pkst + 9 * SM::pk;                     // pt stage s at ptst + s * 3 pt
    unsigned char *lsst = ptst + 9 * SM::pt;                     // loss table stage s at lsst + s * ls

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int quarter = warp & 3, grp = (warp >> 2) & 3;
    const int orow = quarter * 32 + lane;
    const DnItem item = p.items[blockIdx.x];
    const int64_t o0 = (int64_t)item.tile * kDnRows;
    const int64_t qb = item.q0;
    const int nq = item.nq;
    const int nA = p.nA;
    // kDnWarps: GEMM1 warp, kDnWarps + 1: copy warp, kDnWarps + 2: GEMM2 warp
    const bool producer = warp >= kDnWarps;
    // this thread's own row (X-step) or column (Y-step: quarter q of the tile
    // is the 32-column block blocks[4 tile + q]), and its partial slot
    int64_t own = o0 + orow;
    if (!XSTEP) {
        const int32_t b = producer ? -1 : p.blocks[4 * (int64_t)item.tile + quarter];
        own = b < 0 ? p.nown : 32 * (int64_t)b + lane;
    }
    const bool own_ok = !producer && own < p.nown;
    const int64_t slot = own_ok ? (int64_t)p.segchunk[own] + item.part : 0;
    const uint32_t lane_base = (uint32_t)(quarter * 32) << 16;
    const int tb = grp * 16;  // this warp's columns of a chunk

    if (warp == 0) tmem_alloc(&tslot, kDnTmem);
    if (tid == 0) {
        for (int s = 0; s < kDnMaxStages; ++s) mbar_init(&barA[s], 1);
        for (int s = 0; s < 3; ++s) mbar_init(&barP[s], 1);
        for (int s = 0; s < 3; ++s) mbar_init(&barL[s], 1);
        for (int s = 0; s < 3; ++s) mbar_init(&barT[s], 1);
        mbar_init(&barG1[0], 1);
        mbar_init(&barG1[1], 1);
        mbar_init(&barG2[0], 1);
        mbar_init(&barG2[1], 1);
        mbar_init(&barU[0], kDnWarps);
        mbar_init(&barU[1], kDnWarps);
        for (int s = 0; s < 4; ++s) mbar_init(&barE[s], kDnWarps);
    }
    // Y-step: this thread's column loss, and whether the warp shares one kind
    LossF myspec = make_float4(__int_as_float(kLossQuad), 0.f, 0.f, 0.f);
    if (!XSTEP && own_ok) myspec = p.lossf[own];
    // Y-step with column weights: this thread's column's weight
    const float wown = (!XSTEP && WGT && own_ok) ? p.wcol[own] : 1.f;
    int wkind = -1;
    if constexpr (!XSTEP) {
        const int kd = __float_as_int(myspec.x);
        const int k0 = __shfl_sync(0xffffffffu, kd, 0);
        wkind = __all_sync(0xffffffffu, kd == k0) ? k0 : -1;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t taddr = tslot;
    // own rows split in three into tensor memory (GEMM1's A operand, two BF16
    // values per column along k): warps 0 .. 3, one row per thread
    if (grp == 0 && !producer) {
#pragma unroll
        for (int c0 = 0; c0 < KP; c0 += 16) {
            uint32_t hv[8], mv[8], lv[8];
#pragma unroll
            for (int w = 0; w < 16; w += 2) {
                const float v0 = (own_ok && c0 + w < p.k) ? p.F[own * p.k + c0 + w] : 0.f;
                const float v1 = (own_ok && c0 + w + 1 < p.k) ? p.F[own * p.k + c0 + w + 1] : 0.f;
                __nv_bfloat16 h0, m0, l0, h1, m1, l1;
                split3(v0, h0, m0, l0);
                split3(v1, h1, m1, l1);
                hv[w / 2] = bf2_bits(__halves2bfloat162(h0, h1));
                mv[w / 2] = bf2_bits(__halves2bfloat162(m0, m1));
                lv[w / 2] = bf2_bits(__halves2bfloat162(l0, l1));
            }
            tmem_st8(taddr + lane_base + (uint32_t)(kDnColOwn + c0 / 2), hv);
            tmem_st8(taddr + lane_base + (uint32_t)(kDnColOwn + KP / 2 + c0 / 2), mv);
            tmem_st8(taddr + lane_base + (uint32_t)(kDnColOwn + KP + c0 / 2), lv);
        }
        tmem_wait_st();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();

    bool ok = true;
    float lacc = 0.f, lcomp = 0.f;
    // producer bookkeeping (warp kDnWarps, lane 0)
    int p_issued = 0, a_issued = 0, t_issued = 0, l_issued = 0, g1_issued = 0, g2_issued = 0;
    if (producer) {
        if (lane == 0) {
            auto issue_pack = [&](int64_t q) {  // GEMM1's W parts, stage q % 3
                const int s = (int)((q - qb) % 3);
                unsigned char *st = pkst + s * 3 * SM::pk;
                const int64_t t0 = q * kDnNT;
                mbar_expect_tx(&barP[s], (unsigned)(3 * SM::pk));
#pragma unroll
                for (int w = 0; w < 3; ++w)
                    bulk_g2s(st + w * SM::pk, p.pk + w * p.pack_part + t0 * KP, (unsigned)SM::pk, &barP[s]);
                ++p_issued;
            };
            auto issue_ls = [&](int64_t q) {  // X-step: the chunk's column losses, stage q % 3
                const int s = (int)((q - qb) % 3);
                const int64_t t0 = q * kDnNT;
                const int nv = (int)(p.nother - t0 < kDnNT ? p.nother - t0 : kDnNT);
                mbar_expect_tx(&barL[s], (unsigned)(nv * sizeof(LossF)));
                bulk_g2s(lsst + s * SM::ls, p.lossf + t0, (unsigned)(nv * sizeof(LossF)), &barL[s]);
                ++l_issued;
            };
            auto issue_pt = [&](int64_t q) {  // GEMM2's W parts, stage q % 3
                const int s = (int)((q - qb) % 3);
                unsigned char *st = ptst + s * 3 * SM::pt;
                mbar_expect_tx(&barT[s], (unsigned)(3 * SM::pt));
#pragma unroll
                for (int w = 0; w < 3; ++w)
                    bulk_g2s(st + w * SM::pt, p.pt + w * p.pack_part + q * KP * kDnNT, (unsigned)SM::pt, &barT[s]);
                ++t_issued;
            };
            // Y-step: the tile's 32-column blocks (box q of a stage holds block q)
            int32_t blk[4] = {-1, -1, -1, -1};
            unsigned nblk = 0;
            if constexpr (!XSTEP) {
                for (int qd = 0; qd < 4; ++qd) {
                    blk[qd] = p.blocks[4 * (int64_t)item.tile + qd];
                    nblk += blk[qd] >= 0 ? 1u : 0u;
                }
            }
            auto issue_a = [&](int64_t q) {  // the A tile, stage q % nA (out-of-range elements read as 0)
                const int s = (int)((q - qb) % nA);
                unsigned char *dst = ast + s * SM::a;
                const int t0 = (int)(q * kDnNT);
                if constexpr (XSTEP) {
                    mbar_expect_tx(&barA[s], (unsigned)SM::a);
                    tma_load_2d(dst, &amap, t0, (int)o0, &barA[s]);
                    tma_load_2d(dst + SM::a / 2, &amap, t0 + 32, (int)o0, &barA[s]);
                } else {
                    mbar_expect_tx(&barA[s], nblk * (unsigned)(SM::a / 4));
                    for (int qd = 0; qd < 4; ++qd)
                        if (blk[qd] >= 0) tma_load_2d(dst + qd * (SM::a / 4), &amap, 32 * blk[qd], t0, &barA[s]);
                }
                ++a_issued;
            };
            // GEMM1 of chunk q into accumulator buffer (q - qb) % 2, once its W parts are in
            auto issue_gemm1 = [&](int64_t q) -> bool {
                const int c = (int)(q - qb);
                const int s = c % 3, b = c & 1;
                if (!mbar_wait_bounded(&barP[s], (unsigned)(c / 3) & 1u)) return false;
                tc_fence_after();
                const uint32_t idesc = umma_idesc_bf16(kDnRows, kDnNT);
                const unsigned char *w = pkst + s * 3 * SM::pk;
                constexpr uint32_t RB = 2 * KP;  // bytes per W row; a K step of 16 is 32 bytes, 8 own columns
                // (own part, W part), smallest products first; hi . hi last
                const int pa[6] = {1, 0, 2, 0, 1, 0};
                const int pb[6] = {1, 2, 0, 1, 0, 0};
#pragma unroll
                for (int pr = 0; pr < 6; ++pr)
#pragma unroll
                    for (int ks = 0; ks < KP / 16; ++ks)
                        umma_bf16_ta(taddr + (uint32_t)(b * kDnNT),
                                     taddr + (uint32_t)(kDnColOwn + pa[pr] * (KP / 2) + ks * 8),
                                     umma_desc_sw(w + pb[pr] * SM::pk + ks * 32, RB), idesc, pr > 0 || ks > 0);
                umma_commit(&barG1[b]);
                ++g1_issued;
                return true;
            };
            // GEMM2 of chunk q: G += R W, R from tensor memory
            auto issue_gemm2 = [&](int64_t q) -> bool {
                const int c = (int)(q - qb);
                const int s = c % 3, rb = c & 1;
                if (!mbar_wait_bounded(&barT[s], (unsigned)(c / 3) & 1u)) return false;
                tc_fence_after();
                const uint32_t idesc = umma_idesc_bf16(kDnRows, KP);
                const unsigned char *wt = ptst + s * 3 * SM::pt;
                // (R part, W part), smallest products first; a K = 16 step of R is 8 columns
                const int pa[6] = {1, 0, 2, 0, 1, 0};
                const int pb[6] = {1, 2, 0, 1, 0, 0};
                constexpr int P0 = B16 ? 5 : 0;  // the BF16 form: hi . hi only
#pragma unroll
                for (int pr = P0; pr < 6; ++pr)
#pragma unroll
                    for (int ks = 0; ks < kDnNT / 16; ++ks)
                        umma_bf16_ta(taddr + kDnColG, taddr + (uint32_t)(kDnColR + rb * 96 + pa[pr] * 32 + ks * 8),
                                     umma_desc_sw(wt + pb[pr] * SM::pt + ks * 32, 2 * kDnNT), idesc,
                                     c > 0 || pr > P0 || ks > 0);
                umma_commit(&barG2[rb]);
                ++g2_issued;
                return true;
            };
            if (warp == kDnWarps) {
                // GEMM1 warp: W's GEMM1 parts and GEMM1
                for (int s = 0; s < 3 && s < nq; ++s) issue_pack(qb + s);
                ok = issue_gemm1(qb);
                if (ok && nq > 1) ok = issue_gemm1(qb + 1);
                for (int it = 0; ok && it < nq; ++it) {
                    const int64_t q = qb + it;
                    // U of chunk q has been read (so GEMM1 of q is done): its
                    // accumulator buffer takes chunk q + 2, its W stage chunk q + 3
                    if (!mbar_wait_bounded(&barU[it & 1], (unsigned)(it >> 1) & 1u)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    if (it + 3 < nq) issue_pack(q + 3);
                    if (it + 2 < nq && !issue_gemm1(q + 2)) {
                        ok = false;
                        break;
                    }
                }
            } else if (warp == kDnWarps + 2) {
                // GEMM2 warp (gradient passes): G += R W once R of chunk q is written
                for (int it = 0; GRAD && it < nq; ++it) {
                    if (!mbar_wait_bounded(&barE[it & 3], (unsigned)(it >> 2) & 1u)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    if (!issue_gemm2(qb + it)) {
                        ok = false;
                        break;
                    }
                }
            } else {
                // copy warp: A tiles, loss tables and W's GEMM2 parts
                for (int s = 0; s < nA && s < nq; ++s) issue_a(qb + s);
                if (XSTEP)
                    for (int s = 0; s < 3 && s < nq; ++s) issue_ls(qb + s);
                if (GRAD) {
                    issue_pt(qb);
                    if (nq > 1) issue_pt(qb + 1);
                }
                for (int it = 0; it < nq; ++it) {
                    const int64_t q = qb + it;
                    // the entries of chunk q are done: its A stage and loss-table
                    // stage are free, and (the warps having waited for GEMM2 of
                    // q - 2 before writing R of q) so is the GEMM2 stage of q - 2
                    if (!mbar_wait_bounded(&barE[it & 3], (unsigned)(it >> 2) & 1u)) {
                        ok = false;
                        break;
                    }
                    if (it + nA < nq) issue_a(q + nA);
                    if (XSTEP && it + 3 < nq) issue_ls(q + 3);
                    if (GRAD && it >= 1 && it + 1 < nq) issue_pt(q + 1);
                }
            }
        }
    } else {
        for (int it = 0; it < nq; ++it) {
            const int64_t q = qb + it;
            const int b = it & 1;
            const int sA = it % nA;
            ok = ok && mbar_wait_bounded(&barG1[b], (unsigned)(it >> 1) & 1u);
            if (XSTEP) ok = ok && mbar_wait_bounded(&barL[it % 3], (unsigned)(it / 3) & 1u);  // loss table
            ok = ok && mbar_wait_bounded(&barA[sA], (unsigned)(it / nA) & 1u);
            tc_fence_after();
            ok = __all_sync(0xffffffffu, ok);  // tcgen05.ld / st below are warp-collective
            if (!ok) break;
            float lsum = 0.f;
            float rr[16];
            {
                const unsigned char *as = ast + sA * SM::a;
                const int64_t t0 = q * kDnNT;
                float u[16], a[16];
                tmem_ld16(taddr + lane_base + (uint32_t)(b * kDnNT + tb), u);
                // U of this chunk is in registers: its buffer may take the next GEMM1
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&barU[b]);
                if constexpr (XSTEP) {
                    // box tb / 32, row orow: 16-byte units (tb % 32) / 4 .. + 3, swizzled
                    const unsigned char *row = as + (tb >> 5) * (SM::a / 2) + orow * 128;
#pragma unroll
                    for (int w = 0; w < 4; ++w) {
                        const float4 v =
                            *reinterpret_cast<const float4 *>(row + ((((tb & 31) >> 2) + w) ^ (orow & 7)) * 16);
                        a[4 * w] = v.x;
                        a[4 * w + 1] = v.y;
                        a[4 * w + 2] = v.z;
                        a[4 * w + 3] = v.w;
                    }
                } else {
                    // box `quarter`: 64 chunk rows x 32 columns
                    const float *af = reinterpret_cast<const float *>(as) + quarter * (kDnNT * 32);
#pragma unroll
                    for (int w = 0; w < 16; ++w) a[w] = af[(tb + w) * 32 + lane];
                }
                const int64_t nv = p.nother - t0 - tb;  // valid columns from tb on
                const uint32_t valid = !own_ok ? 0u : (nv >= 16 ? 0xffffu : (nv <= 0 ? 0u : (1u << nv) - 1u));
                const LossF *lf = reinterpret_cast<const LossF *>(lsst + (it % 3) * SM::ls) + tb;
                // the kind (and parameters) the 16 entries share, -1 if they do not:
                // X-step, kept in the w of each column's loss; Y-step, the warp's columns
                int kind = wkind;
                float prm = myspec.y, lev = myspec.z;
                if constexpr (XSTEP) {
                    const LossF l0 = lf[0];
                    kind = nv > 0 ? __float_as_int(l0.w) : -1;
                    prm = l0.y;
                    lev = l0.z;
                }
                if constexpr (XSTEP && WGT) {
                    dn_block_w(u, a, lf, p.wcol + t0 + tb, valid, rr, lsum);
                } else if (__all_sync(0xffffffffu, valid == 0xffffu)) {
                    switch (kind) {
                    case kLossQuad: dn_block<kLossQuad, MISS>(u, a, prm, lev, rr, lsum); break;
                    case kLossHuber: dn_block<kLossHuber, MISS>(u, a, prm, lev, rr, lsum); break;
                    case kLossHinge: dn_block<kLossHinge, MISS>(u, a, prm, lev, rr, lsum); break;
                    case kLossLogistic: dn_block<kLossLogistic, MISS>(u, a, prm, lev, rr, lsum); break;
                    case kLossOrdinal: dn_block<kLossOrdinal, MISS>(u, a, prm, lev, rr, lsum); break;
                    default: dn_block_any<XSTEP>(u, a, lf, myspec, valid, rr, lsum); break;
                    }
                } else {
                    dn_block_any<XSTEP>(u, a, lf, myspec, valid, rr, lsum);
                }
                if constexpr (!XSTEP && WGT) {  // the column's weight on its 16 entries
                    lsum *= wown;
#pragma unroll
                    for (int w = 0; w < 16; ++w) rr[w] *= wown;
                }
            }
            // compensated FP32 running sum of the chunk sums
            {
                const float y = lsum - lcomp;
                const float t = lacc + y;
                lcomp = (t - lacc) - y;
                lacc = t;
            }
            if constexpr (GRAD) {
                // R of the previous chunk is no longer read once its GEMM2 is done
                // R buffer it % 2 is free once GEMM2 of it - 2 is done
                if (it > 1) ok = mbar_wait_bounded(&barG2[b], (unsigned)((it - 2) >> 1) & 1u);
                tc_fence_after();
                ok = __all_sync(0xffffffffu, ok);
                if (!ok) break;
                uint32_t hi[8], mi[8], lo[8];
                const unsigned long long m1 = pk2(-1.f, -1.f);
                if constexpr (B16) {
#pragma unroll
                    for (int w = 0; w < 16; w += 2) hi[w / 2] = bf2_bits(__floats2bfloat162_rn(rr[w], rr[w + 1]));
                } else {
#pragma unroll
                for (int w = 0; w < 16; w += 2) {
                    // r = hi + mid + lo, each remainder exact in FP32
                    const __nv_bfloat162 h2 = __floats2bfloat162_rn(rr[w], rr[w + 1]);
                    const float2 hf = __bfloat1622float2(h2);
                    const unsigned long long r1 = ffma2(pk2(hf.x, hf.y), m1, pk2(rr[w], rr[w + 1]));
                    float a0, a1;
                    upk2(r1, a0, a1);
                    const __nv_bfloat162 m2 = __floats2bfloat162_rn(a0, a1);
                    const float2 mf = __bfloat1622float2(m2);
                    float b0, b1;
                    upk2(ffma2(pk2(mf.x, mf.y), m1, r1), b0, b1);
                    hi[w / 2] = bf2_bits(h2);
                    mi[w / 2] = bf2_bits(m2);
                    lo[w / 2] = bf2_bits(__floats2bfloat162_rn(b0, b1));
                }
                }
                const uint32_t rcol = kDnColR + (uint32_t)(b * 96 + tb / 2);
                tmem_st8(taddr + lane_base + rcol, hi);
                if constexpr (!B16) {
                    tmem_st8(taddr + lane_base + rcol + 32, mi);
                    tmem_st8(taddr + lane_base + rcol + 64, lo);
                }
                tmem_wait_st();
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&barE[it & 3]);
        }
        if (GRAD && ok) {
            ok = mbar_wait_bounded(&barG2[(nq - 1) & 1], (unsigned)((nq - 1) >> 1) & 1u);
            if (ok && nq > 1) ok = mbar_wait_bounded(&barG2[nq & 1], (unsigned)((nq - 2) >> 1) & 1u);
            tc_fence_after();
            ok = __all_sync(0xffffffffu, ok);
        }
    }
    const bool fail = __syncthreads_or(!ok) != 0;
    if (!fail && !producer) {
        red[grp][orow] = (double)lacc - (double)lcomp;
        if (GRAD && grp == 0) {
            float *g = p.part_grad + slot * p.k;
#pragma unroll
            for (int bb = 0; bb < KP / 16; ++bb) {
                float v[16];
                tmem_ld16(taddr + lane_base + (uint32_t)(kDnColG + 16 * bb), v);
                if (own_ok) {
#pragma unroll
                    for (int w = 0; w < 16; ++w)
                        if (16 * bb + w < p.k) g[16 * bb + w] = v[w];
                }
            }
        }
    }
    __syncthreads();
    if (!fail && !producer && grp == 0 && own_ok)
        p.part_loss[slot] = red[0][orow] + red[1][orow] + red[2][orow] + red[3][orow];
    if (fail && producer && lane == 0) {  // each producer warp drains what it issued
        atomicOr(p.err, 1);
        // wait (bounded) for the last copy into each stage and the last MMA
        // batches: every earlier one completed before a later one was issued
        for (int c = p_issued - 3 > 0 ? p_issued - 3 : 0; c < p_issued; ++c)
            mbar_wait_bounded(&barP[c % 3], (unsigned)(c / 3) & 1u);
        for (int c = l_issued - 3 > 0 ? l_issued - 3 : 0; c < l_issued; ++c)
            mbar_wait_bounded(&barL[c % 3], (unsigned)(c / 3) & 1u);
        for (int c = a_issued - nA > 0 ? a_issued - nA : 0; c < a_issued; ++c)
            mbar_wait_bounded(&barA[c % nA], (unsigned)(c / nA) & 1u);
        for (int c = t_issued - 3 > 0 ? t_issued - 3 : 0; c < t_issued; ++c)
            mbar_wait_bounded(&barT[c % 3], (unsigned)(c / 3) & 1u);
        for (int c = g1_issued - 2 > 0 ? g1_issued - 2 : 0; c < g1_issued; ++c)
            mbar_wait_bounded(&barG1[c & 1], (unsigned)(c >> 1) & 1u);
        for (int c = g2_issued - 2 > 0 ? g2_issued - 2 : 0; c < g2_issued; ++c)
            mbar_wait_bounded(&barG2[c & 1], (unsigned)(c >> 1) & 1u);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(taddr, kDnTmem);
    }
}

// The other factor W (rows x k, FP32) split x = hi + mid + lo into both packed
// layouts, swizzled K-major (sw_off): over k (row r, coordinate c of part w at
// byte w part 2 + sw_off(r, c, 2 KP)), all three parts; and, per chunk of
// kDnNT rows, over the chunk rows (chunk q, element (c, t) of part w at byte
// w part 2 + q KP kDnNT 2 + sw_off(c, t, 2 kDnNT)), all three parts.  Rows
// from `rows` to rows_pad and coordinates from k to KP are zero.
template <int KP>
__global__ void __launch_bounds__(256) dense_pack_kernel(const float *__restrict__ W, int64_t rows, int k,
                                                         int64_t part, __nv_bfloat16 *__restrict__ pk,
                                                         __nv_bfloat16 *__restrict__ pt)
{
    // one CTA per chunk of kDnNT rows, staged in shared memory; every store
    // is a 16-byte unit of eight BF16 values
    __shared__ float tile[kDnNT][KP + 1];
    const int64_t q = blockIdx.x, r0 = q * kDnNT;
    for (int i = threadIdx.x; i < kDnNT * KP; i += blockDim.x) {
        const int r = i / KP, c = i - r * KP;
        tile[r][c] = (r0 + r < rows && c < k) ? W[(r0 + r) * k + c] : 0.f;
    }
    __syncthreads();
    auto pack8 = [](const float (&v)[8], uint4 &h, uint4 &m, uint4 &l) {
        uint32_t hv[4], mv[4], lv[4];
#pragma unroll
        for (int w = 0; w < 8; w += 2) {
            __nv_bfloat16 h0, m0, l0, h1, m1, l1;
            split3(v[w], h0, m0, l0);
            split3(v[w + 1], h1, m1, l1);
            hv[w / 2] = bf2_bits(__halves2bfloat162(h0, h1));
            mv[w / 2] = bf2_bits(__halves2bfloat162(m0, m1));
            lv[w / 2] = bf2_bits(__halves2bfloat162(l0, l1));
        }
        h = make_uint4(hv[0], hv[1], hv[2], hv[3]);
        m = make_uint4(mv[0], mv[1], mv[2], mv[3]);
        l = make_uint4(lv[0], lv[1], lv[2], lv[3]);
    };
    for (int i = threadIdx.x; i < kDnNT * (KP / 8); i += blockDim.x) {
        // K-major over k: row r, coordinates 8 g .. 8 g + 7
        const int r = i / (KP / 8), g = i - r * (KP / 8);
        float v[8];
#pragma unroll
        for (int w = 0; w < 8; ++w) v[w] = tile[r][8 * g + w];
        uint4 h, m, l;
        pack8(v, h, m, l);
        const int64_t o = r0 * KP + sw_off((uint32_t)r, (uint32_t)(8 * g), 2 * KP) / 2;
        *reinterpret_cast<uint4 *>(pk + o) = h;
        *reinterpret_cast<uint4 *>(pk + part + o) = m;
        *reinterpret_cast<uint4 *>(pk + 2 * part + o) = l;
        // K-major over the chunk rows: coordinate c (= i / 8 here), rows 8 t .. 8 t + 7
        const int c = i / (kDnNT / 8), tg = i - c * (kDnNT / 8);
#pragma unroll
        for (int w = 0; w < 8; ++w) v[w] = tile[8 * tg + w][c];
        pack8(v, h, m, l);
        const int64_t ot = q * KP * kDnNT + sw_off((uint32_t)c, (uint32_t)(8 * tg), 2 * kDnNT) / 2;
        *reinterpret_cast<uint4 *>(pt + ot) = h;
        *reinterpret_cast<uint4 *>(pt + part + ot) = m;
        *reinterpret_cast<uint4 *>(pt + 2 * part + ot) = l;
    }
}

// Values outside a column loss's domain (flag 64) or not finite (flag 8).
static __global__ void dense_validate_kernel(const float *__restrict__ A, int64_t lda, int64_t m, int64_t n,
                                             const LossSpec *__restrict__ loss, int *__restrict__ flag)
{
    int f = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m * n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = i / n, j = i - r * n;
        const float a = A[r * lda + j];
        if (!isfinite(a)) {
            f |= 8;
            continue;
        }
        const LossSpec s = loss[j];
        if ((s.kind == kLossHinge || s.kind == kLossLogistic) && a != 1.f && a != -1.f) f |= 64;
        if (s.kind == kLossOrdinal && (a != floorf(a) || a < 1.f || a > (float)s.levels)) f |= 64;
    }
    if (f) atomicOr(flag, f);
}

// Omega's values (CSR) into a dense table that holds NaN everywhere else:
// one warp per row writes the row's NaN fill, then its entries.
// Rows 0 .. m - 1 of rowptr (which may point into the middle of a pointer
// array: entry indices are absolute) into rows of A; a column index outside
// [0, n) is skipped, so rows whose checks are still running may be scattered.
static __global__ void dense_scatter_kernel(const int32_t *__restrict__ rowptr, const int32_t *__restrict__ colidx,
                                            const float *__restrict__ val, int64_t m, int64_t n, int64_t lda,
                                            float *__restrict__ A)
{
    const int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (i >= m) return;
    float *row = A + i * lda;
    for (int64_t c = threadIdx.x & 31; c < lda; c += 32) row[c] = __int_as_float(0x7fffffff);
    __syncwarp();
    for (int e = rowptr[i] + (threadIdx.x & 31); e < rowptr[i + 1]; e += 32) {
        const int32_t j = colidx[e];
        if (j >= 0 && j < n) row[j] = val[e];
    }
}

static __global__ void dense_alpha_kernel(float *__restrict__ alpha, int64_t nseg, float value)
{
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s < nseg) alpha[s] = value;
}

// Segment s (row s % 128 of own tile s / 128) -> its first partial slot;
// tb holds per tile {first slot, parts}; sc[nseg] = total slots.
static __global__ void dense_segchunk_kernel(int32_t *__restrict__ sc, int64_t nseg, const int64_t *__restrict__ tb,
                                             int64_t total)
{
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s < nseg) {
        const int64_t t = s / kDnRows;
        sc[s] = (int32_t)(tb[2 * t] + (s - t * kDnRows) * tb[2 * t + 1]);
    } else if (s == nseg) {
        sc[s] = (int32_t)total;
    }
}

namespace {

int dense_width(int k)
{
    for (int K : {16, 32, 64})
        if (k <= K) return K;
    return 0;
}

template <bool XSTEP, bool GRAD, int KP, bool MISS, bool B16, bool WGT>
cudaError_t launch_dense_kp(glrm_s *h, const DenseArgs &a, int nA, unsigned items)
{
    const size_t smem = DnSmem<XSTEP, GRAD, KP>::bytes(nA);
    cudaError_t e = cudaFuncSetAttribute(dense_pass_kernel<XSTEP, GRAD, KP, MISS, B16, WGT>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const CUtensorMap *map = reinterpret_cast<const CUtensorMap *>(XSTEP ? h->dn.tmap_x : h->dn.tmap_y);
    dense_pass_kernel<XSTEP, GRAD, KP, MISS, B16, WGT><<<items, kDnThreads, smem, h->stream>>>(a, *map);
    h->launches += 1;
    return cudaGetLastError();
}

// A stages that fit next to the fixed buffers and the kernel's static shared
// memory (at most kDnMaxStages; fewer than 2 is refused by the caller).
template <bool XSTEP, bool GRAD, int KP, bool MISS, bool B16, bool WGT>
int stages_kp(int optin)
{
    using SM = DnSmem<XSTEP, GRAD, KP>;
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, dense_pass_kernel<XSTEP, GRAD, KP, MISS, B16, WGT>) != cudaSuccess) return 0;
    if ((size_t)optin < fa.sharedSizeBytes) return 0;
    const size_t room = (size_t)optin - fa.sharedSizeBytes;
    if (room < SM::bytes(0)) return 0;
    const int n = (int)((room - SM::bytes(0)) / SM::a);
    return n < kDnMaxStages ? n : kDnMaxStages;
}

template <bool XSTEP, bool GRAD>
cudaError_t launch_dense(glrm_s *h, const float *F, float *part_grad, double *part_loss)
{
    const Dense &d = h->dn;
    DenseArgs a;
    a.nown = XSTEP ? h->m : h->n;
    a.nother = XSTEP ? h->n : h->m;
    a.k = h->k;
    a.F = F;
    a.pk = d.pk;
    a.pt = d.pt;
    a.pack_part = d.pack_part;
    a.lossf = d.lossf;
    a.wcol = (const float *)h->lscale;
    a.items = XSTEP ? d.items_x : d.items_y;
    a.blocks = XSTEP ? nullptr : d.blocks_y;
    a.segchunk = XSTEP ? d.segchunk_x : d.segchunk_y;
    a.part_grad = part_grad;
    a.part_loss = part_loss;
    a.err = h->s.err;
    const unsigned tiles = (unsigned)(XSTEP ? d.nitems_x : d.nitems_y);
    int optin = 0;
    cudaError_t e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device);
    if (e != cudaSuccess) return e;
    // the BF16 form's gradient passes take the single-product GEMM2
    const bool b16 = GRAD && h->prec == GLRM_BF16;
#define GLRM_DENSE_GO(KK, MS, B, WG)                                               \
    {                                                                              \
        a.nA = stages_kp<XSTEP, GRAD, KK, MS, B, WG>(optin);                       \
        if (a.nA < 2) return cudaErrorInvalidConfiguration;                        \
        return launch_dense_kp<XSTEP, GRAD, KK, MS, B, WG>(h, a, a.nA, tiles);     \
    }
    // weighted losses (FP32 models only) take the variant that also tests for
    // missing cells, whatever the table: the test never fires on a full one
#define GLRM_DENSE_CASE(KK)                                                        \
    if (d.KP == KK) {                                                              \
        if (a.wcol) GLRM_DENSE_GO(KK, true, false, true)                           \
        if constexpr (GRAD) {                                                      \
            if (b16) {                                                             \
                if (d.missing) GLRM_DENSE_GO(KK, true, true, false)                \
                GLRM_DENSE_GO(KK, false, true, false)                              \
            }                                                                      \
        }                                                                          \
        if (d.missing) GLRM_DENSE_GO(KK, true, false, false)                       \
        GLRM_DENSE_GO(KK, false, false, false)                                     \
    }
    GLRM_DENSE_CASE(16)
    GLRM_DENSE_CASE(32)
    GLRM_DENSE_CASE(64)
#undef GLRM_DENSE_CASE
#undef GLRM_DENSE_GO
    return cudaErrorInvalidValue;
}

cudaError_t dense_pack(glrm_s *h, const float *W, int64_t rows)
{
    const Dense &d = h->dn;
    const int64_t rows_pad = (rows + kDnRows - 1) / kDnRows * kDnRows;
    tmark(h, "dense_pack");
    const unsigned nchunks = (unsigned)(rows_pad / kDnNT);
    if (d.KP == 16)
        dense_pack_kernel<16><<<nchunks, 256, 0, h->stream>>>(W, rows, h->k, d.pack_part, d.pk, d.pt);
    else if (d.KP == 32)
        dense_pack_kernel<32><<<nchunks, 256, 0, h->stream>>>(W, rows, h->k, d.pack_part, d.pk, d.pt);
    else
        dense_pack_kernel<64><<<nchunks, 256, 0, h->stream>>>(W, rows, h->k, d.pack_part, d.pk, d.pt);
    h->launches += 1;
    return cudaGetLastError();
}

// Relative cost of evaluating one entry of a 16- or 32-wide group of columns
// (counted instructions of the loss blocks plus the per-entry load and sum
// work): a group whose columns share one kind takes that kind's block; a
// group that mixes kinds, or runs past the table, takes the per-entry switch
// and pays for every kind present (its lanes diverge).
double group_cost(const std::vector<LossSpec> &loss, int64_t j0, int width)
{
    auto extra = [](int kind) -> double {
        switch (kind) {
        case kLossQuad: return 2;
        case kLossHuber: return 8;
        case kLossHinge: return 4;
        case kLossLogistic: return 22;
        case kLossL1: return 5;
        case kLossQuantile: return 6;
        default: return 16;
        }
    };
    const int64_t n = (int64_t)loss.size();
    bool uniform = j0 + width <= n;
    unsigned seen = 0;
    for (int64_t j = j0; j < j0 + width; ++j) {
        const int kd = j < n ? loss[j].kind : kLossQuad;  // lanes past the table run the quadratic block
        if (j < n && kd != loss[j0].kind) uniform = false;
        seen |= 1u << kd;
    }
    if (uniform) return 6 + extra(loss[j0].kind);
    double c = 10;
    for (int kd = 0; kd < kLossKinds; ++kd)
        if (seen >> kd & 1u) c += extra(kd);
    return c;
}

// Work items of one pass: own tile t (rows t * 128 ..) takes parts_t items,
// each a contiguous range of the other dimension's 64-wide chunks.  Entry
// costs vary with the column losses: along the chunks in the X-step (the
// columns are the other dimension), between the tiles in the Y-step.
//
// Plan: parts sized so items carry about equal cost, about four items per SM
// (no fewer than tiles, none empty), launched in the order of the middle of
// their chunk range (items reading the same chunks of the other factor run
// close together).  One CTA is resident per SM, and a finished CTA's SM takes
// the next item in launch order, so the pass ends when the last SM does:
// the per-item cost target and the number of items split in two (halves
// launched after the rest, to fill the last wave) are chosen by simulating
// that schedule, with each item paying a fixed pipeline fill and drain of
// about 1.3 average chunks on top of its entries.
struct PlanRange {
    int64_t tile, q0, q1;
    bool tail;  // a half of a split item: launched after the others
};

double list_schedule_end(const std::vector<double> &t, int slots)
{
    std::priority_queue<double, std::vector<double>, std::greater<double>> free_at;
    for (int i = 0; i < slots; ++i) free_at.push(0.0);
    double end = 0;
    for (double c : t) {
        const double f = free_at.top() + c;
        free_at.pop();
        free_at.push(f);
        end = std::max(end, f);
    }
    return end;
}

ItemPlan plan_items(int64_t nown, int64_t nother, int sms, const std::vector<double> &tile_cost,
                    const std::vector<double> &chunk_cost)
{
    const int64_t tiles = (nown + kDnRows - 1) / kDnRows;
    const int64_t nch = std::max<int64_t>(1, (nother + kDnNT - 1) / kDnNT);
    std::vector<double> pre(nch + 1, 0.0);
    for (int64_t q = 0; q < nch; ++q) pre[q + 1] = pre[q] + chunk_cost[q];
    double total = 0;
    for (int64_t t = 0; t < tiles; ++t) total += tile_cost[t] * pre[nch];
    const double fill = 1.3 * total / (double)(tiles * nch);
    auto mid = [](const PlanRange &r) { return r.q0 + r.q1; };
    auto order = [&](std::vector<PlanRange> &v) {
        std::stable_sort(v.begin(), v.end(), [&](const PlanRange &a, const PlanRange &b) {
            return a.tail != b.tail ? !a.tail : mid(a) < mid(b);
        });
    };
    // the tile's chunks in np ranges of about equal cost, at least one chunk each
    auto build = [&](double per_item) {
        std::vector<PlanRange> v;
        for (int64_t t = 0; t < tiles; ++t) {
            int64_t np = (int64_t)std::llround(tile_cost[t] * pre[nch] / per_item);
            np = std::max<int64_t>(1, std::min<int64_t>(np, nch));
            int64_t q = 0;
            for (int64_t i = 0; i < np; ++i) {
                int64_t e = nch;
                if (i + 1 < np) {
                    const double goal = pre[nch] * (double)(i + 1) / (double)np;
                    e = std::lower_bound(pre.begin(), pre.end(), goal) - pre.begin();
                    e = std::max<int64_t>(e, q + 1);
                    e = std::min<int64_t>(e, nch - (np - 1 - i));
                }
                v.push_back({t, q, e, false});
                q = e;
            }
        }
        order(v);
        return v;
    };
    // the last `s` items of the launch order split in two at the middle of their cost
    auto split = [&](const std::vector<PlanRange> &v, int64_t s) {
        std::vector<PlanRange> w(v.begin(), v.end() - s);
        for (auto r = v.end() - s; r != v.end(); ++r) {
            if (r->q1 - r->q0 < 2) {
                w.push_back(*r);
                continue;
            }
            const double goal = 0.5 * (pre[r->q0] + pre[r->q1]);
            int64_t e = std::lower_bound(pre.begin() + r->q0, pre.begin() + r->q1, goal) - pre.begin();
            e = std::max<int64_t>(r->q0 + 1, std::min<int64_t>(e, r->q1 - 1));
            w.push_back({r->tile, r->q0, e, true});
            w.push_back({r->tile, e, r->q1, true});
        }
        order(w);
        return w;
    };
    auto finish_time = [&](const std::vector<PlanRange> &v) {
        std::vector<double> t(v.size());
        for (size_t i = 0; i < v.size(); ++i) t[i] = tile_cost[v[i].tile] * (pre[v[i].q1] - pre[v[i].q0]) + fill;
        return list_schedule_end(t, sms);
    };
    const double per0 = total / (double)std::max<int64_t>(tiles, 4LL * sms);
    std::vector<PlanRange> best = build(per0);
    if ((int64_t)best.size() <= 64LL * sms) {  // beyond that the last wave is a small share
        double best_end = finish_time(best);
        for (int f = 0; f <= 10; ++f) {
            const std::vector<PlanRange> v = build(per0 * (1.0 + 0.03 * f));
            const int64_t n = (int64_t)v.size();
            for (int g = 0; g <= 24; ++g) {
                const std::vector<PlanRange> w = g ? split(v, n * g / 24) : v;
                const double end = finish_time(w);
                if (end < best_end * (1.0 - 1e-9)) {
                    best_end = end;
                    best = w;
                }
            }
        }
    }
    // parts per tile in chunk order, slots, items in launch order
    ItemPlan pl;
    pl.tiles.assign(2 * tiles, 0);
    std::vector<std::vector<size_t>> by_tile(tiles);
    for (size_t i = 0; i < best.size(); ++i) by_tile[best[i].tile].push_back(i);
    pl.items.resize(best.size());
    for (int64_t t = 0; t < tiles; ++t) {
        std::vector<size_t> &ix = by_tile[t];
        std::sort(ix.begin(), ix.end(), [&](size_t a, size_t b) { return best[a].q0 < best[b].q0; });
        const int64_t rows = std::min<int64_t>(kDnRows, nown - t * kDnRows);
        pl.tiles[2 * t] = pl.slots;
        pl.tiles[2 * t + 1] = (int64_t)ix.size();
        for (size_t p = 0; p < ix.size(); ++p) {
            const PlanRange &r = best[ix[p]];
            DnItem it{};
            it.tile = (int32_t)t;
            it.part = (int32_t)p;
            it.parts = (int32_t)ix.size();
            it.q0 = (int32_t)r.q0;
            it.nq = (int32_t)(r.q1 - r.q0);
            it.base = pl.slots;
            pl.items[ix[p]] = it;
        }
        pl.slots += rows * (int64_t)ix.size();
    }
    return pl;
}

}  // namespace

bool dense_supported(int k) { return dense_width(k) != 0; }

void dense_free(glrm_s *h)
{
    Dense &d = h->dn;
    for (void *p : {(void *)d.A, (void *)d.pk, (void *)d.pt, (void *)d.lossf, (void *)d.segchunk_x,
                    (void *)d.segchunk_y, (void *)d.items_x, (void *)d.items_y, (void *)d.blocks_y})
        if (p) cudaFreeAsync(p, h->stream);
    d = Dense();
}

namespace {

using EncodeTiled = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                 const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// Tensor maps of A (FP32, dims n x m, row pitch lda): X-step boxes of 32
// columns x 128 rows with the 128-byte swizzle, Y-step boxes of 32 columns x
// 64 rows.  Out-of-range elements load as zero.
cudaError_t encode_maps(glrm_s *h)
{
    static EncodeTiled encode = nullptr;
    if (!encode) {
        cudaDriverEntryPointQueryResult q;
        void *fn = nullptr;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
        if (e != cudaSuccess) return e;
        if (q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
        encode = reinterpret_cast<EncodeTiled>(fn);
    }
    Dense &d = h->dn;
    const cuuint64_t dims[2] = {(cuuint64_t)h->n, (cuuint64_t)h->m};
    const cuuint64_t strides[1] = {(cuuint64_t)d.lda * sizeof(float)};
    const cuuint32_t estr[2] = {1, 1};
    const cuuint32_t box_x[2] = {32, (cuuint32_t)kDnRows};
    const cuuint32_t box_y[2] = {32, (cuuint32_t)kDnNT};
    CUresult r = encode(reinterpret_cast<CUtensorMap *>(d.tmap_x), CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, d.A, dims,
                        strides, box_x, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
    r = encode(reinterpret_cast<CUtensorMap *>(d.tmap_y), CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, d.A, dims, strides,
               box_y, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

}  // namespace

// Packs, work items and the segment -> partial-slot tables the shared prox
// and decide kernels read (segment s owns slots segchunk[s] .. segchunk[s + 1]).
cudaError_t dense_prepare(glrm_s *h)
{
    Dense &d = h->dn;
    d.KP = dense_width(h->k);
    int sms = 0;
    cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device);
    if (e != cudaSuccess) return e;
    const int64_t rows_pad = (std::max(h->m, h->n) + kDnRows - 1) / kDnRows * kDnRows;
    d.pack_part = rows_pad * d.KP;
    if ((e = dalloc(h, &d.pk, 3 * (size_t)d.pack_part * sizeof(__nv_bfloat16))) != cudaSuccess) return e;
    if ((e = dalloc(h, &d.pt, 3 * (size_t)d.pack_part * sizeof(__nv_bfloat16))) != cudaSuccess) return e;
    if ((e = encode_maps(h)) != cudaSuccess) return e;
    // column losses in FP32, each with the kind its 16-column group shares
    // (-1: mixed)
    std::vector<float4> lf(h->n);
    for (int64_t j = 0; j < h->n; ++j) {
        const LossSpec &L = h->loss_host[j];
        int32_t kb = L.kind;
        float kf;
        memcpy(&kf, &kb, sizeof kf);
        lf[j] = make_float4(kf, (float)L.param, (float)L.levels, 0.f);
    }
    const int64_t ngroups = (h->n + kDnNT - 1) / kDnNT * (kDnNT / 16);
    std::vector<int32_t> gk(ngroups, kLossQuad);
    for (int64_t g = 0; g * 16 < h->n; ++g) {
        const LossSpec &L0 = h->loss_host[g * 16];
        int32_t kd = L0.kind;
        for (int64_t j = g * 16; j < std::min<int64_t>(h->n, g * 16 + 16); ++j) {
            const LossSpec &L = h->loss_host[j];
            if (L.kind != L0.kind || (float)L.param != (float)L0.param || L.levels != L0.levels) kd = -1;
        }
        gk[g] = kd;
    }
    for (int64_t j = 0; j < h->n; ++j) {
        const int32_t kd = gk[j / 16];
        memcpy(&lf[j].w, &kd, sizeof kd);
    }
    if ((e = dalloc(h, &d.lossf, (size_t)h->n * sizeof(float4))) != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(d.lossf, lf.data(), lf.size() * sizeof(float4), cudaMemcpyHostToDevice,
                             h->stream)) != cudaSuccess)
        return e;

    // X-step: chunks are 64 columns (four 16-column groups), tiles alike;
    // Y-step: tiles are 128 columns (four 32-column warps), chunks alike
    const int64_t tiles_x = (h->m + kDnRows - 1) / kDnRows, tiles_y = (h->n + kDnRows - 1) / kDnRows;
    const int64_t nch_x = std::max<int64_t>(1, (h->n + kDnNT - 1) / kDnNT);
    const int64_t nch_y = std::max<int64_t>(1, (h->m + kDnNT - 1) / kDnNT);
    DensePlan &pl = h->dnplan;  // depends only on m, n, the losses and the device: made once per handle
    if (!pl.ready) {
        std::vector<double> cx(nch_x, 0.0), cy(tiles_y, 0.0);
        for (int64_t q = 0; q < nch_x; ++q)
            for (int g = 0; g < kDnNT / 16; ++g) cx[q] += 16 * group_cost(h->loss_host, q * kDnNT + 16 * g, 16);
        // Y-step tiles: the 32-column blocks in order of cost (then loss kind),
        // four to a tile.  A tile advances at the pace of its slowest block: a
        // block's four warps (warp indices equal mod 4) share one SM
        // sub-partition, and the four blocks move through the chunks in step;
        // tiles of like blocks leave no sub-partition waiting on another.
        const int64_t nb = (h->n + 31) / 32;
        std::vector<double> bc(nb);
        std::vector<int64_t> order(nb);
        for (int64_t b = 0; b < nb; ++b) {
            bc[b] = group_cost(h->loss_host, 32 * b, 32);
            order[b] = b;
        }
        std::stable_sort(order.begin(), order.end(), [&](int64_t u, int64_t v) {
            return bc[u] != bc[v] ? bc[u] < bc[v] : h->loss_host[32 * u].kind < h->loss_host[32 * v].kind;
        });
        pl.blocks_y.assign(4 * tiles_y, -1);
        std::vector<int64_t> tile_of(nb);
        for (int64_t i = 0; i < nb; ++i) {
            pl.blocks_y[i] = (int32_t)order[i];
            tile_of[order[i]] = i / 4;
            cy[i / 4] = std::max(cy[i / 4], kDnRows * bc[order[i]]);
        }
        pl.x = plan_items(h->m, h->n, sms, std::vector<double>(tiles_x, 1.0), cx);
        pl.y = plan_items(h->n, h->m, sms, cy, std::vector<double>(nch_y, 1.0));
        // Y slots in column order: column j owns parts-of-its-tile slots
        pl.seg_y.resize(h->n + 1);
        int64_t run = 0;
        for (int64_t j = 0; j < h->n; ++j) {
            pl.seg_y[j] = (int32_t)std::min<int64_t>(run, INT32_MAX);
            run += pl.y.tiles[2 * tile_of[j / 32] + 1];
        }
        pl.seg_y[h->n] = (int32_t)std::min<int64_t>(run, INT32_MAX);
        pl.y.slots = run;
        pl.ready = true;
    }
    const ItemPlan &px = pl.x, &py = pl.y;
    if (px.slots > INT32_MAX || py.slots > INT32_MAX) return cudaErrorInvalidValue;
    d.nitems_x = (int64_t)px.items.size();
    d.nitems_y = (int64_t)py.items.size();
    d.slots_x = px.slots;
    d.slots_y = py.slots;
    d.slots = std::max(px.slots, py.slots);
    int64_t *tb = nullptr;
    if ((e = dalloc(h, &d.items_x, px.items.size() * sizeof(DnItem))) != cudaSuccess) return e;
    if ((e = dalloc(h, &d.items_y, py.items.size() * sizeof(DnItem))) != cudaSuccess) return e;
    if ((e = dalloc(h, &d.blocks_y, pl.blocks_y.size() * sizeof(int32_t))) != cudaSuccess) return e;
    if ((e = dalloc(h, &d.segchunk_x, (size_t)(h->m + 1) * sizeof(int32_t))) != cudaSuccess) return e;
    if ((e = dalloc(h, &d.segchunk_y, (size_t)(h->n + 1) * sizeof(int32_t))) != cudaSuccess) return e;
    if ((e = dalloc(h, &tb, px.tiles.size() * sizeof(int64_t))) != cudaSuccess) return e;
    const std::pair<const void *, void *> copies[5] = {{px.items.data(), d.items_x},
                                                       {py.items.data(), d.items_y},
                                                       {pl.blocks_y.data(), d.blocks_y},
                                                       {pl.seg_y.data(), d.segchunk_y},
                                                       {px.tiles.data(), tb}};
    const size_t sizes[5] = {px.items.size() * sizeof(DnItem), py.items.size() * sizeof(DnItem),
                             pl.blocks_y.size() * sizeof(int32_t), pl.seg_y.size() * sizeof(int32_t),
                             px.tiles.size() * sizeof(int64_t)};
    for (int c = 0; c < 5; ++c)
        if ((e = cudaMemcpyAsync(copies[c].second, copies[c].first, sizes[c], cudaMemcpyHostToDevice, h->stream)) !=
            cudaSuccess)
            return e;
    dense_segchunk_kernel<<<(unsigned)((h->m + 256) / 256), 256, 0, h->stream>>>(d.segchunk_x, h->m, tb, px.slots);
    e = cudaGetLastError();
    dfree(tb, h->stream);
    return e;
}

cudaError_t launch_dense_scatter(glrm_s *h, float *A, int64_t lda, cudaStream_t st, int64_t r0, int64_t r1)
{
    if (r1 < 0) r1 = h->m;
    if (r1 <= r0) return cudaSuccess;
    dense_scatter_kernel<<<(unsigned)((r1 - r0 + 7) / 8), 256, 0, st>>>(
        h->csr.ptr + r0, h->csr.idx, (const float *)h->csr.val, r1 - r0, h->n, lda, A + r0 * lda);
    h->launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_dense_validate(const float *A, int64_t lda, int64_t m, int64_t n, const LossSpec *loss,
                                  int *flag, cudaStream_t st)
{
    const int64_t total = m * n;
    const unsigned nb = (unsigned)std::min<int64_t>(4096, std::max<int64_t>(1, (total + 255) / 256));
    dense_validate_kernel<<<nb, 256, 0, st>>>(A, lda, m, n, loss, flag);
    return cudaGetLastError();
}

// alpha = 1 / max(n_i, 1): every row has n observed entries, every column m.
cudaError_t dense_reset_steps(glrm_s *h)
{
    dense_alpha_kernel<<<(unsigned)((h->m + 255) / 256), 256, 0, h->stream>>>(
        (float *)h->alpha_x, h->m, 1.f / (float)std::max<int64_t>(h->n, 1));
    dense_alpha_kernel<<<(unsigned)((h->n + 255) / 256), 256, 0, h->stream>>>(
        (float *)h->alpha_y, h->n, 1.f / (float)std::max<int64_t>(h->m, 1));
    h->launches += 2;
    return cudaGetLastError();
}

cudaError_t dense_half_step(glrm_s *h, bool xstep)
{
    const int64_t nseg = xstep ? h->m : h->n;
    const int32_t *segchunk = xstep ? h->dn.segchunk_x : h->dn.segchunk_y;
    float *F = (float *)(xstep ? h->X : h->Yt);
    const float *W = (const float *)(xstep ? h->Yt : h->X);
    float *alpha = (float *)(xstep ? h->alpha_x : h->alpha_y);
    const int rk = reg_code(h, xstep);
    const float rw = (float)(xstep ? h->rx_w : h->ry_w);
    Scratch &s = h->s;
    cudaStream_t st = h->stream;
    cudaError_t e = dense_pack(h, W, xstep ? h->n : h->m);
    if (e != cudaSuccess) return e;
    tmark(h, xstep ? "dense_grad_x" : "dense_grad_y");
    e = xstep ? launch_dense<true, true>(h, F, (float *)s.part_grad, s.part_loss)
              : launch_dense<false, true>(h, F, (float *)s.part_grad, s.part_loss);
    if (e != cudaSuccess) return e;
    tmark(h, xstep ? "prox_x" : "prox_y");
    e = launch_prox<float>(nseg, segchunk, (const float *)s.part_grad, s.part_loss, F, alpha, h->k, rk, rw,
                           (float *)s.cand, s.f_old, s.r_old, s.r_new, st);
    if (e != cudaSuccess) return e;
    tmark(h, xstep ? "dense_loss_x" : "dense_loss_y");
    e = xstep ? launch_dense<true, false>(h, (const float *)s.cand, nullptr, s.part_loss2)
              : launch_dense<false, false>(h, (const float *)s.cand, nullptr, s.part_loss2);
    if (e != cudaSuccess) return e;
    tmark(h, xstep ? "decide_x" : "decide_y");
    e = launch_decide<float>(nseg, segchunk, s.part_loss2, s.f_old, s.r_old, s.r_new, (const float *)s.cand, F,
                             alpha, h->k, xstep ? s.kept_obj_x : s.kept_obj_y, xstep ? s.kept_reg_x : s.kept_reg_y,
                             xstep ? s.acc_x : s.acc_y, st);
    tmark(h, nullptr);
    h->launches += 2;
    return e;
}

cudaError_t dense_objective_at(glrm_s *h, const float *X, const float *Yt, double *out)
{
    Scratch &s = h->s;
    cudaError_t e = dense_pack(h, Yt, h->n);
    if (e != cudaSuccess) return e;
    tmark(h, "dense_objective");
    if ((e = launch_dense<true, false>(h, X, nullptr, s.part_loss)) != cudaSuccess) return e;
    tmark(h, "reduce_stage1");
    reduce_stage1<float><<<kRedBlocks, 256, 0, h->stream>>>(
        s.part_loss, h->dn.slots_x, nullptr, 0, X, h->m, reg_code(h, true), (float)h->rx_w, Yt, h->n,
        reg_code(h, false), (float)h->ry_w, h->k, nullptr, 0, nullptr, 0, s.red_part, s.red_cnt);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    tmark(h, "reduce_stage2");
    reduce_stage2<<<1, 256, 0, h->stream>>>(s.red_part, s.red_cnt, kRedBlocks, out, nullptr);
    tmark(h, nullptr);
    h->launches += 2;
    return cudaGetLastError();
}

cudaError_t dense_grad_at(glrm_s *h, const float *X, const float *Yt, float *GX, float *GYt, bool reg,
                          const double *scale)
{
    Scratch &s = h->s;
    cudaError_t e = dense_pack(h, Yt, h->n);
    if (e != cudaSuccess) return e;
    tmark(h, "dense_grad_x");
    if ((e = launch_dense<true, true>(h, X, (float *)s.part_grad, s.part_loss)) != cudaSuccess) return e;
    tmark(h, "grad_seg_x");
    seg_grad_kernel<float><<<blocks_for(h->m, kWarpsPerBlock), kWarpsPerBlock * 32, 0, h->stream>>>(
        h->m, h->dn.segchunk_x, (const float *)s.part_grad, X, h->k, reg_code(h, true), (float)h->rx_w, reg, scale, GX);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = dense_pack(h, X, h->m)) != cudaSuccess) return e;
    tmark(h, "dense_grad_y");
    if ((e = launch_dense<false, true>(h, Yt, (float *)s.part_grad, s.part_loss)) != cudaSuccess) return e;
    tmark(h, "grad_seg_y");
    seg_grad_kernel<float><<<blocks_for(h->n, kWarpsPerBlock), kWarpsPerBlock * 32, 0, h->stream>>>(
        h->n, h->dn.segchunk_y, (const float *)s.part_grad, Yt, h->k, reg_code(h, false), (float)h->ry_w, reg, scale,
        GYt);
    tmark(h, nullptr);
    h->launches += 2;
    return cudaGetLastError();
}

}  // namespace glrm
