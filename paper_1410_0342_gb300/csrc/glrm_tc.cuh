// Fifth-generation tensor core (tcgen05) building blocks for the dense,
// fully observed form: D (128 x N, FP32, in tensor memory) += A (128 x K) B^T
// with A and B in BF16, K-major, staged in shared memory in the canonical
// no-swizzle layout of 8-row x 16-byte core matrices.
//
// Layout of an R x K BF16 operand tile in shared memory (R rows, K a multiple
// of 16): element (r, c) sits at
//     ((r / 8) * (K / 8) + c / 8) * 64 + (r % 8) * 8 + c % 8      (elements)
// so the core matrices of one 8-row group follow each other along K
// (leading-dimension byte offset 128) and 8-row groups are K * 16 bytes apart
// (stride-dimension byte offset).
#pragma once

#include <algorithm>

#include "glrm_tiled.cuh"

namespace glrm {

// Shared-memory matrix descriptor (tcgen05): start address, leading and
// stride byte offsets (all >> 4), descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t umma_desc(const void *smem, uint32_t lbo, uint32_t sbo)
{
    const uint64_t a = (uint64_t)((smem_u32(smem) >> 4) & 0x3FFF);
    return a | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) | ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) |
           ((uint64_t)1 << 46);
}

// Instruction descriptor, kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, N and M as given.
__host__ __device__ constexpr uint32_t umma_idesc_bf16(int M, int N)
{
    return (1u << 4)                           // D: FP32
           | (1u << 7)                         // A: BF16
           | (1u << 10)                        // B: BF16
           | ((uint32_t)(N >> 3) << 17)        // N / 8
           | ((uint32_t)(M >> 4) << 24);       // M / 16
}

__device__ __forceinline__ uint32_t tmem_alloc(uint32_t *slot, uint32_t ncols)
{
    // whole warp; the TMEM address lands in shared memory
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    return 0;
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// One MMA, issued by a single thread: D[taddr] (+)= A B^T.
__device__ __forceinline__ void umma_bf16(uint32_t taddr, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          bool accumulate)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(taddr),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"((uint32_t)accumulate)
        : "memory");
}

// The mbarrier arrives once every MMA issued so far by this thread is done.
__device__ __forceinline__ void umma_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(bar))
                 : "memory");
}

// 16 consecutive FP32 columns of this thread's TMEM lane (warp w of the
// warpgroup reads lanes 32 w .. 32 w + 31).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16])
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
        "%14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int q = 0; q < 16; ++q) v[q] = __uint_as_float(r[q]);
}

__host__ __device__ __forceinline__ int64_t core_index(int64_t r, int c, int K)
{
    return ((r >> 3) * (K >> 3) + (c >> 3)) * 64 + (r & 7) * 8 + (c & 7);
}

// Swizzled K-major operand layouts.  Rows of RB = 32, 64 or 128 bytes (16,
// 32 or 64 BF16 values along K), 8-row groups of 8 RB bytes; inside a group
// the 16-byte unit u of row r sits at u ^ (r % 8 >> (3 - log2(RB / 16)))
// (the 32-, 64- and 128-byte swizzles: address bits 4.. are XORed with bits
// 7..).  Every operand buffer starts on a 1024-byte boundary.
__host__ __device__ constexpr uint32_t sw_off(uint32_t r, uint32_t c, uint32_t RB)
{
    const uint32_t off = r * RB + c * 2;
    return off ^ (((off >> 7) & (RB / 16 - 1)) << 4);
}

// Layout-type field of the descriptor for rows of RB bytes.
__host__ __device__ constexpr uint64_t sw_type(uint32_t RB)
{
    return RB == 128 ? 2ull : (RB == 64 ? 4ull : 6ull);
}

// Descriptor of a swizzled K-major operand at smem (the K offset of an MMA
// inside a row is added to the start address): stride between 8-row groups
// 8 RB, leading offset unused (1).
__device__ __forceinline__ uint64_t umma_desc_sw(const void *smem, uint32_t RB)
{
    const uint64_t a = (uint64_t)((smem_u32(smem) >> 4) & 0x3FFF);
    return a | (1ull << 16) | ((uint64_t)(((8 * RB) >> 4) & 0x3FFF) << 32) | (1ull << 46) | (sw_type(RB) << 61);
}

// D (M x N, row-major FP32) = A (M x K, row-major BF16) B^T (B: N x K,
// row-major BF16).  One CTA of 128 threads per 128 x NT tile; M a multiple of
// 128, N of NT, K of 16 and at most kTcMaxK.  Operands in the swizzled K-major
// layout with RB = 2K bytes per row for K <= 64, or (K = 128) two 64-wide
// column blocks of 128-byte rows.
constexpr int kTcMaxK = 128;
constexpr int kTcNT = 64;

static __global__ void __launch_bounds__(128, 1)
tc_gemm_bf16_kernel(const __nv_bfloat16 *__restrict__ A, const __nv_bfloat16 *__restrict__ B,
                    float *__restrict__ D, int M, int N, int K, int *__restrict__ err)
{
    extern __shared__ __align__(1024) unsigned char dsm_tc[];
    __shared__ uint64_t bar;
    __shared__ uint32_t tslot;
    unsigned char *base = dsm_tc + ((1024 - (smem_u32(dsm_tc) & 1023)) & 1023);
    const int KB = K < 64 ? K : 64;           // K values per column block
    const uint32_t RB = (uint32_t)KB * 2;     // bytes per row
    const int nblk = K / KB;
    unsigned char *As = base;                 // block j at As + j * 128 RB
    unsigned char *Bs = base + (size_t)nblk * 128 * RB;  // block j at Bs + j * NT RB
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t r0 = (int64_t)blockIdx.x * 128, n0 = (int64_t)blockIdx.y * kTcNT;
    for (int q = tid; q < 128 * K; q += 128) {
        const int r = q / K, c = q % K;
        *reinterpret_cast<__nv_bfloat16 *>(As + (c / KB) * 128 * RB + sw_off(r, c % KB, RB)) = A[(r0 + r) * K + c];
    }
    for (int q = tid; q < kTcNT * K; q += 128) {
        const int r = q / K, c = q % K;
        *reinterpret_cast<__nv_bfloat16 *>(Bs + (c / KB) * kTcNT * RB + sw_off(r, c % KB, RB)) =
            B[(n0 + r) * K + c];
    }
    if (tid == 0) mbar_init(&bar, 1);
    if (warp == 0) tmem_alloc(&tslot, kTcNT);
    fence_proxy_async();  // shared-memory writes visible to the tensor core
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t taddr = tslot;
    if (tid == 0) {
        const uint32_t idesc = umma_idesc_bf16(128, kTcNT);
        for (int ks = 0; ks < K / 16; ++ks) {
            const int j = ks * 16 / KB, kk = ks * 16 % KB;
            const uint64_t ad = umma_desc_sw(As + j * 128 * RB + kk * 2, RB);
            const uint64_t bd = umma_desc_sw(Bs + j * kTcNT * RB + kk * 2, RB);
            umma_bf16(taddr, ad, bd, idesc, ks > 0);
        }
        umma_commit(&bar);
    }
    bool ok = mbar_wait_bounded(&bar, 0);
    if (!ok) ok = mbar_wait_bounded(&bar, 0);
    tc_fence_after();
    if (__syncthreads_or(!ok)) {
        if (tid == 0) atomicOr(err, 1);
    } else {
        const int row = (int)r0 + warp * 32 + lane;
#pragma unroll
        for (int c = 0; c < kTcNT; c += 16) {
            float v[16];
            tmem_ld16(taddr + ((uint32_t)(warp * 32) << 16) + (uint32_t)c, v);
#pragma unroll
            for (int q = 0; q < 16; ++q) D[(int64_t)row * N + n0 + c + q] = v[q];
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(taddr, kTcNT);
    }
}

}  // namespace glrm
