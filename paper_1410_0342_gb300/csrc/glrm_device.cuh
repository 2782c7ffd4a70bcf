// Device-side pieces of the GLRM sweep: per-entry losses and derivatives,
// per-coordinate proximal operators and regulariser values, factor-row
// loaders and warp reductions.  Section references are to Udell et al.,
// "Generalized Low Rank Models" (arXiv 1410.0342).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <math.h>
#include <stdint.h>

namespace glrm {

constexpr int kLossQuad = 0, kLossHuber = 1, kLossHinge = 2, kLossLogistic = 3, kLossOrdinal = 4;
constexpr int kLossL1 = 5, kLossQuantile = 6, kLossKinds = 7;
constexpr int kRegZero = 0, kRegQuad = 1, kRegL1 = 2, kRegNonneg = 3;
// Internal: the indicator of x = 1 (an offset coordinate of X).
constexpr int kRegFixOne = 4;
// Offset roles carried above the regulariser kind passed to the kernels
// (kind | role << 8): the last coordinate of X is held at 1 and the last
// coordinate of Y is not penalised (Section 3.4, "Offsets and scaling").
constexpr int kOffsetX = 1, kOffsetY = 2;

// The regulariser kind of coordinate c of k under an encoded kind rk.
__host__ __device__ __forceinline__ int reg_kind_at(int rk, int c, int k)
{
    const int role = rk >> 8;
    if (role && c == k - 1) return role == kOffsetX ? kRegFixOne : kRegZero;
    return rk & 0xff;
}

// One column's loss, 16 bytes so that a lane loads it with one instruction.
struct __align__(16) LossSpec {
    int32_t kind;
    int32_t levels;
    double param;
};

__device__ __forceinline__ float xexp(float x) { return expf(x); }
__device__ __forceinline__ double xexp(double x) { return exp(x); }
__device__ __forceinline__ float xlog1p(float x) { return log1pf(x); }
__device__ __forceinline__ double xlog1p(double x) { return log1p(x); }
template <class T> __device__ __forceinline__ T xinf();
template <> __device__ __forceinline__ float xinf<float>() { return __int_as_float(0x7f800000); }
template <> __device__ __forceinline__ double xinf<double>() { return __longlong_as_double(0x7ff0000000000000LL); }

// L(u, a) into *L and dL/du as the return value (a subgradient with the
// kinked term's derivative taken as 0 at its kink).
//   quadratic (u-a)^2                                      eq. qpca
//   Huber with threshold delta = param                     Sec. 4.3
//   hinge (1 - a u)_+                                      Sec. 5.2
//   logistic log(1 + exp(-a u)), overflow-free form        Sec. 5.2
//   ordinal hinge over levels 1..d                         eq. ord-pca
//   l1 |a - u|                                             Sec. 4.2 (robust PCA)
//   quantile alpha (a - u)_+ + (1 - alpha) (u - a)_+        Sec. 4.2 (quantile PCA)
// loss_deriv_k: one kind, its parameters already in T (param: the Huber
// threshold or the quantile alpha; levels: the ordinal level count; others
// ignore them).
template <int KIND, class T>
__device__ __forceinline__ T loss_deriv_k(T u, T a, T param, T levels, T &L)
{
    if constexpr (KIND == kLossQuad) {
        T r = u - a;
        L = r * r;
        return T(2) * r;
    } else if constexpr (KIND == kLossHuber) {
        T x = u - a, d = param, ax = fabs(x);
        if (ax <= d) {
            L = T(0.5) * x * x;
            return x;
        }
        L = d * (ax - T(0.5) * d);
        return x > T(0) ? d : -d;
    } else if constexpr (KIND == kLossHinge) {
        T z = T(1) - a * u;
        if (z > T(0)) {
            L = z;
            return -a;
        }
        L = T(0);
        return T(0);
    } else if constexpr (KIND == kLossLogistic) {
        // z = -a u; log(1 + e^z) = max(z, 0) + log1p(e^{-|z|});
        // derivative -a sigma(z) with sigma evaluated on the stable side.
        T z = -a * u, e = xexp(-fabs(z));
        L = fmax(z, T(0)) + xlog1p(e);
        T sg = z >= T(0) ? T(1) / (T(1) + e) : e / (T(1) + e);
        return -a * sg;
    } else if constexpr (KIND == kLossL1) {
        T x = u - a;
        L = fabs(x);
        return x > T(0) ? T(1) : (x < T(0) ? T(-1) : T(0));
    } else if constexpr (KIND == kLossQuantile) {
        T x = u - a;
        L = x > T(0) ? (T(1) - param) * x : -param * x;
        return x > T(0) ? T(1) - param : (x < T(0) ? -param : T(0));
    } else {
        // Ordinal hinge in closed form.  A term (1 - u + a')_+ with a' < a is
        // active (> 0) exactly for a' >= floor(u); a term (1 + u - a')_+ with
        // a' > a exactly for a' <= ceil(u).  With n1, n2 active terms over the
        // integer ranges [lo1, hi1], [lo2, hi2] the sums are arithmetic series.
        const T d = levels;
        const T lev = fmin(fmax(a, T(1)), d);  // a is validated to 1..d at set-up
        const T lo1 = fmax(T(1), floor(u)), hi1 = lev - T(1);
        const T n1 = fmax(T(0), hi1 - lo1 + T(1));
        const T lo2 = lev + T(1), hi2 = fmin(d, ceil(u));
        const T n2 = fmax(T(0), hi2 - lo2 + T(1));
        L = n1 * (T(1) - u) + T(0.5) * n1 * (lo1 + hi1) + n2 * (T(1) + u) - T(0.5) * n2 * (lo2 + hi2);
        return n2 - n1;
    }
}

// L(u, a) into *L and dL/du as the return value, for a runtime kind.
template <class T>
__device__ __forceinline__ T loss_deriv_kind(int kind, T u, T a, T param, T levels, T &L)
{
    switch (kind) {
    case kLossQuad: return loss_deriv_k<kLossQuad, T>(u, a, param, levels, L);
    case kLossHuber: return loss_deriv_k<kLossHuber, T>(u, a, param, levels, L);
    case kLossHinge: return loss_deriv_k<kLossHinge, T>(u, a, param, levels, L);
    case kLossLogistic: return loss_deriv_k<kLossLogistic, T>(u, a, param, levels, L);
    case kLossL1: return loss_deriv_k<kLossL1, T>(u, a, param, levels, L);
    case kLossQuantile: return loss_deriv_k<kLossQuantile, T>(u, a, param, levels, L);
    default: return loss_deriv_k<kLossOrdinal, T>(u, a, param, levels, L);
    }
}

template <class T>
__device__ __forceinline__ T loss_deriv(const LossSpec &s, T u, T a, T &L)
{
    return loss_deriv_kind<T>(s.kind, u, a, T(s.param), T(s.levels), L);
}

// A column's loss with its parameters already in FP32.  The FP32 kernels read
// this form so that no entry converts the FP64 parameter (a conversion that
// runs on the FP64 pipe, 1/64 of the FP32 rate on this GPU).
struct __align__(16) LossSpecF {
    int32_t kind;
    int32_t levels;
    float param;
    float levelsf;
};
template <class T> struct LossOfT { using type = LossSpec; };
template <> struct LossOfT<float> { using type = LossSpecF; };
// The loss table type the kernels of element type T read.
template <class T> using LossOf = typename LossOfT<T>::type;

template <class T>
__device__ __forceinline__ T loss_deriv(const LossSpecF &s, T u, T a, T &L)
{
    static_assert(sizeof(T) == sizeof(float), "LossSpecF is read by FP32 kernels");
    return loss_deriv_kind<T>(s.kind, u, a, s.param, s.levelsf, L);
}

// argmin_a L(u, a) (Sec. 5.3).  For the ordinal hinge,
// L(u, a+1) - L(u, a) = (1 + a - u)_+ - (u - a)_+ is <= 0 exactly when
// u >= a + 1/2, so the minimiser is 1 + #{a in 1..d-1 : u > a + 1/2} with
// ties at u = a + 1/2 going to the lower level; the comparisons are exact in
// any precision.
template <class T>
__device__ __forceinline__ T decode_value(const LossSpec &s, T u)
{
    switch (s.kind) {
    case kLossHinge:
    case kLossLogistic:
        return u >= T(0) ? T(1) : T(-1);
    case kLossOrdinal: {
        int lev = 1;
        for (int a = 1; a < s.levels; ++a) lev += (u > T(a) + T(0.5)) ? 1 : 0;
        return T(lev);
    }
    default:
        return u;
    }
}

// prox_{alpha r} of one coordinate (every regulariser here is separable):
// z/(1 + 2 alpha w), soft threshold at alpha w, max(z, 0), 1 (an offset
// coordinate of X), identity.
template <class T>
__device__ __forceinline__ T prox1(int kind, T w, T alpha, T z)
{
    switch (kind) {
    case kRegQuad:
        return z / (T(1) + T(2) * alpha * w);
    case kRegL1: {
        T t = alpha * w;
        return z > t ? z - t : (z < -t ? z + t : T(0));
    }
    case kRegNonneg:
        return z > T(0) ? z : T(0);
    case kRegFixOne:
        return T(1);
    default:
        return z;
    }
}

// One coordinate's share of r(x): w x^2, w |x|, 0 or +inf (infeasible), 0.
template <class T>
__device__ __forceinline__ double reg1(int kind, T w, T x)
{
    switch (kind) {
    case kRegQuad:
        return (double)w * (double)x * (double)x;
    case kRegL1:
        return (double)w * fabs((double)x);
    case kRegNonneg:
        return x < T(0) ? xinf<double>() : 0.0;
    case kRegFixOne:
        return x == T(1) ? 0.0 : xinf<double>();
    default:
        return 0.0;
    }
}

// The same in the model's precision (a segment's regulariser for the accept /
// reject test; FP64 only where the segment terms are combined).
template <class T>
__device__ __forceinline__ T reg1t(int kind, T w, T x)
{
    switch (kind) {
    case kRegQuad:
        return w * x * x;
    case kRegL1:
        return w * fabs(x);
    case kRegNonneg:
        return x < T(0) ? xinf<T>() : T(0);
    case kRegFixOne:
        return x == T(1) ? T(0) : xinf<T>();
    default:
        return T(0);
    }
}

// One coordinate of the regulariser's gradient: 2 w x, w sign(x), 0.
template <class T>
__device__ __forceinline__ T reg_grad1(int kind, T w, T x)
{
    switch (kind) {
    case kRegQuad:
        return T(2) * w * x;
    case kRegL1:
        return x > T(0) ? w : (x < T(0) ? -w : T(0));
    default:
        return T(0);
    }
}

// 1/sqrt(d) in FP64 for a positive, finite, normal d; false (and y = 0)
// otherwise: d <= 0, NaN, infinite or subnormal.  d = mant 2^e2 with e2 even
// and mant in [1, 4) (exponent bits), so 1/sqrt(d) = 1/sqrt(mant) 2^(-e2/2):
// a float estimate of 1/sqrt(mant) from rsqrtf refined by two Newton-Raphson
// steps y <- y (3 - mant y^2) / 2 (each squares the relative error: ~1e-7 ->
// ~1e-14 -> below FP64 rounding), then scaled exactly by a power of two.
// Saves the FP64 division and square root, which are slow on this GPU, and
// works for every double exponent, not only float-range ones.
__device__ __forceinline__ bool rsqrt_fp64(double d, double &y)
{
    if (!(d >= 2.2250738585072014e-308 && d <= 1.7976931348623157e308)) {
        y = 0.0;
        return false;
    }
    const long long bits = __double_as_longlong(d);
    const int e2 = ((int)((bits >> 52) & 0x7ff) - 1023) & ~1;
    const double mant = d * __longlong_as_double((long long)(1023 - e2) << 52);
    double r = (double)rsqrtf((float)mant);
    r = r * (1.5 - 0.5 * mant * r * r);
    r = r * (1.5 - 0.5 * mant * r * r);
    y = r * __longlong_as_double((long long)(1023 - e2 / 2) << 52);
    return true;
}

// Solve (C C^T) x = b in place for an SPD matrix G (row-major, leading
// dimension LD, lower triangle used; overwritten by C) and right-hand side b
// (overwritten by x), one warp, K <= 32.  Column by column: lane 0 takes the
// pivot's reciprocal square root, lanes below it scale the column, and the
// trailing update's (row, column) pairs are spread over all 32 lanes (an
// FP64 instruction costs the same issue time however few lanes it has, and
// FP64 runs at 1/64 of the FP32 rate here, so no lane should sit idle in
// it); the two triangular solves are column-oriented.  FP64 throughout.
// Returns (to every lane) false when a pivot was not positive, finite and
// normal: G was not numerically positive definite (or held Inf / NaN); b
// then holds no solution and must not be used.
template <int K, int LD>
__device__ __forceinline__ bool warp_cholesky_factor(double (*G)[LD])
{
    const int lane = threadIdx.x & 31;
    bool ok = true;
    for (int c = 0; c < K; ++c) {
        if (lane == 0) {
            double r;
            ok = rsqrt_fp64(G[c][c], r) && ok;
            G[c][c] = r;  // the pivot slot keeps 1/C[c][c] from here on
        }
        __syncwarp();
        const double r = G[c][c];
        if (lane > c && lane < K) G[lane][c] *= r;
        __syncwarp();
        // pairs (c + 1 + i, c + 1 + j), 0 <= j <= i < n, numbered p = i (i + 1) / 2 + j
        const int n = K - 1 - c;
        for (int p = lane; p < n * (n + 1) / 2; p += 32) {
            int i = (int)((sqrtf(8.f * (float)p + 1.f) - 1.f) * 0.5f);
            while ((i + 1) * (i + 2) / 2 <= p) ++i;
            while (i * (i + 1) / 2 > p) --i;
            const int row = c + 1 + i, col = c + 1 + p - i * (i + 1) / 2;
            G[row][col] -= G[row][c] * G[col][c];
        }
        __syncwarp();
    }
    return __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
}

// b <- (C C^T)^{-1} b with the factor warp_cholesky_factor left in G: C w = b
// (w[c] = b[c] / C[c][c], then b[r] -= C[r][c] w[c] for r > c), then C^T x = w.
template <int K, int LD>
__device__ __forceinline__ void warp_cholesky_subst(double (*G)[LD], double *b)
{
    const int lane = threadIdx.x & 31;
    for (int c = 0; c < K; ++c) {
        if (lane == 0) b[c] *= G[c][c];
        __syncwarp();
        if (lane > c && lane < K) b[lane] -= G[lane][c] * b[c];
        __syncwarp();
    }
    for (int c = K - 1; c >= 0; --c) {
        if (lane == 0) b[c] *= G[c][c];
        __syncwarp();
        if (lane < c) b[lane] -= G[c][lane] * b[c];
        __syncwarp();
    }
}

template <int K, int LD>
__device__ __forceinline__ bool warp_cholesky_solve(double (*G)[LD], double *b)
{
    const bool ok = warp_cholesky_factor<K, LD>(G);
    warp_cholesky_subst<K, LD>(G, b);
    return ok;
}

// Bits of the handle's device status word (Scratch::err).
constexpr int kErrWait = 1;   // a bounded wait hit its iteration limit
constexpr int kErrPivot = 2;  // an ALS Cholesky pivot was not positive and finite

__device__ __forceinline__ float shfl_xor(float v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
__device__ __forceinline__ double shfl_xor(double v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
__device__ __forceinline__ int shfl_xor(int v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }

template <class T>
__device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += shfl_xor(v, o);
    return v;
}

// Load coordinates c0 .. c0+S-1 of a factor row (row-major, k values).
// VEC: the caller guarantees k == the padded width, so the slice is in range,
// and 16-byte alignment, so the slice loads as float4 / double2 vectors.
// Otherwise coordinates at or beyond k read as 0.
template <class T, int S, bool VEC>
__device__ __forceinline__ void load_slice(T (&v)[S], const T *__restrict__ row, int c0, int k)
{
    if constexpr (VEC && sizeof(T) == 4) {
        static_assert(S % 4 == 0, "float slice must be a multiple of 4");
        const float4 *p = reinterpret_cast<const float4 *>(row + c0);
#pragma unroll
        for (int q = 0; q < S / 4; ++q) {
            float4 t = __ldg(p + q);
            v[4 * q + 0] = t.x;
            v[4 * q + 1] = t.y;
            v[4 * q + 2] = t.z;
            v[4 * q + 3] = t.w;
        }
    } else if constexpr (VEC && sizeof(T) == 8) {
        static_assert(S % 2 == 0, "double slice must be a multiple of 2");
        const double2 *p = reinterpret_cast<const double2 *>(row + c0);
#pragma unroll
        for (int q = 0; q < S / 2; ++q) {
            double2 t = __ldg(p + q);
            v[2 * q + 0] = t.x;
            v[2 * q + 1] = t.y;
        }
    } else {
#pragma unroll
        for (int s = 0; s < S; ++s) v[s] = (c0 + s < k) ? __ldg(row + c0 + s) : T(0);
    }
}

}  // namespace glrm
