// Global optimality certificate (Section 7.6, eq. convex-certificate) for a
// model with the quadratic regulariser w (||X||^2 + ||Y||^2):
//     || (1/gamma) G + U V^T ||_2 <= 1,   gamma = 2 w,
// where G (m x n, zero off Omega) holds w_j L_j'(x_i . y_j, A_ij) and U V^T
// is the product of the singular vectors of Z = X Y (nonzero singular
// values).  With ||Z||_* = inf 1/2 (||X||^2 + ||Y||^2) over X Y = Z, the
// regularised problem's convex relaxation is L(Z) + 2 w ||Z||_*, hence
// gamma = 2 w.
//
// U V^T is never formed.  From the k x k Gram matrices X^T X = V_a D_a V_a^T
// and Y Y^T = V_b D_b V_b^T (Jacobi, FP64), X = Q_x S_a V_a^T and
// Y^T = Q_y S_b V_b^T with orthonormal Q_x, Q_y, so Z = Q_x C Q_y^T with
// C = S_a V_a^T V_b S_b (k x k); with C = U_c S V_c^T (one-sided Jacobi),
// U V^T = Q_x (U_c V_c^T) Q_y^T = X K Y, K = V_a S_a^-1 U_c V_c^T S_b^-1 V_b^T.
// The 2-norm of M = G / gamma + X K Y is then found by power iteration on
// M^T M with M v = G v / gamma + X (K (Y v)) and M^T w = G^T w / gamma +
// Y^T (K^T (X^T w)): sparse products over the CSR and CSC orders, k-vector
// reductions and row updates, all in FP64.
#include "glrm_handle.h"

namespace glrm {
namespace {

constexpr int kCertBlocks = 304;  // partial sums of the reductions (2 x 152 SMs)
constexpr int kJacobiSweeps = 60;
constexpr int kSvdMaxL = 96;  // columns of the randomized range finder (k + oversampling)
// Segments averaging this many entries or more take the chunked products.
constexpr int64_t kLongSegment = 2048;

// g[e] = w_j L_j'(u, a) with u = x_i . y_j accumulated in FP64 in coordinate
// order, one warp per segment; the same value in both orders.
template <class T>
__global__ void cert_deriv_kernel(int64_t nseg, const int32_t *__restrict__ ptr, const int32_t *__restrict__ idx,
                                  const T *__restrict__ val, const T *__restrict__ F, const T *__restrict__ W, int k,
                                  const LossSpec *__restrict__ loss, const T *__restrict__ lsc, bool xstep,
                                  double *__restrict__ g)
{
    const int lane = threadIdx.x & 31;
    const int64_t s = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (s >= nseg) return;
    const T *f = F + s * k;
    for (int e = ptr[s] + lane; e < ptr[s + 1]; e += 32) {
        const int32_t j = idx[e];
        const T *w = W + (int64_t)j * k;
        double u = 0.0;
        for (int c = 0; c < k; ++c) u += (double)f[c] * (double)w[c];
        const int64_t col = xstep ? j : s;
        double L;
        double d = loss_deriv<double>(loss[col], u, (double)val[e], L);
        if (lsc) d *= (double)lsc[col];
        g[e] = d;
    }
}

// Partial Gram matrices of the rows of F (rows x k): block b sums rows
// b, b + B, ... for every pair p <= q (threads over pairs), in row order.
template <class T>
__global__ void cert_gram_kernel(int64_t rows, const T *__restrict__ F, int k, double *__restrict__ part)
{
    const int npair = k * (k + 1) / 2;
    for (int t = threadIdx.x; t < npair; t += blockDim.x) {
        int p = 0, rem = t;
        while (rem >= k - p) {
            rem -= k - p;
            ++p;
        }
        const int q = p + rem;
        double acc = 0.0;
        for (int64_t r = blockIdx.x; r < rows; r += gridDim.x) acc += (double)F[r * k + p] * (double)F[r * k + q];
        part[(int64_t)blockIdx.x * npair + t] = acc;
    }
}

// Partial sums over rows of F^T v (k entries per block).
template <class T>
__global__ void cert_kvec_kernel(int64_t rows, const T *__restrict__ F, int k, const double *__restrict__ v,
                                 double *__restrict__ part)
{
    for (int c = threadIdx.x; c < k; c += blockDim.x) {
        double acc = 0.0;
        for (int64_t r = blockIdx.x; r < rows; r += gridDim.x) acc += (double)F[r * k + c] * v[r];
        part[(int64_t)blockIdx.x * k + c] = acc;
    }
}

// Sum of nb partial vectors of length len, in block order (one block).
__global__ void cert_sum_kernel(const double *__restrict__ part, int nb, int len, double *__restrict__ out)
{
    for (int t = threadIdx.x; t < len; t += blockDim.x) {
        double acc = 0.0;
        for (int b = 0; b < nb; ++b) acc += part[(int64_t)b * len + t];
        out[t] = acc;
    }
}

// out[s] = scale * sum_{e in segment s} g[e] x[idx[e]] + F[s] . kv, one warp
// per segment; lane partial sums combined by a fixed butterfly.
template <class T>
__global__ void cert_apply_kernel(int64_t nseg, const int32_t *__restrict__ ptr, const int32_t *__restrict__ idx,
                                  const double *__restrict__ g, const double *__restrict__ x, double scale,
                                  const T *__restrict__ F, int k, const double *__restrict__ kv,
                                  double *__restrict__ out)
{
    const int lane = threadIdx.x & 31;
    const int64_t s = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (s >= nseg) return;
    double acc = 0.0;
    for (int e = ptr[s] + lane; e < ptr[s + 1]; e += 32) acc += g[e] * x[idx[e]];
    double lr = 0.0;
    for (int c = lane; c < k; c += 32) lr += (double)F[s * k + c] * kv[c];
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        acc += __shfl_xor_sync(0xffffffffu, acc, o);
        lr += __shfl_xor_sync(0xffffffffu, lr, o);
    }
    if (lane == 0) out[s] = scale * acc + lr;
}

// The same two products over the chunk table of an orientation (chunks of at
// most 1024 entries), for long segments: one warp per chunk writes a
// partial, one warp per segment adds its chunks' partials in chunk order.
__global__ void chunk_apply_kernel(int64_t nchunks, const int4 *__restrict__ chunks, const int32_t *__restrict__ idx,
                                   const double *__restrict__ g, const double *__restrict__ x,
                                   double *__restrict__ part)
{
    const int lane = threadIdx.x & 31;
    const int64_t c = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (c >= nchunks) return;
    const int4 ch = chunks[c];
    double acc = 0.0;
    for (int e = ch.y + lane; e < ch.z; e += 32) acc += g[e] * x[idx[e]];
#pragma unroll
    for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) part[c] = acc;
}

template <class T>
__global__ void seg_apply_sum_kernel(int64_t nseg, const int32_t *__restrict__ segchunk,
                                     const double *__restrict__ part, double scale, const T *__restrict__ F, int k,
                                     const double *__restrict__ kv, double *__restrict__ out)
{
    const int lane = threadIdx.x & 31;
    const int64_t s = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (s >= nseg) return;
    double lr = 0.0;
    for (int c = lane; c < k; c += 32) lr += (double)F[s * k + c] * kv[c];
#pragma unroll
    for (int o = 16; o; o >>= 1) lr += __shfl_xor_sync(0xffffffffu, lr, o);
    if (lane == 0) {
        double acc = 0.0;
        for (int c = segchunk[s]; c < segchunk[s + 1]; ++c) acc += part[c];
        out[s] = scale * acc + lr;
    }
}

// Partial sums of squares.
__global__ void cert_sq_kernel(int64_t n, const double *__restrict__ v, double *__restrict__ part)
{
    __shared__ double red[256];
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        acc += v[i] * v[i];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int o = 128; o; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// v *= 1 / sqrt(*sq) (no change when *sq is 0).
__global__ void cert_scale_kernel(int64_t n, double *__restrict__ v, const double *__restrict__ sq)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const double s = *sq;
    if (i < n && s > 0.0) v[i] *= 1.0 / sqrt(s);
}

// out = A t (transpose: A^T t) for a k x k row-major A (one block).
__global__ void cert_kmat_kernel(const double *__restrict__ A, int k, bool trans, const double *__restrict__ t,
                                 double *__restrict__ out)
{
    for (int r = threadIdx.x; r < k; r += blockDim.x) {
        double acc = 0.0;
        for (int c = 0; c < k; ++c) acc += (trans ? A[c * k + r] : A[r * k + c]) * t[c];
        out[r] = acc;
    }
}

// ---------------------------------------------------------- small FP64 algebra
// One block of blockDim.x >= k threads; k x k matrices row-major in global
// scratch.  Thread r owns row r where rows are touched independently.

// Cyclic Jacobi eigendecomposition of the symmetric A (overwritten): on
// return diag(A) holds the eigenvalues, V the eigenvectors as columns.
__device__ void jacobi_eig(double *A, double *V, int k)
{
    const int r = threadIdx.x;
    for (int c = 0; c < k && r < k; ++c) V[r * k + c] = r == c ? 1.0 : 0.0;
    __syncthreads();
    for (int sweep = 0; sweep < kJacobiSweeps; ++sweep) {
        double off = 0.0, dia = 0.0;
        for (int p = 0; p < k; ++p)
            for (int q = 0; q < k; ++q) (p == q ? dia : off) += A[p * k + q] * A[p * k + q];
        if (off <= 1e-30 * dia || off == 0.0) break;
        for (int p = 0; p < k - 1; ++p)
            for (int q = p + 1; q < k; ++q) {
                const double apq = A[p * k + q];
                if (apq == 0.0) continue;
                const double app = A[p * k + p], aqq = A[q * k + q];
                const double th = (aqq - app) / (2.0 * apq);
                const double t = (th >= 0.0 ? 1.0 : -1.0) / (fabs(th) + sqrt(1.0 + th * th));
                const double cs = 1.0 / sqrt(1.0 + t * t), sn = t * cs;
                __syncthreads();
                if (r < k) {  // columns p, q
                    const double a = A[r * k + p], b = A[r * k + q];
                    A[r * k + p] = cs * a - sn * b;
                    A[r * k + q] = sn * a + cs * b;
                    const double va = V[r * k + p], vb = V[r * k + q];
                    V[r * k + p] = cs * va - sn * vb;
                    V[r * k + q] = sn * va + cs * vb;
                }
                __syncthreads();
                if (r < k) {  // rows p, q
                    const double a = A[p * k + r], b = A[q * k + r];
                    A[p * k + r] = cs * a - sn * b;
                    A[q * k + r] = sn * a + cs * b;
                }
                __syncthreads();
            }
    }
    __syncthreads();
}

// One-sided Jacobi SVD of C (k x k, overwritten by U S): columns made
// orthogonal by plane rotations that also act on Vc.
__device__ void jacobi_svd(double *C, double *Vc, int k, double *red)
{
    const int r = threadIdx.x;
    for (int c = 0; c < k && r < k; ++c) Vc[r * k + c] = r == c ? 1.0 : 0.0;
    __syncthreads();
    for (int sweep = 0; sweep < kJacobiSweeps; ++sweep) {
        int rotated = 0;
        for (int p = 0; p < k - 1; ++p)
            for (int q = p + 1; q < k; ++q) {
                if (r == 0) {
                    double a = 0.0, b = 0.0, c = 0.0;
                    for (int i = 0; i < k; ++i) {
                        a += C[i * k + p] * C[i * k + p];
                        b += C[i * k + q] * C[i * k + q];
                        c += C[i * k + p] * C[i * k + q];
                    }
                    red[0] = a;
                    red[1] = b;
                    red[2] = c;
                }
                __syncthreads();
                const double a = red[0], b = red[1], c = red[2];
                __syncthreads();
                if (fabs(c) <= 1e-15 * sqrt(a * b) || c == 0.0) continue;
                rotated = 1;
                const double ze = (b - a) / (2.0 * c);
                const double t = (ze >= 0.0 ? 1.0 : -1.0) / (fabs(ze) + sqrt(1.0 + ze * ze));
                const double cs = 1.0 / sqrt(1.0 + t * t), sn = t * cs;
                if (r < k) {
                    const double x = C[r * k + p], y = C[r * k + q];
                    C[r * k + p] = cs * x - sn * y;
                    C[r * k + q] = sn * x + cs * y;
                    const double vx = Vc[r * k + p], vy = Vc[r * k + q];
                    Vc[r * k + p] = cs * vx - sn * vy;
                    Vc[r * k + q] = sn * vx + cs * vy;
                }
                __syncthreads();
            }
        if (!rotated) break;
    }
    __syncthreads();
}

// K = V_a S_a^-1 U_c V_c^T S_b^-1 V_b^T from the two Gram matrices (their
// pairs p <= q in Ga, Gb).  Scratch: 6 k x k matrices and 2k + 4 values.
// rank[0] receives the rank of Z (singular values above rtol times the
// largest); singular values of X or Y below 1e-7 of their largest (the Gram
// matrices resolve no more) count as zero.
__global__ void cert_core_kernel(const double *__restrict__ Ga, const double *__restrict__ Gb, int k, double rtol,
                                 double *__restrict__ scratch, double *__restrict__ K, int *__restrict__ rank)
{
    const int kk = k * k;
    double *A = scratch, *Va = A + kk, *B = Va + kk, *Vb = B + kk, *C = Vb + kk, *Vc = C + kk;
    double *sa = Vc + kk, *sb = sa + k, *red = sb + k;
    const int r = threadIdx.x;
    if (r < k) {
        int t = 0;
        for (int p = 0; p < k; ++p)
            for (int q = p; q < k; ++q, ++t) {
                if (p == r || q == r) {
                    const int o = p == r ? q : p;
                    A[r * k + o] = Ga[t];
                    B[r * k + o] = Gb[t];
                }
            }
    }
    __syncthreads();
    jacobi_eig(A, Va, k);
    jacobi_eig(B, Vb, k);
    if (r == 0) {
        double ma = 0.0, mb = 0.0;
        for (int i = 0; i < k; ++i) {
            sa[i] = sqrt(fmax(A[i * k + i], 0.0));
            sb[i] = sqrt(fmax(B[i * k + i], 0.0));
            ma = fmax(ma, sa[i]);
            mb = fmax(mb, sb[i]);
        }
        for (int i = 0; i < k; ++i) {
            if (!(sa[i] > 1e-7 * ma)) sa[i] = 0.0;
            if (!(sb[i] > 1e-7 * mb)) sb[i] = 0.0;
        }
    }
    __syncthreads();
    if (r < k)  // C = S_a V_a^T V_b S_b
        for (int c = 0; c < k; ++c) {
            double acc = 0.0;
            for (int i = 0; i < k; ++i) acc += Va[i * k + r] * Vb[i * k + c];
            C[r * k + c] = sa[r] * acc * sb[c];
        }
    __syncthreads();
    jacobi_svd(C, Vc, k, red);
    // singular values: column norms of C = U_c S; P = U_c V_c^T over the kept ones
    if (r == 0) {
        double mx = 0.0;
        for (int c = 0; c < k; ++c) {
            double s2 = 0.0;
            for (int i = 0; i < k; ++i) s2 += C[i * k + c] * C[i * k + c];
            A[c] = sqrt(s2);  // A is free now: row 0 keeps the singular values
            mx = fmax(mx, A[c]);
        }
        int rk = 0;
        for (int c = 0; c < k; ++c) {
            if (A[c] > rtol * mx && mx > 0.0) ++rk;
            else A[c] = 0.0;
        }
        rank[0] = rk;
    }
    __syncthreads();
    if (r < k)  // B <- P = sum_c (C[:, c] / s_c) Vc[:, c]^T, row r
        for (int q = 0; q < k; ++q) {
            double acc = 0.0;
            for (int c = 0; c < k; ++c)
                if (A[c] > 0.0) acc += C[r * k + c] / A[c] * Vc[q * k + c];
            B[r * k + q] = acc;
        }
    __syncthreads();
    if (r < k)  // C <- S_a^-1 P S_b^-1 (zero where a singular value was dropped)
        for (int q = 0; q < k; ++q)
            C[r * k + q] = (sa[r] > 0.0 && sb[q] > 0.0) ? B[r * k + q] / (sa[r] * sb[q]) : 0.0;
    __syncthreads();
    if (r < k)  // Vc <- V_a C
        for (int q = 0; q < k; ++q) {
            double acc = 0.0;
            for (int i = 0; i < k; ++i) acc += Va[r * k + i] * C[i * k + q];
            Vc[r * k + q] = acc;
        }
    __syncthreads();
    if (r < k)  // K = (V_a C) V_b^T
        for (int q = 0; q < k; ++q) {
            double acc = 0.0;
            for (int i = 0; i < k; ++i) acc += Vc[r * k + i] * Vb[q * k + i];
            K[r * k + q] = acc;
        }
}

// Deterministic pseudo-random start vector (splitmix64 of the index).
__global__ void cert_start_kernel(int64_t n, double *__restrict__ v)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    unsigned long long z = (unsigned long long)i + 0x9e3779b97f4a7c15ULL;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    z ^= z >> 31;
    v[i] = (double)(z >> 11) * 0x1p-53 - 0.5;
}

inline unsigned nblk(int64_t n, int per) { return (unsigned)((n + per - 1) / per); }

template <class T>
cudaError_t certificate_impl(glrm_s *h, int iters, double tol, double *norm, int *done)
{
    cudaStream_t st = h->stream;
    const int64_t m = h->m, n = h->n, nnz = h->nnz;
    const int k = h->k, npair = k * (k + 1) / 2;
    const T *X = (const T *)h->X, *Yt = (const T *)h->Yt;
    const double scale = 1.0 / (2.0 * h->rx_w);
    double *gr = nullptr, *gc = nullptr, *v = nullptr, *w = nullptr, *part = nullptr, *small = nullptr;
    int *rank = nullptr;
    const size_t part_len = (size_t)kCertBlocks * (size_t)std::max(npair, k);
    const size_t small_len = (size_t)9 * k * k + 8 * (size_t)k + 32;
    cudaError_t e = cudaSuccess;
    auto A = [&](auto **p, size_t bytes) {
        if (e == cudaSuccess) e = dalloc_bytes(h, (void **)p, std::max<size_t>(bytes, 16), st);
    };
    A(&gr, (size_t)nnz * sizeof(double));
    A(&gc, (size_t)nnz * sizeof(double));
    A(&v, (size_t)n * sizeof(double));
    A(&w, (size_t)m * sizeof(double));
    A(&part, part_len * sizeof(double));
    A(&small, small_len * sizeof(double));
    A(&rank, sizeof(int));
    double *cpart = nullptr;  // chunk partials of the long-segment products
    A(&cpart, (size_t)std::max(h->csr.nchunks, h->csc.nchunks) * sizeof(double));
    // small: Ga | Gb | K | t | Kt | scratch (6 k^2 + 2k + 4) | sq
    double *Ga = small, *Gb = Ga + npair, *K = Gb + npair, *t = K + k * k, *kt = t + k, *core = kt + k;
    double *sq = core + 6 * k * k + 2 * k + 4;
    const int core_threads = ((k + 31) / 32) * 32;
    if (e == cudaSuccess) {
        cert_deriv_kernel<T><<<nblk(m, 8), 256, 0, st>>>(m, h->csr.ptr, h->csr.idx, (const T *)h->csr.val, X, Yt,
                                                         k, h->loss_dev, (const T *)h->lscale, true, gr);
        cert_deriv_kernel<T><<<nblk(n, 8), 256, 0, st>>>(n, h->csc.ptr, h->csc.idx, (const T *)h->csc.val, Yt, X,
                                                         k, h->loss_dev, (const T *)h->lscale, false, gc);
        cert_gram_kernel<T><<<kCertBlocks, 256, 0, st>>>(m, X, k, part);
        cert_sum_kernel<<<1, 256, 0, st>>>(part, kCertBlocks, npair, Ga);
        cert_gram_kernel<T><<<kCertBlocks, 256, 0, st>>>(n, Yt, k, part);
        cert_sum_kernel<<<1, 256, 0, st>>>(part, kCertBlocks, npair, Gb);
        cert_core_kernel<<<1, core_threads, 0, st>>>(Ga, Gb, k, 1e-10, core, K, rank);
        cert_start_kernel<<<nblk(n, 256), 256, 0, st>>>(n, v);
        cert_sq_kernel<<<kCertBlocks, 256, 0, st>>>(n, v, part);
        cert_sum_kernel<<<1, 32, 0, st>>>(part, kCertBlocks, 1, sq);
        cert_scale_kernel<<<nblk(n, 256), 256, 0, st>>>(n, v, sq);
        h->launches += 11;
        e = cudaGetLastError();
    }
    // out = scale * G_orient x + F (K-vector kt) over one orientation
    auto apply = [&](const Orient &o, int64_t nseg, const double *g, const double *x, const T *F, double *out) {
        if (o.nchunks > 0 && nnz >= kLongSegment * nseg) {
            chunk_apply_kernel<<<nblk(o.nchunks, 8), 256, 0, st>>>(o.nchunks, o.chunks, o.idx, g, x, cpart);
            seg_apply_sum_kernel<T><<<nblk(nseg, 8), 256, 0, st>>>(nseg, o.segchunk, cpart, scale, F, k, kt, out);
            h->launches += 1;
        } else {
            cert_apply_kernel<T><<<nblk(nseg, 8), 256, 0, st>>>(nseg, o.ptr, o.idx, g, x, scale, F, k, kt, out);
        }
    };
    double est = 0.0, prev = -1.0;
    int it = 0;
    for (; e == cudaSuccess && it < iters; ++it) {
        // w = M v
        cert_kvec_kernel<T><<<kCertBlocks, 64, 0, st>>>(n, Yt, k, v, part);
        cert_sum_kernel<<<1, 64, 0, st>>>(part, kCertBlocks, k, t);
        cert_kmat_kernel<<<1, 64, 0, st>>>(K, k, false, t, kt);
        apply(h->csr, m, gr, v, X, w);
        // v = M^T w
        cert_kvec_kernel<T><<<kCertBlocks, 64, 0, st>>>(m, X, k, w, part);
        cert_sum_kernel<<<1, 64, 0, st>>>(part, kCertBlocks, k, t);
        cert_kmat_kernel<<<1, 64, 0, st>>>(K, k, true, t, kt);
        apply(h->csc, n, gc, w, Yt, v);
        // ||M^T M v|| with ||v|| = 1 is the estimate of sigma^2; normalise v
        cert_sq_kernel<<<kCertBlocks, 256, 0, st>>>(n, v, part);
        cert_sum_kernel<<<1, 32, 0, st>>>(part, kCertBlocks, 1, sq);
        cert_scale_kernel<<<nblk(n, 256), 256, 0, st>>>(n, v, sq);
        h->launches += 11;
        double hs = 0.0;
        e = cudaMemcpyAsync(&hs, sq, sizeof(double), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) break;
        est = sqrt(sqrt(hs));
        if (!std::isfinite(est)) break;
        if (prev >= 0.0 && fabs(est - prev) <= tol * est) {
            ++it;
            break;
        }
        prev = est;
    }
    for (void *p : {(void *)gr, (void *)gc, (void *)v, (void *)w, (void *)part, (void *)small, (void *)rank,
                    (void *)cpart})
        if (p) cudaFreeAsync(p, st);
    *norm = est;
    *done = it;
    return e;
}

// ------------------------------------------------------- SVD initialisation
// Section 7.5: the scaled table A~ (a_e -> (m / (sigma_j m_j)) (a_e - mu_j)
// on Omega, 0 elsewhere), its top k' singular triples by the randomized range
// finder with power iterations (Section 7.5 points to Halko et al.), and
// X = U S^1/2, Y = S^1/2 V^T diag(sigma) (plus the offset column / row).

// Scaled values in one orientation (FP64): column j's factor from its
// statistics; a column without a finite sigma_j > 0 scales to 0.
template <class T>
__global__ void svd_scale_kernel(int64_t nseg, const int32_t *__restrict__ ptr, const int32_t *__restrict__ idx,
                                 const T *__restrict__ val, bool rows, int64_t m, const int32_t *__restrict__ colptr,
                                 const double *__restrict__ mu, const double *__restrict__ s2,
                                 double *__restrict__ out)
{
    const int lane = threadIdx.x & 31;
    const int64_t s = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (s >= nseg) return;
    for (int e = ptr[s] + lane; e < ptr[s + 1]; e += 32) {
        const int64_t j = rows ? idx[e] : s;
        const double sg = sqrt(s2[j]);
        const double mj = (double)(colptr[j + 1] - colptr[j]);
        out[e] = (sg > 0.0 && sg < 1e300) ? (double)m / (sg * mj) * ((double)val[e] - mu[j]) : 0.0;
    }
}

// out (nseg x l) = segment sums of a_e In[idx_e, :] (In: other x l, FP64),
// one warp per segment, lanes over the l columns.
__global__ void svd_spmm_kernel(int64_t nseg, const int32_t *__restrict__ ptr, const int32_t *__restrict__ idx,
                                const double *__restrict__ a, const double *__restrict__ In, int l,
                                double *__restrict__ out)
{
    const int lane = threadIdx.x & 31;
    const int64_t s = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (s >= nseg) return;
    double acc[kSvdMaxL / 32];
#pragma unroll
    for (int q = 0; q < kSvdMaxL / 32; ++q) acc[q] = 0.0;
    for (int e = ptr[s]; e < ptr[s + 1]; ++e) {
        const double av = a[e];
        const double *row = In + (int64_t)idx[e] * l;
#pragma unroll
        for (int q = 0; q < kSvdMaxL / 32; ++q) {
            const int c = q * 32 + lane;
            if (c < l) acc[q] += av * row[c];
        }
    }
#pragma unroll
    for (int q = 0; q < kSvdMaxL / 32; ++q) {
        const int c = q * 32 + lane;
        if (c < l) out[s * l + c] = acc[q];
    }
}

// out rows over the chunk table (see chunk_apply_kernel): partial l-vectors
// per chunk, then per segment the sum of its chunks' partials in chunk order.
__global__ void svd_chunk_spmm_kernel(int64_t nchunks, const int4 *__restrict__ chunks,
                                      const int32_t *__restrict__ idx, const double *__restrict__ a,
                                      const double *__restrict__ In, int l, double *__restrict__ part)
{
    const int lane = threadIdx.x & 31;
    const int64_t c = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (c >= nchunks) return;
    const int4 ch = chunks[c];
    double acc[kSvdMaxL / 32];
#pragma unroll
    for (int q = 0; q < kSvdMaxL / 32; ++q) acc[q] = 0.0;
    for (int e = ch.y; e < ch.z; ++e) {
        const double av = a[e];
        const double *row = In + (int64_t)idx[e] * l;
#pragma unroll
        for (int q = 0; q < kSvdMaxL / 32; ++q) {
            const int col = q * 32 + lane;
            if (col < l) acc[q] += av * row[col];
        }
    }
#pragma unroll
    for (int q = 0; q < kSvdMaxL / 32; ++q) {
        const int col = q * 32 + lane;
        if (col < l) part[c * l + col] = acc[q];
    }
}

__global__ void svd_seg_sum_kernel(int64_t nseg, const int32_t *__restrict__ segchunk,
                                   const double *__restrict__ part, int l, double *__restrict__ out)
{
    const int lane = threadIdx.x & 31;
    const int64_t s = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (s >= nseg) return;
    for (int col = lane; col < l; col += 32) {
        double acc = 0.0;
        for (int c = segchunk[s]; c < segchunk[s + 1]; ++c) acc += part[(int64_t)c * l + col];
        out[s * l + col] = acc;
    }
}

// Pseudo-random start block (splitmix64 of the seed and the index), in [-1/2, 1/2).
__global__ void svd_random_kernel(int64_t cnt, unsigned long long seed, double *__restrict__ out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= cnt) return;
    unsigned long long z = seed + (unsigned long long)i * 0x9e3779b97f4a7c15ULL;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    z ^= z >> 31;
    out[i] = (double)(z >> 11) * 0x1p-53 - 0.5;
}

// Partial Gram matrices (all l x l entries) of a tall FP64 matrix.
__global__ void svd_gram_kernel(int64_t rows, const double *__restrict__ F, int l, double *__restrict__ part)
{
    for (int t = threadIdx.x; t < l * l; t += blockDim.x) {
        const int p = t / l, q = t % l;
        double acc = 0.0;
        if (q >= p)
            for (int64_t r = blockIdx.x; r < rows; r += gridDim.x) acc += F[r * l + p] * F[r * l + q];
        part[(int64_t)blockIdx.x * l * l + t] = acc;
    }
}

// Orthonormalising factor of a Gram matrix (upper triangle of G, l x l):
// G = V D V^T (Jacobi); R = V D^-1/2 keeping eigenvalues above 1e-13 of the
// largest (columns of the others zero), so F R has orthonormal (or zero)
// columns.  One block.
__global__ void svd_orth_kernel(const double *__restrict__ G, int l, double *__restrict__ scratch,
                                double *__restrict__ R)
{
    double *A = scratch, *V = A + l * l;
    const int r = threadIdx.x;
    if (r < l)
        for (int c = 0; c < l; ++c) A[r * l + c] = c >= r ? G[r * l + c] : G[c * l + r];
    __syncthreads();
    jacobi_eig(A, V, l);
    double mx = 0.0;
    for (int c = 0; c < l; ++c) mx = fmax(mx, A[c * l + c]);
    if (r < l)
        for (int c = 0; c < l; ++c) {
            const double d = A[c * l + c];
            R[r * l + c] = d > 1e-13 * mx && d > 0.0 ? V[r * l + c] / sqrt(d) : 0.0;
        }
}

// The top kp eigenpairs of the Gram matrix of B^T (l x l, upper triangle):
// eigenvalues s^2 descending; writes the right factors
// PX = W_top diag(s^1/2) and PY = W_top diag(s^-1/2) (l x kp each; zero for
// s below 1e-13 of the largest s^2).  One block.
__global__ void svd_top_kernel(const double *__restrict__ G, int l, int kp, double *__restrict__ scratch,
                               double *__restrict__ PX, double *__restrict__ PY, double *__restrict__ sv)
{
    double *A = scratch, *V = A + l * l;
    int *order = (int *)(V + l * l);
    const int r = threadIdx.x;
    if (r < l)
        for (int c = 0; c < l; ++c) A[r * l + c] = c >= r ? G[r * l + c] : G[c * l + r];
    __syncthreads();
    jacobi_eig(A, V, l);
    if (r == 0) {
        for (int c = 0; c < l; ++c) order[c] = c;
        for (int a = 0; a < l; ++a)  // selection sort, descending, stable
            for (int b = a + 1; b < l; ++b)
                if (A[order[b] * l + order[b]] > A[order[a] * l + order[a]]) {
                    const int t = order[a];
                    order[a] = order[b];
                    order[b] = t;
                }
    }
    __syncthreads();
    const double mx = A[order[0] * l + order[0]];
    if (r < l)
        for (int c = 0; c < kp; ++c) {
            const double d = A[order[c] * l + order[c]];
            const bool ok = d > 1e-13 * mx && d > 0.0;
            const double s = ok ? sqrt(d) : 0.0;
            PX[r * kp + c] = ok ? V[r * l + order[c]] * sqrt(s) : 0.0;
            PY[r * kp + c] = ok ? V[r * l + order[c]] / sqrt(s) : 0.0;
            if (r == 0) sv[c] = s;
        }
}

// out = In R for row-major In (rows x l) and R (l x l): rows in place.
__global__ void svd_right_kernel(int64_t rows, double *__restrict__ F, int l, const double *__restrict__ R)
{
    const int lane = threadIdx.x & 31;
    const int64_t s = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (s >= rows) return;
    double in[kSvdMaxL / 32], out[kSvdMaxL / 32];
#pragma unroll
    for (int q = 0; q < kSvdMaxL / 32; ++q) {
        const int c = q * 32 + lane;
        in[q] = c < l ? F[s * l + c] : 0.0;
        out[q] = 0.0;
    }
    for (int i = 0; i < l; ++i) {
        const double fi = __shfl_sync(0xffffffffu, in[i / 32], i % 32);
#pragma unroll
        for (int q = 0; q < kSvdMaxL / 32; ++q) {
            const int c = q * 32 + lane;
            if (c < l) out[q] += fi * R[i * l + c];
        }
    }
#pragma unroll
    for (int q = 0; q < kSvdMaxL / 32; ++q) {
        const int c = q * 32 + lane;
        if (c < l) F[s * l + c] = out[q];
    }
}

// Factor rows: dst[s, 0..kp) = scale_s * (In[s, :] P), scale_s = sigma_s (Y)
// or 1 (X); with the offset, dst[s, k-1] = 1 (X) or mu_s (Y; 0 where NaN).
template <class T>
__global__ void svd_factor_kernel(int64_t rows, const double *__restrict__ In, int l, const double *__restrict__ P,
                                  int kp, int k, const double *__restrict__ s2, const double *__restrict__ mu,
                                  bool offset, T *__restrict__ dst)
{
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= rows) return;
    double sc = 1.0;
    if (s2) {
        const double sg = sqrt(s2[s]);
        sc = (sg > 0.0 && sg < 1e300) ? sg : 1.0;
    }
    for (int c = 0; c < kp; ++c) {
        double acc = 0.0;
        for (int i = 0; i < l; ++i) acc += In[s * l + i] * P[i * kp + c];
        dst[s * k + c] = (T)(sc * acc);
    }
    for (int c = kp; c < k; ++c) {
        double v = 0.0;
        if (offset && c == k - 1) v = mu ? (mu[s] == mu[s] ? mu[s] : 0.0) : 1.0;
        dst[s * k + c] = (T)v;
    }
}

template <class T>
cudaError_t svd_init_impl(glrm_s *h, int oversample, int power_iters, unsigned long long seed, double *sv_host)
{
    cudaStream_t st = h->stream;
    const int64_t m = h->m, n = h->n, nnz = h->nnz;
    const int k = h->k, kp = h->offset ? k - 1 : k;
    const int l = std::min(kSvdMaxL, kp + oversample);
    double *mu = nullptr, *s2 = nullptr, *ar = nullptr, *ac = nullptr, *Qm = nullptr, *Qn = nullptr;
    double *part = nullptr, *small = nullptr;
    cudaError_t e = cudaSuccess;
    auto A = [&](double **p, size_t cnt) {
        if (e == cudaSuccess) e = dalloc_bytes(h, (void **)p, std::max<size_t>(cnt, 2) * sizeof(double), st);
    };
    A(&mu, n);
    A(&s2, n);
    A(&ar, nnz);
    A(&ac, nnz);
    A(&Qm, (size_t)m * l);
    A(&Qn, (size_t)n * l);
    A(&part, (size_t)kCertBlocks * l * l);
    A(&small, (size_t)6 * l * l + 3 * (size_t)l + 64);
    double *spart = nullptr;  // chunk partials of the long-segment products
    A(&spart, (size_t)std::max(h->csr.nchunks, h->csc.nchunks) * l);
    double *G = small, *R = G + l * l, *scratch = R + l * l, *PX = scratch + 2 * l * l + l, *PY = PX + l * kp;
    double *sv = PY + l * kp;
    const int bt = ((l + 31) / 32) * 32;
    auto spmm = [&](const Orient &o, int64_t nseg, const double *a, const double *In, double *out) {
        if (o.nchunks > 0 && nnz >= kLongSegment * nseg) {
            svd_chunk_spmm_kernel<<<nblk(o.nchunks, 8), 256, 0, st>>>(o.nchunks, o.chunks, o.idx, a, In, l, spart);
            svd_seg_sum_kernel<<<nblk(nseg, 8), 256, 0, st>>>(nseg, o.segchunk, spart, l, out);
            h->launches += 1;
        } else {
            svd_spmm_kernel<<<nblk(nseg, 8), 256, 0, st>>>(nseg, o.ptr, o.idx, a, In, l, out);
        }
    };
    auto orth = [&](double *F, int64_t rows) {  // F <- F (V D^-1/2) of its Gram
        svd_gram_kernel<<<kCertBlocks, 256, 0, st>>>(rows, F, l, part);
        cert_sum_kernel<<<1, 256, 0, st>>>(part, kCertBlocks, l * l, G);
        svd_orth_kernel<<<1, bt, 0, st>>>(G, l, scratch, R);
        svd_right_kernel<<<nblk(rows, 8), 256, 0, st>>>(rows, F, l, R);
        h->launches += 4;
    };
    if (e == cudaSuccess) {
        e = launch_column_stats(h, mu, s2);
        if (kp > 0) {
            const T *rv = (const T *)h->csr.val, *cv = (const T *)h->csc.val;
            svd_scale_kernel<T><<<nblk(m, 8), 256, 0, st>>>(m, h->csr.ptr, h->csr.idx, rv, true, m, h->csc.ptr, mu,
                                                            s2, ar);
            svd_scale_kernel<T><<<nblk(n, 8), 256, 0, st>>>(n, h->csc.ptr, h->csc.idx, cv, false, m, h->csc.ptr, mu,
                                                            s2, ac);
            svd_random_kernel<<<nblk(n * l, 256), 256, 0, st>>>(n * l, seed, Qn);
            spmm(h->csr, m, ar, Qn, Qm);  // A~ Omega
            h->launches += 4;
            orth(Qm, m);
            for (int it = 0; it < power_iters; ++it) {
                spmm(h->csc, n, ac, Qm, Qn);  // A~^T Q
                orth(Qn, n);
                spmm(h->csr, m, ar, Qn, Qm);  // A~ Q
                orth(Qm, m);
                h->launches += 2;
            }
            // B^T = A~^T Q (n x l); its Gram B B^T = W diag(s^2) W^T
            spmm(h->csc, n, ac, Qm, Qn);
            svd_gram_kernel<<<kCertBlocks, 256, 0, st>>>(n, Qn, l, part);
            cert_sum_kernel<<<1, 256, 0, st>>>(part, kCertBlocks, l * l, G);
            svd_top_kernel<<<1, bt, 0, st>>>(G, l, kp, scratch, PX, PY, sv);
            h->launches += 4;
        }
        // X = Q W S^1/2; Y^T = diag(sigma) B^T W S^-1/2 (A~ ~ (Q W) S (B^T W S^-1)^T)
        svd_factor_kernel<T><<<nblk(m, 256), 256, 0, st>>>(m, Qm, l, PX, kp, k, nullptr, nullptr, h->offset,
                                                           (T *)h->X);
        svd_factor_kernel<T><<<nblk(n, 256), 256, 0, st>>>(n, Qn, l, PY, kp, k, s2, mu, h->offset, (T *)h->Yt);
        h->launches += 2;
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e == cudaSuccess && sv_host && kp > 0)
            e = cudaMemcpyAsync(sv_host, sv, kp * sizeof(double), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    }
    for (double *p : {mu, s2, ar, ac, Qm, Qn, part, small, spart})
        if (p) cudaFreeAsync(p, st);
    return e;
}

}  // namespace

cudaError_t svd_init(glrm_s *h, int oversample, int power_iters, unsigned long long seed, double *sv_host)
{
    return h->prec == GLRM_FP64 ? svd_init_impl<double>(h, oversample, power_iters, seed, sv_host)
                                : svd_init_impl<float>(h, oversample, power_iters, seed, sv_host);
}

cudaError_t certificate_norm(glrm_s *h, int iters, double tol, double *norm, int *done)
{
    return h->prec == GLRM_FP64 ? certificate_impl<double>(h, iters, tol, norm, done)
                                : certificate_impl<float>(h, iters, tol, norm, done);
}

}  // namespace glrm
