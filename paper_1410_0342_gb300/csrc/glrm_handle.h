// Host-side state behind a glrm_t handle and the per-precision engine
// interface.  Everything here is internal to libglrm.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <string>
#include <vector>

#include "glrm.h"
#include "glrm_device.cuh"

namespace glrm {

// Entries of one segment (a row in CSR, a column in CSC) are cut into chunks
// of at most kChunk entries; one warp processes one chunk.
constexpr int kChunk = 1024;
constexpr int kMaxK = 64;
constexpr int kPad = 8;  // zeroed entries after the last one in library copies of Omega
constexpr int kStreamWarps = 8;  // warps per CTA of the staged (fused / blocked / masked) kernels
constexpr int kMaskedWarps = 16;   // warps per CTA of the masked-tile kernels
constexpr int kRingSlotsHost = 8;  // value-stream ring slots per warp (masked kernels)
constexpr int kRingBytes = 1024;   // bytes per ring slot
// Other factors larger than this are walked band by band by the chunked
// passes (chunk launch order, see chunk_order) so that they stay in L2.
constexpr double kBandBytes = 32.0 * 1024 * 1024;

// How a half-step runs over one orientation (chosen at set-up):
// chunked: entries cut into chunks, the other factor gathered from global
//          memory (L1/L2); any size.
// fused:   the whole other factor staged in shared memory per CTA; one kernel.
// blocked: the other factor staged panel by panel; partials per (panel, segment).
// masked:  segments in tiles of 32 (lane = segment), the tile's union of
//          other-indices walked in order with one broadcast load per index.
constexpr int kModeChunked = 0, kModeFused = 1, kModeBlocked = 2, kModeMasked = 3;

// One orientation of Omega: CSR (segments = rows, used by the X-step) or CSC
// (segments = columns, used by the Y-step).
struct Orient {
    int64_t nseg = 0;
    int32_t *ptr = nullptr;       // nseg + 1
    int32_t *idx = nullptr;       // nnz: column (CSR) or row (CSC) of each entry
    void *val = nullptr;          // nnz values, element type of the model
    int4 *chunks = nullptr;       // {segment, begin, end, 0}
    int32_t *segchunk = nullptr;  // nseg + 1: first chunk of each segment
    int32_t *order = nullptr;     // nchunks: launch order of the chunks (null: chunk order)
    int64_t nchunks = 0;
    int32_t maxlen = 0;
    int mode = kModeChunked;
    int R = 0, nb = 0, ngroups = 0;  // blocked: panel rows, panels, segment groups
    int32_t *runptr = nullptr;       // blocked: (nb + 1) x nseg run starts
    int grid = 0;                    // fused / blocked: CTAs per launch
    int cap = 0;                     // fused / blocked: entries per staging buffer
    size_t smem_bytes = 0;           // fused / blocked / masked: dynamic shared memory
    // masked tiles: pair lists per tile of 32 segments, cut into units of at
    // most P pairs (one unit per tile: fused kernel; more: partials)
    int64_t npairs = 0;
    bool full = false;         // other factor resident in shared memory (else gathered)
    int warps = 0;             // warps per CTA of the masked kernel
    int P = 0;                 // pairs per unit
    int64_t nunits = 0;
    int32_t *tptr = nullptr;   // ntiles + 1: first pair of each tile
    int32_t *tidx = nullptr;   // npairs: other-index of each pair
    uint32_t *tmask = nullptr; // npairs: lanes holding it
    void *tval = nullptr;      // nnz + kPad values in (tile, index, lane) order
    int32_t *ubeg = nullptr;   // ntiles + 1: first unit of each tile
    int32_t *utile = nullptr;  // nunits: tile of each unit
    int32_t *uvoff = nullptr;  // nunits: first value of each unit
};

struct Scratch {
    void *part_grad = nullptr;     // max chunks x k, element type
    double *part_loss = nullptr;   // max chunks
    double *part_loss2 = nullptr;  // max chunks
    void *cand = nullptr;          // max(m, n) x k candidate factors
    double *f_old = nullptr, *r_old = nullptr, *r_new = nullptr;  // max(m, n)
    double *kept_obj_x = nullptr, *kept_reg_x = nullptr;         // m
    double *kept_obj_y = nullptr, *kept_reg_y = nullptr;         // n
    int32_t *acc_x = nullptr, *acc_y = nullptr;                  // m, n
    double *red_part = nullptr;     // kRedBlocks partial sums
    long long *red_cnt = nullptr;   // kRedBlocks x 2 partial counts
    double *hist = nullptr;         // hist_cap objective history
    long long *accepts = nullptr;   // 2
    double *scalar = nullptr;       // 1
    int hist_cap = 0;
    void *als_part = nullptr;       // ALS per-chunk Gram partials
    size_t als_bytes = 0;
    int *err = nullptr;             // device status word (kErrWait, kErrPivot bits)
    double *conv = nullptr;         // sweep_until: [0] previous objective, [1] current one
    double *conv_par = nullptr;     // sweep_until: rtol, reference objective, use-reference flag
    int *conv_cnt = nullptr;        // sweep_until: [0] sweeps run, [1] sweep limit, [2] stop flag
    __nv_bfloat16 *x_bf16 = nullptr;   // BF16 form: BF16 copies of the factors
    __nv_bfloat16 *yt_bf16 = nullptr;
};

constexpr int kRedBlocks = 304;  // 2 x 152 SMs

// One CTA's work in a dense pass: chunks q0 .. q0 + nq - 1 of the other
// dimension against own tile `tile`, the tile's part `part` of `parts`.  An
// own row / column s of the tile keeps its partial results in slot
// segchunk[s] + part; for the X-step's tiles of 128 consecutive rows that is
// base + (s - 128 tile) * parts + part (base: the tile's first slot).
struct DnItem {
    int32_t tile, part, parts, q0, nq, pad;
    int64_t base;
};

// The work items of one pass in launch order, per tile {first slot, parts}
// (first slot: X-step tiles only), and the number of partial slots.
struct ItemPlan {
    std::vector<DnItem> items;
    std::vector<int64_t> tiles;
    int64_t slots = 0;
};

struct DensePlan {
    bool ready = false;
    ItemPlan x, y;  // y.items index Y-step tiles of blocks_y; y.slots from seg_y
    std::vector<int32_t> blocks_y;  // per Y-step tile its four 32-column blocks (-1: none)
    std::vector<int32_t> seg_y;     // column -> first partial slot (n + 1 entries)
};

// Dense (fully observed) table and the tensor-core form's buffers.
struct Dense {
    bool on = false;
    bool missing = false;  // A holds NaN at cells outside Omega (a sparse table stored densely)
    float *A = nullptr;    // m x lda, lda = n rounded up to 4 (padding columns are never read)
    int64_t lda = 0;
    int KP = 0;  // k padded to a multiple of 16
    DnItem *items_x = nullptr, *items_y = nullptr;  // per-CTA work items of the X- and Y-step passes
    int32_t *blocks_y = nullptr;                    // per Y-step tile its four 32-column blocks
    int64_t nitems_x = 0, nitems_y = 0;
    __nv_bfloat16 *pk = nullptr;  // packed other factor, K-major over k (parts hi, mid, lo)
    __nv_bfloat16 *pt = nullptr;  // packed other factor, K-major over chunk rows (parts hi, mid, lo)
    int64_t pack_part = 0;        // elements per part
    int32_t *segchunk_x = nullptr, *segchunk_y = nullptr;  // segment -> first partial slot
    int64_t slots_x = 0, slots_y = 0, slots = 0;           // partial slots per half-step, the larger
    float4 *lossf = nullptr;      // n column losses in FP32 {kind bits, param, levels, group kind bits}
    alignas(64) unsigned char tmap_x[128] = {};  // CUtensorMap of A, X-step boxes
    alignas(64) unsigned char tmap_y[128] = {};  // CUtensorMap of A, Y-step boxes
};

// Optional per-launch timing: an event is recorded before every kernel launch
// (tagged with the kernel's name) and after the last one, so consecutive
// events on the handle's stream bracket exactly one kernel.
struct Timer {
    bool on = false;
    std::vector<cudaEvent_t> pool;
    std::vector<std::pair<const char *, size_t>> marks;  // name (null = stop), event
    std::map<std::string, std::pair<double, long long>> acc;  // ms, launches
};

}  // namespace glrm

struct glrm_s {
    int64_t m = 0, n = 0;
    int k = 0;
    int prec = GLRM_FP32;
    int device = 0;
    cudaStream_t stream = nullptr;
    std::vector<glrm::LossSpec> loss_host;
    glrm::LossSpec *loss_dev = nullptr;
    glrm::LossSpecF *loss_f = nullptr;  // the same losses with FP32 parameters (FP32 kernels)
    int rx_kind = 0, ry_kind = 0;
    bool offset = false;  // last coordinate of X held at 1, of Y unpenalised (glrm_set_offset)
    void *lscale = nullptr;  // n per-column loss weights, element type (glrm_set_column_scale); null: all 1
    double rx_w = 0.0, ry_w = 0.0;
    void *X = nullptr, *Yt = nullptr;          // factors
    void *alpha_x = nullptr, *alpha_y = nullptr;  // step sizes, element type
    bool have_omega = false;
    int64_t nnz = 0;
    glrm::Orient csr, csc;
    glrm::Scratch s;
    glrm::Dense dn;
    glrm::DensePlan dnplan;  // dense-pass work items (fixed by m, n and the losses)
    glrm::Timer timer;
    long long launches = 0;  // kernels enqueued since creation
    int64_t sweeps_done = 0;
    int path_x = GLRM_PATH_AUTO, path_y = GLRM_PATH_AUTO;
    std::string err;
    bool pooled = false;  // holds a reference on the device's memory pool
    // set-up helpers: a non-blocking stream for the CSR checks that overlap the
    // CSC copies, and an event to hand work between it and `stream`
    cudaStream_t aux = nullptr;
    cudaEvent_t ev_csr = nullptr, ev_aux = nullptr;
    // glrm_sweep_until: one sweep and the convergence check captured as the
    // body of a conditional WHILE graph node (rebuilt after any change of the
    // buffers or kernel paths it was captured with)
    cudaGraphExec_t conv_exec = nullptr;
    long long conv_launches = 0;  // kernels in one captured sweep
};

namespace glrm {

size_t elem_size(int prec);

// The loss table the kernels of element type T read.
template <class T> inline const LossOf<T> *loss_of(const glrm_s *h);
template <> inline const LossSpec *loss_of<double>(const glrm_s *h) { return h->loss_dev; }
template <> inline const LossSpecF *loss_of<float>(const glrm_s *h) { return h->loss_f; }

// The regulariser kind the kernels of one half-step take: the model's kind
// with the offset role of that factor above it (see reg_kind_at).
inline int reg_code(const glrm_s *h, bool xstep)
{
    const int rk = xstep ? h->rx_kind : h->ry_kind;
    return h->offset ? rk | ((xstep ? kOffsetX : kOffsetY) << 8) : rk;
}

// Handle memory: stream-ordered allocations from a per-device pool (on the
// handle's stream; freeing is ordered after the work queued before it).
cudaError_t pool_acquire(int dev);
void pool_release(int dev);
cudaError_t dalloc_bytes(glrm_s *h, void **p, size_t bytes, cudaStream_t st);
template <class P>
cudaError_t dalloc(glrm_s *h, P **p, size_t bytes)
{
    return dalloc_bytes(h, reinterpret_cast<void **>(p), bytes, h->stream);
}
// The same, ordered on another of the handle's streams.
template <class P>
cudaError_t dalloc_on(glrm_s *h, P **p, size_t bytes, cudaStream_t st)
{
    return dalloc_bytes(h, reinterpret_cast<void **>(p), bytes, st);
}
template <class P>
void dfree(P *&p, cudaStream_t st)
{
    if (p) cudaFreeAsync((void *)p, st);
    p = nullptr;
}

// Record a timing mark before the launch of kernel `name` (null closes the
// last interval).  No-op unless timing is enabled.
void tmark(glrm_s *h, const char *name);

// Per-precision launchers, instantiated for float and double in their own
// translation units.  Each returns a cudaError_t of the launches.
template <class T>
struct Engine {
    static cudaError_t half_step(glrm_s *h, bool xstep);
    static cudaError_t reduce_sweep(glrm_s *h, double *hist_slot);
    static cudaError_t objective_at(glrm_s *h, const T *X, const T *Yt, double *out);
    static cudaError_t grad_at(glrm_s *h, const T *X, const T *Yt, T *GX, T *GYt, bool reg,
                               const double *scale);
    static cudaError_t predict(glrm_s *h, int64_t cnt, const int32_t *rows, const int32_t *cols,
                               T *out, bool decode);
    static cudaError_t reset_steps(glrm_s *h);
    static cudaError_t als_half(glrm_s *h, bool xstep, double gamma);
    static cudaError_t proxprox_half(glrm_s *h, bool xstep, double alpha, int inner);
    static cudaError_t tiled_half_step(glrm_s *h, bool xstep);
    static cudaError_t masked_half_step(glrm_s *h, bool xstep);
};

// Validation of one orientation, writes bit flags into *flag (device int).
cudaError_t launch_validate_ptr(const int32_t *ptr, int64_t nseg, int64_t nnz, int *flag,
                                cudaStream_t st);
// Entry checks of one orientation in one pass (index range and order, finite
// values; loss domains when `loss` is given; the digests into digest[0..1]
// when `digest` is given).  rows: CSR; other: the index bound; n: columns.
cudaError_t launch_check_entries(const Orient &o, bool rows, int64_t other, int64_t n, int64_t nnz, int prec,
                                 const LossSpec *loss, int *flag, unsigned long long *digest, cudaStream_t st);
cudaError_t launch_digest_compare(const unsigned long long *d, int *flag, cudaStream_t st);
cudaError_t bf16_half_step_entry(glrm_s *h, bool xstep);
cudaError_t launch_fill_i32(int32_t *p, int64_t n, int32_t v, cudaStream_t st);
// Per-column statistics mu_j, sigma2_j of the loss scaling (glrm_stats.cu).
cudaError_t launch_column_stats(glrm_s *h, double *mu, double *s2);
// Tables of multi-dimensional features (glrm_features.cu): one feature's
// kind, label / level count, width of its block of Y and first column.
constexpr int kFeatScalar = 0, kFeatCategorical = 1, kFeatOrdinal = 2;
struct FeatDev {
    int32_t kind, levels, width, first;
};
// ||(1/gamma) G + U V^T||_2 by power iteration (glrm_cert.cu).
cudaError_t certificate_norm(glrm_s *h, int iters, double tol, double *norm, int *done);
// SVD initialisation of the factors (glrm_cert.cu).
cudaError_t svd_init(glrm_s *h, int oversample, int power_iters, unsigned long long seed, double *sv_host);
// The CSC arrays (C.ptr, C.idx, C.val allocated) from validated CSR ones (glrm_transpose.cu).
cudaError_t build_csc_from_csr(glrm_s *h, cudaStream_t st, const float *A = nullptr, int64_t lda = 0,
                               cudaEvent_t a_ready = nullptr);
// Raise *flag when an index lies outside [0, bound).
cudaError_t launch_check_index(const int32_t *idx, int64_t n, int64_t bound, int *flag, cudaStream_t st);
cudaError_t launch_embed_rowcount(int64_t m, const int32_t *rowptr, const int32_t *featidx, const FeatDev *F,
                                  int64_t *cnt, cudaStream_t st);
cudaError_t launch_embed(int prec, int64_t m, int64_t nf, int64_t maxcnt, const int32_t *rowptr,
                         const int32_t *featidx, const void *val, const int32_t *colptr, const int32_t *rowidx,
                         const void *cval, const FeatDev *F, const int32_t *e_rowptr, int32_t *e_colidx, void *e_val,
                         const int32_t *e_colptr, int32_t *e_rowidx, void *e_cval, int *flag, cudaStream_t st);
cudaError_t launch_decode_features(glrm_s *h, const FeatDev *F, int32_t nf, int64_t cnt, const int32_t *rows,
                                   const int32_t *feats, void *out);
// Dense, fully observed form (tensor cores, FP32 models).
bool dense_supported(int k);
void dense_free(glrm_s *h);
cudaError_t dense_prepare(glrm_s *h);
cudaError_t launch_dense_validate(const float *A, int64_t lda, int64_t m, int64_t n, const LossSpec *loss,
                                  int *flag, cudaStream_t st);
// The CSR entries of rows r0 .. r1 - 1 (r1 < 0: all rows) into those rows of
// a dense m x lda table A, NaN at every other cell (on st); column indices
// outside [0, n) are skipped.
cudaError_t launch_dense_scatter(glrm_s *h, float *A, int64_t lda, cudaStream_t st, int64_t r0 = 0,
                                 int64_t r1 = -1);
cudaError_t dense_reset_steps(glrm_s *h);
cudaError_t dense_half_step(glrm_s *h, bool xstep);
cudaError_t dense_objective_at(glrm_s *h, const float *X, const float *Yt, double *out);
cudaError_t dense_grad_at(glrm_s *h, const float *X, const float *Yt, float *GX, float *GYt, bool reg,
                          const double *scale);
cudaError_t launch_build_runptr(const Orient &o, cudaStream_t st);
cudaError_t launch_mt_count(const Orient &o, int64_t nother, int32_t *cnt, cudaStream_t st);
cudaError_t launch_mt_build(const Orient &o, int prec, cudaStream_t st);

}  // namespace glrm
