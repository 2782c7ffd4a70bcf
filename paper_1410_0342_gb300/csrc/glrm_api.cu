// C ABI of libglrm (declared in include/glrm.h): handle life cycle, the
// observed set's copy, validation and chunk tables, and the entry points
// that enqueue the per-precision engines.
#include <cuda_runtime.h>
#include <math.h>

#include <cmath>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "glrm_setup.h"

using namespace glrm;

namespace {

thread_local std::string g_error;

int fail(glrm_s *h, int code, const std::string &msg)
{
    if (h) h->err = msg;
    else g_error = msg;
    return code;
}

int cuda_fail(glrm_s *h, cudaError_t e, const char *where)
{
    return fail(h, GLRM_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define CK(call)                                              \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return cuda_fail(h, e_, #call); \
    } while (0)

void free_orient(Orient &o, cudaStream_t st)
{
    dfree(o.ptr, st);
    dfree(o.idx, st);
    dfree(o.val, st);
    dfree(o.chunks, st);
    dfree(o.segchunk, st);
    dfree(o.order, st);
    dfree(o.runptr, st);
    dfree(o.tptr, st);
    dfree(o.tidx, st);
    dfree(o.tmask, st);
    dfree(o.tval, st);
    dfree(o.ubeg, st);
    dfree(o.utile, st);
    dfree(o.uvoff, st);
    o.npairs = 0;
    o.nunits = 0;
    o.nchunks = 0;
    o.maxlen = 0;
    o.mode = kModeChunked;
    o.R = o.nb = o.ngroups = o.grid = 0;
    o.smem_bytes = 0;
}

void free_scratch(Scratch &s, cudaStream_t st)
{
    dfree(s.part_grad, st); dfree(s.part_loss, st); dfree(s.part_loss2, st); dfree(s.cand, st);
    dfree(s.f_old, st); dfree(s.r_old, st); dfree(s.r_new, st);
    dfree(s.kept_obj_x, st); dfree(s.kept_reg_x, st); dfree(s.kept_obj_y, st); dfree(s.kept_reg_y, st);
    dfree(s.acc_x, st); dfree(s.acc_y, st); dfree(s.red_part, st); dfree(s.red_cnt, st);
    dfree(s.hist, st); dfree(s.accepts, st); dfree(s.scalar, st); dfree(s.als_part, st); dfree(s.err, st);
    dfree(s.x_bf16, st); dfree(s.yt_bf16, st);
    dfree(s.conv, st); dfree(s.conv_par, st); dfree(s.conv_cnt, st);
    s.hist_cap = 0;
    s.als_bytes = 0;
}

bool prec_ok(int p) { return p == GLRM_FP64 || p == GLRM_FP32 || p == GLRM_BF16; }

// The handle's device must be current for every call.
struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
        else prev = -1;
    }
    ~DeviceGuard()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

template <class T>
cudaError_t run_half(glrm_s *h, bool xstep) { return Engine<T>::half_step(h, xstep); }

cudaError_t half_step(glrm_s *h, bool xstep)
{
    if (h->dn.on) return dense_half_step(h, xstep);
    // scaled losses (glrm_set_column_scale) on a sparse table run on the chunked path
    if (h->lscale) return h->prec == GLRM_FP64 ? run_half<double>(h, xstep) : run_half<float>(h, xstep);
    const Orient &o = xstep ? h->csr : h->csc;
    if (o.mode == kModeMasked)
        return h->prec == GLRM_FP64 ? Engine<double>::masked_half_step(h, xstep)
                                    : Engine<float>::masked_half_step(h, xstep);
    if (o.mode != kModeChunked)
        return h->prec == GLRM_FP64 ? Engine<double>::tiled_half_step(h, xstep)
                                    : Engine<float>::tiled_half_step(h, xstep);
    return h->prec == GLRM_FP64 ? run_half<double>(h, xstep) : run_half<float>(h, xstep);
}

// Padded width the staged kernels use for k (0: not supported there).
int tiled_width(int k)
{
    for (int K : {4, 8, 12, 16, 20, 24, 32})
        if (k <= K) return K;
    return 0;
}

// Pick fused / blocked / chunked for one orientation: fused when the whole
// other factor (plus, for the X-step, its loss table) fits in one CTA's shared
// memory; blocked when panels of it do and a (panel, segment) run holds 64
// entries or more on average; chunked otherwise.
// Masked tiles: count each tile's pairs; build the layout when forced or when
// a pair averages >= 8 observed lanes.  The other factor is kept whole in
// shared memory when it fits, else gathered per batch (needs k == K).  Tiles
// are split into units of P pairs only when there are too few tiles to give
// every warp of the GPU one.
int plan_masked(glrm_s *h, Orient &o, bool xstep, int force, int K, int sms, size_t budget)
{
    const size_t es = elem_size(h->prec);
    const int64_t nother = xstep ? h->n : h->m;
    const int64_t ntiles = (o.nseg + 31) / 32;
    const bool forced = force != GLRM_PATH_AUTO;
    CK(dalloc(h, &o.tptr, (size_t)(ntiles + 1) * sizeof(int32_t)));
    CK(launch_mt_count(o, nother, o.tptr, h->stream));
    std::vector<int32_t> cnt((size_t)ntiles);
    CK(cudaMemcpyAsync(cnt.data(), o.tptr, (size_t)ntiles * sizeof(int32_t), cudaMemcpyDeviceToHost,
                       h->stream));
    CK(cudaStreamSynchronize(h->stream));
    std::vector<int32_t> off((size_t)ntiles + 1);
    int64_t tot = 0;
    int32_t cmax = 0;
    for (int64_t t = 0; t < ntiles; ++t) {
        off[t] = (int32_t)tot;
        tot += cnt[t];
        cmax = std::max(cmax, cnt[t]);
    }
    off[ntiles] = (int32_t)tot;
    const double lanes = tot ? (double)h->nnz / (double)tot : 0.0;
    auto give_up = [&](const char *why) {
        dfree(o.tptr, h->stream);
        return forced ? fail(h, GLRM_ERR_ARG, why) : GLRM_OK;
    };
    if (!forced && lanes < 8.0) return give_up("");
    const size_t ring = (size_t)kRingSlotsHost * kRingBytes;
    const size_t full_fixed = ((((size_t)nother * K * es) + 15) & ~(size_t)15) +
                              (xstep ? (size_t)nother * sizeof(LossSpec) : 0);
    const size_t gather_warp = ring + 2 * 32 * (size_t)K * es;
    int warps = 0;
    bool full = false;
    for (int w = kMaskedWarps; w >= 4 && !warps; w -= 4) {
        if (full_fixed + w * ring <= budget) {
            warps = w;
            full = true;
        } else if (h->k == K && w * gather_warp <= budget) {
            warps = w;
        }
    }
    if (!warps) return give_up("masked path: the other factor neither fits in shared memory nor can be gathered (k must be a multiple of 4)");
    const int64_t slots = (int64_t)sms * warps;
    int64_t P = std::max<int64_t>(cmax, 1);
    if (force == GLRM_PATH_MASKED_SPLIT) {
        P = std::max<int64_t>(32, ((cmax + 1) / 2 + 31) & ~(int64_t)31);
    } else if (ntiles < slots) {
        P = std::max<int64_t>(256, ((tot / (2 * slots)) + 31) & ~(int64_t)31);
        if (P >= cmax) P = cmax;
    }
    std::vector<int32_t> ubeg((size_t)ntiles + 1);
    std::vector<int32_t> utile;
    int64_t nunits = 0;
    for (int64_t t = 0; t < ntiles; ++t) {
        ubeg[t] = (int32_t)nunits;
        const int64_t nu = cnt[t] ? (cnt[t] + P - 1) / P : 1;  // an empty tile keeps one unit
        for (int64_t q = 0; q < nu; ++q) utile.push_back((int32_t)t);
        nunits += nu;
    }
    ubeg[ntiles] = (int32_t)nunits;
    o.full = full;
    o.warps = warps;
    o.P = (int)P;
    o.nunits = nunits;
    o.npairs = tot;
    CK(cudaMemcpyAsync(o.tptr, off.data(), off.size() * sizeof(int32_t), cudaMemcpyHostToDevice,
                       h->stream));
    CK(dalloc(h, &o.tidx, (size_t)std::max<int64_t>(tot, 1) * sizeof(int32_t)));
    CK(dalloc(h, &o.tmask, (size_t)std::max<int64_t>(tot, 1) * sizeof(uint32_t)));
    CK(dalloc(h, &o.tval, ((size_t)h->nnz + kPad) * es));
    CK(cudaMemsetAsync(o.tval, 0, ((size_t)h->nnz + kPad) * es, h->stream));
    CK(dalloc(h, &o.ubeg, ubeg.size() * sizeof(int32_t)));
    CK(dalloc(h, &o.utile, (size_t)nunits * sizeof(int32_t)));
    CK(dalloc(h, &o.uvoff, (size_t)nunits * sizeof(int32_t)));
    CK(cudaMemcpyAsync(o.ubeg, ubeg.data(), ubeg.size() * sizeof(int32_t), cudaMemcpyHostToDevice,
                       h->stream));
    CK(cudaMemcpyAsync(o.utile, utile.data(), utile.size() * sizeof(int32_t), cudaMemcpyHostToDevice,
                       h->stream));
    // empty tiles never reach the emit loop: their single unit starts at
    // the tile's first value
    std::vector<int32_t> uvoff0((size_t)nunits, 0);
    {
        std::vector<int32_t> ptr((size_t)o.nseg + 1);
        CK(cudaMemcpyAsync(ptr.data(), o.ptr, ptr.size() * sizeof(int32_t), cudaMemcpyDeviceToHost,
                           h->stream));
        CK(cudaStreamSynchronize(h->stream));
        for (int64_t t = 0; t < ntiles; ++t) uvoff0[ubeg[t]] = ptr[(size_t)(t * 32)];
    }
    CK(cudaMemcpyAsync(o.uvoff, uvoff0.data(), uvoff0.size() * sizeof(int32_t), cudaMemcpyHostToDevice,
                       h->stream));
    CK(launch_mt_build(o, h->prec, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    o.mode = kModeMasked;
    o.smem_bytes = full ? full_fixed + (size_t)warps * ring : (size_t)warps * gather_warp;
    o.grid = (int)std::max<int64_t>(1, std::min<int64_t>((nunits + warps - 1) / warps, (int64_t)sms));
    return GLRM_OK;
}

int choose_mode(glrm_s *h, Orient &o, bool xstep, int force)
{
    int dev = h->device, optin = 0, sms = 0;
    CK(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    dfree(o.runptr, h->stream);
    dfree(o.tptr, h->stream);
    dfree(o.tidx, h->stream);
    dfree(o.tmask, h->stream);
    dfree(o.tval, h->stream);
    dfree(o.ubeg, h->stream);
    dfree(o.utile, h->stream);
    dfree(o.uvoff, h->stream);
    const int K = tiled_width(h->k);
    o.mode = kModeChunked;
    if (force == GLRM_PATH_CHUNKED) return GLRM_OK;
    if (h->prec == GLRM_BF16) {  // the BF16 form runs on the chunked path
        if (force == GLRM_PATH_AUTO) return GLRM_OK;
        return fail(h, GLRM_ERR_ARG, "the BF16 form runs on the chunked path only");
    }
    if (K == 0 || h->nnz == 0) {
        if (force == GLRM_PATH_AUTO) return GLRM_OK;
        return fail(h, GLRM_ERR_ARG, "the staged paths need 1 <= k <= 32 and a non-empty Omega");
    }
    const size_t es = elem_size(h->prec);
    const int64_t nother = xstep ? h->n : h->m;
    const size_t per_row = (size_t)K * es + (xstep ? sizeof(LossSpec) : 0);
    const size_t budget = (size_t)optin - 1024;
    if (force == GLRM_PATH_AUTO || force == GLRM_PATH_MASKED || force == GLRM_PATH_MASKED_SPLIT) {
        int rc = plan_masked(h, o, xstep, force, K, sms, budget);
        if (rc != GLRM_OK || o.mode == kModeMasked || force != GLRM_PATH_AUTO) return rc;
    }
    // per warp: two staging buffers of `cap` (index, value) pairs
    const size_t per_cap = (size_t)kStreamWarps * 2 * (sizeof(int32_t) + es);
    const size_t panel_all = ((((size_t)nother * K * es) + 15) & ~(size_t)15) +
                             (xstep ? (size_t)nother * sizeof(LossSpec) : 0);
    const int cap_fused =
        panel_all < budget ? (int)std::min<size_t>(1024, ((budget - panel_all) / per_cap) & ~(size_t)3) : 0;
    const bool fused_ok = cap_fused >= 64;
    if (force == GLRM_PATH_FUSED && !fused_ok)
        return fail(h, GLRM_ERR_ARG, "fused path: the other factor does not fit in shared memory");
    if (force == GLRM_PATH_FUSED || (force == GLRM_PATH_AUTO && fused_ok && o.maxlen <= 8192)) {
        o.mode = kModeFused;
        o.cap = cap_fused;
        o.smem_bytes = panel_all + per_cap * cap_fused;
        const int64_t want = (o.nseg + kStreamWarps - 1) / kStreamWarps;
        o.grid = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)sms));
        return GLRM_OK;
    }
    // blocked: 1024-entry buffers, panels from what is left, runs kept under
    // about 80% of a buffer on average
    const int cap = 1024;
    const double density = (double)h->nnz / ((double)o.nseg * (double)nother);
    const size_t left = budget > per_cap * cap ? budget - per_cap * cap : 0;
    int64_t R = (int64_t)std::min<double>((double)(left / per_row), 0.8 * cap / std::max(density, 1e-12));
    R &= ~(int64_t)31;
    if (force == GLRM_PATH_BLOCKED && R >= 32) {
        // forced: at least two panels when the factor allows, so the partial
        // reduction over panels is exercised
        const int64_t half = ((nother + 1) / 2 + 31) & ~(int64_t)31;
        R = std::max<int64_t>(32, std::min<int64_t>(R, half));
    }
    if (R < 32) {
        if (force == GLRM_PATH_AUTO) return GLRM_OK;
        return fail(h, GLRM_ERR_ARG, "blocked path: shared memory too small");
    }
    const int nb = (int)((nother + R - 1) / R);
    const double avg_run = (double)h->nnz / ((double)nb * (double)o.nseg);
    if (force == GLRM_PATH_AUTO && avg_run < 64.0) return GLRM_OK;
    o.mode = kModeBlocked;
    o.R = (int)R;
    o.nb = nb;
    o.cap = cap;
    o.grid = sms;
    o.ngroups = (int)std::max<int64_t>(1, std::min<int64_t>(o.nseg, (4LL * sms + nb - 1) / nb));
    o.smem_bytes = (((size_t)R * K * es + 15) & ~(size_t)15) + (xstep ? (size_t)R * sizeof(LossSpec) : 0) +
                   per_cap * cap;
    CK(dalloc(h, &o.runptr, (size_t)(nb + 1) * o.nseg * sizeof(int32_t)));
    CK(launch_build_runptr(o, h->stream));
    return GLRM_OK;
}

cudaError_t reduce_sweep(glrm_s *h, double *slot)
{
    return h->prec == GLRM_FP64 ? Engine<double>::reduce_sweep(h, slot)
                                : Engine<float>::reduce_sweep(h, slot);
}

// Chunk table of one orientation from its (host) pointer array.
void build_chunks(const std::vector<int32_t> &ptr, std::vector<int4> &chunks,
                  std::vector<int32_t> &segchunk, int32_t &maxlen)
{
    const int64_t nseg = (int64_t)ptr.size() - 1;
    segchunk.resize(nseg + 1);
    chunks.clear();
    maxlen = 0;
    for (int64_t s = 0; s < nseg; ++s) {
        segchunk[s] = (int32_t)chunks.size();
        const int32_t b = ptr[s], e = ptr[s + 1];
        maxlen = std::max(maxlen, e - b);
        for (int64_t c = b; c < e; c += kChunk)
            chunks.push_back(make_int4((int)s, (int)c, (int)std::min<int64_t>(e, c + kChunk), 0));
    }
    segchunk[nseg] = (int32_t)chunks.size();
}

// Launch order of the chunked passes when the other factor does not stay in
// L2: chunk q of every segment before chunk q + 1 of any.  Within a segment
// the entries are sorted by the other index, so on tables whose segments
// spread alike over the other dimension (uniform sampling) the warps running
// at one time gather rows from one band of the other factor, which then
// stays in L2 instead of being read from HBM once per entry.
std::vector<int32_t> chunk_order(const std::vector<int4> &chunks, const std::vector<int32_t> &segchunk)
{
    std::vector<int32_t> ord(chunks.size());
    std::vector<int32_t> rank(chunks.size());
    for (size_t c = 0; c < chunks.size(); ++c) {
        ord[c] = (int32_t)c;
        rank[c] = (int32_t)c - segchunk[chunks[c].x];
    }
    std::stable_sort(ord.begin(), ord.end(), [&](int32_t a, int32_t b) { return rank[a] < rank[b]; });
    return ord;
}

// Number of partial slots an orientation's passes write (chunks, or
// panels x segments when blocked).
int64_t partial_slots(const Orient &o)
{
    if (o.mode == kModeMasked) return o.nunits * 32;
    return o.mode == kModeBlocked ? (int64_t)o.nb * o.nseg : o.nchunks;
}

// The captured sweep graph holds the buffer pointers and kernel paths of the
// moment it was captured: drop it whenever either changes.
void drop_conv_graph(glrm_s *h)
{
    if (h->conv_exec) cudaGraphExecDestroy(h->conv_exec);
    h->conv_exec = nullptr;
}

int alloc_scratch(glrm_s *h)
{
    Scratch &s = h->s;
    drop_conv_graph(h);
    free_scratch(s, h->stream);
    const size_t es = elem_size(h->prec);
    int64_t nch = std::max<int64_t>(1, std::max(partial_slots(h->csr), partial_slots(h->csc)));
    // the chunked passes (objective, gradient, weighted half-steps) write one
    // slot per chunk whatever path the half-steps take
    nch = std::max<int64_t>(nch, std::max(h->csr.nchunks, h->csc.nchunks));
    if (h->dn.on) nch = std::max<int64_t>(nch, h->dn.slots);
    const int Kt = std::max(h->k, tiled_width(h->k));
    const int64_t mx = std::max(h->m, h->n);
    CK(dalloc(h, &s.part_grad, (size_t)nch * Kt * es));
    CK(dalloc(h, &s.part_loss, (size_t)nch * sizeof(double)));
    CK(dalloc(h, &s.part_loss2, (size_t)nch * sizeof(double)));
    CK(dalloc(h, &s.cand, (size_t)mx * h->k * es));
    CK(dalloc(h, &s.f_old, (size_t)mx * sizeof(double)));
    CK(dalloc(h, &s.r_old, (size_t)mx * sizeof(double)));
    CK(dalloc(h, &s.r_new, (size_t)mx * sizeof(double)));
    CK(dalloc(h, &s.kept_obj_x, (size_t)h->m * sizeof(double)));
    CK(dalloc(h, &s.kept_reg_x, (size_t)h->m * sizeof(double)));
    CK(dalloc(h, &s.kept_obj_y, (size_t)h->n * sizeof(double)));
    CK(dalloc(h, &s.kept_reg_y, (size_t)h->n * sizeof(double)));
    CK(dalloc(h, &s.acc_x, (size_t)h->m * sizeof(int32_t)));
    CK(dalloc(h, &s.acc_y, (size_t)h->n * sizeof(int32_t)));
    CK(dalloc(h, &s.red_part, kRedBlocks * sizeof(double)));
    CK(dalloc(h, &s.red_cnt, 2 * kRedBlocks * sizeof(long long)));
    CK(dalloc(h, &s.accepts, 2 * sizeof(long long)));
    CK(dalloc(h, &s.scalar, sizeof(double)));
    CK(dalloc(h, &s.err, sizeof(int)));
    CK(dalloc(h, &s.conv, 2 * sizeof(double)));
    CK(dalloc(h, &s.conv_par, 4 * sizeof(double)));
    CK(dalloc(h, &s.conv_cnt, 3 * sizeof(int)));
    if (h->prec == GLRM_BF16) {
        CK(dalloc(h, &s.x_bf16, (size_t)h->m * h->k * sizeof(__nv_bfloat16)));
        CK(dalloc(h, &s.yt_bf16, (size_t)h->n * h->k * sizeof(__nv_bfloat16)));
    }
    // every segment's previous step counts as accepted (the BF16 form's first
    // gradients then come from its BF16 rows)
    CK(launch_fill_i32(s.acc_x, h->m, 1, h->stream));
    CK(launch_fill_i32(s.acc_y, h->n, 1, h->stream));
    CK(cudaMemsetAsync(s.accepts, 0, 2 * sizeof(long long), h->stream));
    CK(cudaMemsetAsync(s.err, 0, sizeof(int), h->stream));
    return GLRM_OK;
}

int ensure_hist(glrm_s *h, int n)
{
    if (h->s.hist_cap >= n) return GLRM_OK;
    drop_conv_graph(h);
    dfree(h->s.hist, h->stream);
    CK(dalloc(h, &h->s.hist, (size_t)n * sizeof(double)));
    h->s.hist_cap = n;
    return GLRM_OK;
}

const char *flag_message(int f)
{
    if (f & 1) return "pointer array not monotone, not starting at 0 or not ending at nnz";
    if (f & 2) return "index out of range";
    if (f & 4) return "indices within a row/column not strictly ascending (unsorted or duplicate)";
    if (f & 16) return "a CSC entry has no CSR counterpart";
    if (f & 32) return "CSR and CSC values differ for the same entry";
    if (f & 64) return "a value outside its column loss's domain (Boolean: -1 or +1; ordinal: integer in 1..d)";
    return "invalid observed set";
}

// Density from which an FP32 observed set is stored densely (NaN marking the
// missing cells) and swept by the tensor-core form: the dense passes cost
// about 13 ps per cell against about 30 ps per observed entry for the masked
// sparse path (mixed table, k = 20, measured on GB300).
constexpr double kDenseAutoDensity = 0.4;

// Whether the observed set goes to the dense form: 1 yes, 0 no, else a
// GLRM error code (a dense request the model cannot take).
int dense_choice(glrm_s *h)
{
    const bool force_dense = h->path_x == GLRM_PATH_DENSE || h->path_y == GLRM_PATH_DENSE;
    if (force_dense) {
        if ((h->path_x != GLRM_PATH_DENSE && h->path_x != GLRM_PATH_AUTO) ||
            (h->path_y != GLRM_PATH_DENSE && h->path_y != GLRM_PATH_AUTO))
            return fail(h, GLRM_ERR_ARG, "the dense path runs both half-steps");
        if ((h->prec != GLRM_FP32 && h->prec != GLRM_BF16) || !dense_supported(h->k))
            return fail(h, GLRM_ERR_ARG, "the dense path needs an FP32 or BF16 model with k <= 64");
        return 1;
    }
    if (h->path_x == GLRM_PATH_AUTO && h->path_y == GLRM_PATH_AUTO &&
        (h->prec == GLRM_FP32 || h->prec == GLRM_BF16) &&
        dense_supported(h->k) && (double)h->nnz >= kDenseAutoDensity * (double)h->m * (double)h->n) {
        size_t free_b = 0, total_b = 0;
        CK(cudaMemGetInfo(&free_b, &total_b));
        return (double)h->m * (double)((h->n + 3) / 4 * 4) * 4.0 <= 0.5 * (double)free_b ? 1 : 0;
    }
    return 0;
}

// Set up the kernel paths of an observed set (CSR / CSC and their chunk tables
// already built): the dense form, or a sparse path per half-step.  preA: the
// dense table already built from the CSR arrays (pitch (n + 3) / 4 * 4), taken
// over by the dense form (or freed if the sparse paths are chosen).
int configure_paths(glrm_s *h, float *preA = nullptr)
{
    const int choice = dense_choice(h);
    if (choice < 0) {
        if (preA) cudaFreeAsync(preA, h->stream);
        return choice;
    }
    const bool dense = choice == 1;
    dense_free(h);
    if (preA && !dense) {
        cudaFreeAsync(preA, h->stream);
        preA = nullptr;
    }
    if (!dense) {
        int rc = choose_mode(h, h->csr, true, h->path_x);
        if (rc == GLRM_OK) rc = choose_mode(h, h->csc, false, h->path_y);
        return rc;
    }
    // the chunk tables stay (ALS runs on them); the tile layouts go
    int rc = choose_mode(h, h->csr, true, GLRM_PATH_CHUNKED);
    if (rc == GLRM_OK) rc = choose_mode(h, h->csc, false, GLRM_PATH_CHUNKED);
    if (rc != GLRM_OK) return rc;
    Dense &d = h->dn;
    d.lda = (h->n + 3) / 4 * 4;
    cudaError_t e = cudaSuccess;
    if (preA) {
        d.A = preA;
    } else {
        CK(dalloc(h, &d.A, std::max<size_t>((size_t)h->m * d.lda * sizeof(float), 16)));
        e = launch_dense_scatter(h, d.A, d.lda, h->stream);
    }
    if (e == cudaSuccess) e = dense_prepare(h);
    if (e != cudaSuccess) {
        dense_free(h);
        return cuda_fail(h, e, "dense set-up");
    }
    d.missing = true;
    d.on = true;
    return GLRM_OK;
}

// csc_given false: only the CSR arrays are given; the CSC orientation is
// built from them on the device after they pass validation.
int set_observed_impl(glrm_s *h, int64_t nnz, const int32_t *rp, const int32_t *ci, const void *rv,
                      const int32_t *cp, const int32_t *ri, const void *cv, cudaMemcpyKind kind,
                      bool csc_given = true)
{
    if (!h) return fail(nullptr, GLRM_ERR_ARG, "null handle");
    DeviceGuard dg(h->device);
    if (nnz < 0 || nnz >= (int64_t)INT32_MAX) return fail(h, GLRM_ERR_RANGE, "nnz must be in [0, 2^31)");
    if (!rp || (csc_given && !cp) || (nnz > 0 && (!ci || !rv || (csc_given && (!ri || !cv)))))
        return fail(h, GLRM_ERR_ARG, "null observed-set pointer");
    h->have_omega = false;
    free_orient(h->csr, h->stream);
    free_orient(h->csc, h->stream);
    dense_free(h);
    const size_t es = elem_size(h->prec);
    cudaStream_t st = h->stream;
    Orient &R = h->csr, &C = h->csc;
    R.nseg = h->m;
    C.nseg = h->n;
    h->nnz = nnz;
    // kPad extra zeroed entries let the staged kernels copy 16-byte aligned
    // supersets of any entry range.
    const size_t nz = (size_t)nnz + kPad;
    if (!h->aux) {
        CK(cudaStreamCreateWithFlags(&h->aux, cudaStreamNonBlocking));
        CK(cudaEventCreateWithFlags(&h->ev_csr, cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&h->ev_aux, cudaEventDisableTiming));
    }
    cudaStream_t au = h->aux;
    // the built CSC's column pointers (host copy; an upload source on the
    // auxiliary stream, so declared before the drain below)
    std::vector<int32_t> cpost;
    // every return below waits for the work queued on both streams, so no
    // copy from the caller's arrays is still running when the call returns
    // (an early return on invalid CSR arrays may leave CSC copies queued)
    struct Drain {
        cudaStream_t a, s;
        ~Drain()
        {
            cudaStreamSynchronize(a);
            cudaStreamSynchronize(s);
        }
    } drain{au, st};
    CK(dalloc(h, &R.ptr, (size_t)(h->m + 1) * sizeof(int32_t)));
    CK(dalloc(h, &C.ptr, (size_t)(h->n + 1) * sizeof(int32_t)));
    CK(dalloc(h, &R.idx, nz * sizeof(int32_t)));
    CK(dalloc(h, &C.idx, nz * sizeof(int32_t)));
    CK(dalloc(h, &R.val, nz * es));
    CK(dalloc(h, &C.val, nz * es));
    int *flag = nullptr;                // [0]: CSR checks, [1]: CSC checks
    unsigned long long *dig = nullptr;  // index and value digests: CSR, then CSC
    CK(dalloc(h, &flag, 2 * sizeof(int)));
    CK(dalloc(h, &dig, 4 * sizeof(unsigned long long)));
    CK(cudaMemsetAsync(flag, 0, 2 * sizeof(int), st));
    CK(cudaMemsetAsync(dig, 0, 4 * sizeof(unsigned long long), st));
    // the copies fill entries 0 .. nnz - 1; only the padding is zeroed
    CK(cudaMemsetAsync(R.idx + nnz, 0, kPad * sizeof(int32_t), st));
    CK(cudaMemsetAsync(C.idx + nnz, 0, kPad * sizeof(int32_t), st));
    CK(cudaMemsetAsync((char *)R.val + (size_t)nnz * es, 0, kPad * es, st));
    CK(cudaMemsetAsync((char *)C.val + (size_t)nnz * es, 0, kPad * es, st));
    // CSR first: its checks and chunk table run on the auxiliary stream while
    // the CSC arrays are still being copied.  From host CSR arrays alone the
    // entries come over in pieces of whole row blocks, each checked and counted
    // for the CSC build while the next one is copied (pipe).
    const bool pipe = !csc_given && kind == cudaMemcpyHostToDevice && nnz > 0;
    CK(cudaMemcpyAsync(R.ptr, rp, (size_t)(h->m + 1) * sizeof(int32_t), kind, st));
    if (nnz > 0 && !pipe) {
        CK(cudaMemcpyAsync(R.idx, ci, (size_t)nnz * sizeof(int32_t), kind, st));
        CK(cudaMemcpyAsync(R.val, rv, (size_t)nnz * es, kind, st));
    }
    CK(cudaEventRecord(h->ev_csr, st));
    if (csc_given) {
        CK(cudaMemcpyAsync(C.ptr, cp, (size_t)(h->n + 1) * sizeof(int32_t), kind, st));
        if (nnz > 0) {
            CK(cudaMemcpyAsync(C.idx, ri, (size_t)nnz * sizeof(int32_t), kind, st));
            CK(cudaMemcpyAsync(C.val, cv, (size_t)nnz * es, kind, st));
        }
    }
    CK(cudaStreamWaitEvent(au, h->ev_csr, 0));
    // validation, per orientation: pointers first (the index checks rely on
    // them), then indices, values, the loss domains and the digests; the two
    // orientations' digests are compared last
    int hf[2] = {0, 0};
    auto check = [&](int which, cudaStream_t s) -> int {
        cudaError_t e = cudaMemcpyAsync(&hf[which], flag + which, sizeof(int), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(h, e, "validation");
        return GLRM_OK;
    };
    // chunk table of one orientation, host-built from its validated pointer
    // array (read back, or the host copy when there is one)
    auto chunk_table = [&](Orient &o, int64_t nother, cudaStream_t s, const int32_t *host_ptr = nullptr) -> int {
        std::vector<int32_t> ptr(o.nseg + 1);
        if (host_ptr) {
            std::copy(host_ptr, host_ptr + o.nseg + 1, ptr.begin());
        } else {
            CK(cudaMemcpyAsync(ptr.data(), o.ptr, ptr.size() * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
        }
        std::vector<int4> chunks;
        std::vector<int32_t> segchunk;
        build_chunks(ptr, chunks, segchunk, o.maxlen);
        o.nchunks = (int64_t)chunks.size();
        CK(dalloc_on(h, &o.chunks, std::max<size_t>(1, chunks.size()) * sizeof(int4), s));
        CK(dalloc_on(h, &o.segchunk, segchunk.size() * sizeof(int32_t), s));
        if (!chunks.empty())
            CK(cudaMemcpyAsync(o.chunks, chunks.data(), chunks.size() * sizeof(int4), cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(o.segchunk, segchunk.data(), segchunk.size() * sizeof(int32_t), cudaMemcpyHostToDevice,
                           s));
        std::vector<int32_t> ord;
        if ((double)nother * h->k * (double)es > kBandBytes && !chunks.empty()) {
            ord = chunk_order(chunks, segchunk);
            CK(dalloc_on(h, &o.order, ord.size() * sizeof(int32_t), s));
            CK(cudaMemcpyAsync(o.order, ord.data(), ord.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s));
        }
        CK(cudaStreamSynchronize(s));  // the host tables go out of scope
        return GLRM_OK;
    };
    int rc = GLRM_OK;
    cudaError_t e = launch_validate_ptr(R.ptr, h->m, nnz, flag, au);
    if (e != cudaSuccess) rc = cuda_fail(h, e, "validate_ptr");
    if (rc == GLRM_OK) rc = check(0, au);
    CscBuild cb;
    bool cb_live = false;
    float *preA = nullptr;  // the dense table, when the dense form will be chosen
    const int64_t pre_lda = (h->n + 3) / 4 * 4;
    bool r_chunked = false;  // the CSR chunk table is built
    cudaEvent_t a_ready = nullptr;  // the dense table is written
    if (rc == GLRM_OK && hf[0] == 0 && pipe) {
        // the pointers are valid: pieces of row blocks, copied on the main
        // stream, checked and counted on the auxiliary one as each lands
        const int32_t *hrp = rp;
        e = csc_build_begin(h, cb, au);
        cb_live = e == cudaSuccess;
        // the dense table, when it will be chosen, is scattered piece by piece too
        if (e == cudaSuccess && dense_choice(h) == 1)
            e = dalloc_on(h, &preA, std::max<size_t>((size_t)h->m * pre_lda * sizeof(float), 16), au);
        const int64_t pieces = std::max<int64_t>(1, std::min<int64_t>({8, nnz / (8 << 20) + 1, cb.nblk}));
        const int64_t per = (cb.nblk + pieces - 1) / pieces;
        std::vector<cudaEvent_t> evs;
        for (int64_t b0 = 0; e == cudaSuccess && b0 < cb.nblk; b0 += per) {
            const int64_t b1 = std::min<int64_t>(cb.nblk, b0 + per);
            const int64_t r0 = b0 * cb.RB, r1 = std::min<int64_t>(h->m, b1 * cb.RB);
            const int64_t e0 = hrp[r0], e1 = hrp[r1];
            cudaEvent_t ev = nullptr;
            e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
            if (e != cudaSuccess) break;
            evs.push_back(ev);
            if (e1 > e0) {
                e = cudaMemcpyAsync(R.idx + e0, ci + e0, (size_t)(e1 - e0) * sizeof(int32_t), kind, st);
                if (e == cudaSuccess)
                    e = cudaMemcpyAsync((char *)R.val + (size_t)e0 * es, (const char *)rv + (size_t)e0 * es,
                                        (size_t)(e1 - e0) * es, kind, st);
            }
            if (e == cudaSuccess) e = cudaEventRecord(ev, st);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(au, ev, 0);
            if (e == cudaSuccess)
                e = launch_check_rows(R.ptr + r0, R.idx, R.val, r1 - r0, e1 - e0, h->prec, h->n, h->loss_dev, flag,
                                      au);
            if (e == cudaSuccess) e = csc_build_count(h, cb, b0, b1, au);
            if (e == cudaSuccess && preA) e = launch_dense_scatter(h, preA, pre_lda, au, r0, r1);
        }
        if (e != cudaSuccess) rc = cuda_fail(h, e, "csr pieces");
        // the CSR chunk table from the host's (validated) pointers while the
        // pieces are copied; its upload queues behind them
        if (rc == GLRM_OK) rc = chunk_table(R, h->n, st, rp);
        r_chunked = rc == GLRM_OK;
        if (rc == GLRM_OK) rc = check(0, au);
        for (cudaEvent_t ev : evs) cudaEventDestroy(ev);
    } else if (rc == GLRM_OK && hf[0] == 0) {
        e = launch_check_entries(R, true, h->n, h->n, nnz, h->prec, h->loss_dev, flag, dig, au);
        if (e != cudaSuccess) rc = cuda_fail(h, e, "validate_idx");
        if (rc == GLRM_OK) rc = check(0, au);
    }
    // the dense table needs the CSR arrays only: built here too when it will
    // be chosen and was not scattered piece by piece above (queued before the
    // CSR chunk table, whose host build overlaps it); when the CSC is built
    // here, on the main stream beside the CSC build's prefix pass, which then
    // reads its entries from it
    cudaStream_t ds = csc_given ? au : st;
    if (rc == GLRM_OK && hf[0] == 0 && !preA && dense_choice(h) == 1) {
        e = dalloc_on(h, &preA, std::max<size_t>((size_t)h->m * pre_lda * sizeof(float), 16), ds);
        if (e == cudaSuccess) e = launch_dense_scatter(h, preA, pre_lda, ds);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&a_ready, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventRecord(a_ready, ds);
        if (e != cudaSuccess) {
            if (preA) cudaFreeAsync(preA, ds);
            preA = nullptr;
            rc = cuda_fail(h, e, "dense set-up");
        }
    }
    if (rc == GLRM_OK && hf[0] == 0 && !r_chunked)
        rc = chunk_table(R, h->n, au, kind == cudaMemcpyHostToDevice ? rp : nullptr);
    if (rc == GLRM_OK && hf[0] == 0 && !csc_given) {
        // the CSC orientation from the validated CSR arrays: consistent by
        // construction, so no CSC checks or digests; its entries read from
        // the dense table's tiles when there is one
        if (cb_live) {
            e = csc_build_finish(h, cb, cpost, au, preA, pre_lda, a_ready);
            cb_live = false;
        } else {
            e = build_csc_from_csr(h, au, preA, pre_lda, a_ready);
        }
        if (e == cudaSuccess) e = cudaEventRecord(h->ev_aux, au);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(st, h->ev_aux, 0);
        if (e != cudaSuccess) rc = cuda_fail(h, e, "csc from csr");
    }
    if (rc == GLRM_OK && hf[0] == 0 && csc_given) {
        // the CSC side: on the main stream, after its copies
        e = cudaEventRecord(h->ev_aux, au);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(st, h->ev_aux, 0);
        if (e == cudaSuccess) e = launch_validate_ptr(C.ptr, h->n, nnz, flag + 1, st);
        if (e != cudaSuccess) rc = cuda_fail(h, e, "validate_ptr");
        if (rc == GLRM_OK) rc = check(1, st);
        if (rc == GLRM_OK && hf[1] == 0) {
            e = launch_check_entries(C, false, h->m, h->n, nnz, h->prec, nullptr, flag + 1, dig + 2, st);
            if (e != cudaSuccess) rc = cuda_fail(h, e, "validate_idx");
            if (rc == GLRM_OK) rc = check(1, st);
        }
        if (rc == GLRM_OK && hf[1] == 0) {
            e = launch_digest_compare(dig, flag + 1, st);
            if (e != cudaSuccess) rc = cuda_fail(h, e, "validate_cross");
            if (rc == GLRM_OK) rc = check(1, st);
        }
    }
    if (cb_live) {  // a pipelined build that did not reach its end
        dfree(cb.cnt, au);
        dfree(cb.tot, au);
    }
    dfree(flag, st);
    dfree(dig, st);
    if (a_ready) cudaEventDestroy(a_ready);  // released once its waits are done
    const int hflag = hf[0] | hf[1];
    if (preA && (rc != GLRM_OK || hflag)) {
        cudaStreamSynchronize(au);
        cudaFreeAsync(preA, st);
        preA = nullptr;
    }
    if (rc != GLRM_OK) return rc;
    if (hflag) {
        const int code = (hflag & 8) && !(hflag & ~8) ? GLRM_ERR_NONFINITE : GLRM_ERR_OMEGA;
        free_orient(R, h->stream);
        free_orient(C, h->stream);
        return fail(h, code, (hflag & 8) && !(hflag & ~8) ? "non-finite value in the observed set"
                                                        : flag_message(hflag));
    }
    const int32_t *cpost_host = !cpost.empty() ? cpost.data() : (csc_given && kind == cudaMemcpyHostToDevice ? cp : nullptr);
    if ((rc = chunk_table(C, h->m, st, cpost_host)) != GLRM_OK) {
        if (preA) cudaFreeAsync(preA, st);
        return rc;
    }
    rc = configure_paths(h, preA);
    if (rc == GLRM_OK) rc = alloc_scratch(h);
    if (rc != GLRM_OK) return rc;
    h->have_omega = true;
    e = h->prec == GLRM_FP64 ? Engine<double>::reset_steps(h) : Engine<float>::reset_steps(h);
    if (e != cudaSuccess) return cuda_fail(h, e, "reset_steps");
    CK(cudaStreamSynchronize(st));
    h->err.clear();
    return GLRM_OK;
}

// Fully observed table: Omega = every (i, j).  A copy with rows padded to a
// multiple of 4 floats (16-byte aligned rows for the bulk copies), validated
// like an observed set (finite, inside each column loss's domain).
int set_dense_impl(glrm_s *h, const void *A, int64_t lda, cudaMemcpyKind kind)
{
    if (!h) return fail(nullptr, GLRM_ERR_ARG, "null handle");
    if (!A) return fail(h, GLRM_ERR_ARG, "null table");
    if (h->prec != GLRM_FP32 && h->prec != GLRM_BF16)
        return fail(h, GLRM_ERR_ARG, "the dense form runs on GLRM_FP32 and GLRM_BF16 models");
    if (lda < h->n) return fail(h, GLRM_ERR_ARG, "lda < n");
    if (!dense_supported(h->k)) return fail(h, GLRM_ERR_RANGE, "the dense form supports k <= 64");
    DeviceGuard dg(h->device);
    h->have_omega = false;
    free_orient(h->csr, h->stream);
    free_orient(h->csc, h->stream);
    dense_free(h);
    cudaStream_t st = h->stream;
    Dense &d = h->dn;
    d.lda = (h->n + 3) / 4 * 4;
    const size_t bytes = (size_t)h->m * d.lda * sizeof(float);
    CK(dalloc(h, &d.A, std::max<size_t>(bytes, 16)));
    if (d.lda != h->n) CK(cudaMemsetAsync(d.A, 0, bytes, st));
    CK(cudaMemcpy2DAsync(d.A, (size_t)d.lda * sizeof(float), A, (size_t)lda * sizeof(float),
                         (size_t)h->n * sizeof(float), (size_t)h->m, kind, st));
    int *flag = nullptr;
    CK(dalloc(h, &flag, sizeof(int)));
    int hflag = 0;
    cudaError_t e = cudaMemsetAsync(flag, 0, sizeof(int), st);
    if (e == cudaSuccess) e = launch_dense_validate(d.A, d.lda, h->m, h->n, h->loss_dev, flag, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    dfree(flag, h->stream);
    if (e != cudaSuccess) {
        dense_free(h);
        return cuda_fail(h, e, "dense validation");
    }
    if (hflag) {
        dense_free(h);
        return fail(h, (hflag & 8) ? GLRM_ERR_NONFINITE : GLRM_ERR_OMEGA,
                    (hflag & 8) ? "non-finite value in the table" : flag_message(hflag));
    }
    h->nnz = h->m * h->n;
    h->csr.nseg = h->m;
    h->csc.nseg = h->n;
    e = dense_prepare(h);
    if (e != cudaSuccess) {
        dense_free(h);
        return cuda_fail(h, e, "dense_prepare");
    }
    d.missing = false;
    d.on = true;
    int rc = alloc_scratch(h);
    if (rc != GLRM_OK) return rc;
    h->have_omega = true;
    if ((e = dense_reset_steps(h)) != cudaSuccess) return cuda_fail(h, e, "reset_steps");
    CK(cudaStreamSynchronize(st));
    h->err.clear();
    return GLRM_OK;
}

cudaError_t reset_steps_any(glrm_s *h)
{
    if (h->dn.on && !h->dn.missing) return dense_reset_steps(h);
    return h->prec == GLRM_FP64 ? Engine<double>::reset_steps(h) : Engine<float>::reset_steps(h);
}

}  // namespace

namespace glrm {
size_t elem_size(int prec) { return prec == GLRM_FP64 ? sizeof(double) : sizeof(float); }

// Device memory of the handles: one stream-ordered pool per device that
// keeps freed blocks (a new observed set of the same sizes reuses them
// instead of paying cudaMalloc / cudaFree again); trimmed when the device's
// last handle goes.
namespace {
std::mutex g_pool_mu;
std::map<int, std::pair<cudaMemPool_t, int>> g_pools;  // device -> (pool, live handles)
}  // namespace

cudaError_t pool_acquire(int dev)
{
    std::lock_guard<std::mutex> lk(g_pool_mu);
    auto it = g_pools.find(dev);
    if (it == g_pools.end()) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t pool;
        cudaError_t e = cudaMemPoolCreate(&pool, &props);
        if (e != cudaSuccess) return e;
        uint64_t keep = UINT64_MAX;
        e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        if (e != cudaSuccess) return e;
        it = g_pools.emplace(dev, std::make_pair(pool, 0)).first;
    }
    it->second.second += 1;
    return cudaSuccess;
}

void pool_release(int dev)
{
    std::lock_guard<std::mutex> lk(g_pool_mu);
    auto it = g_pools.find(dev);
    if (it == g_pools.end()) return;
    if (--it->second.second == 0) cudaMemPoolTrimTo(it->second.first, 0);
}

cudaError_t dalloc_bytes(glrm_s *h, void **p, size_t bytes, cudaStream_t st)
{
    cudaMemPool_t pool;
    {
        std::lock_guard<std::mutex> lk(g_pool_mu);
        auto it = g_pools.find(h->device);
        if (it == g_pools.end()) return cudaErrorInitializationError;
        pool = it->second.first;
    }
    return cudaMallocFromPoolAsync(p, bytes, pool, st);
}

void tmark(glrm_s *h, const char *name)
{
    Timer &t = h->timer;
    if (!t.on) return;
    const size_t i = t.marks.size();
    if (i >= t.pool.size()) {
        cudaEvent_t ev;
        if (cudaEventCreate(&ev) != cudaSuccess) return;
        t.pool.push_back(ev);
    }
    if (cudaEventRecord(t.pool[i], h->stream) != cudaSuccess) return;
    t.marks.emplace_back(name, i);
}
}  // namespace glrm

namespace glrm {

// Convergence check after a sweep of glrm_sweep_until, one thread, FP64:
// append the sweep's objective F_t (conv[1]) to the history and stop when
//   use_ref:  F_t - F_ref <= rtol |F_ref|            (within rtol of a reference)
//   else:     F_{t-w} - F_t <= w rtol |F_t|, t >= w   (average relative decrease
//             over the last w sweeps; F_0 = conv[0], the objective at the start)
// or when the sweep limit is reached.  Stopping clears the condition of the
// enclosing WHILE graph node (graph mode) and sets the stop flag cnt[2].
// par = {rtol, F_ref, use_ref, w}; cnt = {sweeps run, sweep limit, stop flag}.
__global__ void converge_check_kernel(cudaGraphConditionalHandle cond, int graph, const double *__restrict__ par,
                                      const double *__restrict__ conv, int *__restrict__ cnt,
                                      double *__restrict__ hist)
{
    const double F = conv[1];
    const int t = cnt[0] + 1;
    hist[t - 1] = F;
    cnt[0] = t;
    const double rtol = par[0], fref = par[1];
    const int w = (int)par[3];
    bool done;
    if (par[2] != 0.0) {
        done = F - fref <= rtol * fabs(fref);
    } else if (t >= w) {
        const double Fw = t == w ? conv[0] : hist[t - w - 1];
        done = Fw - F <= (double)w * rtol * fabs(F);
    } else {
        done = false;
    }
    if (done || t >= cnt[1]) {
        cnt[2] = 1;
        if (graph) cudaGraphSetConditional(cond, 0);
    }
}
}  // namespace glrm

namespace {

// Fold the recorded marks into per-kernel totals (synchronises).
int timer_collect(glrm_s *h)
{
    Timer &t = h->timer;
    if (t.marks.empty()) return GLRM_OK;
    CK(cudaStreamSynchronize(h->stream));
    for (size_t q = 0; q + 1 < t.marks.size(); ++q) {
        if (!t.marks[q].first) continue;
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, t.pool[t.marks[q].second], t.pool[t.marks[q + 1].second]));
        auto &a = t.acc[t.marks[q].first];
        a.first += ms;
        a.second += 1;
    }
    t.marks.clear();
    return GLRM_OK;
}


// One sweep and its convergence check, enqueued on the handle's stream.
cudaError_t sweep_and_check(glrm_s *h, cudaGraphConditionalHandle cond, int graph)
{
    cudaError_t e = half_step(h, true);
    if (e == cudaSuccess) e = half_step(h, false);
    if (e == cudaSuccess) e = reduce_sweep(h, h->s.conv + 1);
    if (e != cudaSuccess) return e;
    converge_check_kernel<<<1, 1, 0, h->stream>>>(cond, graph, h->s.conv_par, h->s.conv, h->s.conv_cnt, h->s.hist);
    h->launches += 1;
    return cudaGetLastError();
}

// Capture one sweep and its check as the body of a conditional WHILE node:
// the body runs again while the check leaves the condition at 1.
cudaError_t build_conv_graph(glrm_s *h)
{
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaGraphCreate(&g, 0);
    if (e != cudaSuccess) return e;
    cudaGraphConditionalHandle cond;
    e = cudaGraphConditionalHandleCreate(&cond, g, 1, cudaGraphCondAssignDefault);
    cudaGraphNodeParams np = {};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = cond;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    if (e == cudaSuccess) e = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np);
    if (e == cudaSuccess) {
        cudaGraph_t body = np.conditional.phGraph_out[0];
        const bool timing = h->timer.on;
        h->timer.on = false;  // no per-kernel events inside the graph
        const long long l0 = h->launches;
        e = cudaStreamBeginCaptureToGraph(h->stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
        if (e == cudaSuccess) {
            const cudaError_t e2 = sweep_and_check(h, cond, 1);
            e = cudaStreamEndCapture(h->stream, &body);
            if (e2 != cudaSuccess) e = e2;
        }
        h->conv_launches = h->launches - l0;
        h->launches = l0;
        h->timer.on = timing;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&h->conv_exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        h->conv_exec = nullptr;
        cudaGetLastError();  // a failed capture leaves no sticky error behind
    }
    return e;
}

}  // namespace

extern "C" {

const char *glrm_global_error(void) { return g_error.c_str(); }

const char *glrm_last_error(glrm_t h) { return h ? h->err.c_str() : g_error.c_str(); }

int glrm_create(int64_t m, int64_t n, int32_t k, const glrm_loss *col_loss, int32_t rx_kind,
                double rx_weight, int32_t ry_kind, double ry_weight, int32_t precision, void *stream,
                glrm_t *out)
{
    g_error.clear();
    if (!out) return fail(nullptr, GLRM_ERR_ARG, "out is null");
    *out = nullptr;
    if (m < 1 || n < 1 || m >= INT32_MAX || n >= INT32_MAX)
        return fail(nullptr, GLRM_ERR_RANGE, "m and n must be in [1, 2^31)");
    if (k < 1 || k > kMaxK) return fail(nullptr, GLRM_ERR_RANGE, "k must be in [1, 64]");
    if (!prec_ok(precision)) return fail(nullptr, GLRM_ERR_ARG, "unsupported precision");
    if (!col_loss) return fail(nullptr, GLRM_ERR_ARG, "col_loss is null");
    for (int r : {rx_kind, ry_kind})
        if (r < kRegZero || r > kRegNonneg) return fail(nullptr, GLRM_ERR_ARG, "bad regulariser kind");
    if (!(rx_weight >= 0.0) || !(ry_weight >= 0.0) || !isfinite(rx_weight) || !isfinite(ry_weight))
        return fail(nullptr, GLRM_ERR_ARG, "regulariser weights must be finite and >= 0");
    std::vector<LossSpec> spec((size_t)n);
    for (int64_t j = 0; j < n; ++j) {
        const glrm_loss &L = col_loss[j];
        if (L.kind < kLossQuad || L.kind >= kLossKinds)
            return fail(nullptr, GLRM_ERR_ARG, "bad loss kind in column " + std::to_string(j));
        if (L.kind == kLossHuber && !(L.param > 0.0 && isfinite(L.param)))
            return fail(nullptr, GLRM_ERR_ARG, "Huber threshold must be > 0 (column " + std::to_string(j) + ")");
        if (L.kind == kLossQuantile && !(L.param > 0.0 && L.param < 1.0))
            return fail(nullptr, GLRM_ERR_ARG, "quantile alpha must be in (0, 1) (column " + std::to_string(j) + ")");
        if (L.kind == kLossOrdinal && (L.levels < 2 || L.levels > 1024))
            return fail(nullptr, GLRM_ERR_ARG, "ordinal levels must be in [2, 1024] (column " + std::to_string(j) + ")");
        spec[j] = LossSpec{L.kind, L.kind == kLossOrdinal ? L.levels : 0,
                           (L.kind == kLossHuber || L.kind == kLossQuantile) ? L.param : 0.0};
    }
    glrm_s *h = new (std::nothrow) glrm_s;
    if (!h) return fail(nullptr, GLRM_ERR_NOMEM, "host allocation failed");
    h->m = m;
    h->n = n;
    h->k = k;
    h->prec = precision;
    h->stream = (cudaStream_t)stream;
    h->loss_host = spec;
    h->rx_kind = rx_kind;
    h->ry_kind = ry_kind;
    h->rx_w = rx_weight;
    h->ry_w = ry_weight;
    cudaError_t e = cudaGetDevice(&h->device);
    if (e == cudaSuccess) e = pool_acquire(h->device);
    if (e == cudaSuccess) h->pooled = true;
    const size_t es = elem_size(precision);
    if (e == cudaSuccess) e = dalloc(h, &h->loss_dev, (size_t)n * sizeof(LossSpec));
    if (e == cudaSuccess) e = dalloc(h, &h->loss_f, (size_t)n * sizeof(LossSpecF));
    if (e == cudaSuccess) e = dalloc(h, &h->X, (size_t)m * k * es);
    if (e == cudaSuccess) e = dalloc(h, &h->Yt, (size_t)n * k * es);
    if (e == cudaSuccess) e = dalloc(h, &h->alpha_x, (size_t)m * es);
    if (e == cudaSuccess) e = dalloc(h, &h->alpha_y, (size_t)n * es);
    std::vector<LossSpecF> specf((size_t)n);
    for (int64_t j = 0; j < n; ++j)
        specf[(size_t)j] = LossSpecF{spec[(size_t)j].kind, spec[(size_t)j].levels, (float)spec[(size_t)j].param,
                                     (float)spec[(size_t)j].levels};
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h->loss_dev, spec.data(), (size_t)n * sizeof(LossSpec),
                            cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h->loss_f, specf.data(), (size_t)n * sizeof(LossSpecF), cudaMemcpyHostToDevice,
                            h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->X, 0, (size_t)m * k * es, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->Yt, 0, (size_t)n * k * es, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) {
        std::string msg = std::string("glrm_create: ") + cudaGetErrorString(e);
        glrm_destroy(h);
        return fail(nullptr, e == cudaErrorMemoryAllocation ? GLRM_ERR_NOMEM : GLRM_ERR_CUDA, msg);
    }
    *out = h;
    return GLRM_OK;
}

int glrm_set_observed(glrm_t h, int64_t nnz, const int32_t *rp, const int32_t *ci, const void *rv,
                      const int32_t *cp, const int32_t *ri, const void *cv)
{
    return set_observed_impl(h, nnz, rp, ci, rv, cp, ri, cv, cudaMemcpyDeviceToDevice);
}

int glrm_set_observed_host(glrm_t h, int64_t nnz, const int32_t *rp, const int32_t *ci,
                           const void *rv, const int32_t *cp, const int32_t *ri, const void *cv)
{
    return set_observed_impl(h, nnz, rp, ci, rv, cp, ri, cv, cudaMemcpyHostToDevice);
}

int glrm_set_observed_csr(glrm_t h, int64_t nnz, const int32_t *rp, const int32_t *ci, const void *rv)
{
    return set_observed_impl(h, nnz, rp, ci, rv, nullptr, nullptr, nullptr, cudaMemcpyDeviceToDevice, false);
}

int glrm_set_observed_csr_host(glrm_t h, int64_t nnz, const int32_t *rp, const int32_t *ci, const void *rv)
{
    return set_observed_impl(h, nnz, rp, ci, rv, nullptr, nullptr, nullptr, cudaMemcpyHostToDevice, false);
}

int glrm_set_dense(glrm_t h, const void *A, int64_t lda)
{
    return set_dense_impl(h, A, lda, cudaMemcpyDeviceToDevice);
}

int glrm_set_dense_host(glrm_t h, const void *A, int64_t lda)
{
    return set_dense_impl(h, A, lda, cudaMemcpyHostToDevice);
}

static int copy_factors(glrm_t h, void *X, void *Yt, const void *Xs, const void *Yts, cudaMemcpyKind kind,
                        bool sync)
{
    if (!h) return fail(nullptr, GLRM_ERR_ARG, "null handle");
    DeviceGuard dg(h->device);
    const size_t es = elem_size(h->prec);
    if (X && Xs) CK(cudaMemcpyAsync(X, Xs, (size_t)h->m * h->k * es, kind, h->stream));
    if (Yt && Yts) CK(cudaMemcpyAsync(Yt, Yts, (size_t)h->n * h->k * es, kind, h->stream));
    if (sync) CK(cudaStreamSynchronize(h->stream));
    return GLRM_OK;
}

int glrm_set_factors(glrm_t h, const void *X, const void *Yt)
{
    return h ? copy_factors(h, h->X, h->Yt, X, Yt, cudaMemcpyDeviceToDevice, false)
             : fail(nullptr, GLRM_ERR_ARG, "null handle");
}

int glrm_get_factors(glrm_t h, void *X, void *Yt)
{
    return h ? copy_factors(h, X, Yt, X ? h->X : nullptr, Yt ? h->Yt : nullptr,
                            cudaMemcpyDeviceToDevice, false)
             : fail(nullptr, GLRM_ERR_ARG, "null handle");
}

int glrm_set_factors_host(glrm_t h, const void *X, const void *Yt)
{
    return h ? copy_factors(h, h->X, h->Yt, X, Yt, cudaMemcpyHostToDevice, true)
             : fail(nullptr, GLRM_ERR_ARG, "null handle");
}

int glrm_get_factors_host(glrm_t h, void *X, void *Yt)
{
    return h ? copy_factors(h, X, Yt, X ? h->X : nullptr, Yt ? h->Yt : nullptr,
                            cudaMemcpyDeviceToHost, true)
             : fail(nullptr, GLRM_ERR_ARG, "null handle");
}

int glrm_set_offset(glrm_t h, int32_t on)
{
    if (!h) return fail(nullptr, GLRM_ERR_ARG, "null handle");
    if (h->offset != (on != 0)) drop_conv_graph(h);  // captured sweeps carry the regulariser codes
    h->offset = on != 0;
    return GLRM_OK;
}

int glrm_set_column_scale(glrm_t h, const double *w_host)
{
    if (!h) return fail(nullptr, GLRM_ERR_ARG, "null handle");
    if (h->prec == GLRM_BF16) return fail(h, GLRM_ERR_ARG, "column loss weights need a GLRM_FP32 or GLRM_FP64 model");
    DeviceGuard dg(h->device);
    drop_conv_graph(h);  // captured sweeps carry the weight pointer
    if (!w_host) {
        dfree(h->lscale, h->stream);
        return GLRM_OK;
    }
    for (int64_t j = 0; j < h->n; ++j)
        if (!(w_host[j] > 0.0) || !std::isfinite(w_host[j]))
            return fail(h, GLRM_ERR_ARG, "column loss weights must be finite and > 0");
    const size_t es = elem_size(h->prec);
    std::vector<unsigned char> buf((size_t)h->n * es);
    for (int64_t j = 0; j < h->n; ++j) {
        if (h->prec == GLRM_FP64) reinterpret_cast<double *>(buf.data())[j] = w_host[j];
        else reinterpret_cast<float *>(buf.data())[j] = (float)w_host[j];
    }
    if (!h->lscale) CK(dalloc_bytes(h, &h->lscale, buf.size(), h->stream));
    CK(cudaMemcpyAsync(h->lscale, buf.data(), buf.size(), cudaMemcpyHostToDevice, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return GLRM_OK;
}

int glrm_column_stats(glrm_t h, double *mu_dev, double *sigma2_dev)
{
    if (!h) return fail(nullptr, GLRM_ERR_ARG, "null handle");
    if (!mu_dev || !sigma2_dev) return fail(h, GLRM_ERR_ARG, "null pointer");
    if (!h->have_omega) return fail(h, GLRM_ERR_STATE, "no observed set");
    DeviceGuard dg(h->device);
    cudaError_t e = launch_column_stats(h, mu_dev, sigma2_dev);
    return e == cudaSuccess ? GLRM_OK : cuda_fail(h, e, "glrm_column_stats");
}

// ------------------------------------- certificate and regularisation path

int glrm_set_reg_weights(glrm_t h, double rx_weight, double ry_weight)
{
    if (!h) return fail(nullptr, GLRM_ERR_ARG, "null handle");
    if (!(rx_weight >= 0.0) || !(ry_weight >= 0.0) || !std::isfinite(rx_weight) || !std::isfinite(ry_weight))
        return fail(h, GLRM_ERR_ARG, "regulariser weights must be finite and >= 0");
    drop_conv_graph(h);  // captured sweeps carry the weights
    h->rx_w = rx_weight;
    h->ry_w = ry_weight;
    return GLRM_OK;
}

int glrm_certificate(glrm_t h, int32_t max_iters, double tol, double *norm_host, int32_t *iters_host)
{
    if (!h) return fail(nullptr, GLRM_ERR_ARG, "null handle");
    if (!norm_host || max_iters < 1 || !(tol >= 0.0)) return fail(h, GLRM_ERR_ARG, "bad arguments");
    if (!h->have_omega) return fail(h, GLRM_ERR_STATE, "no observed set");
    if (h->dn.on && !h->dn.missing)
        return fail(h, GLRM_ERR_STATE, "the certificate runs on an observed set, not on a dense table");
    if (h->rx_kind != kRegQuad || h->ry_kind != kRegQuad || h->rx_w != h->ry_w || !(h->rx_w > 0.0))
        return fail(h, GLRM_ERR_ARG, "the certificate needs one quadratic regulariser weight > 0 on X and Y");
    if (h->offset) return fail(h, GLRM_ERR_ARG, "the certificate does not take an offset");
    DeviceGuard dg(h->device);
    double nrm = 0.0;
    int done = 0;
    cudaError_t e = certificate_norm(h, max_iters, tol, &nrm, &done);
    if (e != cudaSuccess) return cuda_fail(h, e, "glrm_certificate");
    *norm_host = nrm;
    if (iters_host) *iters_host = done;
    return std::isfinite(nrm) ? GLRM_OK : fail(h, GLRM_ERR_NONFINITE, "non-finite certificate");
}

int glrm_regularization_path(glrm_t h, int32_t nvals, const double *gamma_host, int32_t max_sweeps, double rtol,
                             int32_t window, double *objective_host, int32_t *sweeps_host, double *cert_host,
                             int32_t cert_iters)
{
    if (!h) return fail(nullptr, GLRM_ERR_ARG, "null handle");
    if (nvals < 1 || !gamma_host || !objective_host || !sweeps_host || (cert_host && cert_iters < 1))
        return fail(h, GLRM_ERR_ARG, "bad arguments");
    for (int32_t t = 0; t < nvals; ++t)
        if (!(gamma_host[t] >= 0.0) || !std::isfinite(gamma_host[t]))
            return fail(h, GLRM_ERR_ARG, "regularisation weights must be finite and >= 0");
    for (int32_t t = 0; t < nvals; ++t) {
        int rc = glrm_set_reg_weights(h, gamma_host[t], gamma_host[t]);
        if (rc == GLRM_OK) rc = glrm_reset_steps(h);
        int32_t done = 0;
        if (rc == GLRM_OK) rc = glrm_sweep_until(h, max_sweeps, rtol, NAN, window, &done, nullptr);
        if (rc == GLRM_OK) rc = glrm_objective(h, objective_host + t);
        if (rc != GLRM_OK) return rc;
        sweeps_host[t] = done;
        if (cert_host) {
            rc = glrm_certificate(h, cert_iters, 1e-10, cert_host + t, nullptr);
            if (rc != GLRM_OK) return rc;
        }
    }
    return GLRM_OK;
}

int glrm_svd_init(glrm_t h, int32_t oversample, int32_t power_iters, uint64_t seed, double *singular_values_host)
{
    if (!h) return fail(nullptr, GLRM_ERR_ARG, "null handle");
    if (oversample < 0 || power_iters < 0 || power_iters > 100) return fail(h, GLRM_ERR_ARG, "bad arguments");
    if (!h->have_omega) return fail(h, GLRM_ERR_STATE, "no observed set");
    if (h->dn.on && !h->dn.missing)
        return fail(h, GLRM_ERR_STATE, "the SVD initialisation runs on an observed set, not on a dense table");
    if (h->offset && h->k < 1) return fail(h, GLRM_ERR_ARG, "bad rank");
    DeviceGuard dg(h->device);
    cudaError_t e = svd_init(h, oversample, power_iters, (unsigned long long)seed, singular_values_host);
    return e == cudaSuccess ? GLRM_OK : cuda_fail(h, e, "glrm_svd_init");
}

// ------------------------------------------------ multi-dimensional features

namespace {

// The features' device table (kind, levels, width, first column) and the
// embedded width; GLRM_OK or an error for a bad kind or level count.
int feature_table(int32_t nfeat, const glrm_feature *feat, std::vector<FeatDev> &F, int64_t &D, glrm_s *h)
{
    if (nfeat < 1 || !feat) return fail(h, GLRM_ERR_ARG, "need nfeat >= 1 feature descriptors");
    F.resize((size_t)nfeat);
    D = 0;
    for (int32_t j = 0; j < nfeat; ++j) {
        const glrm_feature &f = feat[j];
        int w = 0;
        if (f.kind == GLRM_FEATURE_SCALAR) w = 1;
        else if (f.kind == GLRM_FEATURE_CATEGORICAL && f.levels >= 2 && f.levels <= GLRM_FEATURE_MAX_LEVELS) w = f.levels;
        else if (f.kind == GLRM_FEATURE_ORDINAL && f.levels >= 2 && f.levels <= GLRM_FEATURE_MAX_LEVELS) w = f.levels - 1;
        else return fail(h, GLRM_ERR_ARG, "bad feature kind or level count");
        F[(size_t)j] = FeatDev{f.kind, f.levels, w, (int32_t)D};
        D += w;
        if (D >= (int64_t)INT32_MAX) return fail(h, GLRM_ERR_RANGE, "embedded width must be < 2^31");
    }
    return GLRM_OK;
}

// Embedded column pointers from the features' column pointers (host).
int64_t embedded_colptr(const std::vector<FeatDev> &F, const std::vector<int32_t> &cp, std::vector<int64_t> &ecp)
{
    ecp.assign(1, 0);
    for (size_t j = 0; j < F.size(); ++j) {
        const int64_t c = cp[j + 1] - cp[j];
        for (int l = 0; l < F[j].width; ++l) ecp.push_back(ecp.back() + c);
    }
    return ecp.back();
}

}  // namespace

int glrm_embed_losses(int32_t nfeat, const glrm_feature *feat_host, const glrm_loss *scalar_loss_host,
                      glrm_loss *out_host, int64_t *ncols_host)
{
    std::vector<FeatDev> F;
    int64_t D = 0;
    int rc = feature_table(nfeat, feat_host, F, D, nullptr);
    if (rc != GLRM_OK) return rc;
    if (ncols_host) *ncols_host = D;
    if (!out_host) return GLRM_OK;
    for (int32_t j = 0; j < nfeat; ++j) {
        const FeatDev &f = F[(size_t)j];
        if (f.kind == GLRM_FEATURE_SCALAR) {
            if (!scalar_loss_host) return fail(nullptr, GLRM_ERR_ARG, "scalar features need their losses");
            out_host[f.first] = scalar_loss_host[j];
        } else {
            for (int l = 0; l < f.width; ++l) out_host[f.first + l] = glrm_loss{GLRM_LOSS_HINGE, 0, 0.0};
        }
    }
    return GLRM_OK;
}

int glrm_embed_size(int32_t nfeat, const glrm_feature *feat_host, const int32_t *colptr_dev, int64_t *ncols_host,
                    int64_t *nnz_host, void *stream)
{
    std::vector<FeatDev> F;
    int64_t D = 0;
    int rc = feature_table(nfeat, feat_host, F, D, nullptr);
    if (rc != GLRM_OK) return rc;
    if (!colptr_dev || !ncols_host || !nnz_host) return fail(nullptr, GLRM_ERR_ARG, "null pointer");
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<int32_t> cp((size_t)nfeat + 1);
    cudaError_t e = cudaMemcpyAsync(cp.data(), colptr_dev, cp.size() * sizeof(int32_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail(nullptr, GLRM_ERR_CUDA, std::string("glrm_embed_size: ") + cudaGetErrorString(e));
    for (int32_t j = 0; j < nfeat; ++j)
        if (cp[(size_t)j + 1] < cp[(size_t)j]) return fail(nullptr, GLRM_ERR_OMEGA, "column pointers decrease");
    std::vector<int64_t> ecp;
    *nnz_host = embedded_colptr(F, cp, ecp);
    *ncols_host = D;
    return GLRM_OK;
}

int glrm_embed_features(int32_t nfeat, const glrm_feature *feat_host, int64_t m, int64_t nnz,
                        const int32_t *rowptr_dev, const int32_t *featidx_dev, const void *val_dev,
                        const int32_t *colptr_dev, const int32_t *rowidx_dev, const void *cval_dev,
                        int32_t precision, int32_t *e_rowptr_dev, int32_t *e_colidx_dev, void *e_val_dev,
                        int32_t *e_colptr_dev, int32_t *e_rowidx_dev, void *e_cval_dev, void *stream)
{
    std::vector<FeatDev> F;
    int64_t D = 0;
    int rc = feature_table(nfeat, feat_host, F, D, nullptr);
    if (rc != GLRM_OK) return rc;
    if (!prec_ok(precision)) return fail(nullptr, GLRM_ERR_ARG, "bad precision");
    if (m < 1 || nnz < 0 || nnz >= (int64_t)INT32_MAX) return fail(nullptr, GLRM_ERR_RANGE, "bad m or nnz");
    if (!rowptr_dev || !colptr_dev || !e_rowptr_dev || !e_colptr_dev ||
        (nnz > 0 && (!featidx_dev || !val_dev || !rowidx_dev || !cval_dev || !e_colidx_dev || !e_val_dev ||
                     !e_rowidx_dev || !e_cval_dev)))
        return fail(nullptr, GLRM_ERR_ARG, "null pointer");
    cudaStream_t st = (cudaStream_t)stream;
    auto cuda_err = [](cudaError_t e) {
        return fail(nullptr, e == cudaErrorMemoryAllocation ? GLRM_ERR_NOMEM : GLRM_ERR_CUDA,
                    std::string("glrm_embed_features: ") + cudaGetErrorString(e));
    };
    // host copies of the two pointer arrays: the row / column structure is
    // checked here, the embedded column pointers follow from them
    std::vector<int32_t> rp((size_t)m + 1), cp((size_t)nfeat + 1);
    cudaError_t e = cudaMemcpyAsync(rp.data(), rowptr_dev, rp.size() * sizeof(int32_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(cp.data(), colptr_dev, cp.size() * sizeof(int32_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_err(e);
    if (rp[0] != 0 || cp[0] != 0 || rp[(size_t)m] != nnz || cp[(size_t)nfeat] != nnz)
        return fail(nullptr, GLRM_ERR_OMEGA, "pointer arrays do not span nnz entries");
    int64_t maxcnt = 0;
    for (int64_t i = 0; i < m; ++i)
        if (rp[(size_t)i + 1] < rp[(size_t)i]) return fail(nullptr, GLRM_ERR_OMEGA, "row pointers decrease");
    for (int32_t j = 0; j < nfeat; ++j) {
        if (cp[(size_t)j + 1] < cp[(size_t)j]) return fail(nullptr, GLRM_ERR_OMEGA, "column pointers decrease");
        maxcnt = std::max<int64_t>(maxcnt, cp[(size_t)j + 1] - cp[(size_t)j]);
    }
    std::vector<int64_t> ecp;
    const int64_t ennz = embedded_colptr(F, cp, ecp);
    if (ennz >= (int64_t)INT32_MAX) return fail(nullptr, GLRM_ERR_RANGE, "embedded nnz must be < 2^31");
    // feature indices are checked on the device before the row counts use them
    FeatDev *Fd = nullptr;
    int64_t *cnt = nullptr;
    int *flag = nullptr;
    e = cudaMallocAsync((void **)&Fd, F.size() * sizeof(FeatDev), st);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&cnt, (size_t)m * sizeof(int64_t), st);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&flag, sizeof(int), st);
    auto release = [&]() {
        if (Fd) cudaFreeAsync(Fd, st);
        if (cnt) cudaFreeAsync(cnt, st);
        if (flag) cudaFreeAsync(flag, st);
        cudaStreamSynchronize(st);
    };
    if (e == cudaSuccess) e = cudaMemcpyAsync(Fd, F.data(), F.size() * sizeof(FeatDev), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(flag, 0, sizeof(int), st);
    int hflag = 0;
    if (e == cudaSuccess && nnz > 0) e = launch_check_index(featidx_dev, nnz, nfeat, flag, st);
    if (e == cudaSuccess && nnz > 0) e = launch_check_index(rowidx_dev, nnz, m, flag, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        release();
        return cuda_err(e);
    }
    if (hflag) {
        release();
        return fail(nullptr, GLRM_ERR_OMEGA, "feature or row index out of range");
    }
    std::vector<int64_t> hc((size_t)m);
    e = launch_embed_rowcount(m, rowptr_dev, featidx_dev, Fd, cnt, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hc.data(), cnt, hc.size() * sizeof(int64_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        release();
        return cuda_err(e);
    }
    std::vector<int32_t> erp((size_t)m + 1), ecp32(ecp.size());
    erp[0] = 0;
    for (int64_t i = 0; i < m; ++i) erp[(size_t)i + 1] = erp[(size_t)i] + (int32_t)hc[(size_t)i];
    for (size_t c = 0; c < ecp.size(); ++c) ecp32[c] = (int32_t)ecp[c];
    e = cudaMemcpyAsync(e_rowptr_dev, erp.data(), erp.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(e_colptr_dev, ecp32.data(), ecp32.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && nnz > 0)
        e = launch_embed(precision, m, nfeat, maxcnt, rowptr_dev, featidx_dev, val_dev, colptr_dev, rowidx_dev,
                         cval_dev, Fd, e_rowptr_dev, e_colidx_dev, e_val_dev, e_colptr_dev, e_rowidx_dev, e_cval_dev,
                         flag, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    release();
    if (e != cudaSuccess) return cuda_err(e);
    if (hflag) return fail(nullptr, GLRM_ERR_OMEGA, "a categorical or ordinal value is not a label 1..levels");
    return GLRM_OK;
}

int glrm_decode_features(glrm_t h, int32_t nfeat, const glrm_feature *feat_host, int64_t cnt,
                         const int32_t *rows_dev, const int32_t *feats_dev, void *out_dev)
{
    if (!h) return fail(nullptr, GLRM_ERR_ARG, "null handle");
    std::vector<FeatDev> F;
    int64_t D = 0;
    int rc = feature_table(nfeat, feat_host, F, D, h);
    if (rc != GLRM_OK) return rc;
    if (D != h->n) return fail(h, GLRM_ERR_ARG, "the features' embedded width is not the model's n");
    if (cnt < 0 || (cnt > 0 && (!rows_dev || !feats_dev || !out_dev))) return fail(h, GLRM_ERR_ARG, "bad request arrays");
    if (cnt == 0) return GLRM_OK;
    DeviceGuard dg(h->device);
    FeatDev *Fd = nullptr;
    CK(dalloc(h, &Fd, F.size() * sizeof(FeatDev)));
    cudaError_t e = cudaMemcpyAsync(Fd, F.data(), F.size() * sizeof(FeatDev), cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = launch_decode_features(h, Fd, nfeat, cnt, rows_dev, feats_dev, out_dev);
    // the host table must outlive the copy; the device one is freed in stream order
    cudaError_t e2 = cudaStreamSynchronize(h->stream);
    dfree(Fd, h->stream);
    if (e == cudaSuccess) e = e2;
    return e == cudaSuccess ? GLRM_OK : cuda_fail(h, e, "glrm_decode_features");
}

int glrm_reset_steps(glrm_t h)
{
    if (!h) return fail(nullptr, GLRM_ERR_ARG, "null handle");
    if (!h->have_omega) return fail(h, GLRM_ERR_STATE, "no observed set");
    DeviceGuard dg(h->device);
    cudaError_t e = reset_steps_any(h);
    return e == cudaSuccess ? GLRM_OK : cuda_fail(h, e, "reset_steps");
}

// Read (synchronising) and clear the handle's device status word: a bounded
// wait that expired, or an ALS factorisation that met a pivot that was not
// positive and finite, since the status was last read.
static int read_status(glrm_t h)
{
    int flag = 0;
    CK(cudaMemcpyAsync(&flag, h->s.err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    if (!flag) return GLRM_OK;
    CK(cudaMemsetAsync(h->s.err, 0, sizeof(int), h->stream));
    if (flag & kErrWait)
        return fail(h, GLRM_ERR_TIMEOUT, "a device-side wait (a staged copy or a tensor-core "
                                         "operation) did not complete within its limit; results of "
                                         "this call are invalid");
    return fail(h, GLRM_ERR_NONFINITE, "an ALS row or column system was not numerically positive "
                                       "definite (a Cholesky pivot was not positive and finite: "
                                       "Inf or huge values in the data or factors); those rows or "
                                       "columns kept their previous factor");
}

int glrm_sweep(glrm_t h, int32_t nsweeps, double *history)
{
    if (!h) return fail(nullptr, GLRM_ERR_ARG, "null handle");
    if (!h->have_omega) return fail(h, GLRM_ERR_STATE, "glrm_sweep before glrm_set_observed");
    if (nsweeps < 0) return fail(h, GLRM_ERR_ARG, "nsweeps < 0");
    if (nsweeps == 0) return GLRM_OK;
    DeviceGuard dg(h->device);
    int rc = ensure_hist(h, nsweeps);
    if (rc != GLRM_OK) return rc;
    for (int t = 0; t < nsweeps; ++t) {
        cudaError_t e = half_step(h, true);
        if (e == cudaSuccess) e = half_step(h, false);
        if (e == cudaSuccess) e = reduce_sweep(h, h->s.hist + t);
        if (e != cudaSuccess) return cuda_fail(h, e, "glrm_sweep");
        h->sweeps_done++;
    }
    if (history) {
        CK(cudaMemcpyAsync(history, h->s.hist, (size_t)nsweeps * sizeof(double),
                           cudaMemcpyDeviceToHost, h->stream));
        return read_status(h);
    }
    return GLRM_OK;
}

int glrm_sweep_until(glrm_t h, int32_t max_sweeps, double rtol, double f_ref, int32_t window,
                     int32_t *sweeps_host, double *history_host)
{
    if (!h) return fail(nullptr, GLRM_ERR_ARG, "null handle");
    if (!h->have_omega) return fail(h, GLRM_ERR_STATE, "glrm_sweep_until before glrm_set_observed");
    if (max_sweeps < 1 || !(rtol >= 0.0) || window < 1 || !sweeps_host)
        return fail(h, GLRM_ERR_ARG, "bad arguments");
    DeviceGuard dg(h->device);
    int rc = ensure_hist(h, max_sweeps);
    if (rc != GLRM_OK) return rc;
    const bool use_ref = !std::isnan(f_ref);
    const double par[4] = {rtol, use_ref ? f_ref : 0.0, use_ref ? 1.0 : 0.0, (double)window};
    const int cnt[3] = {0, max_sweeps, 0};
    CK(cudaMemcpyAsync(h->s.conv_par, par, sizeof par, cudaMemcpyHostToDevice, h->stream));
    CK(cudaMemcpyAsync(h->s.conv_cnt, cnt, sizeof cnt, cudaMemcpyHostToDevice, h->stream));
    CK(cudaStreamSynchronize(h->stream));  // the two small copies come from pageable memory
    if (!use_ref) {
        // F_0: the objective before the first sweep
        rc = glrm_objective_at(h, h->X, h->Yt, h->s.conv);
        if (rc != GLRM_OK) return rc;
    }
    int ran = 0;
    if (h->prec != GLRM_BF16 && (h->conv_exec || build_conv_graph(h) == cudaSuccess)) {
        // the whole loop on the device: one graph launch
        CK(cudaGraphLaunch(h->conv_exec, h->stream));
        CK(cudaMemcpyAsync(&ran, h->s.conv_cnt, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
        CK(cudaStreamSynchronize(h->stream));
        h->launches += (long long)ran * h->conv_launches;
    } else {
        // the BF16 form keeps host-side state between sweeps (refresh
        // schedule): the device's decision is read back after every sweep
        int host_cnt[3] = {0, 0, 0};
        for (int t = 0; t < max_sweeps; ++t) {
            const cudaError_t e = sweep_and_check(h, cudaGraphConditionalHandle(), 0);
            if (e != cudaSuccess) return cuda_fail(h, e, "glrm_sweep_until");
            CK(cudaMemcpyAsync(host_cnt, h->s.conv_cnt, sizeof host_cnt, cudaMemcpyDeviceToHost, h->stream));
            CK(cudaStreamSynchronize(h->stream));
            if (host_cnt[2]) break;
        }
        ran = host_cnt[0];
    }
    h->sweeps_done += ran;
    *sweeps_host = ran;
    if (history_host && ran > 0)
        CK(cudaMemcpyAsync(history_host, h->s.hist, (size_t)ran * sizeof(double), cudaMemcpyDeviceToHost,
                           h->stream));
    return read_status(h);
}

int glrm_last_accepts(glrm_t h, int64_t *acc)
{
    if (!h || !acc) return fail(h, GLRM_ERR_ARG, "null argument");
    if (!h->have_omega) return fail(h, GLRM_ERR_STATE, "no observed set");
    DeviceGuard dg(h->device);
    long long tmp[2];
    CK(cudaMemcpyAsync(tmp, h->s.accepts, sizeof tmp, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    acc[0] = tmp[0];
    acc[1] = tmp[1];
    return GLRM_OK;
}

int glrm_objective_at(glrm_t h, const void *X, const void *Yt, double *out)
{
    if (!h) return fail(nullptr, GLRM_ERR_ARG, "null handle");
    if (!X || !Yt || !out) return fail(h, GLRM_ERR_ARG, "null pointer");
    if (!h->have_omega) return fail(h, GLRM_ERR_STATE, "no observed set");
    DeviceGuard dg(h->device);
    cudaError_t e = h->dn.on ? dense_objective_at(h, (const float *)X, (const float *)Yt, out)
                    : h->prec == GLRM_FP64
                        ? Engine<double>::objective_at(h, (const double *)X, (const double *)Yt, out)
                        : Engine<float>::objective_at(h, (const float *)X, (const float *)Yt, out);
    return e == cudaSuccess ? GLRM_OK : cuda_fail(h, e, "glrm_objective_at");
}

int glrm_objective(glrm_t h, double *out)
{
    if (!h || !out) return fail(h, GLRM_ERR_ARG, "null argument");
    if (!h->have_omega) return fail(h, GLRM_ERR_STATE, "no observed set");
    int rc = glrm_objective_at(h, h->X, h->Yt, h->s.scalar);
    if (rc != GLRM_OK) return rc;
    DeviceGuard dg(h->device);
    CK(cudaMemcpyAsync(out, h->s.scalar, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return GLRM_OK;
}

int glrm_grad_at(glrm_t h, const void *X, const void *Yt, void *GX, void *GYt, int32_t include_reg,
                 const double *scale)
{
    if (!h) return fail(nullptr, GLRM_ERR_ARG, "null handle");
    if (!X || !Yt || !GX || !GYt) return fail(h, GLRM_ERR_ARG, "null pointer");
    if (!h->have_omega) return fail(h, GLRM_ERR_STATE, "no observed set");
    if (include_reg && (h->rx_kind == kRegNonneg || h->ry_kind == kRegNonneg))
        return fail(h, GLRM_ERR_ARG, "the nonnegativity indicator has no gradient");
    DeviceGuard dg(h->device);
    cudaError_t e = h->dn.on ? dense_grad_at(h, (const float *)X, (const float *)Yt, (float *)GX, (float *)GYt,
                                             include_reg != 0, scale)
                    : h->prec == GLRM_FP64
                        ? Engine<double>::grad_at(h, (const double *)X, (const double *)Yt,
                                                  (double *)GX, (double *)GYt, include_reg != 0, scale)
                        : Engine<float>::grad_at(h, (const float *)X, (const float *)Yt, (float *)GX,
                                                 (float *)GYt, include_reg != 0, scale);
    return e == cudaSuccess ? GLRM_OK : cuda_fail(h, e, "glrm_grad_at");
}

int glrm_grad(glrm_t h, void *GX, void *GYt)
{
    if (!h) return fail(nullptr, GLRM_ERR_ARG, "null handle");
    return glrm_grad_at(h, h->X, h->Yt, GX, GYt, 0, nullptr);
}

int glrm_predict(glrm_t h, int64_t cnt, const int32_t *rows, const int32_t *cols, void *out,
                 int32_t decode)
{
    if (!h) return fail(nullptr, GLRM_ERR_ARG, "null handle");
    if (cnt < 0 || (cnt > 0 && (!rows || !cols || !out))) return fail(h, GLRM_ERR_ARG, "bad arguments");
    DeviceGuard dg(h->device);
    cudaError_t e = h->prec == GLRM_FP64
                        ? Engine<double>::predict(h, cnt, rows, cols, (double *)out, decode != 0)
                        : Engine<float>::predict(h, cnt, rows, cols, (float *)out, decode != 0);
    return e == cudaSuccess ? GLRM_OK : cuda_fail(h, e, "glrm_predict");
}

int glrm_als_sweep(glrm_t h, int32_t nsweeps, double *history)
{
    if (!h) return fail(nullptr, GLRM_ERR_ARG, "null handle");
    if (!h->have_omega) return fail(h, GLRM_ERR_STATE, "glrm_als_sweep before glrm_set_observed");
    if (nsweeps < 0) return fail(h, GLRM_ERR_ARG, "nsweeps < 0");
    if (h->dn.on && !h->dn.missing)
        return fail(h, GLRM_ERR_STATE, "ALS runs on an observed set, not on a dense table");
    if (h->offset) return fail(h, GLRM_ERR_ARG, "ALS does not take an offset (glrm_set_offset)");
    if (h->lscale) return fail(h, GLRM_ERR_ARG, "ALS does not take column loss weights (glrm_set_column_scale)");
    if (h->rx_kind != kRegQuad || h->ry_kind != kRegQuad || h->rx_w != h->ry_w || !(h->rx_w > 0.0))
        return fail(h, GLRM_ERR_ARG,
                    "ALS needs quadratic regularisers of equal weight gamma > 0 on X and Y");
    if (h->k > 32) return fail(h, GLRM_ERR_RANGE, "ALS supports k <= 32");
    for (const LossSpec &L : h->loss_host)
        if (L.kind != kLossQuad) return fail(h, GLRM_ERR_ARG, "ALS needs quadratic loss in every column");
    if (nsweeps == 0) return GLRM_OK;
    DeviceGuard dg(h->device);
    int rc = ensure_hist(h, nsweeps);
    if (rc != GLRM_OK) return rc;
    for (int t = 0; t < nsweeps; ++t) {
        cudaError_t e = h->prec == GLRM_FP64 ? Engine<double>::als_half(h, true, h->rx_w)
                                             : Engine<float>::als_half(h, true, h->rx_w);
        if (e == cudaSuccess)
            e = h->prec == GLRM_FP64 ? Engine<double>::als_half(h, false, h->ry_w)
                                     : Engine<float>::als_half(h, false, h->ry_w);
        if (e == cudaSuccess)
            e = h->prec == GLRM_FP64
                    ? Engine<double>::objective_at(h, (const double *)h->X, (const double *)h->Yt, h->s.hist + t)
                    : Engine<float>::objective_at(h, (const float *)h->X, (const float *)h->Yt, h->s.hist + t);
        if (e != cudaSuccess) return cuda_fail(h, e, "glrm_als_sweep");
        h->sweeps_done++;
    }
    if (history) {
        CK(cudaMemcpyAsync(history, h->s.hist, (size_t)nsweeps * sizeof(double),
                           cudaMemcpyDeviceToHost, h->stream));
        return read_status(h);
    }
    return GLRM_OK;
}

int glrm_proxprox_sweep(glrm_t h, int32_t nsweeps, double alpha, int32_t inner, double *history)
{
    if (!h) return fail(nullptr, GLRM_ERR_ARG, "null handle");
    if (!h->have_omega) return fail(h, GLRM_ERR_STATE, "glrm_proxprox_sweep before glrm_set_observed");
    if (nsweeps < 0 || inner < 1 || !(alpha > 0.0) || !std::isfinite(alpha))
        return fail(h, GLRM_ERR_ARG, "nsweeps >= 0, inner >= 1 and a finite alpha > 0 are required");
    if (h->dn.on && !h->dn.missing)
        return fail(h, GLRM_ERR_STATE, "prox-prox runs on an observed set, not on a dense table");
    if (h->k > 32) return fail(h, GLRM_ERR_RANGE, "prox-prox supports k <= 32");
    if (h->offset || h->lscale)
        return fail(h, GLRM_ERR_ARG, "prox-prox takes neither an offset nor column loss weights");
    for (const LossSpec &L : h->loss_host)
        if (L.kind != kLossQuad) return fail(h, GLRM_ERR_ARG, "prox-prox needs quadratic loss in every column");
    if (nsweeps == 0) return GLRM_OK;
    DeviceGuard dg(h->device);
    int rc = ensure_hist(h, nsweeps);
    if (rc != GLRM_OK) return rc;
    const bool f64 = h->prec == GLRM_FP64;
    for (int t = 0; t < nsweeps; ++t) {
        cudaError_t e = f64 ? Engine<double>::proxprox_half(h, true, alpha, inner)
                            : Engine<float>::proxprox_half(h, true, alpha, inner);
        if (e == cudaSuccess)
            e = f64 ? Engine<double>::proxprox_half(h, false, alpha, inner)
                    : Engine<float>::proxprox_half(h, false, alpha, inner);
        if (e == cudaSuccess)
            e = f64 ? Engine<double>::objective_at(h, (const double *)h->X, (const double *)h->Yt, h->s.hist + t)
                    : Engine<float>::objective_at(h, (const float *)h->X, (const float *)h->Yt, h->s.hist + t);
        if (e != cudaSuccess) return cuda_fail(h, e, "glrm_proxprox_sweep");
        h->sweeps_done++;
    }
    if (history) {
        CK(cudaMemcpyAsync(history, h->s.hist, (size_t)nsweeps * sizeof(double), cudaMemcpyDeviceToHost,
                           h->stream));
        return read_status(h);
    }
    return GLRM_OK;
}

// State layout: 8 int64 header words {magic, version, m, n, k, prec, sweeps, 0}
// then X, Yt, alpha_x, alpha_y in the model's element type.
static const int64_t kStateMagic = 0x4d524c47;  // "GLRM"

int glrm_get_state(glrm_t h, void *buf, size_t *len)
{
    if (!h || !len) return fail(h, GLRM_ERR_ARG, "null argument");
    const size_t es = elem_size(h->prec);
    const size_t need = 8 * sizeof(int64_t) + es * (size_t)((h->m + h->n) * h->k + h->m + h->n);
    if (!buf) {
        *len = need;
        return GLRM_OK;
    }
    if (*len < need) return fail(h, GLRM_ERR_ARG, "state buffer too small");
    DeviceGuard dg(h->device);
    int64_t hdr[8] = {kStateMagic, 1, h->m, h->n, h->k, h->prec, h->sweeps_done, 0};
    char *p = (char *)buf;
    memcpy(p, hdr, sizeof hdr);
    p += sizeof hdr;
    CK(cudaMemcpyAsync(p, h->X, es * h->m * h->k, cudaMemcpyDeviceToHost, h->stream));
    p += es * h->m * h->k;
    CK(cudaMemcpyAsync(p, h->Yt, es * h->n * h->k, cudaMemcpyDeviceToHost, h->stream));
    p += es * h->n * h->k;
    CK(cudaMemcpyAsync(p, h->alpha_x, es * h->m, cudaMemcpyDeviceToHost, h->stream));
    p += es * h->m;
    CK(cudaMemcpyAsync(p, h->alpha_y, es * h->n, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    *len = need;
    return GLRM_OK;
}

int glrm_set_state(glrm_t h, const void *buf, size_t len)
{
    if (!h || !buf) return fail(h, GLRM_ERR_ARG, "null argument");
    const size_t es = elem_size(h->prec);
    const size_t need = 8 * sizeof(int64_t) + es * (size_t)((h->m + h->n) * h->k + h->m + h->n);
    if (len < need) return fail(h, GLRM_ERR_ARG, "state buffer too small");
    int64_t hdr[8];
    memcpy(hdr, buf, sizeof hdr);
    if (hdr[0] != kStateMagic || hdr[1] != 1 || hdr[2] != h->m || hdr[3] != h->n || hdr[4] != h->k ||
        hdr[5] != h->prec)
        return fail(h, GLRM_ERR_ARG, "state does not match this model");
    DeviceGuard dg(h->device);
    const char *p = (const char *)buf + sizeof hdr;
    CK(cudaMemcpyAsync(h->X, p, es * h->m * h->k, cudaMemcpyHostToDevice, h->stream));
    p += es * h->m * h->k;
    CK(cudaMemcpyAsync(h->Yt, p, es * h->n * h->k, cudaMemcpyHostToDevice, h->stream));
    p += es * h->n * h->k;
    CK(cudaMemcpyAsync(h->alpha_x, p, es * h->m, cudaMemcpyHostToDevice, h->stream));
    p += es * h->m;
    CK(cudaMemcpyAsync(h->alpha_y, p, es * h->n, cudaMemcpyHostToDevice, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    h->sweeps_done = hdr[6];
    return GLRM_OK;
}

int glrm_set_path(glrm_t h, int32_t xstep_path, int32_t ystep_path)
{
    if (!h) return fail(nullptr, GLRM_ERR_ARG, "null handle");
    for (int p : {xstep_path, ystep_path})
        if (p < GLRM_PATH_AUTO || p > GLRM_PATH_DENSE) return fail(h, GLRM_ERR_ARG, "bad path");
    if (h->dn.on && !h->dn.missing) {
        for (int p : {xstep_path, ystep_path})
            if (p != GLRM_PATH_AUTO && p != GLRM_PATH_DENSE)
                return fail(h, GLRM_ERR_STATE, "a fully observed table (glrm_set_dense) has the dense path only");
        return GLRM_OK;
    }
    h->path_x = xstep_path;
    h->path_y = ystep_path;
    if (!h->have_omega) return GLRM_OK;
    DeviceGuard dg(h->device);
    CK(cudaStreamSynchronize(h->stream));
    int rc = configure_paths(h);
    if (rc == GLRM_OK) {
        // keep the fit state; only scratch depends on the paths
        const int hist_cap = h->s.hist_cap;
        rc = alloc_scratch(h);
        if (rc == GLRM_OK && hist_cap) rc = ensure_hist(h, hist_cap);
    }
    if (rc != GLRM_OK) {
        h->path_x = h->path_y = GLRM_PATH_AUTO;
        configure_paths(h);
        alloc_scratch(h);
        return rc;
    }
    CK(cudaStreamSynchronize(h->stream));
    return GLRM_OK;
}

int glrm_get_path(glrm_t h, int32_t *paths_host)
{
    if (!h || !paths_host) return fail(h, GLRM_ERR_ARG, "null argument");
    if (!h->have_omega) return fail(h, GLRM_ERR_STATE, "no observed set");
    if (h->lscale && !h->dn.on) {
        paths_host[0] = paths_host[1] = GLRM_PATH_CHUNKED;
        return GLRM_OK;
    }
    if (h->dn.on) {
        paths_host[0] = paths_host[1] = GLRM_PATH_DENSE;
        return GLRM_OK;
    }
    auto code = [](const Orient &o) {
        if (o.mode == kModeMasked)
            return o.nunits == (o.nseg + 31) / 32 ? GLRM_PATH_MASKED : GLRM_PATH_MASKED_SPLIT;
        return o.mode == kModeFused ? GLRM_PATH_FUSED
                                    : (o.mode == kModeBlocked ? GLRM_PATH_BLOCKED : GLRM_PATH_CHUNKED);
    };
    paths_host[0] = code(h->csr);
    paths_host[1] = code(h->csc);
    return GLRM_OK;
}

int glrm_timing_enable(glrm_t h, int32_t on)
{
    if (!h) return fail(nullptr, GLRM_ERR_ARG, "null handle");
    DeviceGuard dg(h->device);
    int rc = timer_collect(h);
    if (rc != GLRM_OK) return rc;
    h->timer.acc.clear();
    h->timer.on = on != 0;
    return GLRM_OK;
}

int glrm_timing_read(glrm_t h, int32_t max_kernels, char *names_host, double *ms_host,
                     int64_t *launches_host, int32_t *count_host)
{
    if (!h || !count_host) return fail(h, GLRM_ERR_ARG, "null argument");
    DeviceGuard dg(h->device);
    int rc = timer_collect(h);
    if (rc != GLRM_OK) return rc;
    int q = 0;
    for (const auto &kv : h->timer.acc) {
        if (q >= max_kernels) break;
        if (names_host) {
            strncpy(names_host + 32 * q, kv.first.c_str(), 31);
            names_host[32 * q + 31] = 0;
        }
        if (ms_host) ms_host[q] = kv.second.first;
        if (launches_host) launches_host[q] = kv.second.second;
        ++q;
    }
    *count_host = q;
    return GLRM_OK;
}

int glrm_launch_count(glrm_t h, int64_t *count_host)
{
    if (!h || !count_host) return fail(h, GLRM_ERR_ARG, "null argument");
    *count_host = h->launches;
    return GLRM_OK;
}

void glrm_destroy(glrm_t h)
{
    if (!h) return;
    {
        DeviceGuard dg(h->device);
        cudaStreamSynchronize(h->stream);
        for (cudaEvent_t ev : h->timer.pool) cudaEventDestroy(ev);
        free_orient(h->csr, h->stream);
        free_orient(h->csc, h->stream);
        dense_free(h);
        free_scratch(h->s, h->stream);
        dfree(h->loss_dev, h->stream);
        dfree(h->loss_f, h->stream);
        dfree(h->lscale, h->stream);
        dfree(h->X, h->stream);
        dfree(h->Yt, h->stream);
        dfree(h->alpha_x, h->stream);
        dfree(h->alpha_y, h->stream);
        cudaStreamSynchronize(h->stream);
        if (h->aux) cudaStreamDestroy(h->aux);
        if (h->ev_csr) cudaEventDestroy(h->ev_csr);
        if (h->ev_aux) cudaEventDestroy(h->ev_aux);
        if (h->pooled) pool_release(h->device);
    }
    delete h;
}

}  // extern "C"
