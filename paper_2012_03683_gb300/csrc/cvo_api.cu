// C ABI of libcvo (declared in include/cvo.h): argument checking, device
// scratch, the per-pair setup, and the drivers of evaluation, registration
// and batched registration.  Every step of the computation runs in this
// library's CUDA kernels; the host only orders launches and copies results.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "cvo.h"
#include "cvo_internal.cuh"

using namespace cvo;

std::atomic<long long> cvo::g_launch_count{0};
static_assert(CVO_SHARD_STATS == cvo::kShardStats, "shard statistics: header and kernels disagree");

namespace cvo {
void set_error_message(const char* msg);
}

namespace {

thread_local std::string g_err;

cvo_status fail(cvo_status s, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return s;
}

#define CVO_CUDA(call)                                                                          \
    do {                                                                                        \
        cudaError_t e_ = (call);                                                                \
        if (e_ != cudaSuccess)                                                                  \
            return fail(e_ == cudaErrorMemoryAllocation ? CVO_ERR_OOM : CVO_ERR_CUDA, "%s: %s (%s:%d)", \
                        #call, cudaGetErrorString(e_), __FILE__, __LINE__);                     \
    } while (0)

#define CVO_TRY(expr)                 \
    do {                              \
        cvo_status s_ = (expr);       \
        if (s_ < 0) return s_;        \
    } while (0)

struct DevBuf {
    void* p = nullptr;
    size_t cap = 0;
};

// A stream with its own setup scratch: the pairs of a batch are set up on
// several of these at once (their kernels are small and overlap).
constexpr int kSetupLanes = 8;
struct SetupLane {
    cudaStream_t s = nullptr;
    cudaEvent_t ev = nullptr;
    DevBuf keys, vals, keys2, vals2, sort_tmp, flags, gidx;
};

cudaError_t ensure(DevBuf& b, size_t bytes)
{
    if (bytes <= b.cap && b.p) return cudaSuccess;
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.cap = 0;
    const size_t nb = std::max<size_t>(bytes, 256);
    cudaError_t e = cudaMalloc(&b.p, nb);
    if (e == cudaSuccess) b.cap = nb;
    return e;
}

void release(DevBuf& b)
{
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.cap = 0;
}

struct LevelHost {
    double h;         // cell edge (y and z)
    double hx;        // cell edge along x (h / cell_xdiv)
    double rdesign;   // cutoff radius the level is built for (cell edge = cell_factor * rdesign)
    int nx, ny, nz;
    float ox, oy, oz;
    long long ncells;
    int shift;
    int ngroups;
    int nitems;
};

constexpr long long kMaxCells = 1LL << 26;
constexpr int kMiscWords = 64;   // bbox (12), bad flag (1), group totals (<= kMaxLevels), Z's moments (10)
constexpr int kZStatsWord = 48;  // Z's centroid, mean squared and largest radius: 5 raw 8-byte words from here
static_assert(kZStatsWord % 2 == 0 && kZStatsWord + 10 <= kMiscWords, "Z's moments must fit the scratch slot");

float decode_orderable(unsigned u)
{
    const unsigned b = (u & 0x80000000u) ? (u & 0x7fffffffu) : ~u;
    float f;
    std::memcpy(&f, &b, 4);
    return f;
}

// Device resources of one prepared pair: grid levels of Z, Hilbert-ordered
// queries of X and their groups, the iteration state.
struct PairRes {
    DevBuf xrec, hkeys, levels_dev, state;
    DevBuf in_xyz[2], in_feat[2];   // a batch's device copies of host-resident inputs (X, Z)
    DevBuf zrec[kMaxLevels], cell_start[kMaxLevels], groups[kMaxLevels], items[kMaxLevels];
    int n = 0, m = 0, nlevels = 0;
    LevelHost lv[kMaxLevels];
    LevelDesc ld[kMaxLevels];   // host copy of levels_dev
    double zc[3] = {0, 0, 0};   // centroid of Z (the lever centre)
    double zr2 = 0.0, zrmax = 0.0;
    int max_items = 1;

    void free_all()
    {
        DevBuf* bufs[] = {&xrec, &hkeys, &levels_dev, &state, &in_xyz[0], &in_xyz[1], &in_feat[0], &in_feat[1]};
        for (DevBuf* b : bufs) release(*b);
        for (int k = 0; k < kMaxLevels; ++k) {
            release(zrec[k]);
            release(cell_start[k]);
            release(groups[k]);
            release(items[k]);
        }
    }
};

}  // namespace

// Lets other translation units report an error through cvo_last_error().
void cvo::set_error_message(const char* msg) { g_err = msg ? msg : ""; }

struct cvo_handle_s {
    cvo_params p{};
    cudaStream_t s = nullptr;
    int device = 0;
    int num_sms = 152;
    int timing = 0;
    int loop_mode = 1;   // registration loop: 0 queued from the host, 1 CUDA graph, 2 persistent kernel
    // scratch shared by every pair's setup (used one pair at a time)
    DevBuf stage_xyz[2], stage_feat[2];
    DevBuf keys, vals, keys2, vals2, sort_tmp, flags, gidx, misc;
    // a batch sets its pairs up on kSetupLanes streams, each with its own
    // copy of the setup scratch (created on first use)
    SetupLane lanes[kSetupLanes];
    // sweep / finalize scratch
    DevBuf part_stats, part_cnt, grp_stats, grp_cnt, grp_arrivals, pairs_dev, counters, trace;
    DevBuf batch_work;   // per pair of a batch: work items left (the batched step re-splits the grid by them)
    DevBuf item_rows;    // a batch's work queue: one statistics row per work item
    DevBuf queue_buf;    // a batch's work queue: [0] next item, [1] items, then ibase (pairs + 1 ints)
    DevBuf batch_scratch;   // a batch's set-up: every pair's segment of the sort and scan scratch
    // many small host <-> device copies through one staging copy (upload_blocks, fetch_states)
    DevBuf d_stage;
    unsigned char* h_stage = nullptr;   // pinned, h_stage_cap bytes
    size_t h_stage_cap = 0;
    cudaEvent_t stage_ev = nullptr;     // after the last copy out of h_stage
    // gradients with respect to the inputs: device outputs for host callers,
    // per-query terms of dF/dl and their sum
    DevBuf bw_out[4], bw_tq, bw_dell, bw_part;

    std::vector<PairRes> pr;
    IterState* h_state = nullptr;   // pinned mirror(s)
    int h_state_cap = 0;
    unsigned* h_misc = nullptr;     // pinned, h_misc_cap words
    int h_misc_cap = 0;
    int last_iters = 0;
    double sweep_ms = 0.0;
    int sweep_n = 0;
    std::vector<cudaEvent_t> evs;
    // shared by the pairs of one call
    int dense = 0, rs = 1, rec_bf16 = 0, D = 0;
    FeatConst fc{};
    double kappa = 1.0;
    int sweep_blocks = 1;
    // tuning: grid cell edge = cell_factor * cutoff radius; query groups live in
    // octree super-cells about 2^super_delta cutoff radii wide
    double cell_factor = 0.5;
    int super_delta = 2;
    // work split: each query group's candidate stream is split into chunks
    // of about chunk_len candidates (work items), so up to stream / chunk_len
    // lanes of different warps serve one query
    int chunk_len = kChunkLen;
    // lanes per query in the sweep (1, 2 or 4): query groups of 32 / query_lanes
    // queries, each query's candidates shared among its lanes
    int query_lanes = 1;
    // grid cells along x (the rows whose runs the sweep streams) up to
    // cell_xdiv times shorter than across: the runs' ends trim closer to the
    // query group's ball-grown box, and the number of runs stays the same
    int cell_xdiv = 4;
    // an X-row shard registration in progress (cvo_shard_begin .. cvo_shard_end)
    int shard_active = 0;
    // failure injection for the next persistent registration (cvo_inject_barrier_stall)
    int inj_leave_at = -1;
    unsigned inj_polls = 0;
    int shard_nb = 0;
    SweepArgs shard_a{};
    LevelDesc* shard_levels = nullptr;   // non-NULL: the items are re-planned beside every step
};

namespace {

cvo_status check_params(const cvo_params* p)
{
    if (!p) return fail(CVO_ERR_INVALID_ARG, "params is NULL");
    if (!(p->ell > 0.0) || !std::isfinite(p->ell)) return fail(CVO_ERR_INVALID_ARG, "ell must be > 0");
    if (!(p->sigma > 0.0) || !std::isfinite(p->sigma)) return fail(CVO_ERR_INVALID_ARG, "sigma must be > 0");
    if (!std::isfinite(p->cutoff_mult)) return fail(CVO_ERR_INVALID_ARG, "cutoff_mult must be finite");
    if (p->n_blocks < 0 || p->n_blocks > CVO_MAX_BLOCKS)
        return fail(CVO_ERR_INVALID_ARG, "n_blocks must be in [0, %d]", CVO_MAX_BLOCKS);
    int D = 0;
    for (int b = 0; b < p->n_blocks; ++b) {
        const cvo_feat_block& fb = p->blocks[b];
        if (fb.dim < 1) return fail(CVO_ERR_INVALID_ARG, "block %d: dim must be >= 1", b);
        if (fb.kind != CVO_FEAT_SE && fb.kind != CVO_FEAT_DOT)
            return fail(CVO_ERR_INVALID_ARG, "block %d: unknown kind %d", b, fb.kind);
        if (fb.kind == CVO_FEAT_SE && (!(fb.scale > 0.0) || !std::isfinite(fb.scale) || !std::isfinite(fb.sigma)))
            return fail(CVO_ERR_INVALID_ARG, "block %d: scale must be > 0 and sigma finite", b);
        D += fb.dim;
    }
    if (D > CVO_MAX_FEAT_DIM) return fail(CVO_ERR_INVALID_ARG, "total feature dim %d > %d", D, CVO_MAX_FEAT_DIM);
    if (p->max_iters < 0) return fail(CVO_ERR_INVALID_ARG, "max_iters must be >= 0");
    if (p->anneal) {
        if (!(p->ell_min > 0.0) || p->ell_min > p->ell)
            return fail(CVO_ERR_INVALID_ARG, "annealing needs 0 < ell_min <= ell");
        if (!(p->decay > 0.0) || p->decay > 1.0) return fail(CVO_ERR_INVALID_ARG, "decay must be in (0, 1]");
        if (!(p->indicator_tol >= 0.0)) return fail(CVO_ERR_INVALID_ARG, "indicator_tol must be >= 0");
    }
    if (!(p->max_step_rot > 0.0)) return fail(CVO_ERR_INVALID_ARG, "max_step_rot must be > 0");
    if (!(p->step_tol_rot >= 0.0) || !(p->step_tol_trans >= 0.0))
        return fail(CVO_ERR_INVALID_ARG, "step tolerances must be >= 0");
    if (!std::isfinite(p->max_step_trans)) return fail(CVO_ERR_INVALID_ARG, "max_step_trans must be finite");
    if (!std::isfinite(p->feat_cutoff_mult)) return fail(CVO_ERR_INVALID_ARG, "feat_cutoff_mult must be finite");
    return CVO_OK;
}

cvo_status check_pose(const double* T, const char* name)
{
    if (!T) return fail(CVO_ERR_INVALID_ARG, "%s is NULL", name);
    for (int k = 0; k < 16; ++k)
        if (!std::isfinite(T[k])) return fail(CVO_ERR_INVALID_ARG, "%s has a non-finite entry", name);
    if (T[12] != 0.0 || T[13] != 0.0 || T[14] != 0.0 || T[15] != 1.0)
        return fail(CVO_ERR_INVALID_ARG, "%s: last row must be (0, 0, 0, 1)", name);
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            double d = 0.0;
            for (int k = 0; k < 3; ++k) d += T[4 * k + a] * T[4 * k + b];
            if (std::fabs(d - (a == b ? 1.0 : 0.0)) > 1e-6)
                return fail(CVO_ERR_INVALID_ARG, "%s: rotation is not orthonormal within 1e-6", name);
        }
    const double det = T[0] * (T[5] * T[10] - T[6] * T[9]) - T[1] * (T[4] * T[10] - T[6] * T[8]) +
                       T[2] * (T[4] * T[9] - T[5] * T[8]);
    if (det < 0.0) return fail(CVO_ERR_INVALID_ARG, "%s: rotation has determinant -1", name);
    return CVO_OK;
}

int feat_dim(const cvo_params& p)
{
    int D = 0;
    for (int b = 0; b < p.n_blocks; ++b) D += p.blocks[b].dim;
    return D;
}

cvo_status check_cloud(const cvo_cloud* c, const char* name, int D)
{
    if (!c) return fail(CVO_ERR_INVALID_ARG, "%s is NULL", name);
    if (c->n < 0) return fail(CVO_ERR_INVALID_ARG, "%s.n < 0", name);
    if (c->n > 0 && !c->xyz) return fail(CVO_ERR_INVALID_ARG, "%s.xyz is NULL", name);
    if (c->n > 0 && D > 0 && !c->feat) return fail(CVO_ERR_INVALID_ARG, "%s.feat is NULL but D = %d", name, D);
    if (c->feat_dtype != CVO_F32 && c->feat_dtype != CVO_BF16)
        return fail(CVO_ERR_INVALID_ARG, "%s.feat_dtype unknown", name);
    if (c->on_device && c->n > 0) {
        const void* ptrs[2] = {c->xyz, D > 0 ? c->feat : nullptr};
        for (const void* ptr : ptrs) {
            if (!ptr) continue;
            cudaPointerAttributes at;
            if (cudaPointerGetAttributes(&at, ptr) != cudaSuccess) {
                cudaGetLastError();
                return fail(CVO_ERR_INVALID_ARG, "%s: pointer is not known to CUDA", name);
            }
            if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged)
                return fail(CVO_ERR_INVALID_ARG, "%s: on_device = 1 but the pointer is not device memory", name);
        }
    }
    return CVO_OK;
}

// Device copies (or the caller's device pointers) of one cloud.
cvo_status stage(cvo_handle h, const cvo_cloud* c, int slot, int D, const float** xyz, const void** feat)
{
    *xyz = c->xyz;
    *feat = c->feat;
    if (c->on_device || c->n == 0) return CVO_OK;
    const size_t bx = (size_t)c->n * 3 * sizeof(float);
    CVO_CUDA(ensure(h->stage_xyz[slot], bx));
    CVO_CUDA(cudaMemcpyAsync(h->stage_xyz[slot].p, c->xyz, bx, cudaMemcpyHostToDevice, h->s));
    *xyz = (const float*)h->stage_xyz[slot].p;
    if (D > 0) {
        const size_t bf = (size_t)c->n * D * (c->feat_dtype == CVO_BF16 ? 2 : 4);
        CVO_CUDA(ensure(h->stage_feat[slot], bf));
        CVO_CUDA(cudaMemcpyAsync(h->stage_feat[slot].p, c->feat, bf, cudaMemcpyHostToDevice, h->s));
        *feat = h->stage_feat[slot].p;
    }
    return CVO_OK;
}

int bits_for(long long v)
{
    int b = 1;
    while (b < 32 && (1LL << b) < v) ++b;
    return b;
}

// Sorts (keys, vals) of length n; returns pointers to the sorted arrays.
cvo_status sort_pairs(cvo_handle h, int n, int nbits, unsigned** ks, unsigned** vs)
{
    int alt = 0;
    CVO_CUDA(ensure(h->sort_tmp, radix_sort_temp_bytes(n)));
    CVO_CUDA(radix_sort_pairs((unsigned*)h->keys.p, (unsigned*)h->vals.p, (unsigned*)h->keys2.p,
                              (unsigned*)h->vals2.p, n, nbits, h->sort_tmp.p, &alt, h->s));
    *ks = (unsigned*)(alt ? h->keys2.p : h->keys.p);
    *vs = (unsigned*)(alt ? h->vals2.p : h->vals.p);
    return CVO_OK;
}

// Feature constants and kappa = sigma^2 prod sigma_b^2 (shared by all pairs).
void set_features(cvo_handle h, int rec_bf16)
{
    const cvo_params& p = h->p;
    FeatConst& fc = h->fc;
    std::memset(&fc, 0, sizeof(fc));
    fc.n_blocks = p.n_blocks;
    int off = 0;
    double kappa = p.sigma * p.sigma;
    for (int b = 0; b < p.n_blocks; ++b) {
        fc.dim[b] = p.blocks[b].dim;
        fc.kind[b] = p.blocks[b].kind;
        fc.off[b] = off;
        off += p.blocks[b].dim;
        fc.fcut2[b] = 3.0e38f;
        if (p.blocks[b].kind == CVO_FEAT_SE) {
            const double sc = p.blocks[b].scale;
            fc.s[b] = (float)(-1.4426950408889634 / (2.0 * sc * sc));
            kappa *= p.blocks[b].sigma * p.blocks[b].sigma;
            if (p.feat_cutoff_mult > 0.0) fc.fcut2[b] = (float)((p.feat_cutoff_mult * sc) * (p.feat_cutoff_mult * sc));
        }
    }
    fc.D = off;
    fc.bf16 = rec_bf16;
    h->kappa = kappa;
    h->D = off;
    h->rec_bf16 = rec_bf16;
    h->rs = 1 + (off * (rec_bf16 ? 2 : 4) + 15) / 16;
    h->dense = !(p.cutoff_mult > 0.0);
}

// Exchanges the handle's stream and setup scratch with a lane's, so that the
// setup functions run on the lane; a second call restores them.
void swap_lane(cvo_handle h, SetupLane& L)
{
    std::swap(h->s, L.s);
    std::swap(h->keys, L.keys);
    std::swap(h->vals, L.vals);
    std::swap(h->keys2, L.keys2);
    std::swap(h->vals2, L.vals2);
    std::swap(h->sort_tmp, L.sort_tmp);
    std::swap(h->flags, L.flags);
    std::swap(h->gidx, L.gidx);
}

cvo_status ensure_lanes(cvo_handle h)
{
    for (SetupLane& L : h->lanes) {
        if (!L.s) CVO_CUDA(cudaStreamCreateWithFlags(&L.s, cudaStreamNonBlocking));
        if (!L.ev) CVO_CUDA(cudaEventCreateWithFlags(&L.ev, cudaEventDisableTiming));
    }
    return CVO_OK;
}

// The handle's stream waits for every lane's work so far.
cvo_status join_lanes(cvo_handle h)
{
    for (SetupLane& L : h->lanes) {
        CVO_CUDA(cudaEventRecord(L.ev, L.s));
        CVO_CUDA(cudaStreamWaitEvent(h->s, L.ev, 0));
    }
    return CVO_OK;
}

// Device pointers of a pair's inputs (the caller's, or staged copies).
struct Staged {
    const float* xyz_x = nullptr;
    const float* xyz_z = nullptr;
    const void* feat_x = nullptr;
    const void* feat_z = nullptr;
};

// A pair's phase-1 results (its scratch slot hm): the boxes of X and Z and
// Z's moments (into P); an error if a coordinate or feature was not finite.
cvo_status decode_slot(PairRes& P, const unsigned* hm, float xmin[3], float xmax[3], float zmin[3], float zmax[3])
{
    if (hm[12]) return fail(CVO_ERR_INVALID_ARG, "non-finite coordinate or feature");
    for (int a = 0; a < 3; ++a) {
        xmin[a] = decode_orderable(hm[a]);
        xmax[a] = decode_orderable(hm[3 + a]);
        zmin[a] = decode_orderable(hm[6 + a]);
        zmax[a] = decode_orderable(hm[9 + a]);
    }
    long long raw[5];
    std::memcpy(raw, hm + kZStatsWord, sizeof(raw));
    double zs[5];
    decode_zstats(raw, P.m, zs);
    for (int a = 0; a < 3; ++a) P.zc[a] = zs[a];
    P.zr2 = zs[3];
    P.zrmax = zs[4];
    return CVO_OK;
}

// The grid levels of Z for lengthscales in [ell_lo, ell_hi] from Z's box:
// one per factor sqrt(2) of the cutoff radius, cell edge cell_factor times
// the level's radius (grown until the grid has at most kMaxCells cells).
void set_levels(cvo_handle h, PairRes& P, const float zmin[3], const float zmax[3], double ell_hi, double ell_lo)
{
    const cvo_params& p = h->p;
    if (h->dense) {
        P.nlevels = 1;
        LevelHost& L = P.lv[0];
        L.h = 1.0;
        L.hx = 1.0;
        L.rdesign = 1.0;
        L.nx = L.ny = L.nz = 1;
        L.ox = zmin[0]; L.oy = zmin[1]; L.oz = zmin[2];
        L.ncells = 1;
    } else {
        const double rc_hi = p.cutoff_mult * ell_hi, rc_lo = p.cutoff_mult * ell_lo;
        int nl = 1 + (int)std::floor(std::log(rc_hi / rc_lo) / std::log(std::sqrt(2.0)) + 1e-9);
        nl = std::max(1, std::min(nl, kMaxLevels));
        P.nlevels = nl;
        for (int k = 0; k < nl; ++k) {
            LevelHost& L = P.lv[k];
            L.rdesign = rc_hi * 1.0002 / std::pow(std::sqrt(2.0), k);
            double hh = h->cell_factor * L.rdesign;
            // the x division first falls back to fewer parts, then the cells
            // grow, until the grid has at most kMaxCells cells
            int xdiv = h->cell_xdiv;
            for (;;) {
                // cell counts in double first: a cloud far wider than the
                // cutoff would overflow an int before the size check
                const double cx = std::floor(((double)zmax[0] - zmin[0]) / (hh / xdiv)) + 1.0;
                const double cy = std::floor(((double)zmax[1] - zmin[1]) / hh) + 1.0;
                const double cz = std::floor(((double)zmax[2] - zmin[2]) / hh) + 1.0;
                if (cx * cy * cz <= (double)kMaxCells) {
                    L.nx = (int)cx;
                    L.ny = (int)cy;
                    L.nz = (int)cz;
                    L.ncells = (long long)L.nx * L.ny * L.nz;
                    break;
                }
                if (xdiv > 1) xdiv /= 2;
                else hh *= 1.26;
            }
            L.h = hh;
            L.hx = hh / xdiv;
            L.ox = zmin[0]; L.oy = zmin[1]; L.oz = zmin[2];
        }
    }
}

// octree super-cells of edge about 2^super_delta times the level's cutoff
// radius hold the query groups (the dense sum: one super-cell)
int group_shift(cvo_handle h, const LevelHost& L, double cell0)
{
    if (h->dense) return 30;
    const int e = (int)std::floor(std::log2(L.rdesign / cell0)) + h->super_delta;
    return 3 * std::max(0, std::min(10, e));
}

// prepare() in three phases, each ending where the host needs a device
// result, so that a batch can run every pair's phase before one wait:
// dev / hm are the pair's kMiscWords slot of scratch on the device and its
// host copy.
// Phase 1: inputs staged; bounding boxes and the finiteness flag into dev.
cvo_status prepare_bbox(cvo_handle h, PairRes& P, const cvo_cloud* X, const cvo_cloud* Z, unsigned* dev, Staged* sg)
{
    const int D = h->D;
    const int n = X->n, m = Z->n;
    P.n = n;
    P.m = m;
    CVO_TRY(stage(h, X, 0, D, &sg->xyz_x, &sg->feat_x));
    CVO_TRY(stage(h, Z, 1, D, &sg->xyz_z, &sg->feat_z));
    CVO_CUDA(cudaMemsetAsync(dev, 0, kMiscWords * sizeof(unsigned), h->s));
    CVO_CUDA(cudaMemsetAsync(dev + 0, 0xff, 3 * sizeof(unsigned), h->s));
    CVO_CUDA(cudaMemsetAsync(dev + 6, 0xff, 3 * sizeof(unsigned), h->s));
    int* bad = (int*)(dev + 12);
    CVO_CUDA(launch_bbox(sg->xyz_x, n, dev + 0, bad, h->s));
    CVO_CUDA(launch_bbox(sg->xyz_z, m, dev + 6, bad, h->s));
    CVO_CUDA(launch_zstats(sg->xyz_z, m, (long long*)(dev + kZStatsWord), h->s));
    if (D > 0) {
        CVO_CUDA(launch_check_feat(sg->feat_x, (long long)n * D, X->feat_dtype == CVO_BF16, bad, h->s));
        CVO_CUDA(launch_check_feat(sg->feat_z, (long long)m * D, Z->feat_dtype == CVO_BF16, bad, h->s));
    }
    return CVO_OK;
}

// Phase 2: from the boxes (hm), the grid levels of Z, the Hilbert-ordered
// queries of X and their groups (group counts into dev + 16 + level).
cvo_status prepare_build(cvo_handle h, PairRes& P, const cvo_cloud* X, const cvo_cloud* Z, double ell_hi,
                         double ell_lo, const Staged& sg, const unsigned* hm, unsigned* dev, bool fan_out)
{
    const int D = h->D;
    const int n = X->n, m = Z->n;
    const float* xyz_x = sg.xyz_x;
    const float* xyz_z = sg.xyz_z;
    const void* feat_x = sg.feat_x;
    const void* feat_z = sg.feat_z;
    float xmin[3], xmax[3], zmin[3], zmax[3];
    CVO_TRY(decode_slot(P, hm, xmin, xmax, zmin, zmax));
    const int rs = h->rs;
    const int nmax = std::max(n, m);
    // the handle's own setup scratch, which the work plan uses after this
    // (with fan_out the builds below run on the lanes' copies)
    CVO_CUDA(ensure(h->keys, (size_t)nmax * 4));
    CVO_CUDA(ensure(h->vals, (size_t)nmax * 4));
    CVO_CUDA(ensure(h->keys2, (size_t)nmax * 4));
    CVO_CUDA(ensure(h->vals2, (size_t)nmax * 4));
    CVO_CUDA(ensure(h->flags, (size_t)std::max(n, 1) * 4));
    CVO_CUDA(ensure(h->gidx, (size_t)std::max(n, 1) * 4));

    set_levels(h, P, zmin, zmax, ell_hi, ell_lo);
    // with fan_out, the grid levels and the queries are built on the setup
    // lanes at once (each lane its own scratch), joined at the end
    if (fan_out) {
        CVO_TRY(ensure_lanes(h));
        for (SetupLane& L : h->lanes) {
            for (DevBuf* b : {&L.keys, &L.vals, &L.keys2, &L.vals2, &L.flags, &L.gidx})
                CVO_CUDA(ensure(*b, (size_t)std::max(nmax, 1) * 4));
            CVO_CUDA(ensure(L.sort_tmp, radix_sort_temp_bytes(nmax)));
            CVO_CUDA(cudaEventRecord(L.ev, h->s));   // after the inputs' staging and the boxes
            CVO_CUDA(cudaStreamWaitEvent(L.s, L.ev, 0));
        }
    }
    // the lane whose stream and scratch the handle holds now; given back on
    // every way out of this function
    struct Held {
        cvo_handle h;
        SetupLane* lane = nullptr;
        void drop()
        {
            if (lane) swap_lane(h, *lane);
            lane = nullptr;
        }
        ~Held() { drop(); }
    } held{h};
    auto use_lane = [&](int i) {
        if (!fan_out) return;
        held.drop();
        held.lane = &h->lanes[i % kSetupLanes];
        swap_lane(h, *held.lane);
    };
    for (int k = 0; k < P.nlevels; ++k) {
        LevelHost& L = P.lv[k];
        use_lane(1 + k % (kSetupLanes - 1));
        CVO_CUDA(ensure(P.zrec[k], (size_t)std::max(m, 1) * rs * sizeof(float4)));
        CVO_CUDA(ensure(P.cell_start[k], (size_t)(L.ncells + 1) * sizeof(int)));
        if (h->dense) {
            const int cs[2] = {0, m};
            CVO_CUDA(cudaMemcpyAsync(P.cell_start[k].p, cs, sizeof(cs), cudaMemcpyHostToDevice, h->s));
            CVO_CUDA(launch_pack(xyz_z, feat_z, Z->feat_dtype == CVO_BF16, D, nullptr, m, (float4*)P.zrec[k].p, rs,
                                 h->rec_bf16, h->s));
        } else {
            CVO_CUDA(launch_cell_keys(xyz_z, m, L.ox, L.oy, L.oz, (float)(1.0 / L.h), (float)(1.0 / L.hx), L.nx, L.ny,
                                      L.nz, (unsigned*)h->keys.p, (unsigned*)h->vals.p, h->s));
            unsigned *ks, *vs;
            CVO_TRY(sort_pairs(h, m, bits_for(L.ncells), &ks, &vs));
            CVO_CUDA(launch_cell_start(ks, m, (int)L.ncells, (int*)P.cell_start[k].p, h->s));
            CVO_CUDA(launch_pack(xyz_z, feat_z, Z->feat_dtype == CVO_BF16, D, vs, m, (float4*)P.zrec[k].p, rs,
                                 h->rec_bf16, h->s));
        }
    }

    // queries: Hilbert order of X in its own frame
    use_lane(0);
    double ext = 0.0;
    for (int a = 0; a < 3; ++a) ext = std::max(ext, (double)xmax[a] - xmin[a]);
    const double cell0 = std::max(ext / 1024.0, 1e-6);
    CVO_CUDA(ensure(P.xrec, (size_t)std::max(n, 1) * rs * sizeof(float4)));
    CVO_CUDA(ensure(P.hkeys, (size_t)std::max(n, 1) * 4));
    CVO_CUDA(launch_hilbert_keys(xyz_x, n, xmin[0], xmin[1], xmin[2], (float)(1.0 / cell0), (unsigned*)h->keys.p,
                                (unsigned*)h->vals.p, h->s));
    {
        unsigned *ks, *vs;
        CVO_TRY(sort_pairs(h, n, 30, &ks, &vs));
        CVO_CUDA(launch_pack(xyz_x, feat_x, X->feat_dtype == CVO_BF16, D, vs, n, (float4*)P.xrec.p, rs, h->rec_bf16,
                             h->s));
        CVO_CUDA(cudaMemcpyAsync(P.hkeys.p, ks, (size_t)n * 4, cudaMemcpyDeviceToDevice, h->s));
    }
    // query groups per level
    CVO_CUDA(ensure(h->flags, (size_t)std::max(n, 1) * 4));
    CVO_CUDA(ensure(h->gidx, (size_t)std::max(n, 1) * 4));
    for (int k = 0; k < P.nlevels; ++k) {
        LevelHost& L = P.lv[k];
        const int sh = group_shift(h, L, cell0);
        L.shift = sh;
        CVO_CUDA(ensure(P.groups[k], (size_t)std::max(n, 1) * sizeof(int2)));
        CVO_CUDA(launch_group_flags((const unsigned*)P.hkeys.p, n, sh, 32 / h->query_lanes, (unsigned*)h->flags.p,
                                    h->s));
        CVO_CUDA(exclusive_scan_u32((const unsigned*)h->flags.p, (unsigned*)h->gidx.p, n, dev + 16 + k, h->s));
        CVO_CUDA(launch_group_write((const unsigned*)P.hkeys.p, (const unsigned*)h->flags.p,
                                    (const unsigned*)h->gidx.p, n, sh, 32 / h->query_lanes, (int2*)P.groups[k].p,
                                    h->s));
    }
    held.drop();
    if (fan_out) CVO_TRY(join_lanes(h));
    return CVO_OK;
}

// Phase 3: the level descriptors, with the group counts (hm).
// The level descriptors on the host (P.ld), with the group counts (hm); the
// device copy's buffer ensured.
cvo_status level_descs(cvo_handle h, PairRes& P, const unsigned* hm)
{
    const int n = P.n;
    for (int k = 0; k < P.nlevels; ++k) {
        LevelHost& L = P.lv[k];
        L.ngroups = n > 0 ? (int)hm[16 + k] : 0;
        L.nitems = 0;
        LevelDesc& d = P.ld[k];
        d.h = (float)L.h;
        d.inv_h = (float)(1.0 / L.h);
        d.inv_hx = (float)(1.0 / L.hx);
        d.ox = L.ox; d.oy = L.oy; d.oz = L.oz;
        d.nx = L.nx; d.ny = L.ny; d.nz = L.nz;
        d.cell_start = (const int*)P.cell_start[k].p;
        d.zrec = (const float4*)P.zrec[k].p;
        d.groups = (const int2*)P.groups[k].p;
        d.items = nullptr;
        d.ngroups = L.ngroups;
        d.nitems = 0;
        d.chunk_min = 0;
        // trimming the rows by each query pays only where a work item is long
        // enough to carry it (the trim is per item, the saving per candidate)
        d.trim = h->chunk_len >= kTrimChunkLen ? 1 : 0;
    }
    P.max_items = 1;
    CVO_CUDA(ensure(P.levels_dev, sizeof(P.ld)));
    return CVO_OK;
}

cvo_status prepare_finish(cvo_handle h, PairRes& P, const unsigned* hm)
{
    CVO_TRY(level_descs(h, P, hm));
    CVO_CUDA(cudaMemcpyAsync(P.levels_dev.p, P.ld, P.nlevels * sizeof(LevelDesc), cudaMemcpyHostToDevice, h->s));
    return CVO_OK;
}

// Builds the grid levels of Z, the Hilbert-ordered queries of X and their groups
// for lengthscales in [ell_lo, ell_hi].  Uses the handle's shared scratch.
// The work items are planned by init_state, once the start pose is known.
cvo_status prepare(cvo_handle h, PairRes& P, const cvo_cloud* X, const cvo_cloud* Z, double ell_hi, double ell_lo)
{
    CVO_CUDA(ensure(h->misc, kMiscWords * sizeof(unsigned)));
    unsigned* dev = (unsigned*)h->misc.p;
    Staged sg;
    CVO_TRY(prepare_bbox(h, P, X, Z, dev, &sg));
    CVO_CUDA(cudaMemcpyAsync(h->h_misc, dev, (kZStatsWord + 10) * sizeof(unsigned), cudaMemcpyDeviceToHost, h->s));
    CVO_CUDA(cudaStreamSynchronize(h->s));
    CVO_TRY(prepare_build(h, P, X, Z, ell_hi, ell_lo, sg, h->h_misc, dev, true));
    CVO_CUDA(cudaMemcpyAsync(h->h_misc + 16, dev + 16, P.nlevels * sizeof(unsigned), cudaMemcpyDeviceToHost, h->s));
    CVO_CUDA(cudaStreamSynchronize(h->s));
    return prepare_finish(h, P, h->h_misc);
}

// Work items of every level of a prepared pair.  planned: at the pose of
// its state (after k_init_state), per query group the candidate-stream
// length at the level's design cutoff radius, groups sorted longest first,
// each split into ceil(length / chunk_len) chunks (at most kMaxChunks) --
// exact for an evaluation, and good for a batch of pairs whose poses stay
// near their starts.  Otherwise uniform: kChunks per group in Hilbert order,
// cut at run time: the first sweep of each grid level of a registration
// with a cutoff, whose later sweeps take the items k_layout lays out from
// the stream lengths the previous sweep recorded.
// In two phases (the item counts go to dev + 16 + level, then are read from
// their host copy hm), so that a batch waits once for all its pairs.
cvo_status plan_launch(cvo_handle h, PairRes& P, bool planned, unsigned* dev)
{
    if (P.n == 0) return CVO_OK;
    for (int k = 0; k < P.nlevels; ++k) {
        LevelHost& L = P.lv[k];
        const int ng = L.ngroups;
        CVO_CUDA(ensure(P.items[k], (size_t)std::max(ng, 1) * kMaxChunks * sizeof(int4)));
        CVO_CUDA(launch_group_cost((const LevelDesc*)P.levels_dev.p, k, ng, (const float4*)P.xrec.p, P.m, h->rs, h->dense,
                                   (const IterState*)P.state.p, h->dense ? -1.0f : (float)L.rdesign,
                                   planned ? h->chunk_len : 0, (unsigned*)h->keys.p, (unsigned*)h->vals.p,
                                   (unsigned*)h->flags.p, h->s));
        unsigned* ks = (unsigned*)h->keys.p;
        unsigned* vs = (unsigned*)h->vals.p;
        if (planned) CVO_TRY(sort_pairs(h, ng, 32, &ks, &vs));
        CVO_CUDA(launch_gather_u32((const unsigned*)h->flags.p, vs, ng, (unsigned*)h->gidx.p, h->s));
        CVO_CUDA(exclusive_scan_u32((const unsigned*)h->gidx.p, ks, ng, dev + 16 + k, h->s));
        CVO_CUDA(launch_write_items((const LevelDesc*)P.levels_dev.p, k, vs, (const unsigned*)h->flags.p, ks, ng,
                                    (int4*)P.items[k].p, h->s));
    }
    return CVO_OK;
}

// The planned items into the level descriptors on the host (P.ld), with the
// item counts (hm).
void plan_descs(PairRes& P, bool planned, const unsigned* hm)
{
    int max_items = 1;
    for (int k = 0; k < P.nlevels; ++k) {
        P.lv[k].nitems = (int)hm[16 + k];
        P.ld[k].items = (const int4*)P.items[k].p;
        P.ld[k].nitems = P.lv[k].nitems;
        P.ld[k].chunk_min = planned ? 0 : kChunkMin;
        max_items = std::max(max_items, P.lv[k].nitems);
    }
    P.max_items = max_items;
}

cvo_status plan_finish(cvo_handle h, PairRes& P, bool planned, const unsigned* hm)
{
    if (P.n == 0) return CVO_OK;
    plan_descs(P, planned, hm);
    CVO_CUDA(cudaMemcpyAsync(P.levels_dev.p, P.ld, P.nlevels * sizeof(LevelDesc), cudaMemcpyHostToDevice, h->s));
    return CVO_OK;
}

cvo_status plan_items(cvo_handle h, PairRes& P, bool planned)
{
    if (P.n == 0) return CVO_OK;
    unsigned* dev = (unsigned*)h->misc.p;
    CVO_TRY(plan_launch(h, P, planned, dev));
    if (planned) {
        CVO_CUDA(cudaMemcpyAsync(h->h_misc + 16, dev + 16, P.nlevels * sizeof(unsigned), cudaMemcpyDeviceToHost, h->s));
        CVO_CUDA(cudaStreamSynchronize(h->s));
    } else {   // uniform: kChunks items for every group, known without a wait
        for (int k = 0; k < P.nlevels; ++k) h->h_misc[16 + k] = (unsigned)(kChunks * P.lv[k].ngroups);
    }
    return plan_finish(h, P, planned, h->h_misc);
}

cvo_status ensure_host_misc(cvo_handle h, int words)
{
    if (words <= h->h_misc_cap) return CVO_OK;
    unsigned* p = nullptr;
    if (cudaMallocHost((void**)&p, (size_t)words * sizeof(unsigned)) != cudaSuccess) {
        cudaGetLastError();
        return fail(CVO_ERR_OOM, "cudaMallocHost failed");
    }
    cudaFreeHost(h->h_misc);
    h->h_misc = p;
    h->h_misc_cap = words;
    return CVO_OK;
}

cvo_status ensure_host_states(cvo_handle h, int n)
{
    if (n <= h->h_state_cap) return CVO_OK;
    if (h->h_state) cudaFreeHost(h->h_state);
    h->h_state = nullptr;
    h->h_state_cap = 0;
    CVO_CUDA(cudaMallocHost((void**)&h->h_state, (size_t)n * sizeof(IterState)));
    h->h_state_cap = n;
    return CVO_OK;
}

// Initial state of one pair; host copy in h->h_state[slot].
enum PlanMode { kNoPlan = 0, kUniform = 1, kPlanned = 2 };

// The state filled on the host (h->h_state[slot]), its device buffer
// ensured; fill_state also copies it to the device.  Its derived constants
// are k_init_state's.
cvo_status state_host(cvo_handle h, PairRes& P, int slot, const double* T, double ell, int mode)
{
    IterState* st = h->h_state + slot;
    std::memset(st, 0, sizeof(IterState));
    std::memcpy(st->T, T, 16 * sizeof(double));
    const cvo_params& p = h->p;
    st->ell = ell;
    st->ell_last = ell;
    st->mode = mode;
    st->kappa = h->kappa;
    st->norm = (P.n > 0 && P.m > 0) ? 1.0 / std::sqrt((double)P.n * (double)P.m) : 0.0;
    st->cutoff_mult = p.cutoff_mult;
    st->ell_min = p.anneal ? p.ell_min : ell;
    st->decay = p.decay;
    st->indicator_tol = p.indicator_tol;
    st->step_tol_rot = p.step_tol_rot;
    st->step_tol_trans = p.step_tol_trans;
    st->max_step_rot = p.max_step_rot;
    st->max_step_trans = p.max_step_trans;
    st->max_iters = p.max_iters;
    st->anneal = p.anneal;
    st->status = 1;
    for (int a = 0; a < 3; ++a) st->c[a] = P.zc[a];
    st->rho2 = P.zr2;
    st->rmax = P.zrmax;
    st->nlevels = P.nlevels;
    for (int k = 0; k < P.nlevels; ++k) st->level_h[k] = (float)P.lv[k].rdesign;
    if (mode == 1 && p.max_iters == 0) st->done = 1;
    CVO_CUDA(ensure(P.state, sizeof(IterState)));
    return CVO_OK;
}

cvo_status fill_state(cvo_handle h, PairRes& P, int slot, const double* T, double ell, int mode)
{
    CVO_TRY(state_host(h, P, slot, T, ell, mode));
    CVO_CUDA(cudaMemcpyAsync(P.state.p, h->h_state + slot, sizeof(IterState), cudaMemcpyHostToDevice, h->s));
    return CVO_OK;
}

cvo_status init_state(cvo_handle h, PairRes& P, int slot, const double* T, double ell, int mode, int plan)
{
    CVO_TRY(fill_state(h, P, slot, T, ell, mode));
    CVO_CUDA(launch_init_state((IterState*)P.state.p, h->s));
    if (plan != kNoPlan) CVO_TRY(plan_items(h, P, plan == kPlanned));
    return CVO_OK;
}

// The set-up of a batch whose inputs are on the device: prepare, init_state
// and plan_items (planned) for every pair, each stage one launch for all
// pairs (the batched launchers) rather than a few dozen launches per pair,
// with one wait after each of the three phases.  The results are those of
// the pair-by-pair set-up: the same kernel bodies on the same data, and
// stable sorts (a pair whose keys need fewer digits than another's takes
// extra passes on zero digits, which keep its order).
double reachable_ell_lo(const cvo_params& p);

// Host blocks to device destinations in one host-to-device copy (through the
// pinned staging buffer) and one copy kernel, instead of a copy per block.
// Sizes are multiples of 4 bytes.  The staging buffer is rewritten only
// after the previous copy out of it has completed.
struct HostBlock {
    const void* src;
    void* dst;
    size_t bytes;
};

cvo_status upload_blocks(cvo_handle h, const std::vector<HostBlock>& blocks)
{
    size_t total = 0;
    for (const HostBlock& b : blocks) total += (b.bytes + 15) & ~(size_t)15;
    if (total == 0) return CVO_OK;
    if (h->stage_ev) CVO_CUDA(cudaEventSynchronize(h->stage_ev));
    else CVO_CUDA(cudaEventCreateWithFlags(&h->stage_ev, cudaEventDisableTiming));
    if (total > h->h_stage_cap) {
        unsigned char* q = nullptr;
        if (cudaMallocHost((void**)&q, total) != cudaSuccess) {
            cudaGetLastError();
            return fail(CVO_ERR_OOM, "cudaMallocHost failed");
        }
        if (h->h_stage) cudaFreeHost(h->h_stage);
        h->h_stage = q;
        h->h_stage_cap = total;
    }
    CVO_CUDA(ensure(h->d_stage, total));
    std::vector<CopyJob> jobs;
    size_t off = 0;
    for (const HostBlock& b : blocks) {
        std::memcpy(h->h_stage + off, b.src, b.bytes);
        jobs.push_back(CopyJob{(const unsigned char*)h->d_stage.p + off, b.dst, (int)b.bytes});
        off += (b.bytes + 15) & ~(size_t)15;
    }
    CVO_CUDA(cudaMemcpyAsync(h->d_stage.p, h->h_stage, total, cudaMemcpyHostToDevice, h->s));
    CVO_CUDA(cudaEventRecord(h->stage_ev, h->s));
    CVO_CUDA(launch_copy_batch(jobs.data(), (int)jobs.size(), h->s));
    return CVO_OK;
}

struct BatchSeg {   // a pair's segment of the batch scratch
    unsigned *keys, *vals, *keys2, *vals2, *flags, *gidx, *temp;
};

cvo_status prepare_batch(cvo_handle h, const std::vector<int>& live, const cvo_cloud* X, const cvo_cloud* Z,
                         const double* T_init, long long* work)
{
    const cvo_params& p = h->p;
    const int nl = (int)live.size();
    const int D = h->D, rs = h->rs;
    const double ell_lo = reachable_ell_lo(p);
    CVO_CUDA(ensure(h->misc, (size_t)nl * kMiscWords * sizeof(unsigned)));
    CVO_TRY(ensure_host_misc(h, nl * kMiscWords));
    unsigned* dev = (unsigned*)h->misc.p;
    unsigned* hm = h->h_misc;
    auto slot = [&](int i) { return dev + (size_t)i * kMiscWords; };
    auto hslot = [&](int i) { return hm + (size_t)i * kMiscWords; };
    auto fetch = [&]() -> cvo_status {
        CVO_CUDA(cudaMemcpyAsync(hm, dev, (size_t)nl * kMiscWords * sizeof(unsigned), cudaMemcpyDeviceToHost, h->s));
        CVO_CUDA(cudaStreamSynchronize(h->s));
        return CVO_OK;
    };

    // phase 1: boxes, finiteness, Z's moments
    std::vector<BoxJob> box(nl);
    for (int i = 0; i < nl; ++i) {
        const cvo_cloud& x = X[live[i]];
        const cvo_cloud& z = Z[live[i]];
        PairRes& P = h->pr[i];
        P.n = x.n;
        P.m = z.n;
        BoxJob& b = box[i];
        b.xyz_x = x.xyz;
        b.xyz_z = z.xyz;
        b.feat_x = x.feat;
        b.feat_z = z.feat;
        b.nfx = D > 0 ? (long long)x.n * D : 0;
        b.nfz = D > 0 ? (long long)z.n * D : 0;
        b.n = x.n;
        b.m = z.n;
        b.fx_bf16 = x.feat_dtype == CVO_BF16;
        b.fz_bf16 = z.feat_dtype == CVO_BF16;
        b.box_x = slot(i);
        b.box_z = slot(i) + 6;
        b.bad = (int*)(slot(i) + 12);
        b.zstats = (long long*)(slot(i) + kZStatsWord);
    }
    CVO_CUDA(launch_boxes_batch(box.data(), nl, h->s));
    CVO_TRY(fetch());

    // the scratch: per pair max(n, m) words in each of six arrays, and the
    // sorts' temporary words
    std::vector<size_t> cap(nl), tw(nl);
    size_t sum_cap = 0, sum_tw = 0;
    for (int i = 0; i < nl; ++i) {
        cap[i] = (size_t)std::max(1, std::max(h->pr[i].n, h->pr[i].m));
        tw[i] = sort_batch_temp_words((int)cap[i]);
        sum_cap += cap[i];
        sum_tw += tw[i];
    }
    CVO_CUDA(ensure(h->batch_scratch, (6 * sum_cap + sum_tw) * sizeof(unsigned)));
    std::vector<BatchSeg> seg(nl);
    {
        unsigned* base = (unsigned*)h->batch_scratch.p;
        size_t off = 0, toff = 6 * sum_cap;
        for (int i = 0; i < nl; ++i) {
            unsigned** arrays[6] = {&seg[i].keys, &seg[i].vals, &seg[i].keys2, &seg[i].vals2, &seg[i].flags,
                                    &seg[i].gidx};
            for (int a = 0; a < 6; ++a) *arrays[a] = base + (size_t)a * sum_cap + off;
            seg[i].temp = base + toff;
            off += cap[i];
            toff += tw[i];
        }
    }

    // phase 2: grid levels of Z, the Hilbert order of X, query groups
    std::vector<double> cell0(nl);
    std::vector<std::array<float, 3>> xlo(nl);
    int nlev = 0;
    for (int i = 0; i < nl; ++i) {
        PairRes& P = h->pr[i];
        float xmin[3], xmax[3], zmin[3], zmax[3];
        CVO_TRY(decode_slot(P, hslot(i), xmin, xmax, zmin, zmax));
        set_levels(h, P, zmin, zmax, p.ell, ell_lo);
        nlev = std::max(nlev, P.nlevels);
        double ext = 0.0;
        for (int a = 0; a < 3; ++a) ext = std::max(ext, (double)xmax[a] - xmin[a]);
        cell0[i] = std::max(ext / 1024.0, 1e-6);
        xlo[i] = {xmin[0], xmin[1], xmin[2]};
        CVO_CUDA(ensure(P.xrec, (size_t)std::max(P.n, 1) * rs * sizeof(float4)));
        CVO_CUDA(ensure(P.hkeys, (size_t)std::max(P.n, 1) * 4));
        for (int k = 0; k < P.nlevels; ++k) {
            LevelHost& L = P.lv[k];
            L.shift = group_shift(h, L, cell0[i]);
            CVO_CUDA(ensure(P.zrec[k], (size_t)std::max(P.m, 1) * rs * sizeof(float4)));
            CVO_CUDA(ensure(P.cell_start[k], (size_t)(L.ncells + 1) * sizeof(int)));
            CVO_CUDA(ensure(P.groups[k], (size_t)std::max(P.n, 1) * sizeof(int2)));
        }
    }
    // pairs i of a job list: idx[j]
    std::vector<int> idx;
    auto pairs_with_level = [&](int k) {
        idx.clear();
        for (int i = 0; i < nl; ++i)
            if (h->pr[i].nlevels > k) idx.push_back(i);
    };
    // sorted (keys, vals) of pair i after a batched sort: in place or in the alternates
    auto sorted_keys = [&](int i, int alt) { return alt ? seg[i].keys2 : seg[i].keys; };
    auto sorted_vals = [&](int i, int alt) { return alt ? seg[i].vals2 : seg[i].vals; };
    auto sort_jobs = [&](const std::vector<int>& ids, auto&& count_of) {
        std::vector<SortJob> sj(ids.size());
        for (size_t j = 0; j < ids.size(); ++j) {
            const BatchSeg& g = seg[ids[j]];
            sj[j] = SortJob{g.keys, g.vals, g.keys2, g.vals2, g.temp, count_of(ids[j])};
        }
        return sj;
    };
    for (int k = 0; k < nlev; ++k) {
        pairs_with_level(k);
        const int cnt = (int)idx.size();
        std::vector<PackJob> pj(cnt);
        if (h->dense) {
            for (int j = 0; j < cnt; ++j) {
                PairRes& P = h->pr[idx[j]];
                const cvo_cloud& z = Z[live[idx[j]]];
                const int cs[2] = {0, P.m};
                CVO_CUDA(cudaMemcpyAsync(P.cell_start[k].p, cs, sizeof(cs), cudaMemcpyHostToDevice, h->s));
                pj[j] = PackJob{z.xyz, z.feat, nullptr, nullptr, nullptr, (float4*)P.zrec[k].p, P.m,
                                z.feat_dtype == CVO_BF16};
            }
        } else {
            std::vector<KeyJob> kj(cnt);
            int nbits = 1;
            for (int j = 0; j < cnt; ++j) {
                const PairRes& P = h->pr[idx[j]];
                const LevelHost& L = P.lv[k];
                kj[j] = KeyJob{Z[live[idx[j]]].xyz, seg[idx[j]].keys, seg[idx[j]].vals, L.ox, L.oy, L.oz,
                               (float)(1.0 / L.h), (float)(1.0 / L.hx), P.m, L.nx, L.ny, L.nz};
                nbits = std::max(nbits, bits_for(L.ncells));
            }
            CVO_CUDA(launch_cell_keys_batch(kj.data(), cnt, h->s));
            const std::vector<SortJob> sj = sort_jobs(idx, [&](int i) { return h->pr[i].m; });
            int alt = 0;
            CVO_CUDA(radix_sort_batch(sj.data(), cnt, nbits, &alt, h->s));
            std::vector<CellStartJob> cj(cnt);
            for (int j = 0; j < cnt; ++j) {
                PairRes& P = h->pr[idx[j]];
                const cvo_cloud& z = Z[live[idx[j]]];
                cj[j] = CellStartJob{sorted_keys(idx[j], alt), (int*)P.cell_start[k].p, P.m, (int)P.lv[k].ncells};
                pj[j] = PackJob{z.xyz, z.feat, sorted_vals(idx[j], alt), nullptr, nullptr, (float4*)P.zrec[k].p, P.m,
                                z.feat_dtype == CVO_BF16};
            }
            CVO_CUDA(launch_cell_start_batch(cj.data(), cnt, h->s));
        }
        CVO_CUDA(launch_pack_batch(pj.data(), cnt, D, rs, h->rec_bf16, h->s));
    }
    {   // queries: Hilbert order of X in its own frame
        std::vector<int> all(nl);
        for (int i = 0; i < nl; ++i) all[i] = i;
        std::vector<KeyJob> kj(nl);
        for (int i = 0; i < nl; ++i)
            kj[i] = KeyJob{X[live[i]].xyz, seg[i].keys, seg[i].vals, xlo[i][0], xlo[i][1], xlo[i][2],
                           (float)(1.0 / cell0[i]), (float)(1.0 / cell0[i]), h->pr[i].n, 0, 0, 0};
        CVO_CUDA(launch_hilbert_keys_batch(kj.data(), nl, h->s));
        const std::vector<SortJob> sj = sort_jobs(all, [&](int i) { return h->pr[i].n; });
        int alt = 0;
        CVO_CUDA(radix_sort_batch(sj.data(), nl, 30, &alt, h->s));
        std::vector<PackJob> pj(nl);
        for (int i = 0; i < nl; ++i) {
            PairRes& P = h->pr[i];
            const cvo_cloud& x = X[live[i]];
            pj[i] = PackJob{x.xyz, x.feat, sorted_vals(i, alt), sorted_keys(i, alt), (unsigned*)P.hkeys.p,
                            (float4*)P.xrec.p, P.n, x.feat_dtype == CVO_BF16};
        }
        CVO_CUDA(launch_pack_batch(pj.data(), nl, D, rs, h->rec_bf16, h->s));
    }
    for (int k = 0; k < nlev; ++k) {   // query groups per level; their counts into the slots
        pairs_with_level(k);
        const int cnt = (int)idx.size();
        std::vector<GroupJob> gj(cnt);
        std::vector<ScanJob> sc(cnt);
        for (int j = 0; j < cnt; ++j) {
            const int i = idx[j];
            PairRes& P = h->pr[i];
            gj[j] = GroupJob{(const unsigned*)P.hkeys.p, seg[i].flags, seg[i].gidx, (int2*)P.groups[k].p, P.n,
                             P.lv[k].shift, 32 / h->query_lanes};
            sc[j] = ScanJob{seg[i].flags, seg[i].gidx, slot(i) + 16 + k, P.n};
        }
        CVO_CUDA(launch_group_flags_batch(gj.data(), cnt, h->s));
        CVO_CUDA(launch_scan_batch(sc.data(), cnt, h->s));
        CVO_CUDA(launch_group_write_batch(gj.data(), cnt, h->s));
    }
    CVO_TRY(fetch());

    // phase 3: level descriptors, start states, the planned work items
    std::vector<StateJob> stj(nl);
    std::vector<HostBlock> up;
    for (int i = 0; i < nl; ++i) {
        PairRes& P = h->pr[i];
        CVO_TRY(level_descs(h, P, hslot(i)));
        CVO_TRY(state_host(h, P, i, T_init + 16 * live[i], p.ell, 1));
        up.push_back(HostBlock{P.ld, P.levels_dev.p, P.nlevels * sizeof(LevelDesc)});
        up.push_back(HostBlock{h->h_state + i, P.state.p, sizeof(IterState)});
        stj[i] = StateJob{(IterState*)P.state.p};
    }
    CVO_TRY(upload_blocks(h, up));
    CVO_CUDA(launch_init_state_batch(stj.data(), nl, h->s));
    for (int k = 0; k < nlev; ++k) {
        pairs_with_level(k);
        const int cnt = (int)idx.size();
        std::vector<CostJob> cj(cnt);
        for (int j = 0; j < cnt; ++j) {
            const int i = idx[j];
            PairRes& P = h->pr[i];
            const LevelHost& L = P.lv[k];
            CVO_CUDA(ensure(P.items[k], (size_t)std::max(L.ngroups, 1) * kMaxChunks * sizeof(int4)));
            cj[j] = CostJob{(const LevelDesc*)P.levels_dev.p, (const float4*)P.xrec.p, (const IterState*)P.state.p,
                            seg[i].keys, seg[i].vals, seg[i].flags, k, L.ngroups, P.m,
                            h->dense ? -1.0f : (float)L.rdesign};
        }
        CVO_CUDA(launch_group_cost_batch(cj.data(), cnt, rs, h->dense, h->chunk_len, h->s));
        const std::vector<SortJob> sj = sort_jobs(idx, [&](int i) { return h->pr[i].lv[k].ngroups; });
        int alt = 0;
        CVO_CUDA(radix_sort_batch(sj.data(), cnt, 32, &alt, h->s));
        std::vector<GatherJob> gj(cnt);
        std::vector<ScanJob> sc(cnt);
        std::vector<ItemsJob> it(cnt);
        for (int j = 0; j < cnt; ++j) {
            const int i = idx[j];
            PairRes& P = h->pr[i];
            const int ng = P.lv[k].ngroups;
            // chunk counts in sorted order, their scan (into the sorted keys'
            // place, no longer needed) and the items
            gj[j] = GatherJob{seg[i].flags, sorted_vals(i, alt), seg[i].gidx, ng};
            sc[j] = ScanJob{seg[i].gidx, sorted_keys(i, alt), slot(i) + 16 + k, ng};
            it[j] = ItemsJob{(const LevelDesc*)P.levels_dev.p, sorted_vals(i, alt), seg[i].flags, sorted_keys(i, alt),
                             (int4*)P.items[k].p, k, ng};
        }
        CVO_CUDA(launch_gather_batch(gj.data(), cnt, h->s));
        CVO_CUDA(launch_scan_batch(sc.data(), cnt, h->s));
        CVO_CUDA(launch_write_items_batch(it.data(), cnt, h->s));
    }
    CVO_TRY(fetch());
    up.clear();
    for (int i = 0; i < nl; ++i) {
        PairRes& P = h->pr[i];
        plan_descs(P, true, hslot(i));
        up.push_back(HostBlock{P.ld, P.levels_dev.p, P.nlevels * sizeof(LevelDesc)});
        *work += P.max_items;
    }
    return upload_blocks(h, up);
}


// Sweep scratch sized for nblocks blocks; the pair table uploaded.
cvo_status setup_sweep(cvo_handle h, const std::vector<PairDesc>& table, int nblocks, SweepArgs* a, bool groups)
{
    if (groups && nblocks > kGroupBlocks * kMaxGroups)
        return fail(CVO_ERR_CUDA, "sweep grid of %d blocks exceeds the %d the group sums hold", nblocks,
                    kGroupBlocks * kMaxGroups);
    h->sweep_blocks = nblocks;
    CVO_CUDA(ensure(h->part_stats, (size_t)kStatN * nblocks * sizeof(float2)));
    CVO_CUDA(ensure(h->part_cnt, (size_t)2 * nblocks * sizeof(unsigned long long)));
    CVO_CUDA(ensure(h->grp_stats, (size_t)kStatN * kMaxGroups * sizeof(float2)));
    CVO_CUDA(ensure(h->grp_cnt, (size_t)2 * kMaxGroups * sizeof(unsigned long long)));
    CVO_CUDA(ensure(h->grp_arrivals, (size_t)kMaxGroups * sizeof(unsigned)));
    CVO_CUDA(ensure(h->counters, 16 * sizeof(unsigned)));
    CVO_CUDA(cudaMemsetAsync(h->grp_arrivals.p, 0, (size_t)kMaxGroups * sizeof(unsigned), h->s));
    CVO_CUDA(cudaMemsetAsync(h->counters.p, 0, 16 * sizeof(unsigned), h->s));
    CVO_CUDA(ensure(h->pairs_dev, table.size() * sizeof(PairDesc)));
    CVO_CUDA(cudaMemcpyAsync(h->pairs_dev.p, table.data(), table.size() * sizeof(PairDesc), cudaMemcpyHostToDevice,
                             h->s));
    a->pairs = (const PairDesc*)h->pairs_dev.p;
    a->npairs = (int)table.size();
    a->rs = h->rs;
    a->dense = h->dense;
    a->part_stats = (float2*)h->part_stats.p;
    a->part_cnt = (unsigned long long*)h->part_cnt.p;
    a->part_cap = nblocks;
    a->grp_stats = (float2*)h->grp_stats.p;
    a->grp_cnt = (unsigned long long*)h->grp_cnt.p;
    a->grp_arrivals = groups ? (unsigned*)h->grp_arrivals.p : nullptr;
    a->fc = h->fc;
    a->nch_next = nullptr;
    a->swept_level = (int*)h->counters.p + 10;
    a->chunk_len = h->chunk_len;
    a->lanes = h->query_lanes;
    return CVO_OK;
}

PairDesc pair_desc(const PairRes& P, int b0, int b1)
{
    PairDesc d;
    d.levels = (const LevelDesc*)P.levels_dev.p;
    d.xrec = (const float4*)P.xrec.p;
    d.st = (IterState*)P.state.p;
    d.n = P.n;
    d.m = P.m;
    d.b0 = b0;
    d.b1 = b1;
    d.bmax = b1 - b0;
    return d;
}

// Sweep blocks resident at once on the device for the handle's feature policy.
// queue_pairs > 0: the work-queue sweep of a batch of that many pairs.
cvo_status resident_sweep_blocks(cvo_handle h, int* out, int queue_pairs = 0)
{
    SweepLaunch sl;
    CVO_CUDA(sweep_launch_info(h->fc, h->rs, h->query_lanes, &sl, queue_pairs > 0));
    const size_t smem = sl.smem + (queue_pairs > 0 ? queue_smem(queue_pairs) : 0);
    int per_sm = 0;
    CVO_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sl.func, sl.threads, smem));
    *out = std::max(per_sm, 1) * h->num_sms;
    return CVO_OK;
}

int single_pair_blocks(cvo_handle h, const PairRes& P)
{
    return std::max(1, std::min((P.max_items + kSweepWarps - 1) / kSweepWarps, h->num_sms * kSweepBlocksPerSm));
}

// The pairs' states into h->h_state: gathered on the device and copied back
// at once (one pair: copied directly).
cvo_status fetch_states(cvo_handle h, int npairs)
{
    if (npairs > 1) {
        CVO_CUDA(ensure(h->d_stage, (size_t)npairs * sizeof(IterState)));
        std::vector<CopyJob> jobs(npairs);
        for (int k = 0; k < npairs; ++k)
            jobs[k] = CopyJob{h->pr[k].state.p, (unsigned char*)h->d_stage.p + (size_t)k * sizeof(IterState),
                              (int)sizeof(IterState)};
        CVO_CUDA(launch_copy_batch(jobs.data(), npairs, h->s));
        CVO_CUDA(cudaMemcpyAsync(h->h_state, h->d_stage.p, (size_t)npairs * sizeof(IterState), cudaMemcpyDeviceToHost,
                                 h->s));
    } else {
        for (int k = 0; k < npairs; ++k)
            CVO_CUDA(cudaMemcpyAsync(h->h_state + k, h->pr[k].state.p, sizeof(IterState), cudaMemcpyDeviceToHost,
                                     h->s));
    }
    CVO_CUDA(cudaStreamSynchronize(h->s));
    return CVO_OK;
}

void fill_info(const IterState* st, cvo_info* inf)
{
    inf->iters = st->iter;
    inf->status = st->status == 0 ? CVO_OK : CVO_NOT_CONVERGED;
    inf->ell_final = st->ell_last;
    inf->F = st->F;
    inf->i_theta = st->i_theta;
    inf->last_step_rot = st->srot;
    inf->last_step_trans = st->strans;
    inf->pairs = st->pairs_total;
    inf->candidates = st->cands_total;
}

cvo_status begin_call(cvo_handle h, int rec_bf16, int npairs)
{
    set_features(h, rec_bf16);
    if ((int)h->pr.size() < npairs) h->pr.resize(npairs);
    CVO_TRY(ensure_host_states(h, npairs));
    return CVO_OK;
}

int rec_bf16_of(const cvo_params& p, const cvo_cloud* X, const cvo_cloud* Z)
{
    return (feat_dim(p) > 0 && X->feat_dtype == CVO_BF16 && Z->feat_dtype == CVO_BF16) ? 1 : 0;
}

cvo_status run_eval(cvo_handle h, const cvo_cloud* X, const cvo_cloud* Z, const double* T, cvo_eval* out)
{
    std::memset(out, 0, sizeof(*out));
    if (X->n == 0 || Z->n == 0) return CVO_OK;
    CVO_TRY(begin_call(h, rec_bf16_of(h->p, X, Z), 1));
    PairRes& P = h->pr[0];
    CVO_TRY(prepare(h, P, X, Z, h->p.ell, h->p.ell));
    CVO_TRY(init_state(h, P, 0, T, h->p.ell, 0, kPlanned));
    const int nb = single_pair_blocks(h, P);
    SweepArgs a{};
    CVO_TRY(setup_sweep(h, std::vector<PairDesc>{pair_desc(P, 0, nb)}, nb, &a, true));
    CVO_CUDA(launch_sweep(a, nb, h->s));
    CVO_CUDA(launch_finalize((IterState*)P.state.p, a.grp_stats, a.grp_cnt, nb, nullptr, h->s));
    CVO_TRY(fetch_states(h, 1));
    const IterState* st = h->h_state;
    out->F = st->F;
    for (int q = 0; q < 6; ++q) out->grad[q] = st->grad[q];
    for (int q = 0; q < 36; ++q) out->hess[q] = st->hess[q];
    out->i_theta = st->i_theta;
    out->pairs = st->pairs;
    out->candidates = st->cands;
    return CVO_OK;
}

// Builds, instantiates and launches the graph of a registration loop: a WHILE
// conditional node whose body is (sweep, finalize, sweep, finalize); the
// finalize (single pair) or the batched finalize's last block (batch) clears
// the condition.
cvo_status run_graph_loop(cvo_handle h, const SweepArgs& a, bool batch, IterState* st_single, double* trace,
                          long long trace_stride, LevelDesc* levels)
{
    SweepLaunch sl;
    CVO_CUDA(sweep_launch_info(a.fc, a.rs, a.lanes, &sl, a.item_rows != nullptr));
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ge = nullptr;
    cvo_status status = CVO_OK;
    auto cleanup = [&]() {
        if (ge) cudaGraphExecDestroy(ge);
        if (g) cudaGraphDestroy(g);
    };
    auto check = [&](cudaError_t e, const char* what) {
        if (e != cudaSuccess && status == CVO_OK)
            status = fail(CVO_ERR_CUDA, "registration graph: %s: %s", what, cudaGetErrorString(e));
        return e == cudaSuccess;
    };
    if (!check(cudaGraphCreate(&g, 0), "cudaGraphCreate")) return cleanup(), status;
    cudaGraphConditionalHandle cond;
    if (!check(cudaGraphConditionalHandleCreate(&cond, g, 1u, cudaGraphCondAssignDefault), "conditional handle"))
        return cleanup(), status;
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = cond;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t cn;
    if (!check(cudaGraphAddNode(&cn, g, nullptr, nullptr, 0, &cp), "conditional node")) return cleanup(), status;
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    SweepArgs sargs = a;
    void* sp[1] = {&sargs};
    cudaGraphNodeParams kp = {};
    kp.type = cudaGraphNodeTypeKernel;
    kp.kernel.func = (void*)sl.func;
    kp.kernel.gridDim = dim3(h->sweep_blocks);
    kp.kernel.blockDim = dim3(sl.threads);
    kp.kernel.sharedMemBytes = (unsigned)(sl.smem + (a.item_rows != nullptr ? queue_smem(a.npairs) : 0));
    kp.kernel.kernelParams = sp;
    cudaGraphNode_t sn;
    if (!check(cudaGraphAddNode(&sn, body, nullptr, nullptr, 0, &kp), "sweep node")) return cleanup(), status;
    int use_cond = 1;
    double* tr = trace;
    cudaGraphNodeParams fpn = {};
    fpn.type = cudaGraphNodeTypeKernel;
    fpn.kernel.blockDim = dim3(kFinalizeThreads);
    fpn.kernel.sharedMemBytes = 0;
    // single pair
    IterState* st = st_single;
    const float2* gs = a.grp_stats;
    const unsigned long long* gcn = a.grp_cnt;
    int ngroups = (h->sweep_blocks + kGroupBlocks - 1) / kGroupBlocks;
    void* fp1[7] = {&st, &gs, &gcn, &ngroups, &tr, &cond, &use_cond};
    // single pair with a cutoff: the next sweep's items laid out beside each step
    const bool lay = !batch && a.nch_next != nullptr;
    LevelDesc* lv = levels;
    const int* swl = a.swept_level;
    const unsigned* nn = a.nch_next;
    void* lp[3] = {&lv, &swl, &nn};
    cudaGraphNodeParams lpn = {};
    lpn.type = cudaGraphNodeTypeKernel;
    lpn.kernel.func = (void*)layout_kernel();
    lpn.kernel.gridDim = dim3(1);
    lpn.kernel.blockDim = dim3(kLayoutThreads);
    lpn.kernel.kernelParams = lp;
    // batch
    PairDesc* pairs = const_cast<PairDesc*>(a.pairs);   // the batched step re-splits the grid in place
    int npairs = a.npairs;
    const float2* ps = a.part_stats;
    const unsigned long long* pc = a.part_cnt;
    int cap = a.part_cap;
    long long tstride = trace_stride;
    unsigned* counters = (unsigned*)h->counters.p;
    unsigned* work = (unsigned*)h->batch_work.p;
    void* fpb[11] = {&pairs, &npairs, &ps, &pc, &cap, &tr, &tstride, &counters, &work, &cond, &use_cond};
    BatchQueue bq{a.item_rows, const_cast<int*>(a.ibase), a.queue};
    void* fpq[9] = {&pairs, &npairs, &tr, &tstride, &counters, &work, &bq, &cond, &use_cond};
    if (batch && a.item_rows != nullptr) {
        fpn.kernel.func = (void*)finalize_batch_queue_kernel();
        fpn.kernel.gridDim = dim3(npairs * kStepCluster);
        fpn.kernel.kernelParams = fpq;
    } else if (batch) {
        fpn.kernel.func = (void*)finalize_batch_kernel();
        fpn.kernel.gridDim = dim3(npairs);
        fpn.kernel.kernelParams = fpb;
    } else {
        fpn.kernel.func = (void*)finalize_kernel();
        fpn.kernel.gridDim = dim3(1);
        fpn.kernel.blockDim = dim3(kStepThreads);
        fpn.kernel.kernelParams = fp1;
    }
    // two iterations per pass of the loop body (halves the conditional
    // node's per-pass overhead; a sweep or step after the last iteration
    // sees the state done and returns at once)
    cudaGraphNode_t fn, sn2, fn2, ln[2];
    if (!check(cudaGraphAddNode(&fn, body, &sn, nullptr, 1, &fpn), "finalize node")) return cleanup(), status;
    if (lay && !check(cudaGraphAddNode(&ln[0], body, &sn, nullptr, 1, &lpn), "layout node")) return cleanup(), status;
    cudaGraphNode_t dep2[2] = {fn, lay ? ln[0] : fn};
    if (!check(cudaGraphAddNode(&sn2, body, dep2, nullptr, lay ? 2 : 1, &kp), "sweep node")) return cleanup(), status;
    if (!check(cudaGraphAddNode(&fn2, body, &sn2, nullptr, 1, &fpn), "finalize node")) return cleanup(), status;
    if (lay && !check(cudaGraphAddNode(&ln[1], body, &sn2, nullptr, 1, &lpn), "layout node")) return cleanup(), status;
    if (!check(cudaGraphInstantiate(&ge, g, 0), "instantiate")) return cleanup(), status;
    if (!check(cudaGraphLaunch(ge, h->s), "launch")) return cleanup(), status;
    check(cudaStreamSynchronize(h->s), "synchronize");
    cleanup();
    return status;
}

void ensure_events(cvo_handle h, int iters)
{
    const size_t need = (size_t)2 * iters;
    while (h->evs.size() < need) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) break;
        h->evs.push_back(e);
    }
}

double sum_sweep_events(cvo_handle h, int iters)
{
    double tot = 0.0;
    for (int it = 0; it < iters && 2 * it + 1 < (int)h->evs.size(); ++it) {
        float ms = 0.0f;
        if (cudaEventElapsedTime(&ms, h->evs[2 * it], h->evs[2 * it + 1]) == cudaSuccess) tot += ms;
    }
    return tot;
}

// lengthscales a registration can reach: a decay needs a reference indicator
// from the previous iteration at the same lengthscale, so at most one decay
// happens every two iterations and no grid level below this one is used
double reachable_ell_lo(const cvo_params& p)
{
    if (!p.anneal) return p.ell;
    return std::max(p.ell_min, p.ell * std::pow(p.decay, (double)(p.max_iters / 2)) * 0.9999);
}

cvo_status run_register(cvo_handle h, const cvo_cloud* X, const cvo_cloud* Z, const double* T_init, double* T_out,
                        cvo_info* info)
{
    const cvo_params& p = h->p;
    cvo_info inf;
    std::memset(&inf, 0, sizeof(inf));
    h->last_iters = 0;
    h->sweep_ms = 0.0;
    h->sweep_n = 0;
    if (X->n == 0 || Z->n == 0 || p.max_iters == 0) {
        std::memcpy(T_out, T_init, 16 * sizeof(double));
        inf.status = (X->n == 0 || Z->n == 0) ? CVO_OK : CVO_NOT_CONVERGED;
        inf.ell_final = p.ell;
        if (info) *info = inf;
        return (cvo_status)inf.status;
    }
    CVO_TRY(begin_call(h, rec_bf16_of(p, X, Z), 1));
    PairRes& P = h->pr[0];
    CVO_TRY(prepare(h, P, X, Z, p.ell, reachable_ell_lo(p)));
    // the dense sum streams all of Z for every group whatever the pose, so a
    // plan made at the start holds; with a cutoff the streams follow the pose:
    // the first sweep of a level takes uniform items, and each sweep records
    // every group's stream length, from which a kernel beside the step lays
    // out the next sweep's items, at most chunk_len candidates each (a plan
    // made once at the start pose for every level measured slower)
    CVO_TRY(init_state(h, P, 0, T_init, p.ell, 1, h->dense ? kPlanned : kUniform));
    CVO_CUDA(ensure(h->trace, (size_t)p.max_iters * CVO_TRACE_STRIDE * sizeof(double)));
    const bool persistent = h->loop_mode == 2;
    const bool replan = !h->dense && !persistent;
    // re-planned items: two waves of four blocks per SM dealt round robin
    // (one wave measured 1 % faster on street-20k and 4 % slower on
    // box80-200k)
    const int nb = replan ? h->num_sms * kSweepBlocksPerSm : single_pair_blocks(h, P);
    SweepArgs a{};
    CVO_TRY(setup_sweep(h, std::vector<PairDesc>{pair_desc(P, 0, nb)}, nb, &a, true));
    double* trace = (double*)h->trace.p;
    IterState* dst = (IterState*)P.state.p;
    int max_groups = 1;
    for (int k = 0; k < P.nlevels; ++k) max_groups = std::max(max_groups, P.lv[k].ngroups);
    CVO_CUDA(ensure(h->gidx, (size_t)std::max(max_groups, P.n) * sizeof(unsigned)));
    LevelDesc* levels = replan ? (LevelDesc*)P.levels_dev.p : nullptr;
    unsigned* nch_next = replan ? (unsigned*)h->gidx.p : nullptr;
    a.nch_next = nch_next;
    a.chunk_len = h->chunk_len;
    const bool graph = !persistent && !h->timing && h->loop_mode == 1;
    if (persistent) {
        // one cooperative launch for the whole loop (events around it when timing)
        int grid = 0;
        CVO_CUDA(persistent_grid(a, &grid));
        if (grid < 1) return fail(CVO_ERR_CUDA, "persistent loop: no resident block fits");
        grid = std::min(grid, kGroupBlocks * kMaxGroups);
        if (grid > a.part_cap) CVO_TRY(setup_sweep(h, std::vector<PairDesc>{pair_desc(P, 0, grid)}, grid, &a, true));
        if (h->timing) {
            ensure_events(h, 1);
            CVO_CUDA(cudaEventRecord(h->evs[0], h->s));
        }
        const int leave_at = h->inj_leave_at;
        const unsigned polls = h->inj_polls;
        h->inj_leave_at = -1;   // one registration only
        h->inj_polls = 0;
        CVO_CUDA(launch_register_persistent(a, (unsigned*)h->counters.p, (unsigned*)h->gidx.p, h->chunk_len, trace,
                                            grid, leave_at, polls, h->s));
        if (h->timing) CVO_CUDA(cudaEventRecord(h->evs[1], h->s));
        CVO_CUDA(cudaMemcpyAsync(h->h_misc + 40, (unsigned*)h->counters.p + 4, sizeof(unsigned), cudaMemcpyDeviceToHost,
                                 h->s));
        CVO_CUDA(cudaStreamSynchronize(h->s));
        if (h->h_misc[40] != 0u) return fail(CVO_ERR_TIMEOUT, "persistent loop: a grid barrier gave up waiting");
    } else if (graph) {
        CVO_TRY(run_graph_loop(h, a, false, dst, trace, 0, levels));
    } else {
        // iterations queued from the host in batches (CUDA events around each
        // sweep when timing); the device-side state stops the kernels once the
        // registration is done, and the host checks between batches
        if (h->timing) ensure_events(h, p.max_iters);
        const int batch = 8;
        int launched = 0;
        while (launched < p.max_iters) {
            const int n = std::min(batch, p.max_iters - launched);
            for (int k = 0; k < n; ++k) {
                const int it = launched + k;
                const bool ev = h->timing && 2 * it + 1 < (int)h->evs.size();
                if (ev) CVO_CUDA(cudaEventRecord(h->evs[2 * it], h->s));
                CVO_CUDA(launch_sweep(a, nb, h->s));
                if (ev) CVO_CUDA(cudaEventRecord(h->evs[2 * it + 1], h->s));
                if (replan) CVO_CUDA(launch_layout(levels, a.swept_level, nch_next, h->s));
                CVO_CUDA(launch_finalize(dst, a.grp_stats, a.grp_cnt, nb, trace, h->s));
            }
            launched += n;
            if (launched >= p.max_iters) break;
            CVO_CUDA(cudaMemcpyAsync(&h->h_state->done, &dst->done, sizeof(int), cudaMemcpyDeviceToHost, h->s));
            CVO_CUDA(cudaStreamSynchronize(h->s));
            if (h->h_state->done) break;
        }
    }
    CVO_TRY(fetch_states(h, 1));
    const IterState* st = h->h_state;
    std::memcpy(T_out, st->T, 16 * sizeof(double));
    fill_info(st, &inf);
    h->last_iters = st->iter;
    // four kernels (six with the layout) per pass of the graph's loop body, two iterations a pass
    if (graph) g_launch_count.fetch_add((replan ? 6LL : 4LL) * ((st->iter + 1) / 2), std::memory_order_relaxed);
    if (h->timing && persistent) {
        // the persistent kernel as a whole (sweeps and steps), per iteration
        float ms = 0.0f;
        if (cudaEventElapsedTime(&ms, h->evs[0], h->evs[1]) == cudaSuccess && st->iter > 0) {
            h->sweep_ms = ms;
            h->sweep_n = st->iter;
        }
    } else if (h->timing) {
        h->sweep_ms = sum_sweep_events(h, st->iter);
        h->sweep_n = st->iter;
    }
    if (info) *info = inf;
    return (cvo_status)inf.status;
}

cvo_status run_register_batch(cvo_handle h, int npairs, const cvo_cloud* X, const cvo_cloud* Z, const double* T_init,
                              double* T_out, cvo_info* infos)
{
    const cvo_params& p = h->p;
    h->last_iters = 0;
    h->sweep_ms = 0.0;
    h->sweep_n = 0;
    // pairs that need iterations; the rest return T_init
    std::vector<int> live;
    for (int k = 0; k < npairs; ++k) {
        const bool empty = X[k].n == 0 || Z[k].n == 0;
        if (empty || p.max_iters == 0) {
            std::memcpy(T_out + 16 * k, T_init + 16 * k, 16 * sizeof(double));
            if (infos) {
                std::memset(infos + k, 0, sizeof(cvo_info));
                infos[k].status = empty ? CVO_OK : CVO_NOT_CONVERGED;
                infos[k].ell_final = p.ell;
            }
        } else {
            live.push_back(k);
        }
    }
    const int nl = (int)live.size();
    if (nl == 0) return p.max_iters == 0 && npairs > 0 ? CVO_NOT_CONVERGED : CVO_OK;
    // the pairs in order of Z's size, largest first: the sweep's blocks (and
    // the work queue's items) go to them in this order, so every sweep ends on
    // small pairs' short items instead of waiting for a large pair's long
    // ones started last (batch-64: block split 28.7 -> 26.9 ms, work queue
    // 27.9 -> 27.2 ms); a pair's result does not depend on its place
    std::stable_sort(live.begin(), live.end(), [&](int x, int y) { return Z[x].n > Z[y].n; });
    int bf = 1;
    for (int k : live) bf &= rec_bf16_of(p, X + k, Z + k);
    CVO_TRY(begin_call(h, bf, nl));
    const double ell_lo = reachable_ell_lo(p);
    long long work = 0;
    // host-resident inputs first copied to the pairs' own device buffers, so
    // that every batch takes the batched set-up (unless CVO_BATCH_SETUP=pairs
    // in the environment selects the pair-by-pair one, for comparison)
    const char* mode = std::getenv("CVO_BATCH_SETUP");
    const bool batched = nl > 1 && !(mode && std::strcmp(mode, "pairs") == 0);
    std::vector<cvo_cloud> Xd, Zd;
    if (batched) {
        Xd.assign(X, X + npairs);
        Zd.assign(Z, Z + npairs);
        const int D = h->D;
        // page-locked host inputs pulled by one kernel launch per 64 arrays
        // (the SMs read the mapped host memory at the link's rate: batch-64's
        // 256 arrays, 224 MB, add 1.05 ms to the batch against 1.6 ms as
        // copy-engine copies); pageable ones copied by the driver
        std::vector<PullJob> pulls;
        auto copy_in = [&](void* dst, const void* src, size_t bytes) -> cvo_status {
            if (bytes == 0) return CVO_OK;
            cudaPointerAttributes at;
            if (cudaPointerGetAttributes(&at, src) == cudaSuccess && at.type == cudaMemoryTypeHost &&
                at.devicePointer != nullptr) {
                pulls.push_back(PullJob{at.devicePointer, dst, (long long)bytes});
                return CVO_OK;
            }
            (void)cudaGetLastError();   // an unregistered pointer's query leaves no error behind
            CVO_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, h->s));
            return CVO_OK;
        };
        for (int i = 0; i < nl; ++i) {
            const int k = live[i];
            cvo_cloud* c[2] = {&Xd[k], &Zd[k]};
            for (int side = 0; side < 2; ++side) {
                cvo_cloud& cl = *c[side];
                if (cl.on_device) continue;
                PairRes& P = h->pr[i];
                const size_t bx = (size_t)cl.n * 3 * sizeof(float);
                CVO_CUDA(ensure(P.in_xyz[side], bx));
                CVO_TRY(copy_in(P.in_xyz[side].p, cl.xyz, bx));
                cl.xyz = (const float*)P.in_xyz[side].p;
                if (D > 0) {
                    const size_t bf = (size_t)cl.n * D * (cl.feat_dtype == CVO_BF16 ? 2 : 4);
                    CVO_CUDA(ensure(P.in_feat[side], bf));
                    CVO_TRY(copy_in(P.in_feat[side].p, cl.feat, bf));
                    cl.feat = P.in_feat[side].p;
                }
                cl.on_device = 1;
            }
        }
        if (!pulls.empty()) CVO_CUDA(launch_pull_batch(pulls.data(), (int)pulls.size(), h->s));
        // every pair's set-up stage in one launch for all pairs
        CVO_TRY(prepare_batch(h, live, Xd.data(), Zd.data(), T_init, &work));
    } else {
        for (int i = 0; i < nl; ++i) {
            CVO_TRY(prepare(h, h->pr[i], X + live[i], Z + live[i], p.ell, ell_lo));
            CVO_TRY(init_state(h, h->pr[i], i, T_init + 16 * live[i], p.ell, 1, kPlanned));
            work += h->pr[i].max_items;
        }
    }
    // split eight waves of resident blocks among the pairs in proportion to
    // their work items (largest remainders, at least one item per warp): the
    // blocks then balance dynamically as they retire.  Measured on 64 cube
    // pairs (608 resident blocks): 878 blocks (two waves, the second partly
    // filled) 131 ms per batch; one wave 143 ms (no balancing within it);
    // 2, 4, 8, 16, 32 waves 131, 117, 113, 113, 116 ms
    // the block split below, or with CVO_BATCH_QUEUE=1 in the environment the
    // work queue: one resident wave whose warps take the items of all running
    // pairs from a counter (its results do not depend on the grid; with the
    // pairs largest first the block split measured 0.8 % faster)
    const char* qmode = std::getenv("CVO_BATCH_QUEUE");
    const bool queue = qmode && std::strcmp(qmode, "1") == 0 && queue_smem(nl) <= 16384;   // ibase in shared memory
    int resident = 0;
    CVO_TRY(resident_sweep_blocks(h, &resident, queue ? nl : 0));
    const int budget = queue ? std::max(nl, resident) : std::max(nl, 8 * resident);
    std::vector<int> nbs(nl), cap(nl);
    std::vector<std::pair<double, int>> rem;
    int used = 0;
    for (int i = 0; i < nl; ++i) {
        const PairRes& P = h->pr[i];
        const double quota = (double)budget * P.max_items / (double)std::max(work, 1LL);
        cap[i] = std::max(1, (P.max_items + kSweepWarps - 1) / kSweepWarps);
        nbs[i] = std::max(1, std::min(cap[i], (int)quota));
        used += nbs[i];
        rem.push_back({quota - (double)nbs[i], i});
    }
    std::sort(rem.begin(), rem.end(), [](const std::pair<double, int>& x, const std::pair<double, int>& y) {
        return x.first > y.first || (x.first == y.first && x.second < y.second);
    });
    for (size_t r = 0; r < rem.size() && used < budget; ++r) {
        const int i = rem[r].second;
        if (rem[r].first > 0.0 && nbs[i] < cap[i]) {
            ++nbs[i];
            ++used;
        }
    }
    std::vector<PairDesc> table;
    int b = 0;
    for (int i = 0; i < nl; ++i) {
        table.push_back(pair_desc(h->pr[i], b, b + nbs[i]));
        // as pairs stop, the batched step hands their blocks to the pairs
        // still running: each up to 8 times its first share, and never more
        // blocks than it has work items for
        table.back().bmax = std::max(1, std::min(cap[i], 8 * nbs[i]));
        b += nbs[i];
    }
    if (queue) b = budget;   // the block ranges are not used
    SweepArgs a{};
    CVO_TRY(setup_sweep(h, table, b, &a, false));
    CVO_CUDA(ensure(h->batch_work, (size_t)nl * sizeof(unsigned)));
    if (queue) {
        // a row per work item of each pair's largest grid level
        size_t rows = 0;
        for (int i = 0; i < nl; ++i) rows += (size_t)std::max(h->pr[i].max_items, 1);
        CVO_CUDA(ensure(h->item_rows, rows * kRowFloats * sizeof(float)));
        CVO_CUDA(ensure(h->queue_buf, (size_t)(4 + nl + 1) * sizeof(unsigned)));
        a.item_rows = (float*)h->item_rows.p;
        a.queue = (unsigned*)h->queue_buf.p;
        a.ibase = (const int*)((unsigned*)h->queue_buf.p + 4);
        CVO_CUDA(launch_queue_init(a.pairs, nl, (unsigned*)h->batch_work.p, const_cast<int*>(a.ibase), a.queue, h->s));
    }
    const long long tstride = (long long)p.max_iters * CVO_TRACE_STRIDE;
    CVO_CUDA(ensure(h->trace, (size_t)nl * tstride * sizeof(double)));
    double* traces = (double*)h->trace.p;
    const bool graph = !h->timing && h->loop_mode != 0;
    if (graph) {
        CVO_TRY(run_graph_loop(h, a, true, nullptr, traces, tstride, nullptr));
    } else {
        if (h->timing) ensure_events(h, p.max_iters);
        unsigned* counters = (unsigned*)h->counters.p;
        const int batch = 8;
        int launched = 0;
        while (launched < p.max_iters) {
            const int n = std::min(batch, p.max_iters - launched);
            for (int k = 0; k < n; ++k) {
                const int it = launched + k;
                const bool ev = h->timing && 2 * it + 1 < (int)h->evs.size();
                if (ev) CVO_CUDA(cudaEventRecord(h->evs[2 * it], h->s));
                CVO_CUDA(launch_sweep(a, b, h->s));
                if (ev) CVO_CUDA(cudaEventRecord(h->evs[2 * it + 1], h->s));
                CVO_CUDA(launch_finalize_batch(const_cast<PairDesc*>(a.pairs), nl, a.part_stats, a.part_cnt,
                                               a.part_cap, traces, tstride, counters, (unsigned*)h->batch_work.p,
                                               BatchQueue{a.item_rows, const_cast<int*>(a.ibase), a.queue}, h->s));
            }
            launched += n;
            if (launched >= p.max_iters) break;
            CVO_CUDA(cudaMemcpyAsync(h->h_misc + 40, counters + 2, sizeof(unsigned), cudaMemcpyDeviceToHost, h->s));
            CVO_CUDA(cudaStreamSynchronize(h->s));
            if (h->h_misc[40] == 0) break;
        }
    }
    CVO_TRY(fetch_states(h, nl));
    cvo_status worst = CVO_OK;
    int max_it = 0;
    for (int i = 0; i < nl; ++i) {
        const IterState* st = h->h_state + i;
        const int k = live[i];
        std::memcpy(T_out + 16 * k, st->T, 16 * sizeof(double));
        if (infos) {
            std::memset(infos + k, 0, sizeof(cvo_info));
            fill_info(st, infos + k);
        }
        if (st->status != 0) worst = CVO_NOT_CONVERGED;
        max_it = std::max(max_it, st->iter);
    }
    if (graph) g_launch_count.fetch_add(4LL * ((max_it + 1) / 2), std::memory_order_relaxed);
    if (h->timing) {
        h->sweep_ms = sum_sweep_events(h, max_it);
        h->sweep_n = max_it;
    }
    h->last_iters = 0;   // per-pair traces are not exposed through cvo_get_trace
    return worst;
}

// X-row shard of one registration (the multi-GPU design of partitioning X
// by rows; the paper uses one GPU): this handle holds rows of X and all of
// Z, and its sweeps' statistics are summed with the other shards' before
// every step, so every shard takes the same step.  The set-up is that of
// run_register, with the indicator normalised by the whole cloud's size.
cvo_status run_shard_begin(cvo_handle h, const cvo_cloud* X, const cvo_cloud* Z, long long n_total, const double* T_init)
{
    const cvo_params& p = h->p;
    h->shard_active = 0;
    h->last_iters = 0;
    CVO_TRY(begin_call(h, rec_bf16_of(p, X, Z), 1));
    PairRes& P = h->pr[0];
    CVO_TRY(prepare(h, P, X, Z, p.ell, reachable_ell_lo(p)));
    CVO_TRY(init_state(h, P, 0, T_init, p.ell, 1, h->dense ? kPlanned : kUniform));
    // i_theta = F / sqrt(N M) with N the rows of every shard (Eq. indicator_actual)
    IterState* dst = (IterState*)P.state.p;
    h->h_state->norm = 1.0 / std::sqrt((double)n_total * (double)P.m);
    CVO_CUDA(cudaMemcpyAsync(&dst->norm, &h->h_state->norm, sizeof(double), cudaMemcpyHostToDevice, h->s));
    CVO_CUDA(ensure(h->trace, (size_t)std::max(p.max_iters, 1) * CVO_TRACE_STRIDE * sizeof(double)));
    const bool replan = !h->dense;
    const int nb = replan ? h->num_sms * kSweepBlocksPerSm : single_pair_blocks(h, P);
    SweepArgs a{};
    CVO_TRY(setup_sweep(h, std::vector<PairDesc>{pair_desc(P, 0, nb)}, nb, &a, true));
    int max_groups = 1;
    for (int k = 0; k < P.nlevels; ++k) max_groups = std::max(max_groups, P.lv[k].ngroups);
    CVO_CUDA(ensure(h->gidx, (size_t)std::max(max_groups, P.n) * sizeof(unsigned)));
    a.nch_next = replan ? (unsigned*)h->gidx.p : nullptr;
    a.chunk_len = h->chunk_len;
    h->shard_a = a;
    h->shard_nb = nb;
    h->shard_levels = replan ? (LevelDesc*)P.levels_dev.p : nullptr;
    CVO_CUDA(cudaStreamSynchronize(h->s));
    h->shard_active = 1;
    return CVO_OK;
}

// Gradients of F(T) with respect to both clouds' points and features and to
// the lengthscale: one gradient sweep per cloud, each with that cloud as the
// queries over a grid of the other (no atomics, so the result is
// deterministic), and a fixed-order sum for dF/dl.
cvo_status run_backward(cvo_handle h, const cvo_cloud* X, const cvo_cloud* Z, const double* T, double dF, float* dX,
                        float* dFX, float* dZ, float* dFZ, double* dell, int on_dev)
{
    const cvo_params& p = h->p;
    const int D = feat_dim(p);
    const int n = X->n, m = Z->n;
    float* outs[4] = {dX, dFX, dZ, dFZ};
    const size_t bytes[4] = {(size_t)n * 3 * sizeof(float), (size_t)n * D * sizeof(float),
                             (size_t)m * 3 * sizeof(float), (size_t)m * D * sizeof(float)};
    if (dell) *dell = 0.0;
    if (n == 0 || m == 0) {
        // no pair: every gradient is zero
        for (int k = 0; k < 4; ++k) {
            if (!outs[k] || bytes[k] == 0) continue;
            if (on_dev) CVO_CUDA(cudaMemsetAsync(outs[k], 0, bytes[k], h->s));
            else std::memset(outs[k], 0, bytes[k]);
        }
        CVO_CUDA(cudaStreamSynchronize(h->s));
        return CVO_OK;
    }
    CVO_TRY(begin_call(h, rec_bf16_of(p, X, Z), 2));
    // device destinations
    float* dev[4];
    for (int k = 0; k < 4; ++k) {
        dev[k] = nullptr;
        if (!outs[k] || bytes[k] == 0) continue;
        if (on_dev) {
            dev[k] = outs[k];
        } else {
            CVO_CUDA(ensure(h->bw_out[k], bytes[k]));
            dev[k] = (float*)h->bw_out[k].p;
        }
    }
    const double ell = p.ell;
    const double sc = dF * h->kappa;
    GradArgs g;
    std::memset(&g, 0, sizeof(g));
    g.rs = h->rs;
    g.dense = h->dense;
    g.fc = h->fc;
    g.scale_pos = (float)(sc / (ell * ell));
    g.scale_ell = (float)(sc / (ell * ell * ell));
    for (int b = 0, col = 0; b < p.n_blocks; ++b)
        for (int j = 0; j < p.blocks[b].dim; ++j, ++col)
            g.feat_scale[col] = p.blocks[b].kind == CVO_FEAT_SE
                                    ? (float)(-sc / (p.blocks[b].scale * p.blocks[b].scale))
                                    : (float)sc;
    auto sweep = [&](int slot, const cvo_cloud* Q, const cvo_cloud* G, const double* Tq, bool rout_transpose,
                     float* pos, float* feat, float* tq) -> cvo_status {
        PairRes& P = h->pr[slot];
        CVO_TRY(prepare(h, P, Q, G, ell, ell));
        CVO_TRY(init_state(h, P, slot, Tq, ell, 0, kPlanned));
        g.levels = (const LevelDesc*)P.levels_dev.p;
        g.xrec = (const float4*)P.xrec.p;
        g.st = (const IterState*)P.state.p;
        g.m = P.m;
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) g.Rout[3 * r + c] = (float)(rout_transpose ? T[4 * c + r] : T[4 * r + c]);
        g.out_pos = pos;
        g.out_feat = D > 0 ? feat : nullptr;
        g.out_tq = tq;
        const int nitems = P.lv[0].nitems;
        CVO_CUDA(ensure(h->bw_part, (size_t)std::max(nitems, 1) * 32 * (4 + D) * sizeof(float)));
        g.part = (float*)h->bw_part.p;
        const int nb = std::max(1, std::min((nitems + kSweepWarps - 1) / kSweepWarps, h->num_sms * 2 * kSweepBlocksPerSm));
        const int ev = h->timing ? 2 * h->sweep_n : -1;   // events around each gradient sweep when timing
        if (ev >= 0) CVO_CUDA(cudaEventRecord(h->evs[ev], h->s));
        CVO_CUDA(launch_grad(g, nb, h->s));
        if (ev >= 0) {
            CVO_CUDA(cudaEventRecord(h->evs[ev + 1], h->s));
            ++h->sweep_n;
        }
        return CVO_OK;
    };
    h->sweep_ms = 0.0;
    h->sweep_n = 0;
    if (h->timing) {
        ensure_events(h, 2);
        if (h->evs.size() < 4) return fail(CVO_ERR_CUDA, "cudaEventCreate failed");
    }
    if (dev[0] || dev[1] || dell) {
        float* tq = nullptr;
        if (dell) {
            CVO_CUDA(ensure(h->bw_tq, (size_t)n * sizeof(float)));
            CVO_CUDA(ensure(h->bw_dell, sizeof(double)));
            tq = (float*)h->bw_tq.p;
        }
        CVO_TRY(sweep(0, X, Z, T, false, dev[0], dev[1], tq));
        if (dell) {
            CVO_CUDA(launch_sum_f32(tq, n, (double*)h->bw_dell.p, h->s));
            CVO_CUDA(cudaMemcpyAsync(dell, h->bw_dell.p, sizeof(double), cudaMemcpyDeviceToHost, h->s));
        }
    }
    if (dev[2] || dev[3]) {
        // Z as the queries over the grid of X: the query transform is T itself
        // (T^-1 of the inverse pose), and dF/dz = R^T dF/dy
        double Ti[16];
        for (int r = 0; r < 3; ++r) {
            for (int c = 0; c < 3; ++c) Ti[4 * r + c] = T[4 * c + r];
            Ti[4 * r + 3] = -(T[r] * T[3] + T[4 + r] * T[7] + T[8 + r] * T[11]);
        }
        Ti[12] = Ti[13] = Ti[14] = 0.0;
        Ti[15] = 1.0;
        CVO_TRY(sweep(1, Z, X, Ti, true, dev[2], dev[3], nullptr));
    }
    if (!on_dev)
        for (int k = 0; k < 4; ++k)
            if (dev[k]) CVO_CUDA(cudaMemcpyAsync(outs[k], dev[k], bytes[k], cudaMemcpyDeviceToHost, h->s));
    CVO_CUDA(cudaStreamSynchronize(h->s));
    if (h->timing) h->sweep_ms = sum_sweep_events(h, h->sweep_n);
    return CVO_OK;
}

// Autotuner: a workload (one registration, or one batched registration) run
// under every tuning of a small grid, timed on the host clock as a caller
// sees it (setup, iterations, result copies; best of two runs); the fastest
// is kept.  First the grid cell and query-group extent (with a cutoff), then,
// for the best of those, the work-item length.  The results must not depend
// on the tuning beyond rounding: run() returns a value (F) that every tuning
// must give to 1e-4 relative of the first one's.
template <class Run>
cvo_status tune_grid(cvo_handle h, Run&& run, cvo_tuning* out)
{
    static const double kCell[] = {0.35, 0.5, 0.7, 1.0};
    static const int kSuper[] = {1, 2, 3};
    static const int kLanes[] = {1, 2, 4};
    static const int kItemLens[] = {64, 96, 128, 192, 384, 768, 1536};
    const double cf0 = h->cell_factor;
    const int sd0 = h->super_delta, ip0 = h->chunk_len, ql0 = h->query_lanes;
    cvo_tuning best{cf0, sd0, ip0, 1e30, ql0};
    double F_ref = 0.0;
    bool have_ref = false;
    cvo_status st = CVO_OK;
    auto try_one = [&](double cf, int sd, int ip, int ql) {
        h->cell_factor = cf;
        h->super_delta = sd;
        h->chunk_len = ip;
        h->query_lanes = ql;
        double ms = 1e30, F = 0.0;
        for (int rep = 0; rep < 2; ++rep) {
            const auto t0 = std::chrono::steady_clock::now();
            st = run(&F);
            if (st < 0) return;
            const auto t1 = std::chrono::steady_clock::now();
            ms = std::min(ms, std::chrono::duration<double, std::milli>(t1 - t0).count());
        }
        st = CVO_OK;
        if (!have_ref) {
            F_ref = F;
            have_ref = true;
        } else if (std::fabs(F - F_ref) > 1e-4 * std::fabs(F_ref) + 1e-300) {
            st = fail(CVO_ERR_CUDA, "autotune: F differs between tunings (%g vs %g)", F, F_ref);
            return;
        }
        if (ms < best.measured_ms) best = cvo_tuning{cf, sd, ip, ms, ql};
    };
    // the dense sum has no grid and no super-cells: only the work split is tuned
    if (!(h->p.cutoff_mult > 0.0)) {
        try_one(cf0, sd0, ip0, ql0);
    } else {
        for (double cf : kCell) {
            for (int sd : kSuper) {
                try_one(cf, sd, ip0, ql0);
                if (st < 0) break;
            }
            if (st < 0) break;
        }
    }
    // then the lanes per query, then the work-item length, for the best so far
    for (int ql : kLanes) {
        if (st < 0 || ql == ql0) continue;
        try_one(best.cell_factor, best.super_delta, ip0, ql);
    }
    for (int ip : kItemLens) {
        if (st < 0 || ip == ip0) continue;
        try_one(best.cell_factor, best.super_delta, ip, best.query_lanes);
    }
    if (st < 0) {
        h->cell_factor = cf0;
        h->super_delta = sd0;
        h->chunk_len = ip0;
        h->query_lanes = ql0;
        return st;
    }
    h->cell_factor = best.cell_factor;
    h->super_delta = best.super_delta;
    h->chunk_len = best.chunk_len;
    h->query_lanes = best.query_lanes;
    *out = best;
    return CVO_OK;
}

// One registration of (X, Z) from T; the check value is F at the start pose
// (the first iteration's).
cvo_status run_autotune(cvo_handle h, const cvo_cloud* X, const cvo_cloud* Z, const double* T, cvo_tuning* out)
{
    std::memset(out, 0, sizeof(*out));
    if (X->n == 0 || Z->n == 0 || h->p.max_iters == 0) {
        *out = cvo_tuning{h->cell_factor, h->super_delta, h->chunk_len, 0.0, h->query_lanes};
        return CVO_OK;
    }
    double T_out[16];
    cvo_info inf;
    return tune_grid(
        h,
        [&](double* F) -> cvo_status {
            CVO_TRY(run_register(h, X, Z, T, T_out, &inf));
            double row[2] = {0.0, 0.0};   // l and F of the first iteration
            if (cudaMemcpy(row, h->trace.p, sizeof(row), cudaMemcpyDeviceToHost) != cudaSuccess)
                return fail(CVO_ERR_CUDA, "autotune: trace copy failed");
            *F = row[1];
            return CVO_OK;
        },
        out);
}

// One batched registration of the npairs pairs; the check value is the sum of
// the pairs' F at their start poses (the first row of each running pair's
// trace).
cvo_status run_autotune_batch(cvo_handle h, int npairs, const cvo_cloud* X, const cvo_cloud* Z, const double* T_init,
                              cvo_tuning* out)
{
    std::memset(out, 0, sizeof(*out));
    int nl = 0;   // pairs that run (both clouds non-empty)
    for (int k = 0; k < npairs; ++k) nl += (X[k].n > 0 && Z[k].n > 0) ? 1 : 0;
    if (nl == 0 || h->p.max_iters == 0) {
        *out = cvo_tuning{h->cell_factor, h->super_delta, h->chunk_len, 0.0, h->query_lanes};
        return CVO_OK;
    }
    std::vector<double> T_out((size_t)16 * npairs), rows((size_t)2 * nl);
    const size_t tstride = (size_t)h->p.max_iters * CVO_TRACE_STRIDE * sizeof(double);
    return tune_grid(
        h,
        [&](double* F) -> cvo_status {
            CVO_TRY(run_register_batch(h, npairs, X, Z, T_init, T_out.data(), nullptr));
            // (l, F) of each running pair's first iteration
            if (cudaMemcpy2D(rows.data(), 2 * sizeof(double), h->trace.p, tstride, 2 * sizeof(double), (size_t)nl,
                             cudaMemcpyDeviceToHost) != cudaSuccess)
                return fail(CVO_ERR_CUDA, "autotune: trace copy failed");
            double sum = 0.0;
            for (int i = 0; i < nl; ++i) sum += rows[(size_t)2 * i + 1];
            *F = sum;
            return CVO_OK;
        },
        out);
}

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

}  // namespace

extern "C" {

const char* cvo_last_error(void) { return g_err.c_str(); }

const char* cvo_version(void) { return "cvo-gb300 0.1 (sm_103a)"; }

long long cvo_kernel_launches(void) { return g_launch_count.load(); }

cvo_status cvo_create(const cvo_params* params, void* cuda_stream, cvo_handle* out)
{
    g_err.clear();
    if (!out) return fail(CVO_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    CVO_TRY(check_params(params));
    int dev = 0;
    CVO_CUDA(cudaGetDevice(&dev));
    cvo_handle h = new cvo_handle_s();
    h->p = *params;
    h->s = (cudaStream_t)cuda_stream;
    h->device = dev;
    // The registration loop of one pair runs as a CUDA graph of (sweep,
    // step) kernels by default.  CVO_LOOP=persistent runs it as one
    // persistent kernel, and CVO_LOOP=host (or CVO_GRAPH=0) queues the
    // kernels from the host, so that a profiler can attribute time to each
    // (it cannot for the kernel nodes of a graph with conditional nodes).
    // Batches always use the graph (or the host queue).
    {
        const char* lv = std::getenv("CVO_LOOP");
        const char* gv = std::getenv("CVO_GRAPH");
        if (lv && std::strcmp(lv, "host") == 0) h->loop_mode = 0;
        else if (lv && std::strcmp(lv, "graph") == 0) h->loop_mode = 1;
        else if (gv && gv[0] == '0') h->loop_mode = 0;
        else if (lv && std::strcmp(lv, "persistent") == 0) h->loop_mode = 2;
        else h->loop_mode = 1;
    }
    cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (ensure_host_states(h, 1) != CVO_OK ||
        cudaMallocHost((void**)&h->h_misc, kMiscWords * sizeof(unsigned)) != cudaSuccess) {
        cudaGetLastError();
        if (h->h_state) cudaFreeHost(h->h_state);
        delete h;
        return fail(CVO_ERR_OOM, "cudaMallocHost failed");
    }
    h->h_misc_cap = kMiscWords;
    *out = h;
    return CVO_OK;
}

cvo_status cvo_destroy(cvo_handle h)
{
    if (!h) return CVO_OK;
    DeviceGuard g(h->device);
    cudaStreamSynchronize(h->s);
    DevBuf* bufs[] = {&h->stage_xyz[0], &h->stage_xyz[1], &h->stage_feat[0], &h->stage_feat[1], &h->keys, &h->vals,
                      &h->keys2, &h->vals2, &h->sort_tmp, &h->flags, &h->gidx, &h->misc, &h->part_stats, &h->part_cnt,
                      &h->grp_stats, &h->grp_cnt, &h->grp_arrivals, &h->pairs_dev, &h->counters, &h->trace,
                      &h->batch_work, &h->item_rows, &h->queue_buf, &h->batch_scratch, &h->d_stage,
                      &h->bw_out[0], &h->bw_out[1], &h->bw_out[2], &h->bw_out[3], &h->bw_tq, &h->bw_dell, &h->bw_part};
    for (DevBuf* b : bufs) release(*b);
    for (SetupLane& L : h->lanes) {
        if (L.s) cudaStreamSynchronize(L.s);
        for (DevBuf* b : {&L.keys, &L.vals, &L.keys2, &L.vals2, &L.sort_tmp, &L.flags, &L.gidx}) release(*b);
        if (L.ev) cudaEventDestroy(L.ev);
        if (L.s) cudaStreamDestroy(L.s);
    }
    for (PairRes& P : h->pr) P.free_all();
    for (cudaEvent_t e : h->evs) cudaEventDestroy(e);
    if (h->h_state) cudaFreeHost(h->h_state);
    if (h->h_misc) cudaFreeHost(h->h_misc);
    if (h->h_stage) cudaFreeHost(h->h_stage);
    if (h->stage_ev) cudaEventDestroy(h->stage_ev);
    delete h;
    return CVO_OK;
}

cvo_status cvo_set_params(cvo_handle h, const cvo_params* params)
{
    g_err.clear();
    if (!h) return fail(CVO_ERR_INVALID_ARG, "handle is NULL");
    CVO_TRY(check_params(params));
    h->p = *params;
    return CVO_OK;
}

cvo_status cvo_evaluate(cvo_handle h, const cvo_cloud* X, const cvo_cloud* Z, const double T[16], cvo_eval* out)
{
    g_err.clear();
    if (!h) return fail(CVO_ERR_INVALID_ARG, "handle is NULL");
    if (!out) return fail(CVO_ERR_INVALID_ARG, "out is NULL");
    const int D = feat_dim(h->p);
    CVO_TRY(check_cloud(X, "X", D));
    CVO_TRY(check_cloud(Z, "Z", D));
    CVO_TRY(check_pose(T, "T"));
    DeviceGuard g(h->device);
    return run_eval(h, X, Z, T, out);
}

cvo_status cvo_backward(cvo_handle h, const cvo_cloud* X, const cvo_cloud* Z, const double T[16], double dF,
                        float* dX, float* dFX, float* dZ, float* dFZ, double* dell, int outputs_on_device)
{
    g_err.clear();
    if (!h) return fail(CVO_ERR_INVALID_ARG, "handle is NULL");
    if (!std::isfinite(dF)) return fail(CVO_ERR_INVALID_ARG, "dF must be finite");
    const int D = feat_dim(h->p);
    CVO_TRY(check_cloud(X, "X", D));
    CVO_TRY(check_cloud(Z, "Z", D));
    CVO_TRY(check_pose(T, "T"));
    DeviceGuard g(h->device);
    if (outputs_on_device) {
        float* outs[4] = {dX, dFX, dZ, dFZ};
        for (float* o : outs) {
            if (!o) continue;
            cudaPointerAttributes at;
            if (cudaPointerGetAttributes(&at, o) != cudaSuccess) {
                cudaGetLastError();
                return fail(CVO_ERR_INVALID_ARG, "output pointer is not known to CUDA");
            }
            if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged)
                return fail(CVO_ERR_INVALID_ARG, "outputs_on_device = 1 but an output is not device memory");
        }
    }
    return run_backward(h, X, Z, T, dF, dX, dFX, dZ, dFZ, dell, outputs_on_device ? 1 : 0);
}

cvo_status cvo_metric_backward(cvo_handle h, const cvo_cloud* X, const cvo_cloud* Z, const double T[16], double di,
                               float* dX, float* dFX, float* dZ, float* dFZ, double* dell, int outputs_on_device)
{
    g_err.clear();
    if (!h) return fail(CVO_ERR_INVALID_ARG, "handle is NULL");
    if (!std::isfinite(di)) return fail(CVO_ERR_INVALID_ARG, "di must be finite");
    if (!X || !Z) return fail(CVO_ERR_INVALID_ARG, "X or Z is NULL");
    // i_theta = F / sqrt(N M) (Eq. indicator_actual): the upstream gradient of
    // F is di / sqrt(N M); an empty cloud has i_theta = 0 and zero gradients
    const double norm = (X->n > 0 && Z->n > 0) ? 1.0 / std::sqrt((double)X->n * (double)Z->n) : 0.0;
    return cvo_backward(h, X, Z, T, di * norm, dX, dFX, dZ, dFZ, dell, outputs_on_device);
}

cvo_status cvo_cosine(cvo_handle h, const cvo_cloud* X, const cvo_cloud* Z, const double T[16],
                      const double* norms2_in, double* cos_theta, double* norms2_out)
{
    g_err.clear();
    if (!h) return fail(CVO_ERR_INVALID_ARG, "handle is NULL");
    if (!cos_theta) return fail(CVO_ERR_INVALID_ARG, "cos_theta is NULL");
    const int D = feat_dim(h->p);
    CVO_TRY(check_cloud(X, "X", D));
    CVO_TRY(check_cloud(Z, "Z", D));
    CVO_TRY(check_pose(T, "T"));
    DeviceGuard g(h->device);
    double nn[2];
    if (norms2_in) {
        if (!(norms2_in[0] >= 0.0) || !(norms2_in[1] >= 0.0))
            return fail(CVO_ERR_INVALID_ARG, "norms2_in must be two values >= 0");
        nn[0] = norms2_in[0];
        nn[1] = norms2_in[1];
    } else {
        // self inner products at the identity: independent of T, so callers
        // that evaluate many poses pass them back in through norms2_in
        static const double I[16] = {1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1};
        cvo_eval e;
        CVO_TRY(run_eval(h, X, X, I, &e));
        nn[0] = e.F;
        CVO_TRY(run_eval(h, Z, Z, I, &e));
        nn[1] = e.F;
    }
    cvo_eval e;
    CVO_TRY(run_eval(h, X, Z, T, &e));
    const double den = std::sqrt(nn[0] * nn[1]);
    *cos_theta = den > 0.0 ? e.F / den : 0.0;
    if (norms2_out) {
        norms2_out[0] = nn[0];
        norms2_out[1] = nn[1];
    }
    return CVO_OK;
}

cvo_status cvo_cosine_dell(cvo_handle h, const cvo_cloud* X, const cvo_cloud* Z, const double T[16], double* cos_theta,
                           double* dcos_dell)
{
    g_err.clear();
    if (!h) return fail(CVO_ERR_INVALID_ARG, "handle is NULL");
    if (!cos_theta || !dcos_dell) return fail(CVO_ERR_INVALID_ARG, "cos_theta or dcos_dell is NULL");
    const int D = feat_dim(h->p);
    CVO_TRY(check_cloud(X, "X", D));
    CVO_TRY(check_cloud(Z, "Z", D));
    CVO_TRY(check_pose(T, "T"));
    DeviceGuard g(h->device);
    *cos_theta = 0.0;
    *dcos_dell = 0.0;
    if (X->n == 0 || Z->n == 0) return CVO_OK;
    static const double I[16] = {1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1};
    // the three double sums of Eq. (indicator) and their l-derivatives (the
    // gradient sweep of one cloud gives dF/dl = sum w d^2 / l^3)
    const cvo_cloud* A[3] = {X, X, Z};
    const cvo_cloud* B[3] = {Z, X, Z};
    const double* P[3] = {T, I, I};
    double F[3], dF[3];
    for (int k = 0; k < 3; ++k) {
        cvo_eval e;
        CVO_TRY(run_eval(h, A[k], B[k], P[k], &e));
        F[k] = e.F;
        CVO_TRY(run_backward(h, A[k], B[k], P[k], 1.0, nullptr, nullptr, nullptr, nullptr, &dF[k], 0));
    }
    if (!(F[1] > 0.0) || !(F[2] > 0.0) || F[0] == 0.0) {
        *cos_theta = (F[1] > 0.0 && F[2] > 0.0) ? F[0] / std::sqrt(F[1] * F[2]) : 0.0;
        return CVO_OK;
    }
    const double c = F[0] / std::sqrt(F[1] * F[2]);
    *cos_theta = c;
    *dcos_dell = c * (dF[0] / F[0] - 0.5 * (dF[1] / F[1] + dF[2] / F[2]));
    return CVO_OK;
}

cvo_status cvo_inner_product(cvo_handle h, const cvo_cloud* X, const cvo_cloud* Z, const double T[16], double* F)
{
    if (!F) return fail(CVO_ERR_INVALID_ARG, "F is NULL");
    cvo_eval e;
    CVO_TRY(cvo_evaluate(h, X, Z, T, &e));
    *F = e.F;
    return CVO_OK;
}

cvo_status cvo_gradient(cvo_handle h, const cvo_cloud* X, const cvo_cloud* Z, const double T[16], double grad[6],
                        double* F)
{
    if (!grad) return fail(CVO_ERR_INVALID_ARG, "grad is NULL");
    cvo_eval e;
    CVO_TRY(cvo_evaluate(h, X, Z, T, &e));
    for (int q = 0; q < 6; ++q) grad[q] = e.grad[q];
    if (F) *F = e.F;
    return CVO_OK;
}

cvo_status cvo_metric(cvo_handle h, const cvo_cloud* X, const cvo_cloud* Z, const double T[16], double* i_theta)
{
    if (!i_theta) return fail(CVO_ERR_INVALID_ARG, "i_theta is NULL");
    cvo_eval e;
    CVO_TRY(cvo_evaluate(h, X, Z, T, &e));
    *i_theta = e.i_theta;
    return CVO_OK;
}

cvo_status cvo_register_pair(cvo_handle h, const cvo_cloud* X, const cvo_cloud* Z, const double T_init[16],
                             double T_out[16], cvo_info* info)
{
    g_err.clear();
    if (!h) return fail(CVO_ERR_INVALID_ARG, "handle is NULL");
    if (!T_out) return fail(CVO_ERR_INVALID_ARG, "T_out is NULL");
    const int D = feat_dim(h->p);
    CVO_TRY(check_cloud(X, "X", D));
    CVO_TRY(check_cloud(Z, "Z", D));
    CVO_TRY(check_pose(T_init, "T_init"));
    DeviceGuard g(h->device);
    return run_register(h, X, Z, T_init, T_out, info);
}

cvo_status cvo_register_batch(cvo_handle h, int npairs, const cvo_cloud* X, const cvo_cloud* Z, const double* T_init,
                              double* T_out, cvo_info* infos)
{
    g_err.clear();
    if (!h) return fail(CVO_ERR_INVALID_ARG, "handle is NULL");
    if (npairs < 0) return fail(CVO_ERR_INVALID_ARG, "npairs < 0");
    if (npairs == 0) return CVO_OK;
    if (!X || !Z || !T_init || !T_out) return fail(CVO_ERR_INVALID_ARG, "NULL array");
    const int D = feat_dim(h->p);
    for (int k = 0; k < npairs; ++k) {
        CVO_TRY(check_cloud(X + k, "X[k]", D));
        CVO_TRY(check_cloud(Z + k, "Z[k]", D));
        CVO_TRY(check_pose(T_init + 16 * k, "T_init[k]"));
    }
    DeviceGuard g(h->device);
    return run_register_batch(h, npairs, X, Z, T_init, T_out, infos);
}

cvo_status cvo_register_sequence(cvo_handle h, int nframes, const cvo_cloud* frames, double ell_first,
                                 const double T_first[16], double* T_rel, double* T_abs, cvo_info* infos)
{
    g_err.clear();
    if (!h) return fail(CVO_ERR_INVALID_ARG, "handle is NULL");
    if (nframes < 0) return fail(CVO_ERR_INVALID_ARG, "nframes < 0");
    if (nframes > 0 && !frames) return fail(CVO_ERR_INVALID_ARG, "frames is NULL");
    if (nframes > 1 && !T_rel) return fail(CVO_ERR_INVALID_ARG, "T_rel is NULL");
    if (!(ell_first > 0.0) || !std::isfinite(ell_first)) return fail(CVO_ERR_INVALID_ARG, "ell_first must be > 0");
    const cvo_params base = h->p;
    if (base.anneal && ell_first < base.ell_min)
        return fail(CVO_ERR_INVALID_ARG, "ell_first must be >= ell_min when annealing");
    const int D = feat_dim(base);
    for (int k = 0; k < nframes; ++k) CVO_TRY(check_cloud(frames + k, "frames[k]", D));
    static const double I[16] = {1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1};
    if (T_first) CVO_TRY(check_pose(T_first, "T_first"));
    DeviceGuard g(h->device);
    if (T_abs && nframes > 0) std::memcpy(T_abs, I, sizeof(I));
    cvo_status worst = CVO_OK;
    for (int k = 0; k + 1 < nframes; ++k) {
        // the first pair has no prior: start from T_first with the larger
        // lengthscale; every later pair starts from the previous relative
        // motion (constant velocity) with params.ell
        h->p = base;
        if (k == 0) h->p.ell = ell_first;
        const double* init = (k == 0) ? (T_first ? T_first : I) : T_rel + 16 * (k - 1);
        cvo_info inf;
        const cvo_status s = run_register(h, frames + k, frames + k + 1, init, T_rel + 16 * k, &inf);
        h->p = base;
        if (s < 0) return s;
        if (s == CVO_NOT_CONVERGED) worst = CVO_NOT_CONVERGED;
        if (infos) infos[k] = inf;
        if (T_abs) {
            // T_abs[k+1] = T_abs[k] T_rel[k] (maps frame k+1 into frame 0)
            const double* A = T_abs + 16 * k;
            const double* B = T_rel + 16 * k;
            double* C = T_abs + 16 * (k + 1);
            for (int r = 0; r < 4; ++r)
                for (int c = 0; c < 4; ++c) {
                    double acc = 0.0;
                    for (int q = 0; q < 4; ++q) acc += A[4 * r + q] * B[4 * q + c];
                    C[4 * r + c] = acc;
                }
        }
    }
    return worst;
}

cvo_status cvo_shard_begin(cvo_handle h, const cvo_cloud* X_rows, const cvo_cloud* Z, long long n_total,
                           const double T_init[16])
{
    g_err.clear();
    if (!h) return fail(CVO_ERR_INVALID_ARG, "handle is NULL");
    const int D = feat_dim(h->p);
    CVO_TRY(check_cloud(X_rows, "X_rows", D));
    CVO_TRY(check_cloud(Z, "Z", D));
    CVO_TRY(check_pose(T_init, "T_init"));
    if (X_rows->n < 1 || Z->n < 1) return fail(CVO_ERR_INVALID_ARG, "a shard needs at least one row of X and one point of Z");
    if (n_total < X_rows->n) return fail(CVO_ERR_INVALID_ARG, "n_total (%lld) < the shard's rows (%d)", n_total, X_rows->n);
    if (h->p.max_iters < 1) return fail(CVO_ERR_INVALID_ARG, "max_iters must be >= 1 for a shard registration");
    DeviceGuard g(h->device);
    return run_shard_begin(h, X_rows, Z, n_total, T_init);
}

cvo_status cvo_shard_sweep(cvo_handle h, double* stats_device)
{
    g_err.clear();
    if (!h) return fail(CVO_ERR_INVALID_ARG, "handle is NULL");
    if (!stats_device) return fail(CVO_ERR_INVALID_ARG, "stats_device is NULL");
    if (!h->shard_active) return fail(CVO_ERR_INVALID_ARG, "no shard registration in progress (cvo_shard_begin)");
    DeviceGuard g(h->device);
    const SweepArgs& a = h->shard_a;
    CVO_CUDA(launch_sweep(a, h->shard_nb, h->s));
    if (h->shard_levels) CVO_CUDA(launch_layout(h->shard_levels, a.swept_level, a.nch_next, h->s));
    CVO_CUDA(launch_stats_out(a.grp_stats, a.grp_cnt, h->shard_nb, stats_device, h->s));
    return CVO_OK;
}

cvo_status cvo_shard_step(cvo_handle h, const double* stats_device, int* done)
{
    g_err.clear();
    if (!h) return fail(CVO_ERR_INVALID_ARG, "handle is NULL");
    if (!stats_device) return fail(CVO_ERR_INVALID_ARG, "stats_device is NULL");
    if (!h->shard_active) return fail(CVO_ERR_INVALID_ARG, "no shard registration in progress (cvo_shard_begin)");
    DeviceGuard g(h->device);
    IterState* dst = (IterState*)h->pr[0].state.p;
    CVO_CUDA(launch_finalize_stats(dst, stats_device, (double*)h->trace.p, h->s));
    if (done) {
        CVO_CUDA(cudaMemcpyAsync(&h->h_state->done, &dst->done, sizeof(int), cudaMemcpyDeviceToHost, h->s));
        CVO_CUDA(cudaStreamSynchronize(h->s));
        *done = h->h_state->done ? 1 : 0;
    }
    return CVO_OK;
}

cvo_status cvo_shard_end(cvo_handle h, double T_out[16], cvo_info* info)
{
    g_err.clear();
    if (!h) return fail(CVO_ERR_INVALID_ARG, "handle is NULL");
    if (!T_out) return fail(CVO_ERR_INVALID_ARG, "T_out is NULL");
    if (!h->shard_active) return fail(CVO_ERR_INVALID_ARG, "no shard registration in progress (cvo_shard_begin)");
    DeviceGuard g(h->device);
    h->shard_active = 0;
    CVO_TRY(fetch_states(h, 1));
    const IterState* st = h->h_state;
    std::memcpy(T_out, st->T, 16 * sizeof(double));
    cvo_info inf;
    std::memset(&inf, 0, sizeof(inf));
    fill_info(st, &inf);
    h->last_iters = st->iter;
    if (info) *info = inf;
    return (cvo_status)inf.status;
}

int cvo_get_trace(cvo_handle h, double* out, int cap)
{
    if (!h) return fail(CVO_ERR_INVALID_ARG, "handle is NULL");
    if (cap < 0 || (cap > 0 && !out)) return fail(CVO_ERR_INVALID_ARG, "bad output buffer");
    const int n = std::min(cap, h->last_iters);
    if (n > 0) {
        DeviceGuard g(h->device);
        if (cudaMemcpy(out, h->trace.p, (size_t)n * CVO_TRACE_STRIDE * sizeof(double), cudaMemcpyDeviceToHost) !=
            cudaSuccess)
            return fail(CVO_ERR_CUDA, "trace copy failed");
    }
    return h->last_iters;
}

cvo_status cvo_set_tuning(cvo_handle h, double cell_factor, int super_delta)
{
    if (!h) return fail(CVO_ERR_INVALID_ARG, "handle is NULL");
    if (!(cell_factor >= 0.25 && cell_factor <= 4.0)) return fail(CVO_ERR_INVALID_ARG, "cell_factor must be in [0.25, 4]");
    if (super_delta < -2 || super_delta > 6) return fail(CVO_ERR_INVALID_ARG, "super_delta must be in [-2, 6]");
    h->cell_factor = cell_factor;
    h->super_delta = super_delta;
    return CVO_OK;
}

cvo_status cvo_autotune(cvo_handle h, const cvo_cloud* X, const cvo_cloud* Z, const double T[16], cvo_tuning* out)
{
    g_err.clear();
    if (!h) return fail(CVO_ERR_INVALID_ARG, "handle is NULL");
    if (!out) return fail(CVO_ERR_INVALID_ARG, "out is NULL");
    const int D = feat_dim(h->p);
    CVO_TRY(check_cloud(X, "X", D));
    CVO_TRY(check_cloud(Z, "Z", D));
    CVO_TRY(check_pose(T, "T"));
    DeviceGuard g(h->device);
    return run_autotune(h, X, Z, T, out);
}

cvo_status cvo_autotune_batch(cvo_handle h, int npairs, const cvo_cloud* X, const cvo_cloud* Z, const double* T_init,
                              cvo_tuning* out)
{
    g_err.clear();
    if (!h) return fail(CVO_ERR_INVALID_ARG, "handle is NULL");
    if (!out) return fail(CVO_ERR_INVALID_ARG, "out is NULL");
    if (npairs < 0) return fail(CVO_ERR_INVALID_ARG, "npairs < 0");
    if (npairs > 0 && (!X || !Z || !T_init)) return fail(CVO_ERR_INVALID_ARG, "NULL array");
    const int D = feat_dim(h->p);
    for (int k = 0; k < npairs; ++k) {
        CVO_TRY(check_cloud(X + k, "X[k]", D));
        CVO_TRY(check_cloud(Z + k, "Z[k]", D));
        CVO_TRY(check_pose(T_init + 16 * k, "T_init[k]"));
    }
    DeviceGuard g(h->device);
    return run_autotune_batch(h, npairs, X, Z, T_init, out);
}

cvo_status cvo_get_tuning(cvo_handle h, cvo_tuning* out)
{
    if (!h || !out) return fail(CVO_ERR_INVALID_ARG, "NULL argument");
    *out = cvo_tuning{h->cell_factor, h->super_delta, h->chunk_len, 0.0, h->query_lanes};
    return CVO_OK;
}

cvo_status cvo_apply_tuning(cvo_handle h, const cvo_tuning* t)
{
    if (!h || !t) return fail(CVO_ERR_INVALID_ARG, "NULL argument");
    if (t->chunk_len < 16 || t->chunk_len > 4096) return fail(CVO_ERR_INVALID_ARG, "chunk_len must be in [16, 4096]");
    const int ql = t->query_lanes == 0 ? 1 : t->query_lanes;   // 0: a tuning from before the field (one lane)
    if (ql != 1 && ql != 2 && ql != 4) return fail(CVO_ERR_INVALID_ARG, "query_lanes must be 1, 2 or 4");
    CVO_TRY(cvo_set_tuning(h, t->cell_factor, t->super_delta));
    h->chunk_len = t->chunk_len;
    h->query_lanes = ql;
    return CVO_OK;
}

cvo_status cvo_set_loop(cvo_handle h, int mode)
{
    if (!h) return fail(CVO_ERR_INVALID_ARG, "handle is NULL");
    if (mode < CVO_LOOP_HOST || mode > CVO_LOOP_PERSISTENT) return fail(CVO_ERR_INVALID_ARG, "unknown loop mode %d", mode);
    h->loop_mode = mode;
    return CVO_OK;
}

cvo_status cvo_inject_barrier_stall(cvo_handle h, int barrier, unsigned poll_limit)
{
    g_err.clear();
    if (!h) return fail(CVO_ERR_INVALID_ARG, "handle is NULL");
    if (barrier >= 0 && poll_limit == 0) return fail(CVO_ERR_INVALID_ARG, "poll_limit must be > 0 with a barrier");
    h->inj_leave_at = barrier >= 0 ? barrier : -1;
    h->inj_polls = barrier >= 0 ? poll_limit : 0;
    return CVO_OK;
}

cvo_status cvo_set_timing(cvo_handle h, int on)
{
    if (!h) return fail(CVO_ERR_INVALID_ARG, "handle is NULL");
    h->timing = on ? 1 : 0;
    return CVO_OK;
}

cvo_status cvo_sweep_time(cvo_handle h, double* avg_ms, int* launches)
{
    if (!h || !avg_ms || !launches) return fail(CVO_ERR_INVALID_ARG, "NULL argument");
    *launches = h->sweep_n;
    *avg_ms = h->sweep_n > 0 ? h->sweep_ms / h->sweep_n : 0.0;
    return CVO_OK;
}

}  // extern "C"
