// Allocation-free dense evaluation: cvo_evaluate_dense_noalloc (include/cvo.h).
//
// This is an addition of this library; the paper has no counterpart.  Some
// callers must not allocate device memory once they are running: a real-time
// odometry loop that fixed its memory budget at start-up (a cudaMalloc or
// cudaFree can synchronise the device and stall the loop, or fail half way
// through a run), or a plugin inside a host application whose memory pool
// owns the GPU.  The handle-based entry points allocate their scratch on
// demand (and pinned host memory when the handle is created), so they cannot
// serve such callers.  This entry point needs no handle and allocates nothing:
// it runs the same pack, sweep and finalize kernels as cvo_evaluate in dense
// mode, with every byte of scratch carved out of one fixed array that lives in
// the library's device image.  Every GPU that loads the library holds that
// array (kScratchBytes, 4.5 MiB) until the process exits.
//
// Limits: dense sum only (cutoff_mult <= 0), at most kNoAllocMaxPoints points
// per cloud and kNoAllocMaxFeat feature entries per point (records of at most
// kNoAllocMaxRec float4).  Larger requests are rejected with
// CVO_ERR_INVALID_ARG and a message naming the limit.
//
// Sharing: all calls use the same array, which keeps the previous call's
// contents.  Everything a call reads is written earlier in the same call (the
// state block and groups by the set-up kernel, the bounding box counters are
// reset there, records by the pack kernels, one partial per launched sweep
// block), so nothing stale is ever read.  Calls that overlap on the GPU (two
// streams, or two host threads, on one device) race on the array: serialise
// them.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

#include "cvo.h"
#include "cvo_internal.cuh"

namespace cvo {
void set_error_message(const char* msg);
}

using namespace cvo;

namespace {

constexpr int kNoAllocMaxPoints = 16384;
constexpr int kNoAllocMaxRec = 7;                          // float4 per record
constexpr int kNoAllocMaxFeat = (kNoAllocMaxRec - 1) * 4;  // float32 feature entries
constexpr int kNoAllocBlocks = 1216;                       // most sweep blocks (partial sums in the array); a
                                                           // launch takes at most kSweepBlocksPerSm per SM
constexpr int kMaxDevices = 64;
constexpr int kNoAllocMaxChunks = 16;                      // work items per query group

constexpr size_t align256(size_t v) { return (v + 255) & ~size_t(255); }
constexpr size_t kOffState = 0;
constexpr size_t kOffLevel = align256(kOffState + sizeof(IterState));
constexpr size_t kOffPair = align256(kOffLevel + sizeof(LevelDesc));
constexpr size_t kOffMisc = align256(kOffPair + sizeof(PairDesc));
constexpr size_t kOffGroups = align256(kOffMisc + 16 * sizeof(unsigned));
constexpr size_t kOffStats = align256(kOffGroups + sizeof(int2) * (kNoAllocMaxPoints / 32));
constexpr size_t kOffCnt = align256(kOffStats + sizeof(float2) * kStatN * kNoAllocBlocks);
constexpr size_t kOffGStats = align256(kOffCnt + sizeof(unsigned long long) * 2 * kNoAllocBlocks);
constexpr size_t kOffGCnt = align256(kOffGStats + sizeof(float2) * kStatN * kMaxGroups);
constexpr size_t kOffGArr = align256(kOffGCnt + sizeof(unsigned long long) * 2 * kMaxGroups);
constexpr size_t kOffItems = align256(kOffGArr + sizeof(unsigned) * kMaxGroups);
constexpr size_t kOffX = align256(kOffItems + sizeof(int4) * (kNoAllocMaxPoints / 32) * kNoAllocMaxChunks);
constexpr size_t kOffZ = align256(kOffX + sizeof(float4) * kNoAllocMaxRec * kNoAllocMaxPoints);
constexpr size_t kUsedBytes = align256(kOffZ + sizeof(float4) * kNoAllocMaxRec * kNoAllocMaxPoints);
constexpr size_t kScratchBytes = 4608 * 1024;   // 4.5 MiB
static_assert(kUsedBytes <= kScratchBytes, "allocation-free scratch layout exceeds its array");

}  // namespace

// The scratch of every cvo_evaluate_dense_noalloc call.  In host code this
// name is only a host-side stand-in for the device array: kernels receive the
// device address that cudaGetSymbolAddress returns for the current device.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

namespace {

std::mutex g_addr_mu;
unsigned char* g_addr[kMaxDevices] = {};
int g_sms[kMaxDevices] = {};

cvo_status na_fail(cvo_status s, const char* msg)
{
    set_error_message(msg);
    return s;
}

// Device address of the scratch array on the current device, looked up once
// per device with that device current, and the device's SM count.
cvo_status scratch_address(unsigned char** out, int* sms)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return na_fail(CVO_ERR_CUDA, "cvo_evaluate_dense_noalloc: no current CUDA device");
    }
    if (dev < 0 || dev >= kMaxDevices) return na_fail(CVO_ERR_CUDA, "cvo_evaluate_dense_noalloc: device ordinal too large");
    std::lock_guard<std::mutex> lk(g_addr_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return na_fail(CVO_ERR_CUDA, "cvo_evaluate_dense_noalloc: cudaGetSymbolAddress of the scratch array failed");
        }
        int count = 0;
        if (cudaDeviceGetAttribute(&count, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || count <= 0) {
            cudaGetLastError();
            return na_fail(CVO_ERR_CUDA, "cvo_evaluate_dense_noalloc: cannot read the device's SM count");
        }
        g_sms[dev] = count;
        g_addr[dev] = (unsigned char*)p;
    }
    *out = g_addr[dev];
    *sms = g_sms[dev];
    return CVO_OK;
}

bool is_device_pointer(const void* p)
{
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Writes the state block, the level descriptor and the query groups, and
// resets the bounding-box counters (min to all ones, max and flag to zero).
__global__ void k_na_setup(IterState init, LevelDesc ld, PairDesc pd, int n, int nch, IterState* st, LevelDesc* lv,
                           PairDesc* pair, int2* groups, int4* items, unsigned* misc, unsigned* arrivals)
{
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    if (tid < kMaxGroups) arrivals[tid] = 0u;   // the sweep's group counters start at zero
    if (tid == 0) {
        *st = init;
        *lv = ld;
        *pair = pd;
        for (int a = 0; a < 3; ++a) {
            misc[a] = 0xffffffffu;       // Z box minimum
            misc[3 + a] = 0u;            // Z box maximum
            misc[8 + a] = 0xffffffffu;   // X box minimum (only its finiteness flag is used)
            misc[11 + a] = 0u;
        }
        misc[6] = 0u;                    // non-finite flag
    }
    const int ng = (n + 31) / 32;
    for (int g = tid; g < ng; g += gridDim.x * blockDim.x) groups[g] = make_int2(32 * g, min(32, n - 32 * g));
    // every group streams all of Z (dense), so every group gets nch chunks
    for (int i = tid; i < ng * nch; i += gridDim.x * blockDim.x) {
        const int g = i / nch;
        items[i] = make_int4(32 * g, min(32, n - 32 * g), (i - g * nch) | (nch << 16), g);
    }
}

__device__ float na_decode(unsigned u)
{
    const unsigned b = (u & 0x80000000u) ? (u & 0x7fffffffu) : ~u;
    return __uint_as_float(b);
}

// Lever centre c = centre of Z's bounding box (as cvo_evaluate uses).
__global__ void k_na_center(const unsigned* misc, IterState* st)
{
    for (int a = 0; a < 3; ++a) st->c[a] = 0.5 * ((double)na_decode(misc[a]) + (double)na_decode(misc[3 + a]));
}

__global__ void k_na_output(const IterState* st, const unsigned* misc, cvo_eval* out)
{
    const bool bad = misc[6] != 0u;
    const double nan = __longlong_as_double(0x7ff8000000000000LL);
    const int t = threadIdx.x;
    if (t == 0) {
        out->F = bad ? nan : st->F;
        out->i_theta = bad ? nan : st->i_theta;
        out->pairs = st->pairs;
        out->candidates = st->cands;
    }
    if (t < 6) out->grad[t] = bad ? nan : st->grad[t];
    if (t < 36) out->hess[t] = bad ? nan : st->hess[t];
}

__global__ void k_na_zero(cvo_eval* out)
{
    const int t = threadIdx.x;
    if (t == 0) {
        out->F = 0.0;
        out->i_theta = 0.0;
        out->pairs = 0;
        out->candidates = 0;
    }
    if (t < 6) out->grad[t] = 0.0;
    if (t < 36) out->hess[t] = 0.0;
}

cvo_status check_pose_na(const double* T)
{
    if (!T) return na_fail(CVO_ERR_INVALID_ARG, "cvo_evaluate_dense_noalloc: T is NULL");
    for (int k = 0; k < 16; ++k)
        if (!std::isfinite(T[k])) return na_fail(CVO_ERR_INVALID_ARG, "cvo_evaluate_dense_noalloc: T is not finite");
    if (T[12] != 0.0 || T[13] != 0.0 || T[14] != 0.0 || T[15] != 1.0)
        return na_fail(CVO_ERR_INVALID_ARG, "cvo_evaluate_dense_noalloc: last row of T must be (0, 0, 0, 1)");
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            double d = 0.0;
            for (int k = 0; k < 3; ++k) d += T[4 * k + a] * T[4 * k + b];
            if (std::fabs(d - (a == b ? 1.0 : 0.0)) > 1e-6)
                return na_fail(CVO_ERR_INVALID_ARG, "cvo_evaluate_dense_noalloc: rotation of T is not orthonormal");
        }
    return CVO_OK;
}

#define NA_CUDA(call)                                                              \
    do {                                                                           \
        if ((call) != cudaSuccess) {                                               \
            cudaGetLastError();                                                    \
            return na_fail(CVO_ERR_CUDA, "cvo_evaluate_dense_noalloc: " #call " failed"); \
        }                                                                          \
    } while (0)

}  // namespace

extern "C" cvo_status cvo_evaluate_dense_noalloc(const cvo_params* p, void* cuda_stream, const cvo_cloud* X,
                                                 const cvo_cloud* Z, const double T[16], cvo_eval* out_device)
{
    set_error_message("");
    if (!p || !X || !Z || !out_device) return na_fail(CVO_ERR_INVALID_ARG, "cvo_evaluate_dense_noalloc: NULL argument");
    if (!(p->ell > 0.0) || !std::isfinite(p->ell) || !(p->sigma > 0.0) || !std::isfinite(p->sigma))
        return na_fail(CVO_ERR_INVALID_ARG, "cvo_evaluate_dense_noalloc: ell and sigma must be > 0");
    if (p->cutoff_mult > 0.0)
        return na_fail(CVO_ERR_INVALID_ARG,
                       "cvo_evaluate_dense_noalloc: evaluates the dense sum only (cutoff_mult must be <= 0)");
    if (p->n_blocks < 0 || p->n_blocks > CVO_MAX_BLOCKS)
        return na_fail(CVO_ERR_INVALID_ARG, "cvo_evaluate_dense_noalloc: n_blocks out of range");
    if (!std::isfinite(p->feat_cutoff_mult))
        return na_fail(CVO_ERR_INVALID_ARG, "cvo_evaluate_dense_noalloc: feat_cutoff_mult must be finite");
    FeatConst fc;
    std::memset(&fc, 0, sizeof(fc));
    double kappa = p->sigma * p->sigma;
    int D = 0;
    for (int b = 0; b < p->n_blocks; ++b) {
        const cvo_feat_block& fb = p->blocks[b];
        // the checks of cvo_create: a squared-exponential block needs a finite
        // scale > 0 and a finite sigma
        if (fb.dim < 1 || (fb.kind != CVO_FEAT_SE && fb.kind != CVO_FEAT_DOT) ||
            (fb.kind == CVO_FEAT_SE && (!(fb.scale > 0.0) || !std::isfinite(fb.scale) || !std::isfinite(fb.sigma))))
            return na_fail(CVO_ERR_INVALID_ARG,
                           "cvo_evaluate_dense_noalloc: invalid feature block (dim >= 1, a known kind; "
                           "squared exponential: scale > 0 and sigma finite)");
        fc.dim[b] = fb.dim;
        fc.kind[b] = fb.kind;
        fc.off[b] = D;
        fc.fcut2[b] = 3.0e38f;
        if (fb.kind == CVO_FEAT_SE) {
            fc.s[b] = (float)(-1.4426950408889634 / (2.0 * fb.scale * fb.scale));
            kappa *= fb.sigma * fb.sigma;
            if (p->feat_cutoff_mult > 0.0)
                fc.fcut2[b] = (float)((p->feat_cutoff_mult * fb.scale) * (p->feat_cutoff_mult * fb.scale));
        }
        D += fb.dim;
    }
    fc.n_blocks = p->n_blocks;
    fc.D = D;
    fc.bf16 = 0;
    if (D > kNoAllocMaxFeat)
        return na_fail(CVO_ERR_INVALID_ARG,
                       "cvo_evaluate_dense_noalloc: at most 24 feature entries per point (fixed scratch)");
    const int n = X->n, m = Z->n;
    if (n < 0 || m < 0 || n > kNoAllocMaxPoints || m > kNoAllocMaxPoints)
        return na_fail(CVO_ERR_INVALID_ARG,
                       "cvo_evaluate_dense_noalloc: each cloud must have 0..16384 points (fixed scratch)");
    const cvo_cloud* cl[2] = {X, Z};
    for (const cvo_cloud* c : cl) {
        if (c->n == 0) continue;
        if (!c->on_device || !c->xyz || !is_device_pointer(c->xyz))
            return na_fail(CVO_ERR_INVALID_ARG, "cvo_evaluate_dense_noalloc: xyz must be a device pointer");
        if (D > 0 && (!c->feat || !is_device_pointer(c->feat)))
            return na_fail(CVO_ERR_INVALID_ARG, "cvo_evaluate_dense_noalloc: features must be a device pointer");
        if (c->feat_dtype != CVO_F32 && c->feat_dtype != CVO_BF16)
            return na_fail(CVO_ERR_INVALID_ARG, "cvo_evaluate_dense_noalloc: unknown feature dtype");
    }
    if (!is_device_pointer(out_device))
        return na_fail(CVO_ERR_INVALID_ARG, "cvo_evaluate_dense_noalloc: out_device must be a device pointer");
    {
        const cvo_status s = check_pose_na(T);
        if (s != CVO_OK) return s;
    }
    unsigned char* base = nullptr;
    int sms = 0;
    {
        const cvo_status s = scratch_address(&base, &sms);
        if (s != CVO_OK) return s;
    }
    cudaStream_t s = (cudaStream_t)cuda_stream;
    if (n == 0 || m == 0) {
        g_launch_count.fetch_add(1, std::memory_order_relaxed);
        k_na_zero<<<1, 64, 0, s>>>(out_device);
        NA_CUDA(cudaGetLastError());
        return CVO_OK;
    }
    IterState* st = (IterState*)(base + kOffState);
    LevelDesc* lv = (LevelDesc*)(base + kOffLevel);
    unsigned* misc = (unsigned*)(base + kOffMisc);
    int2* groups = (int2*)(base + kOffGroups);
    int4* items = (int4*)(base + kOffItems);
    float2* stats = (float2*)(base + kOffStats);
    unsigned long long* cnt = (unsigned long long*)(base + kOffCnt);
    float2* gstats = (float2*)(base + kOffGStats);
    unsigned long long* gcnt = (unsigned long long*)(base + kOffGCnt);
    unsigned* garr = (unsigned*)(base + kOffGArr);
    float4* xrec = (float4*)(base + kOffX);
    float4* zrec = (float4*)(base + kOffZ);
    const int rs = 1 + (D * 4 + 15) / 16;

    IterState init;
    std::memset(&init, 0, sizeof(init));
    std::memcpy(init.T, T, sizeof(init.T));
    init.ell = p->ell;
    init.ell_last = p->ell;
    init.mode = 0;
    init.kappa = kappa;
    init.norm = 1.0 / std::sqrt((double)n * (double)m);
    init.cutoff_mult = p->cutoff_mult;
    init.ell_min = p->ell;
    init.status = 1;
    init.nlevels = 1;
    init.level_h[0] = 1.0f;
    LevelDesc ld;
    std::memset(&ld, 0, sizeof(ld));
    ld.h = 1.0f;
    ld.inv_h = 1.0f;
    ld.inv_hx = 1.0f;
    ld.trim = 0;
    ld.nx = ld.ny = ld.nz = 1;
    ld.cell_start = nullptr;   // the dense sweep reads every record in order
    ld.zrec = zrec;
    ld.groups = groups;
    ld.ngroups = (n + 31) / 32;
    const int nch = std::max(1, std::min(kNoAllocMaxChunks, (m + kChunkLen - 1) / kChunkLen));
    ld.items = items;
    ld.nitems = ld.ngroups * nch;

    const int nblocks = std::max(1, std::min({(ld.nitems + kSweepWarps - 1) / kSweepWarps, kNoAllocBlocks,
                                              sms * kSweepBlocksPerSm}));
    PairDesc pd;
    pd.levels = lv;
    pd.xrec = xrec;
    pd.st = st;
    pd.n = n;
    pd.m = m;
    pd.b0 = 0;
    pd.b1 = nblocks;
    pd.bmax = nblocks;
    PairDesc* pair = (PairDesc*)(base + kOffPair);

    g_launch_count.fetch_add(2, std::memory_order_relaxed);
    k_na_setup<<<(ld.nitems + 255) / 256, 256, 0, s>>>(init, ld, pd, n, nch, st, lv, pair, groups, items, misc, garr);
    NA_CUDA(cudaGetLastError());
    NA_CUDA(launch_bbox(Z->xyz, m, misc, (int*)(misc + 6), s));
    NA_CUDA(launch_bbox(X->xyz, n, misc + 8, (int*)(misc + 6), s));   // finiteness of X (box unused)
    if (D > 0) {
        NA_CUDA(launch_check_feat(X->feat, (long long)n * D, X->feat_dtype == CVO_BF16, (int*)(misc + 6), s));
        NA_CUDA(launch_check_feat(Z->feat, (long long)m * D, Z->feat_dtype == CVO_BF16, (int*)(misc + 6), s));
    }
    k_na_center<<<1, 1, 0, s>>>(misc, st);
    NA_CUDA(cudaGetLastError());
    NA_CUDA(launch_init_state(st, s));
    NA_CUDA(launch_pack(X->xyz, X->feat, X->feat_dtype == CVO_BF16, D, nullptr, n, xrec, rs, 0, s));
    NA_CUDA(launch_pack(Z->xyz, Z->feat, Z->feat_dtype == CVO_BF16, D, nullptr, m, zrec, rs, 0, s));
    SweepArgs a{};
    a.pairs = pair;
    a.npairs = 1;
    a.rs = rs;
    a.dense = 1;
    a.part_stats = stats;
    a.part_cnt = cnt;
    a.part_cap = kNoAllocBlocks;
    a.grp_stats = gstats;
    a.grp_cnt = gcnt;
    a.grp_arrivals = garr;
    a.fc = fc;
    a.nch_next = nullptr;   // no re-planning: the dense plan holds
    a.swept_level = nullptr;
    NA_CUDA(launch_sweep(a, nblocks, s));
    NA_CUDA(launch_finalize(st, gstats, gcnt, nblocks, nullptr, s));
    g_launch_count.fetch_add(1, std::memory_order_relaxed);
    k_na_output<<<1, 64, 0, s>>>(st, misc, out_device);
    NA_CUDA(cudaGetLastError());
    return CVO_OK;
}
