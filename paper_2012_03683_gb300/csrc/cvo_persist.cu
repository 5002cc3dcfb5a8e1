// The registration loop of one pair as a single persistent kernel.
//
// The graph-launched loop pays two kernel boundaries per iteration (sweep ->
// step -> next sweep, about 12 us on GB300 against an 80 us sweep), and its
// work items, planned once at the start pose, go stale as the pose moves:
// a group whose stream has grown becomes one long item that the rest of the
// grid waits for.  Here one cooperative launch keeps one wave of blocks
// resident for the whole registration and re-plans every iteration:
//
//   for each iteration, until the state says done:
//     plan          one warp per query group: the length of its candidate
//                   stream at the current pose, and its chunk count
//                   ceil(length / chunk_len) (at most kMaxChunks)
//     grid barrier
//     sweep         the chunks in chunk-major order (every group's chunk
//                   0, then every chunk 1, ...) dealt round robin to the
//                   grid's warps; per-lane statistics, block and group sums
//                   as in k_sweep (fixed order, deterministic)
//     grid barrier
//     step          block 0 sums the group partials in order and takes the
//                   step of k_finalize (FP64 pose update, annealing,
//                   derived constants)
//     grid barrier
//
// The grid barrier spins on a generation word with an iteration limit: a
// block that gives up sets an error flag, every block leaves the loop on that
// flag, and the host reports CVO_ERR_TIMEOUT.  (The cooperative launch
// guarantees that all blocks are resident, so the limit is a guard, not a
// path; cvo_inject_barrier_stall makes one block leave instead of arriving,
// with a short limit, so that a test can take that path.)
#include "cvo_step_dev.cuh"
#include "cvo_sweep_dev.cuh"

namespace cvo {
namespace {

constexpr unsigned kSpinLimit = 1u << 24;   // polls of a barrier before it gives up (seconds)

struct PersistArgs {
    SweepArgs sw;                 // one pair: sw.pairs[0]; part_cap >= the grid
    unsigned* ctl;                // [2] barrier count, [3] barrier generation, [4] error flag, [5] largest chunk
                                  // count of the iteration; zero before the launch
    unsigned* nch;                // chunk count per query group (the largest level's group count)
    int chunk_len;
    double* trace;
    unsigned spin_limit;          // polls of a barrier before it gives up
    int leave_at;                 // failure injection: >= 0, the last block leaves the kernel at this
                                  // grid barrier (counted from 0) instead of arriving; -1: off
};

// Grid barrier over all blocks of a cooperative launch.  Returns false if
// the wait gave up or another block has (the error flag is set).
__device__ bool grid_barrier(unsigned* ctl, unsigned nblocks, unsigned spin_limit)
{
    __syncthreads();
    __shared__ int ok;
    if (threadIdx.x == 0) {
        volatile unsigned* gen = ctl + 3;
        volatile unsigned* err = ctl + 4;
        const unsigned g = *gen;
        __threadfence();
        const unsigned arrived = atomicAdd(ctl + 2, 1u);
        int good = 1;
        if (arrived == nblocks - 1) {
            ctl[2] = 0u;
            __threadfence();
            atomicAdd(ctl + 3, 1u);
        } else {
            unsigned polls = 0;
            while (*gen == g) {
                if (*err) {
                    good = 0;
                    break;
                }
                if (++polls > spin_limit) {
                    atomicExch(ctl + 4, 1u);
                    good = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        ok = good && (*err == 0u);
    }
    __syncthreads();
    return ok != 0;
}

template <class Feat>
__global__ void __launch_bounds__(kSweepWarps * 32, 4) k_register(PersistArgs a)
{
    extern __shared__ float4 stage_mem[];   // [kSweepWarps][2][32][rs]
    __shared__ float cst[30];
    __shared__ double S[kStatN];
    __shared__ float Shi[kStatN], Slo[kStatN];
    __shared__ unsigned long long cs[2];
    constexpr int kWords = (int)(sizeof(IterState) / 8);
    __shared__ unsigned long long sbuf[kWords];
    __shared__ int s_done;

    const PairDesc P = a.sw.pairs[0];
    IterState* st = P.st;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int rs = rec_stride<Feat>(a.sw.rs);
    const bool dense = a.sw.dense != 0;
    const FeatConst fc = a.sw.fc;
    float4* stage = stage_mem + (size_t)warp * 2 * 32 * rs;
    const unsigned nblocks = gridDim.x;
    const int ngroups = ((int)nblocks + kGroupBlocks - 1) / kGroupBlocks;
    int barrier = 0;   // grid barriers passed (the failure injection counts them)
    auto sync_grid = [&]() {
        if (a.leave_at == barrier++ && blockIdx.x == nblocks - 1) return false;   // leaves without arriving
        return grid_barrier(a.ctl, nblocks, a.spin_limit);
    };

    for (;;) {
        // the state as block 0 left it (read around the L1: another SM wrote it)
        if (threadIdx.x == 0) s_done = (int)__ldcg(&st->done);
        if (threadIdx.x < 30) cst[threadIdx.x] = __ldcg(&st->Ahi[0] + threadIdx.x);
        __syncthreads();
        StatAcc acc;
        stat_acc_init(acc, lane);
        if (s_done) break;
        const int level = __ldcg(&st->level);
        const float sg = __ldcg(&st->sg), rc = __ldcg(&st->rc), rc2 = __ldcg(&st->rc2);
        const LevelDesc L = P.levels[level];

        const int gw = (int)blockIdx.x * kSweepWarps + warp;   // this warp in the grid
        const int nw = (int)nblocks * kSweepWarps;

        // ---- plan: chunk counts at the current pose -------------------------
        for (int g = gw; g < L.ngroups; g += nw) {
            const int2 grp = L.groups[g];
            const bool act = lane < grp.y;
            const float4 q = P.xrec[(size_t)(grp.x + (act ? lane : 0)) * rs];
            const float xq[3] = {q.x, q.y, q.z};
            float xh[3], xl[3];
            transform_df(xq, cst, cst + 9, cst + 18, cst + 21, xh, xl);
            Stream sm;
            const int total = stream_setup(L, P.m, dense, act, xh, rc, lane, sm) ? sm.total : 0;
            if (lane == 0) {
                const int c = total == 0 ? 0 : max(1, min(kMaxChunks, (total + a.chunk_len - 1) / a.chunk_len));
                a.nch[g] = (unsigned)c;
                atomicMax(a.ctl + 5, (unsigned)c);
            }
        }
        if (!sync_grid()) return;

        // ---- sweep: chunk-major slots round robin over the grid's warps -----
        unsigned npairs = 0, ncand = 0;
        const int maxc = (int)__ldcg(a.ctl + 5);
        const int nslots = L.ngroups * maxc;
        for (int s = gw; s < nslots; s += nw) {
            const int k = s / L.ngroups;
            const int g = s - k * L.ngroups;
            const int n = (int)__ldcg(a.nch + g);
            if (k >= n) continue;
            Moments mo;
            float p[3];
            bool act;
            if (!sweep_chunk<Feat>(P, L, L.groups[g], k, n, cst, rs, dense, sg, rc, rc2, fc, stage, nullptr, lane, mo, p,
                                   act, npairs, ncand))
                continue;
            stat_acc_add(acc, mo, p, act, lane);
        }
        sweep_epilogue(acc, npairs, ncand, a.sw, (int)blockIdx.x, (int)nblocks);
        if (!sync_grid()) return;

        // ---- step (block 0) ---------------------------------------------------
        if (blockIdx.x == 0) {
            for (int i = threadIdx.x; i < kWords; i += blockDim.x)
                sbuf[i] = __ldcg(reinterpret_cast<const unsigned long long*>(st) + i);
            if (threadIdx.x < kStatN) {
                const float2* row = a.sw.grp_stats + (size_t)threadIdx.x * kMaxGroups;
                float hi = 0.0f, lo = 0.0f;
                for (int g0 = 0; g0 < ngroups; g0 += 8) {   // eight loads in flight
                    float2 x[8];
#pragma unroll
                    for (int j = 0; j < 8; ++j) x[j] = g0 + j < ngroups ? __ldcg(row + g0 + j) : make_float2(0.0f, 0.0f);
#pragma unroll
                    for (int j = 0; j < 8; ++j) df_add(hi, lo, x[j].x, x[j].y);
                }
                S[threadIdx.x] = (double)hi + (double)lo;
                Shi[threadIdx.x] = hi;
                Slo[threadIdx.x] = lo;
            } else if (threadIdx.x == kStatN || threadIdx.x == kStatN + 1) {
                const int c = threadIdx.x - kStatN;
                unsigned long long t = 0;
                for (int g = 0; g < ngroups; ++g) t += __ldcg(a.sw.grp_cnt + (size_t)c * kMaxGroups + g);
                cs[c] = t;
            } else if (threadIdx.x == kStatN + 2) {
                a.ctl[5] = 0u;   // the next plan's largest chunk count
            }
            __syncthreads();
            IterState* sst = reinterpret_cast<IterState*>(sbuf);
            if (threadIdx.x < 32) step_warp(sst, S, Shi, Slo, cs[0], cs[1], a.trace);
            __syncthreads();
            for (int i = threadIdx.x; i < kWords; i += blockDim.x)
                reinterpret_cast<unsigned long long*>(st)[i] = sbuf[i];
            __threadfence();
        }
        if (!sync_grid()) return;
    }
}

template <class Feat>
cudaError_t persist_t(const PersistArgs& a, int* nblocks, size_t* smem_out, bool query, cudaStream_t s)
{
    if (Feat::kRs > 0 && Feat::kRs != a.sw.rs) return cudaErrorInvalidValue;   // the policy's record layout
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(k_register<Feat>, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    const size_t smem = (size_t)kSweepWarps * 2 * 32 * a.sw.rs * sizeof(float4);
    if (query) {
        int per_sm = 0, dev = 0, sms = 0;
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_register<Feat>, kSweepWarps * 32, smem);
        if (e != cudaSuccess) return e;
        e = cudaGetDevice(&dev);
        if (e != cudaSuccess) return e;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        *nblocks = per_sm * sms;
        *smem_out = smem;
        return cudaSuccess;
    }
    PersistArgs args = a;
    void* params[1] = {&args};
    g_launch_count.fetch_add(1, std::memory_order_relaxed);
    return cudaLaunchCooperativeKernel((const void*)k_register<Feat>, dim3(*nblocks), dim3(kSweepWarps * 32), params,
                                       smem, s);
}

template <class... T>
cudaError_t dispatch(const FeatConst& f, T&&... args)
{
    // the feature-space cutoff's test is compiled in (the persistent loop is
    // an option, so one instance per block list serves both settings)
    if (f.n_blocks == 0) return persist_t<FeatNone>(args...);
    const bool se3 = f.n_blocks >= 1 && f.kind[0] == 0 && f.dim[0] == 3;
    if (f.n_blocks == 1 && se3)
        return f.bf16 ? persist_t<FeatFixed<3, 0, true, true>>(args...) : persist_t<FeatFixed<3, 0, false, true>>(args...);
    if (f.n_blocks == 2 && se3 && f.kind[1] == 1 && f.dim[1] == 19)
        return f.bf16 ? persist_t<FeatFixed<3, 19, true, true>>(args...)
                      : persist_t<FeatFixed<3, 19, false, true>>(args...);
    if (f.n_blocks == 1 && f.kind[0] == 1 && f.dim[0] == 19)
        return f.bf16 ? persist_t<FeatFixed<0, 19, true, false>>(args...)
                      : persist_t<FeatFixed<0, 19, false, false>>(args...);
    return persist_t<FeatGeneric>(args...);
}

}  // namespace

cudaError_t persistent_grid(const SweepArgs& sw, int* nblocks)
{
    PersistArgs a{};
    a.sw = sw;
    size_t smem = 0;
    return dispatch(sw.fc, a, nblocks, &smem, true, (cudaStream_t)0);
}

cudaError_t launch_register_persistent(const SweepArgs& sw, unsigned* ctl, unsigned* nch, int chunk_len, double* trace,
                                       int nblocks, int leave_at, unsigned spin_limit, cudaStream_t s)
{
    PersistArgs a{};
    a.sw = sw;
    a.ctl = ctl;
    a.nch = nch;
    a.chunk_len = chunk_len;
    a.trace = trace;
    a.leave_at = leave_at;
    a.spin_limit = spin_limit > 0 ? spin_limit : kSpinLimit;
    size_t smem = 0;
    int nb = nblocks;
    return dispatch(sw.fc, a, &nb, &smem, false, s);
}

}  // namespace cvo
