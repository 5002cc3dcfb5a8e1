// One block per iteration: reduces the sweep's per-block statistics and takes
// the step on the device, so a registration never waits on the host.
//
// 1. Sums the 43 statistics over the sweep's group sums (each the sum of
//    kGroupBlocks block partials, added by the group's last block) in
//    double-float (hi + lo FP32 pairs, error-free two-sum): a warp per
//    statistic, each lane over every 32nd group in group order, then a
//    butterfly over the lanes; a fixed order, so deterministic, and as
//    accurate as FP64 accumulation at FP32 speed.
// 2. In FP64 (one thread): F = kappa S_W; the gradient of
//    eta -> F(T exp(eta^)) about the lever centre c in Z's frame, mapped to
//    the left perturbation exp(xi^) T.  With gc = (gc_w, gc_v) the centred
//    gradient, R, t the pose:  g_v = R gc_v,  g_w = R (gc_w + c x gc_v) + t x g_v.
//    The indicator of Eq. (indicator_actual) is F / sqrt(N M).
// 3. Registration (the method is gradient ascent on SE(3), Sec. I): the
//    ascent direction in a metric about Z's moved centroid, the Newton step
//    along it inside a trust region on the motion of Z's points (see
//    step_warp); T <- exp(t xi^) T (closed-form SE(3) exponential, Rodrigues
//    + left Jacobian); Gram-Schmidt on R every 16 iterations; the stopping
//    test; the lengthscale annealing of Sec. IV (l <- max(decay l, l_min)
//    once the indicator at the current l changes by less than indicator_tol
//    relative).  F'' is the quadratic form of the centred Hessian at the
//    direction's centred coordinates (w~, v~).
// 4. Writes the derived constants of the next sweep (double-float T^-1,
//    exponent scale, cutoff, grid level).
// An evaluation (no step) also assembles the full 6x6 Hessian.
//
// GB300 runs FP64 at 1/72 of the FP32 rate, so this serial code is kept to
// closed forms (no 6x6 products on the registration path).
#include <cooperative_groups.h>

#include "cvo_step_dev.cuh"

namespace cvo {
namespace {

__global__ void k_init_state(IterState* st)
{
    for (int r = 0; r < 3; ++r) split_df(st->c[r], st->chi[r], st->clo[r]);
    update_derived(st);
}

// the same for many pairs: thread i of the job list's states
__global__ void k_init_state_b(JobList<StateJob> J)
{
    const int i = threadIdx.x;
    if (i >= J.count) return;
    IterState* st = J.j[i].st;
    for (int r = 0; r < 3; ++r) split_df(st->c[r], st->chi[r], st->clo[r]);
    update_derived(st);
}

// The 43 statistics and the two counts of a sweep from its group sums, by a
// block of kStepThreads threads: statistic k by warp k % warps, each lane
// adding every 32nd group sum in group order (all its loads first), then the
// lanes' sums combined by a butterfly (lane 0's result is kept); fixed
// order, so deterministic.  S as doubles, Shi / Slo as double-float pairs.
__device__ void reduce_group_sums(const float2* __restrict__ gs, const unsigned long long* __restrict__ gc_,
                                  int ngroups, double* S, float* Shi, float* Slo, unsigned long long* cs)
{
    constexpr int kWarps = kStepThreads / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int kPerLane = kMaxGroups / 32;
    for (int k = warp; k < kStatN; k += kWarps) {
        const float2* row = gs + (size_t)k * kMaxGroups;
        float2 v[kPerLane];
#pragma unroll
        for (int j = 0; j < kPerLane; ++j) v[j] = lane + 32 * j < ngroups ? row[lane + 32 * j] : make_float2(0.0f, 0.0f);
        float hi = 0.0f, lo = 0.0f;
#pragma unroll
        for (int j = 0; j < kPerLane; ++j) df_add(hi, lo, v[j].x, v[j].y);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float oh = __shfl_xor_sync(0xffffffffu, hi, o), ol = __shfl_xor_sync(0xffffffffu, lo, o);
            df_add(hi, lo, oh, ol);
        }
        if (lane == 0) {
            S[k] = (double)hi + (double)lo;
            Shi[k] = hi;
            Slo[k] = lo;
        }
    }
    if (warp == kWarps - 1) {   // pair and candidate counts
        for (int c = 0; c < 2; ++c) {
            unsigned long long t = 0;
            for (int g = lane; g < ngroups; g += 32) t += gc_[(size_t)c * kMaxGroups + g];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
            if (lane == 0) cs[c] = t;
        }
    }
}

// The step on the block's shared copy of the state (sbuf), from the summed
// statistics, then the state written back.  Called by all kStepThreads
// threads after the statistics are in shared memory.
__device__ void finalize_tail(IterState* st, unsigned long long* sbuf, const double* S, const float* Shi,
                              const float* Slo, const unsigned long long* cs, double* trace,
                              cudaGraphConditionalHandle cond, int use_cond)
{
    constexpr int kWords = (int)(sizeof(IterState) / 8);
    IterState* sst = reinterpret_cast<IterState*>(sbuf);
    if (sst->done) {   // the sweep did nothing; inside a graph's loop: stop it
        if (use_cond && threadIdx.x == 0) cudaGraphSetConditional(cond, 0u);
        return;
    }
    if (sst->mode == 0) {
        if (threadIdx.x == 0) take_step(sst, S, cs[0], cs[1]);
    } else if (threadIdx.x < 32) {
        step_warp(sst, S, Shi, Slo, cs[0], cs[1], trace);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kWords; i += kStepThreads) reinterpret_cast<unsigned long long*>(st)[i] = sbuf[i];
    if (use_cond && threadIdx.x == 0) cudaGraphSetConditional(cond, sst->done ? 0u : 1u);
}

__global__ void __launch_bounds__(kStepThreads)
k_finalize(IterState* st, const float2* __restrict__ gs, const unsigned long long* __restrict__ gc_, int ngroups,
           double* trace, cudaGraphConditionalHandle cond, int use_cond)
{
    static_assert(sizeof(IterState) % 8 == 0, "state is copied in 8-byte words");
    constexpr int kWords = (int)(sizeof(IterState) / 8);
    __shared__ double S[kStatN];
    __shared__ float Shi[kStatN], Slo[kStatN];
    __shared__ unsigned long long cs[2];
    __shared__ unsigned long long sbuf[kWords];
    for (int i = threadIdx.x; i < kWords; i += kStepThreads) sbuf[i] = reinterpret_cast<const unsigned long long*>(st)[i];
    reduce_group_sums(gs, gc_, ngroups, S, Shi, Slo, cs);
    __syncthreads();
    finalize_tail(st, sbuf, S, Shi, Slo, cs, trace, cond, use_cond);
}

// A shard's sweep statistics as kShardStats doubles: the 43 statistics, the
// pair count and the candidate count (the counts are exact in a double up to
// 2^53).  Summed over the shards of one registration, they are what one
// sweep over all of X would give, up to rounding.
__global__ void __launch_bounds__(kStepThreads)
k_stats_out(const float2* __restrict__ gs, const unsigned long long* __restrict__ gc_, int ngroups, double* out)
{
    __shared__ double S[kStatN];
    __shared__ float Shi[kStatN], Slo[kStatN];
    __shared__ unsigned long long cs[2];
    reduce_group_sums(gs, gc_, ngroups, S, Shi, Slo, cs);
    __syncthreads();
    if (threadIdx.x < kStatN) out[threadIdx.x] = S[threadIdx.x];
    else if (threadIdx.x < kStatN + 2) out[threadIdx.x] = (double)cs[threadIdx.x - kStatN];
}

// The step from statistics summed over the shards of a registration (the
// output of k_stats_out added over the shards): the same step as k_finalize.
__global__ void __launch_bounds__(kStepThreads) k_finalize_stats(IterState* st, const double* __restrict__ in, double* trace)
{
    constexpr int kWords = (int)(sizeof(IterState) / 8);
    __shared__ double S[kStatN];
    __shared__ float Shi[kStatN], Slo[kStatN];
    __shared__ unsigned long long cs[2];
    __shared__ unsigned long long sbuf[kWords];
    for (int i = threadIdx.x; i < kWords; i += kStepThreads) sbuf[i] = reinterpret_cast<const unsigned long long*>(st)[i];
    if (threadIdx.x < kStatN) {
        const double v = in[threadIdx.x];
        S[threadIdx.x] = v;
        split_df(v, Shi[threadIdx.x], Slo[threadIdx.x]);
    } else if (threadIdx.x < kStatN + 2) {
        cs[threadIdx.x - kStatN] = (unsigned long long)in[threadIdx.x];
    }
    __syncthreads();
    finalize_tail(st, sbuf, S, Shi, Slo, cs, trace, cudaGraphConditionalHandle{}, 0);
}

// The last finalize block of a batch re-splits the sweep grid among the
// pairs still running, for the next sweep: pair k gets blocks [b0, b1) with
// b0 = a_k + floor((B - A) W_k / W) (a_k running pairs and W_k work before
// it, A and W in all, B the grid), b1 = b0 + 1 + the proportional share of
// its own work, then at most bmax.  Blocks between a capped pair's b1 and
// the next pair's b0 find no work (the sweep returns at once for them).  A
// fixed-order scan over the pairs in chunks of the block's threads.
__device__ void resplit_grid(PairDesc* pairs, int npairs, int nblocks, const unsigned* work)
{
    __shared__ unsigned long long s_w[kFinalizeThreads];
    __shared__ unsigned s_a[kFinalizeThreads];
    __shared__ unsigned long long tot_w;
    __shared__ unsigned tot_a;
    const int t = threadIdx.x;
    // totals
    unsigned long long w = 0;
    unsigned a = 0;
    for (int k = t; k < npairs; k += kFinalizeThreads) {
        const unsigned v = __ldcg(work + k);
        w += v;
        a += v > 0u ? 1u : 0u;
    }
    s_w[t] = w;
    s_a[t] = a;
    __syncthreads();
    if (t < 32) {   // integer sums: any order gives the same totals
        unsigned long long tw = 0;
        unsigned ta = 0;
        for (int i = t; i < kFinalizeThreads; i += 32) {
            tw += s_w[i];
            ta += s_a[i];
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            tw += __shfl_xor_sync(0xffffffffu, tw, o);
            ta += __shfl_xor_sync(0xffffffffu, ta, o);
        }
        if (t == 0) {
            tot_w = tw > 0 ? tw : 1;
            tot_a = ta;
        }
    }
    __syncthreads();
    const unsigned long long W = tot_w;
    const long long rem = (long long)nblocks - (long long)tot_a;
    if (tot_a == 0 || rem < 0) return;   // nothing runs (or more pairs than blocks: keep the split)
    unsigned long long carry_w = 0;
    unsigned carry_a = 0;
    for (int base = 0; base < npairs; base += kFinalizeThreads) {
        const int k = base + t;
        const unsigned v = k < npairs ? __ldcg(work + k) : 0u;
        __syncthreads();
        s_w[t] = v;
        s_a[t] = v > 0u ? 1u : 0u;
        __syncthreads();
        // inclusive scan of the chunk (Hillis-Steele, fixed order)
        for (int o = 1; o < kFinalizeThreads; o <<= 1) {
            const unsigned long long pw = t >= o ? s_w[t - o] : 0ull;
            const unsigned pa = t >= o ? s_a[t - o] : 0u;
            __syncthreads();
            s_w[t] += pw;
            s_a[t] += pa;
            __syncthreads();
        }
        if (k < npairs) {
            const unsigned long long wb = carry_w + s_w[t] - v;   // work before pair k
            const unsigned ab = carry_a + s_a[t] - (v > 0u ? 1u : 0u);
            const int b0 = (int)(ab + (unsigned long long)rem * wb / W);
            int b1 = b0;
            if (v > 0u) {
                const int b1p = (int)(ab + 1u + (unsigned long long)rem * (wb + v) / W);
                b1 = min(b1p, b0 + max(pairs[k].bmax, 1));
            }
            pairs[k].b0 = b0;
            pairs[k].b1 = b1;
        }
        carry_w += s_w[kFinalizeThreads - 1];
        carry_a += s_a[kFinalizeThreads - 1];
    }
}

// The sum of a batch's work-queue rows [i0, i1) (statistics in
// double-float bh + bl, counts in bc), in a fixed order: the block reads the rows as float4 columns,
// thread (r, c) of kRowGroups x kCols adding column c (statistics 4 c ..
// 4 c + 3; the counts at 43 and 44 as integers) of rows i0 + r, i0 + r +
// kRowGroups, ... in double-float, several rows' loads in flight; the
// kRowGroups partial sums of each statistic are then added in row-group
// order.  The order depends on the item numbers only, not on which warp
// swept an item.
__device__ void reduce_item_rows(const float* __restrict__ rows, int i0, int i1, float* bh, float* bl,
                                 unsigned long long* bc)
{
    constexpr int kCols = kRowFloats / 4;                  // 12 float4 per row
    constexpr int kRowGroups = kFinalizeThreads / kCols;   // 21
    constexpr int kUnroll = 12;
    __shared__ float ph[kRowGroups][kRowFloats], pl[kRowGroups][kRowFloats];
    __shared__ unsigned long long pc2[kRowGroups][2];
    const int t = threadIdx.x;
    if (t < kRowGroups * kCols) {
        const int c = t % kCols, r = t / kCols;
        float h[4] = {0.0f, 0.0f, 0.0f, 0.0f}, l[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        unsigned long long cnt0 = 0ull, cnt1 = 0ull;
        auto add = [&](const float4 v) {
            const float x[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int k = 4 * c + e;
                if (k < kStatN) df_add(h[e], l[e], x[e], 0.0f);
                else if (k == kStatN) cnt0 += __float_as_uint(x[e]);
                else if (k == kStatN + 1) cnt1 += __float_as_uint(x[e]);
            }
        };
        const float4* base = reinterpret_cast<const float4*>(rows) + c;
        int i = i0 + r;
        for (; i + (kUnroll - 1) * kRowGroups < i1; i += kUnroll * kRowGroups) {
            float4 v[kUnroll];
#pragma unroll
            for (int u = 0; u < kUnroll; ++u) v[u] = __ldcg(base + (size_t)(i + u * kRowGroups) * kCols);
#pragma unroll
            for (int u = 0; u < kUnroll; ++u) add(v[u]);
        }
        for (; i < i1; i += kRowGroups) add(__ldcg(base + (size_t)i * kCols));
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            ph[r][4 * c + e] = h[e];
            pl[r][4 * c + e] = l[e];
        }
        if (4 * c <= kStatN && kStatN < 4 * c + 4) pc2[r][0] = cnt0;
        if (4 * c <= kStatN + 1 && kStatN + 1 < 4 * c + 4) pc2[r][1] = cnt1;
    }
    __syncthreads();
    if (t < kStatN) {
        float hi = 0.0f, lo = 0.0f;
        for (int r = 0; r < kRowGroups; ++r) df_add(hi, lo, ph[r][t], pl[r][t]);
        bh[t] = hi;
        bl[t] = lo;
    } else if (t < kStatN + 2) {
        unsigned long long v = 0;
        for (int r = 0; r < kRowGroups; ++r) v += pc2[r][t - kStatN];
        bc[t - kStatN] = v;
    }
}

// The next sweep's first item of each pair: the exclusive prefix sum of the
// pairs' work (work[p] items, 0 for a stopped pair), by one block.
__device__ void queue_bases(const unsigned* work, int npairs, int* ibase, unsigned* queue)
{
    __shared__ unsigned wsum[kFinalizeThreads / 32];
    __shared__ unsigned carry;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) carry = 0u;
    __syncthreads();
    for (int k0 = 0; k0 < npairs; k0 += kFinalizeThreads) {
        const int k = k0 + (int)threadIdx.x;
        const unsigned v = k < npairs ? __ldcg(work + k) : 0u;
        unsigned incl = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) wsum[warp] = incl;
        __syncthreads();
        unsigned before = carry;
        for (int w = 0; w < warp; ++w) before += wsum[w];
        if (k < npairs) ibase[k] = (int)(before + incl - v);
        __syncthreads();
        if (threadIdx.x == kFinalizeThreads - 1) carry = before + incl;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        ibase[npairs] = (int)carry;
        queue[0] = 0u;
        queue[1] = carry;
    }
}

__global__ void __launch_bounds__(kFinalizeThreads)
k_finalize_batch(PairDesc* __restrict__ pairs, int npairs, const float2* __restrict__ ps,
                 const unsigned long long* __restrict__ pc, int cap, double* traces, long long trace_stride,
                 unsigned* counters, unsigned* work, cudaGraphConditionalHandle cond, int use_cond)
{
    constexpr int kWords = (int)(sizeof(IterState) / 8);
    __shared__ double S[kStatN];
    __shared__ float Shi[kStatN], Slo[kStatN];
    __shared__ unsigned long long cs[2];
    __shared__ unsigned long long sbuf[kWords];
    __shared__ int is_last;
    const PairDesc P = pairs[blockIdx.x];
    IterState* st = P.st;
    const bool was_done = st->done != 0;
    IterState* sst = reinterpret_cast<IterState*>(sbuf);
    if (!was_done) {
        for (int i = threadIdx.x; i < kWords; i += kFinalizeThreads)
            sbuf[i] = reinterpret_cast<const unsigned long long*>(st)[i];
        // statistic k by warp k % warps: lane l adds the pair's block
        // partials l, l + 32, ... (coalesced, all of a lane's loads issued
        // before its adds), then a butterfly over the lanes; a fixed order
        constexpr int kWarps = kFinalizeThreads / 32;
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        for (int k = warp; k < kStatN; k += kWarps) {
            const float2* row = ps + (size_t)k * cap;
            float hi = 0.0f, lo = 0.0f;
            int b = P.b0 + lane;
            for (; b + 96 < P.b1; b += 128) {
                const float2 v0 = row[b], v1 = row[b + 32], v2 = row[b + 64], v3 = row[b + 96];
                df_add(hi, lo, v0.x, v0.y);
                df_add(hi, lo, v1.x, v1.y);
                df_add(hi, lo, v2.x, v2.y);
                df_add(hi, lo, v3.x, v3.y);
            }
            for (; b < P.b1; b += 32) df_add(hi, lo, row[b].x, row[b].y);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const float oh = __shfl_xor_sync(0xffffffffu, hi, o), ol = __shfl_xor_sync(0xffffffffu, lo, o);
                df_add(hi, lo, oh, ol);
            }
            if (lane == 0) {
                S[k] = (double)hi + (double)lo;
                Shi[k] = hi;
                Slo[k] = lo;
            }
        }
        if (warp == kWarps - 1) {   // pair and candidate counts (integer sums: any order)
            for (int c = 0; c < 2; ++c) {
                const unsigned long long* row = pc + (size_t)c * cap;
                unsigned long long t = 0;
                for (int b = P.b0 + lane; b < P.b1; b += 32) t += row[b];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
                if (lane == 0) cs[c] = t;
            }
        }
        __syncthreads();
        if (threadIdx.x < 32)
            step_warp(sst, S, Shi, Slo, cs[0], cs[1], traces ? traces + (size_t)blockIdx.x * trace_stride : nullptr);
        __syncthreads();
        for (int i = threadIdx.x; i < kWords; i += kFinalizeThreads)
            reinterpret_cast<unsigned long long*>(st)[i] = sbuf[i];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const bool running = !was_done && !sst->done;
        // the work this pair has left: its items at its (next) grid level
        work[blockIdx.x] = running ? (unsigned)max(P.levels[sst->level].nitems, 1) : 0u;
        if (running) atomicAdd(&counters[1], 1u);
        __threadfence();
        is_last = atomicAdd(&counters[0], 1u) == (unsigned)(npairs - 1);
    }
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    resplit_grid(pairs, npairs, cap, work);
    if (threadIdx.x == 0) {
        const unsigned active = atomicAdd(&counters[1], 0u);
        counters[2] = active;
        counters[0] = 0u;
        counters[1] = 0u;
        if (use_cond) cudaGraphSetConditional(cond, active > 0u ? 1u : 0u);
    }
}

// The batched step with a work queue: a cluster of kStepCluster blocks per
// pair.  Block r of the cluster sums the r-th of kStepCluster equal slices
// of the pair's item rows (reduce_item_rows), block 0 adds the slices' sums
// in rank order through distributed shared memory and takes the step, so
// the order is fixed by the item numbers and the pair's rows are read by
// kStepCluster SMs at once.  Block 0 then records the pair's work at its
// next grid level (0 once stopped); the last pair to finish lays out the
// next sweep's queue (queue_bases) and, inside a graph, sets the loop's
// condition.
__global__ void __cluster_dims__(kStepCluster, 1, 1) __launch_bounds__(kFinalizeThreads)
k_finalize_batch_q(PairDesc* __restrict__ pairs, int npairs, double* traces, long long trace_stride,
                   unsigned* counters, unsigned* work, BatchQueue bq, cudaGraphConditionalHandle cond, int use_cond)
{
    namespace cg = cooperative_groups;
    constexpr int kWords = (int)(sizeof(IterState) / 8);
    __shared__ double S[kStatN];
    __shared__ float Shi[kStatN], Slo[kStatN];
    __shared__ unsigned long long cs[2];
    __shared__ unsigned long long sbuf[kWords];
    __shared__ float bh[kStatN], bl[kStatN];          // this block's slice sums
    __shared__ unsigned long long bc[2];
    __shared__ int is_last;
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank();
    const int pi = (int)blockIdx.x / kStepCluster;
    const PairDesc P = pairs[pi];
    IterState* st = P.st;
    const bool was_done = st->done != 0;   // the same for every block of the cluster
    if (!was_done) {
        const int i0 = bq.ibase[pi], n = bq.ibase[pi + 1] - i0;
        const int a = i0 + (int)(((long long)n * rank) / kStepCluster);
        const int b = i0 + (int)(((long long)n * (rank + 1)) / kStepCluster);
        reduce_item_rows(bq.rows, a, b, bh, bl, bc);
    }
    cluster.sync();
    IterState* sst = reinterpret_cast<IterState*>(sbuf);
    if (rank == 0 && !was_done) {
        const int t = threadIdx.x;
        if (t < kStatN) {
            float hi = 0.0f, lo = 0.0f;
            for (int r = 0; r < kStepCluster; ++r) {
                const float* rh = cluster.map_shared_rank(bh, r);
                const float* rl = cluster.map_shared_rank(bl, r);
                df_add(hi, lo, rh[t], rl[t]);
            }
            S[t] = (double)hi + (double)lo;
            Shi[t] = hi;
            Slo[t] = lo;
        } else if (t < kStatN + 2) {
            unsigned long long v = 0;
            for (int r = 0; r < kStepCluster; ++r) v += cluster.map_shared_rank(bc, r)[t - kStatN];
            cs[t - kStatN] = v;
        }
        for (int i = t; i < kWords; i += kFinalizeThreads) sbuf[i] = reinterpret_cast<const unsigned long long*>(st)[i];
    }
    cluster.sync();   // the other blocks' slice sums stay readable until block 0 has them
    if (rank != 0) return;
    if (!was_done) {
        if (threadIdx.x < 32)
            step_warp(sst, S, Shi, Slo, cs[0], cs[1], traces ? traces + (size_t)pi * trace_stride : nullptr);
        __syncthreads();
        for (int i = threadIdx.x; i < kWords; i += kFinalizeThreads)
            reinterpret_cast<unsigned long long*>(st)[i] = sbuf[i];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const bool running = !was_done && !sst->done;
        work[pi] = running ? (unsigned)P.levels[sst->level].nitems : 0u;
        if (running) atomicAdd(&counters[1], 1u);
        __threadfence();
        is_last = atomicAdd(&counters[0], 1u) == (unsigned)(npairs - 1);
    }
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    queue_bases(work, npairs, bq.ibase, bq.queue);
    if (threadIdx.x == 0) {
        const unsigned active = atomicAdd(&counters[1], 0u);
        counters[2] = active;
        counters[0] = 0u;
        counters[1] = 0u;
        if (use_cond) cudaGraphSetConditional(cond, active > 0u ? 1u : 0u);
    }
}

// The first sweep's work queue of a batch: each pair's items at the grid
// level its state starts on (none once stopped), their first-item numbers
// and the queue's counter.  One block.
__global__ void __launch_bounds__(kFinalizeThreads)
k_queue_init(const PairDesc* __restrict__ pairs, int npairs, unsigned* work, int* ibase, unsigned* queue)
{
    for (int k = threadIdx.x; k < npairs; k += kFinalizeThreads) {
        const IterState* st = pairs[k].st;
        work[k] = st->done ? 0u : (unsigned)pairs[k].levels[st->level].nitems;
    }
    __syncthreads();
    queue_bases(work, npairs, ibase, queue);
}

}  // namespace

cudaError_t launch_queue_init(const PairDesc* pairs, int npairs, unsigned* work, int* ibase, unsigned* queue,
                              cudaStream_t s)
{
    g_launch_count.fetch_add(1, std::memory_order_relaxed);
    k_queue_init<<<1, kFinalizeThreads, 0, s>>>(pairs, npairs, work, ibase, queue);
    return cudaGetLastError();
}

const void* finalize_kernel() { return (const void*)k_finalize; }
const void* finalize_batch_kernel() { return (const void*)k_finalize_batch; }
const void* finalize_batch_queue_kernel() { return (const void*)k_finalize_batch_q; }

cudaError_t launch_finalize_batch(PairDesc* pairs, int npairs, const float2* part_stats,
                                  const unsigned long long* part_cnt, int part_cap, double* traces,
                                  long long trace_stride, unsigned* counters, unsigned* work, BatchQueue bq,
                                  cudaStream_t s)
{
    g_launch_count.fetch_add(1, std::memory_order_relaxed);
    if (bq.rows != nullptr) {
        k_finalize_batch_q<<<npairs * kStepCluster, kFinalizeThreads, 0, s>>>(pairs, npairs, traces, trace_stride,
                                                                              counters, work, bq,
                                                                              cudaGraphConditionalHandle{}, 0);
        return cudaGetLastError();
    }
    k_finalize_batch<<<npairs, kFinalizeThreads, 0, s>>>(pairs, npairs, part_stats, part_cnt, part_cap, traces,
                                                         trace_stride, counters, work,
                                                         cudaGraphConditionalHandle{}, 0);
    return cudaGetLastError();
}

cudaError_t launch_init_state(IterState* st, cudaStream_t s)
{
    g_launch_count.fetch_add(1, std::memory_order_relaxed);
    k_init_state<<<1, 1, 0, s>>>(st);
    return cudaGetLastError();
}

cudaError_t launch_init_state_batch(const StateJob* jobs, int count, cudaStream_t s)
{
    for (int c0 = 0; c0 < count; c0 += kJobsPerLaunch) {
        JobList<StateJob> L;
        L.count = count - c0 < kJobsPerLaunch ? count - c0 : kJobsPerLaunch;
        for (int i = 0; i < L.count; ++i) L.j[i] = jobs[c0 + i];
        g_launch_count.fetch_add(1, std::memory_order_relaxed);
        k_init_state_b<<<1, kJobsPerLaunch, 0, s>>>(L);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_stats_out(const float2* grp_stats, const unsigned long long* grp_cnt, int nblocks, double* out,
                             cudaStream_t s)
{
    g_launch_count.fetch_add(1, std::memory_order_relaxed);
    const int ngroups = (nblocks + kGroupBlocks - 1) / kGroupBlocks;
    k_stats_out<<<1, kStepThreads, 0, s>>>(grp_stats, grp_cnt, ngroups, out);
    return cudaGetLastError();
}

cudaError_t launch_finalize_stats(IterState* st, const double* stats, double* trace, cudaStream_t s)
{
    g_launch_count.fetch_add(1, std::memory_order_relaxed);
    k_finalize_stats<<<1, kStepThreads, 0, s>>>(st, stats, trace);
    return cudaGetLastError();
}

cudaError_t launch_finalize(IterState* st, const float2* grp_stats, const unsigned long long* grp_cnt, int nblocks,
                            double* trace, cudaStream_t s)
{
    g_launch_count.fetch_add(1, std::memory_order_relaxed);
    const int ngroups = (nblocks + kGroupBlocks - 1) / kGroupBlocks;
    k_finalize<<<1, kStepThreads, 0, s>>>(st, grp_stats, grp_cnt, ngroups, trace, cudaGraphConditionalHandle{}, 0);
    return cudaGetLastError();
}

}  // namespace cvo
