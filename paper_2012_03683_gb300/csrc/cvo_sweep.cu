// The fused neighbour sweep: the hot loop of the double sum of Eq. (double_sum)
//
//   F = sum_{i,j} sigma^2 exp(-|x_i - T z_j|^2 / (2 l^2)) * c_ij
//
// evaluated in Z's frame, |x_i - T z_j| = |x'_i - z_j| with x'_i = T^-1 x_i.
//
// Work decomposition.  A warp owns one query group: up to 32 queries,
// consecutive in Hilbert order, that lie in one octree super-cell of X (so
// they stay spatially compact under any rigid motion), one query per lane.
// The group's candidate stream is every Z point in the grid cells that
// overlap the group's bounding box in Z's frame, grown by the cutoff radius;
// since the grid sorts Z by cell with x fastest, the stream is a short list
// of contiguous runs (one per (y, z) cell row).
// A group's stream is split into chunks, each its own work item (see the
// item layouts in cvo_internal.cuh).
//
// Staging.  The warp copies its stream into shared memory 32 records at a
// time with cp.async (one record per lane, so the copies are independent and
// in flight together), double buffered: while the warp evaluates batch b
// from shared memory, batch b + 1 is on its way.  Every lane then reads the
// same record (a broadcast), tests its own cutoff, and the warp skips the
// kernel evaluation when no lane is in range.
//
// Per pair: one ex2 (the geometric and squared-exponential feature exponents
// are added in log2 units), the inner products of the label blocks, and the
// moments W = sum w, E = sum w e, Q = sum w e e^T (e = z_j - x'_i) in FP32
// registers.  Per work item, the lanes' moments become 43 linear statistics
// (a warp butterfly after each item; running double-float sums per lane),
// summed per block and per group of blocks, from which the step kernel
// assembles F, the se(3) gradient and the Hessian.
//
// Precision.  x'_i is formed in double-float (hi + lo FP32 pair) from the
// FP32 input coordinates and a double-float copy of T^-1, so the offset
// e = (z - x'_hi) - x'_lo keeps the coordinates' full precision even 80 m
// from the origin (GB300's FP64 rate, 1/72 of FP32, rules out FP64 here).
#include "cvo_sweep_dev.cuh"

namespace cvo {
namespace {

template <class Feat, int S>
__global__ void __launch_bounds__(kSweepWarps * 32) k_sweep(SweepArgs a)
{
    extern __shared__ float4 stage_mem[];   // [kSweepWarps][2][32][rs]
    __shared__ float cst[30];               // Ahi, Alo, bhi, blo, chi, clo
    // the pair this block works on (blocks [b0, b1) of pair pi)
    int pi = 0;
    if (a.npairs > 1) {
        int lo = 0, hi = a.npairs - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (a.pairs[mid].b0 <= (int)blockIdx.x) lo = mid;
            else hi = mid - 1;
        }
        pi = lo;
    }
    const PairDesc P = a.pairs[pi];
    const IterState* st = P.st;
    if (st->done) return;   // uniform per pair; a single pair's blocks all return together
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x < 30) cst[threadIdx.x] = (&st->Ahi[0])[threadIdx.x];
    if (a.nch_next != nullptr && blockIdx.x == 0 && threadIdx.x == 0) *a.swept_level = st->level;
    __syncthreads();
    StatAcc acc;
    stat_acc_init(acc, lane);
    const LevelDesc L = P.levels[st->level];
    const int rs = rec_stride<Feat>(a.rs);
    const bool dense = a.dense != 0;
    const float sg = st->sg, rc = st->rc, rc2 = st->rc2;
    const FeatConst fc = a.fc;
    float4* stage = stage_mem + (size_t)warp * 2 * 32 * rs;
    unsigned char* scratch =
        reinterpret_cast<unsigned char*>(stage_mem + (size_t)kSweepWarps * 2 * 32 * rs) + (size_t)warp * Feat::kScratch;
    unsigned npairs = 0, ncand = 0;

    const int nitems = L.nitems;
    const int nblk = P.b1 - P.b0, bloc = (int)blockIdx.x - P.b0;
    // a batch that re-split its grid may leave blocks past a pair's range
    // (the pair has fewer items than blocks): they have no work, and no
    // finalize reads their partials (a single pair's range is the whole grid)
    if (bloc >= nblk) return;
    for (int item = bloc * kSweepWarps + warp; item < nitems; item += nblk * kSweepWarps) {
        Moments mo;
        float p[3];
        bool act;
        if (!sweep_item<Feat, S>(P, L, item, cst, rs, dense, sg, rc, rc2, fc, stage, scratch, lane, mo, p, act, npairs,
                              ncand, a.nch_next, a.chunk_len))
            continue;
        stat_acc_add(acc, mo, p, act, lane);
    }

    sweep_epilogue(acc, npairs, ncand, a, (int)blockIdx.x, (int)gridDim.x);
}

// The batched sweep as a work queue.  One resident wave of blocks of
// kQueueWarps warps; each warp takes the batch's next work item from a
// counter (a.queue[0]) until the ibase[npairs] items of this sweep are
// gone, so no warp waits for the others of its block and no slot waits for
// a block to be launched (the block split of k_sweep kept about 84 % of the
// warp slots busy on a 64-pair batch).  Item i belongs to the pair p with
// ibase[p] <= i < ibase[p + 1] (the running pairs' items in pair order,
// each pair's longest first); the warp keeps that pair's descriptor, grid
// level, state constants and transform in shared memory while its items
// follow one another.  Each item's 43 statistics and two counts go to its
// own row of a.item_rows, which the batched step sums in item order: the
// result does not depend on which warp took which item, so it is the same
// bits run after run.
template <class Feat, int S>
__global__ void __launch_bounds__(kQueueWarps * 32) k_sweep_q(SweepArgs a)
{
    extern __shared__ float4 stage_mem[];   // [kQueueWarps][2][32][rs], the warps' scratch, ibase
    __shared__ float cstw[kQueueWarps][32];         // per warp: Ahi, Alo, bhi, blo, chi, clo of its pair
    __shared__ PairDesc pairw[kQueueWarps];
    __shared__ LevelDesc levelw[kQueueWarps];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int np = a.npairs;
    const int rs = rec_stride<Feat>(a.rs);
    int* sib = reinterpret_cast<int*>(reinterpret_cast<unsigned char*>(stage_mem + (size_t)kQueueWarps * 2 * 32 * rs) +
                                      (size_t)kQueueWarps * Feat::kScratch);
    for (int k = threadIdx.x; k <= np; k += blockDim.x) sib[k] = __ldg(a.ibase + k);
    __syncthreads();
    const int total = sib[np];
    const bool dense = a.dense != 0;
    const FeatConst fc = a.fc;
    float4* stage = stage_mem + (size_t)warp * 2 * 32 * rs;
    unsigned char* scratch =
        reinterpret_cast<unsigned char*>(stage_mem + (size_t)kQueueWarps * 2 * 32 * rs) + (size_t)warp * Feat::kScratch;
    float* cst = cstw[warp];
    StatAcc idx;
    stat_acc_init(idx, lane);
    int pi = -1;
    float sg = 0.0f, rc = 0.0f, rc2 = 0.0f;
    for (;;) {
        int item = 0;
        if (lane == 0) item = (int)atomicAdd(a.queue, 1u);
        item = __shfl_sync(kFull, item, 0);
        if (item >= total) break;
        int lo = 0, hi = np - 1;   // the last pair whose first item is at or before this one
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (sib[mid] <= item) lo = mid;
            else hi = mid - 1;
        }
        if (lo != pi) {
            pi = lo;
            __syncwarp();
            const PairDesc P = a.pairs[pi];
            const IterState* st = P.st;
            if (lane == 0) {
                pairw[warp] = P;
                levelw[warp] = P.levels[__ldg(&st->level)];
            }
            if (lane < 30) cst[lane] = __ldg(&st->Ahi[0] + lane);
            sg = __ldg(&st->sg);
            rc = __ldg(&st->rc);
            rc2 = __ldg(&st->rc2);
            __syncwarp();
        }
        Moments mo;
        float p[3];
        bool act = false;
        unsigned npairs = 0, ncand = 0;
        const bool ok = sweep_item<Feat, S>(pairw[warp], levelw[warp], item - sib[pi], cst, rs, dense, sg, rc, rc2, fc,
                                            stage, scratch, lane, mo, p, act, npairs, ncand);
        stat_row_write(a.item_rows + (size_t)item * kRowFloats, idx, mo, p, ok && act, npairs, ncand, lane);
    }
}

// ---- gradients with respect to the inputs -----------------------------------
//
// For the pairs inside the cutoff (the pair set held fixed) and the weight
// w = kappa * 2^(arg) * prod(inner products) of one pair, e = z - x' in the
// sweep frame, d^2 = |e|^2:
//   dF/dx      = Rout * sum w e / l^2          (x the query point)
//   dF/dl      = sum w d^2 / l^3
//   dF/du_SE   = -sum w (u - v) / l_b^2        (squared-exponential block)
//   dF/du_DOT  = sum w_(b) v                   (inner-product block; w_(b)
//                                               is w without that block's factor)
// The same kernel serves both clouds: with X as the queries (Rout = R) and
// with Z as the queries over the grid of X (Rout = R^T).
// A policy per block list supplies the per-candidate feature work.

template <int DSE, int DDOT, bool BF16>
struct GradFixed {
    using F = FeatFixed<DSE, DDOT, BF16, true>;
    static constexpr int D = F::D;
    static constexpr bool kSharedAcc = false;
    using Q = typename F::Q;
    struct V {
        float v[D];
    };
    struct Acc {
        float a[D > 0 ? D : 1];   // SE entries: sum w (u - v); inner-product entries: sum w_(b) v
    };
    __device__ static void load_query(Q& q, const float4* rec, const FeatConst& fc) { F::load_query(q, rec, fc, nullptr, 0); }
    __device__ static void zero(Acc& a, float*, const FeatConst&)
    {
#pragma unroll
        for (int k = 0; k < D; ++k) a.a[k] = 0.0f;
    }
    // adds the feature exponent to arg, clears in when the feature-space
    // cutoff excludes the pair; returns the inner-product factor
    __device__ static float pair(const Q& q, const float4* rec, float& arg, bool& in, V& c, const FeatConst& fc)
    {
        F::unpack(rec + 1, c.v);
        if constexpr (DSE > 0) {
            float du2 = 0.0f;
#pragma unroll
            for (int k = 0; k < DSE; ++k) {
                const float d = q.v[k] - c.v[k];
                du2 = fmaf(d, d, du2);
            }
            arg = fmaf(du2, fc.s[0], arg);
            if (du2 > fc.fcut2[0]) in = false;
        }
        if constexpr (DDOT > 0) {
            float dot = 0.0f;
#pragma unroll
            for (int k = 0; k < DDOT; ++k) dot = fmaf(q.v[DSE + k], c.v[DSE + k], dot);
            return dot;
        }
        return 1.0f;
    }
    // base: the weight without the inner-product factor; w: the full weight
    __device__ static void accum(Acc& a, const Q& q, const float4*, const V& c, float base, float w, float*,
                                 const FeatConst&)
    {
#pragma unroll
        for (int k = 0; k < DSE; ++k) a.a[k] = fmaf(w, q.v[k] - c.v[k], a.a[k]);
#pragma unroll
        for (int k = 0; k < DDOT; ++k) a.a[DSE + k] = fmaf(base, c.v[DSE + k], a.a[DSE + k]);
    }
    __device__ static void store(const Acc& a, const float*, const FeatConst&, float* out)
    {
#pragma unroll
        for (int k = 0; k < D; ++k) out[k] = a.a[k];
    }
};

// Geometric kernel only (Eq. geometric_only): no feature outputs.
struct GradNone {
    static constexpr bool kSharedAcc = false;
    struct Q {};
    struct V {};
    struct Acc {};
    __device__ static void load_query(Q&, const float4*, const FeatConst&) {}
    __device__ static void zero(Acc&, float*, const FeatConst&) {}
    __device__ static float pair(const Q&, const float4*, float&, bool&, V&, const FeatConst&) { return 1.0f; }
    __device__ static void accum(Acc&, const Q&, const float4*, const V&, float, float, float*, const FeatConst&) {}
    __device__ static void store(const Acc&, const float*, const FeatConst&, float*) {}
};

// Any block list: per-lane feature accumulators in shared memory (stride 32).
struct GradGeneric {
    static constexpr bool kSharedAcc = true;
    struct Q {
        const float4* rec;
    };
    struct V {
        float val[4];   // per block: squared distance (SE) or inner product (DOT)
    };
    struct Acc {};
    __device__ static float get(const float4* rec, int k, int bf16)
    {
        if (bf16) return __uint_as_float(((unsigned)reinterpret_cast<const unsigned short*>(rec + 1)[k]) << 16);
        return reinterpret_cast<const float*>(rec + 1)[k];
    }
    __device__ static void load_query(Q& q, const float4* rec, const FeatConst&) { q.rec = rec; }
    __device__ static void zero(Acc&, float* sacc, const FeatConst& fc)
    {
        for (int k = 0; k < fc.D; ++k) sacc[32 * k] = 0.0f;
    }
    __device__ static float pair(const Q& q, const float4* rec, float& arg, bool& in, V& c, const FeatConst& fc)
    {
        float mult = 1.0f;
        for (int b = 0; b < fc.n_blocks; ++b) {
            float acc = 0.0f;
            for (int k = 0; k < fc.dim[b]; ++k) {
                const float u = get(q.rec, fc.off[b] + k, fc.bf16);
                const float v = get(rec, fc.off[b] + k, fc.bf16);
                if (fc.kind[b] == 0) {
                    const float d = u - v;
                    acc = fmaf(d, d, acc);
                } else {
                    acc = fmaf(u, v, acc);
                }
            }
            c.val[b] = acc;
            if (fc.kind[b] == 0) {
                arg = fmaf(acc, fc.s[b], arg);
                if (acc > fc.fcut2[b]) in = false;
            } else {
                mult *= acc;
            }
        }
        return mult;
    }
    __device__ static void accum(Acc&, const Q& q, const float4* rec, const V& c, float base, float w, float* sacc,
                                 const FeatConst& fc)
    {
        for (int b = 0; b < fc.n_blocks; ++b) {
            const int off = fc.off[b];
            if (fc.kind[b] == 0) {
                for (int k = 0; k < fc.dim[b]; ++k)
                    sacc[32 * (off + k)] = fmaf(w, get(q.rec, off + k, fc.bf16) - get(rec, off + k, fc.bf16),
                                                sacc[32 * (off + k)]);
            } else {
                float wb = base;
                for (int b2 = 0; b2 < fc.n_blocks; ++b2)
                    if (b2 != b && fc.kind[b2] == 1) wb *= c.val[b2];
                for (int k = 0; k < fc.dim[b]; ++k)
                    sacc[32 * (off + k)] = fmaf(wb, get(rec, off + k, fc.bf16), sacc[32 * (off + k)]);
            }
        }
    }
    __device__ static void store(const Acc&, const float* sacc, const FeatConst& fc, float* out)
    {
        for (int k = 0; k < fc.D; ++k) out[k] = sacc[32 * k];
    }
};

// One warp per work item (chunk k of n of one query group's stream, from the
// level's planned item table): every lane's raw sums over the chunk -- E (3),
// sum w d^2, and the feature accumulators (D) -- go to the item's rows of
// g.part; k_grad_reduce adds a group's chunks in chunk order.
template <class G>
__global__ void __launch_bounds__(kSweepWarps * 32) k_grad(GradArgs g)
{
    extern __shared__ float4 stage_mem[];   // [kSweepWarps][2][32][rs], then (generic) [kSweepWarps][D][32] floats
    __shared__ float cst[30];
    const IterState* st = g.st;
    if (threadIdx.x < 30) cst[threadIdx.x] = (&st->Ahi[0])[threadIdx.x];
    __syncthreads();
    const float* Ahi = cst;
    const float* Alo = cst + 9;
    const float* bhi = cst + 18;
    const float* blo = cst + 21;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const LevelDesc L = g.levels[st->level];
    const int rs = g.rs;
    const bool dense = g.dense != 0;
    const float sg = st->sg, rc = st->rc, rc2 = st->rc2;
    const FeatConst& fc = g.fc;
    const int stride = 4 + fc.D;
    float4* stage = stage_mem + (size_t)warp * 2 * 32 * rs;
    float* sacc = nullptr;
    if constexpr (G::kSharedAcc)
        sacc = reinterpret_cast<float*>(stage_mem + (size_t)kSweepWarps * 2 * 32 * rs) + (size_t)warp * fc.D * 32 +
               lane;

    for (int item = blockIdx.x * kSweepWarps + warp; item < L.nitems; item += gridDim.x * kSweepWarps) {
        const int4 w4 = L.items[item];
        const int2 grp = make_int2(w4.x, w4.y);
        const int k = w4.z & 0xffff, nch = w4.z >> 16;
        const bool act = lane < grp.y;
        const int qi = grp.x + (act ? lane : 0);
        const float4* qrec = g.xrec + (size_t)qi * rs;
        const float4 xq4 = qrec[0];
        const float xq[3] = {xq4.x, xq4.y, xq4.z};
        float xh[3], xl[3];
        transform_df(xq, Ahi, Alo, bhi, blo, xh, xl);

        typename G::Q qf;
        G::load_query(qf, qrec, fc);
        typename G::Acc fa;
        G::zero(fa, sacc, fc);
        float E0 = 0.0f, E1 = 0.0f, E2 = 0.0f, TQ = 0.0f;

        Stream sm;
        if (stream_setup(L, g.m, dense, act, xh, rc, lane, sm) && sm.total > 0) {
            const int clo_ = (int)(((long long)sm.total * k) / nch);
            const int chi_ = (int)(((long long)sm.total * (k + 1)) / nch);
            stream_walk(L, g.m, dense, sm, clo_, chi_, rs, stage, lane, [&](const float4* sb, int cnt) {
#pragma unroll 1
                for (int c = 0; c < cnt; ++c) {
                    const float4* zr = sb + c * rs;
                    const float4 z = zr[0];
                    const float dx = __fsub_rn(__fsub_rn(z.x, xh[0]), xl[0]);
                    const float dy = __fsub_rn(__fsub_rn(z.y, xh[1]), xl[1]);
                    const float dz = __fsub_rn(__fsub_rn(z.z, xh[2]), xl[2]);
                    const float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                    bool in = act && (dense || d2 <= rc2);
                    if (!__any_sync(kFull, in)) continue;
                    float arg = d2 * sg;
                    typename G::V cv;
                    const float mult = G::pair(qf, zr, arg, in, cv, fc);
                    const float base = in ? ex2(arg) : 0.0f;
                    const float w = base * mult;
                    E0 = fmaf(w, dx, E0);
                    E1 = fmaf(w, dy, E1);
                    E2 = fmaf(w, dz, E2);
                    TQ = fmaf(w, d2, TQ);
                    if (in) G::accum(fa, qf, zr, cv, base, w, sacc, fc);
                }
            });
        }
        float* row = g.part + ((size_t)item * 32 + lane) * stride;
        row[0] = E0;
        row[1] = E1;
        row[2] = E2;
        row[3] = TQ;
        G::store(fa, sacc, fc, row + 4);
        __syncwarp();
    }
}

// One warp per query group (the items with chunk 0): each lane adds its
// query's chunk rows in chunk order and writes the gradients at the query's
// index in the caller's order: dpos = scale_pos R_out E, the per-query term
// of dF/dl = scale_ell sum w d^2, and the feature columns times their scale.
__global__ void __launch_bounds__(128) k_grad_reduce(GradArgs g)
{
    const int lane = threadIdx.x & 31;
    const int stride = 4 + g.fc.D;
    const LevelDesc L = g.levels[g.st->level];
    for (int item = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; item < L.nitems; item += (gridDim.x * blockDim.x) >> 5) {
        const int4 w4 = L.items[item];
        if ((w4.z & 0xffff) != 0) continue;   // warp-uniform
        const int nch = w4.z >> 16;
        if (lane >= w4.y) continue;
        const int idx = __float_as_int(g.xrec[(size_t)(w4.x + lane) * g.rs].w);
        float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        for (int c = 0; c < nch; ++c) {
            const float* row = g.part + ((size_t)(item + c) * 32 + lane) * stride;
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[j] += row[j];
        }
        if (g.out_pos) {
#pragma unroll
            for (int r = 0; r < 3; ++r)
                g.out_pos[3 * (size_t)idx + r] =
                    g.scale_pos * fmaf(g.Rout[3 * r], acc[0], fmaf(g.Rout[3 * r + 1], acc[1], g.Rout[3 * r + 2] * acc[2]));
        }
        if (g.out_tq) g.out_tq[idx] = g.scale_ell * acc[3];
        if (g.out_feat) {
            for (int j = 0; j < g.fc.D; ++j) {
                float f = 0.0f;
                for (int c = 0; c < nch; ++c) f += g.part[((size_t)(item + c) * 32 + lane) * stride + 4 + j];
                g.out_feat[(size_t)idx * g.fc.D + j] = g.feat_scale[j] * f;
            }
        }
    }
}

template <class G>
cudaError_t grad_t(const GradArgs& g, int nblocks, cudaStream_t s)
{
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(k_grad<G>, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    size_t smem = (size_t)kSweepWarps * 2 * 32 * g.rs * sizeof(float4);
    if (G::kSharedAcc) smem += (size_t)kSweepWarps * g.fc.D * 32 * sizeof(float);
    g_launch_count.fetch_add(2, std::memory_order_relaxed);
    k_grad<G><<<nblocks, kSweepWarps * 32, smem, s>>>(g);
    k_grad_reduce<<<nblocks, 128, 0, s>>>(g);
    return cudaGetLastError();
}

// ---- work-item planning ------------------------------------------------------

// One warp per query group: the length of the group's candidate stream at the
// state's pose and cutoff radius rc, and the group's chunk count.
__device__ __forceinline__ void group_cost_body(const LevelDesc* __restrict__ levels, int level, int ngroups,
                                                const float4* __restrict__ xrec, int m, int rs, int dense,
                                                const IterState* __restrict__ st, float rc, int chunk_len,
                                                unsigned* keys, unsigned* vals, unsigned* nch, int g, int lane)
{
    if (g >= ngroups) return;   // warp-uniform
    if (chunk_len <= 0) {       // uniform items: Hilbert order, kChunks each
        if (lane == 0) {
            keys[g] = (unsigned)g;
            vals[g] = (unsigned)g;
            nch[g] = (unsigned)kChunks;
        }
        return;
    }
    const LevelDesc L = levels[level];
    const int2 grp = L.groups[g];
    const bool act = lane < grp.y;
    const float4 q = xrec[(size_t)(grp.x + (act ? lane : 0)) * rs];
    const float xq[3] = {q.x, q.y, q.z};
    float xh[3], xl[3];
    transform_df(xq, st->Ahi, st->Alo, st->bhi, st->blo, xh, xl);
    Stream sm;
    const int total = stream_setup(L, m, dense != 0, act, xh, rc, lane, sm) ? sm.total : 0;
    if (lane == 0) {
        const int c = (total + chunk_len - 1) / chunk_len;
        keys[g] = 0xffffffffu - (unsigned)total;   // ascending sort = longest stream first
        vals[g] = (unsigned)g;
        nch[g] = (unsigned)max(1, min(kMaxChunks, c));
    }
}

__global__ void __launch_bounds__(128) k_group_cost(const LevelDesc* __restrict__ levels, int level, int ngroups,
                                                    const float4* __restrict__ xrec, int m, int rs, int dense,
                                                    const IterState* __restrict__ st, float rc, int chunk_len,
                                                    unsigned* keys, unsigned* vals, unsigned* nch)
{
    group_cost_body(levels, level, ngroups, xrec, m, rs, dense, st, rc, chunk_len, keys, vals, nch,
                    (blockIdx.x * blockDim.x + threadIdx.x) >> 5, threadIdx.x & 31);
}

// the same for many pairs (blockIdx.y: the job)
__global__ void __launch_bounds__(128) k_group_cost_b(JobList<CostJob> J, int rs, int dense, int chunk_len)
{
    const CostJob& q = J.j[blockIdx.y];
    group_cost_body(q.levels, q.level, q.ngroups, q.xrec, q.m, rs, dense, q.st, q.rc, chunk_len, q.keys, q.vals, q.nch,
                    (blockIdx.x * blockDim.x + threadIdx.x) >> 5, threadIdx.x & 31);
}

// Work items of level Ld for the next sweep, group after group in group
// order, from the chunk counts the sweep recorded per group.  Warps
// 0 .. nw - 1 of the caller (w, lane) each own a contiguous range of groups,
// handled 32 * kLayAhead groups per round: all loads of a round first, the
// round's count to the other warps through part[] behind a barrier of their
// own (named barrier 1, nw warps), then a warp scan for the offsets and each
// lane writes its own group's items (a warp-wide loop over the groups with
// shuffles measured seven times slower).
constexpr int kLayAhead = 4;
__device__ void lay_out_items(LevelDesc* Ld, const unsigned* __restrict__ nch_next, int w, int nw, int lane,
                              unsigned* part)
{
    const unsigned full = 0xffffffffu;
    const int ng = Ld->ngroups;
    const int2* groups = Ld->groups;
    int4* items = const_cast<int4*>(Ld->items);
    constexpr int kRound = 32 * kLayAhead;
    const int rounds = (ng + kRound * nw - 1) / (kRound * nw);
    unsigned base = 0;   // items before this round's range of warp w
    for (int r = 0; r < rounds; ++r) {
        const int g0 = (r * nw + w) * kRound;
        int2 grp[kLayAhead];
        unsigned n[kLayAhead];
        unsigned s = 0;
#pragma unroll
        for (int a = 0; a < kLayAhead; ++a) {
            const int g = g0 + 32 * a + lane;
            grp[a] = g < ng ? groups[g] : make_int2(0, 0);
            n[a] = g < ng ? nch_next[g] : 0u;
        }
#pragma unroll
        for (int a = 0; a < kLayAhead; ++a) s += n[a];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(full, s, o);
        if (lane == 0) part[w] = s;
        asm volatile("bar.sync 1, %0;" ::"r"(nw * 32) : "memory");
        unsigned before = 0, all = 0;
        for (int k = 0; k < nw; ++k) {
            const unsigned v = part[k];
            before += k < w ? v : 0u;
            all += v;
        }
        asm volatile("bar.sync 1, %0;" ::"r"(nw * 32) : "memory");   // part[] is reused next round
        unsigned off0 = base + before;
#pragma unroll
        for (int a = 0; a < kLayAhead; ++a) {
            unsigned incl = n[a];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned t = __shfl_up_sync(full, incl, o);
                if (lane >= o) incl += t;
            }
            const unsigned off = off0 + incl - n[a];
            const int gbase = g0 + 32 * a;
            for (unsigned c = 0; c < n[a]; ++c)
                items[off + c] = make_int4(grp[a].x, grp[a].y, (int)(c | (n[a] << 16)), gbase + lane);
            off0 += __shfl_sync(full, incl, 31);
        }
        base += all;
    }
    if (w == 0 && lane == 0) {
        Ld->nitems = (int)base;
        Ld->chunk_min = 0;
    }
}

__global__ void __launch_bounds__(kLayoutThreads) k_layout(LevelDesc* levels, const int* swept_level,
                                                        const unsigned* __restrict__ nch_next)
{
    __shared__ unsigned part[kLayoutThreads / 32];
    lay_out_items(levels + *swept_level, nch_next, threadIdx.x >> 5, kLayoutThreads / 32, threadIdx.x & 31, part);
}

__global__ void k_gather_u32(const unsigned* __restrict__ src, const unsigned* __restrict__ idx, int n, unsigned* dst)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = src[idx[i]];
}

// Sorted group i (original index sorted_groups[i]) owns items
// [offsets[i], offsets[i] + nch[g]).
__global__ void k_write_items(const LevelDesc* __restrict__ levels, int level, const unsigned* __restrict__ sorted_groups,
                              const unsigned* __restrict__ nch, const unsigned* __restrict__ offsets, int ngroups,
                              int4* items)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ngroups) return;
    const int g = (int)sorted_groups[i];
    const int2 grp = levels[level].groups[g];
    const int n = (int)nch[g];
    const unsigned off = offsets[i];
    for (int k = 0; k < n; ++k) items[off + k] = make_int4(grp.x, grp.y, k | (n << 16), g);
}

__global__ void k_gather_b(JobList<GatherJob> J)
{
    const GatherJob& q = J.j[blockIdx.y];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < q.n) q.dst[i] = q.src[q.idx[i]];
}

__global__ void k_write_items_b(JobList<ItemsJob> J)
{
    const ItemsJob& q = J.j[blockIdx.y];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= q.ngroups) return;
    const int g = (int)q.sorted_groups[i];
    const int2 grp = q.levels[q.level].groups[g];
    const int n = (int)q.nch[g];
    const unsigned off = q.offsets[i];
    for (int k = 0; k < n; ++k) q.items[off + k] = make_int4(grp.x, grp.y, k | (n << 16), g);
}

template <class J, class F>
cudaError_t each_chunk(const J* jobs, int count, F&& f)
{
    for (int c0 = 0; c0 < count; c0 += kJobsPerLaunch) {
        JobList<J> L;
        L.count = min(kJobsPerLaunch, count - c0);
        for (int i = 0; i < L.count; ++i) L.j[i] = jobs[c0 + i];
        const cudaError_t e = f(L);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

template <class Feat, int S = 1>
cudaError_t info_t(int rs, SweepLaunch* out, bool queue = false)
{
    if (Feat::kRs > 0 && Feat::kRs != rs) return cudaErrorInvalidValue;   // the policy's record layout
    static bool attr_set = false;   // one-time opt-in above the 48 KB default
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(k_sweep<Feat, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_sweep_q<Feat, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    out->func = queue ? (const void*)k_sweep_q<Feat, S> : (const void*)k_sweep<Feat, S>;
    const int warps = queue ? kQueueWarps : kSweepWarps;
    out->smem = (size_t)warps * 2 * 32 * rs * sizeof(float4) + (size_t)warps * Feat::kScratch;
    out->threads = warps * 32;
    return cudaSuccess;
}

}  // namespace

// The sweep specialisation for a block list: kernel and dynamic shared memory.
template <bool Cut>
cudaError_t sweep_info_se3(const FeatConst& f, int rs, SweepLaunch* out, bool queue)
{
    if (f.n_blocks == 1)
        return f.bf16 ? info_t<FeatFixed<3, 0, true, Cut>>(rs, out, queue)
                      : info_t<FeatFixed<3, 0, false, Cut>>(rs, out, queue);
    // bfloat16 labels: the label inner products on the tensor cores
    return f.bf16 ? info_t<FeatMMA<3, Cut>>(rs, out, queue) : info_t<FeatFixed<3, 19, false, Cut>>(rs, out, queue);
}

// RGB + 19 labels with S lanes per query (the feature-space cutoff off)
template <int S>
cudaError_t sweep_info_lanes(const FeatConst& f, int rs, SweepLaunch* out, bool queue)
{
    return f.bf16 ? info_t<FeatMMA<3, false, S>, S>(rs, out, queue)
                  : info_t<FeatFixed<3, 19, false, false>, S>(rs, out, queue);
}

cudaError_t sweep_launch_info(const FeatConst& f, int rs, int lanes, SweepLaunch* out, bool queue)
{
    if (f.n_blocks == 0) return info_t<FeatNone>(rs, out, queue);
    const bool se3 = f.n_blocks >= 1 && f.kind[0] == 0 && f.dim[0] == 3;
    const bool labels = f.n_blocks == 2 && f.kind[1] == 1 && f.dim[1] == 19;
    // query groups of 32 / lanes queries: RGB + labels take each query's
    // candidates on that many lanes; any other block list (or the
    // feature-space cutoff) takes them on one lane, the group's other lanes
    // idle, which is correct but slower
    if (se3 && labels && f.fcut2[0] >= 1.0e38f) {
        if (lanes == 2) return sweep_info_lanes<2>(f, rs, out, queue);
        if (lanes == 4) return sweep_info_lanes<4>(f, rs, out, queue);
    }
    if (se3 && (f.n_blocks == 1 || labels)) {
        // the feature-space cutoff's test only where it is on (the colour block's limit is finite)
        return f.fcut2[0] < 1.0e38f ? sweep_info_se3<true>(f, rs, out, queue) : sweep_info_se3<false>(f, rs, out, queue);
    }
    if (f.n_blocks == 1 && f.kind[0] == 1 && f.dim[0] == 19)
        return f.bf16 ? info_t<FeatMMA<0, false>>(rs, out, queue)
                      : info_t<FeatFixed<0, 19, false, false>>(rs, out, queue);
    return info_t<FeatGeneric>(rs, out, queue);
}

// Gradient sweep specialisation for the block list (the same families as the
// sweep; any other block list takes the generic policy).
cudaError_t launch_grad(const GradArgs& g, int nblocks, cudaStream_t s)
{
    const FeatConst& f = g.fc;
    if (f.n_blocks == 0) return grad_t<GradNone>(g, nblocks, s);
    const bool se3 = f.n_blocks >= 1 && f.kind[0] == 0 && f.dim[0] == 3;
    if (f.n_blocks == 1 && se3)
        return f.bf16 ? grad_t<GradFixed<3, 0, true>>(g, nblocks, s) : grad_t<GradFixed<3, 0, false>>(g, nblocks, s);
    if (f.n_blocks == 2 && se3 && f.kind[1] == 1 && f.dim[1] == 19)
        return f.bf16 ? grad_t<GradFixed<3, 19, true>>(g, nblocks, s)
                      : grad_t<GradFixed<3, 19, false>>(g, nblocks, s);
    if (f.n_blocks == 1 && f.kind[0] == 1 && f.dim[0] == 19)
        return f.bf16 ? grad_t<GradFixed<0, 19, true>>(g, nblocks, s)
                      : grad_t<GradFixed<0, 19, false>>(g, nblocks, s);
    return grad_t<GradGeneric>(g, nblocks, s);
}

cudaError_t launch_group_cost(const LevelDesc* levels, int level, int ngroups, const float4* xrec, int m, int rs,
                              int dense, const IterState* st, float rc, int chunk_len, unsigned* keys, unsigned* vals,
                              unsigned* nch, cudaStream_t s)
{
    if (ngroups <= 0) return cudaSuccess;
    g_launch_count.fetch_add(1, std::memory_order_relaxed);
    k_group_cost<<<(ngroups + 3) / 4, 128, 0, s>>>(levels, level, ngroups, xrec, m, rs, dense, st, rc, chunk_len, keys,
                                                   vals, nch);
    return cudaGetLastError();
}

const void* layout_kernel() { return (const void*)k_layout; }

cudaError_t launch_layout(LevelDesc* levels, const int* swept_level, const unsigned* nch_next, cudaStream_t s)
{
    g_launch_count.fetch_add(1, std::memory_order_relaxed);
    k_layout<<<1, kLayoutThreads, 0, s>>>(levels, swept_level, nch_next);
    return cudaGetLastError();
}

cudaError_t launch_gather_u32(const unsigned* src, const unsigned* idx, int n, unsigned* dst, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    g_launch_count.fetch_add(1, std::memory_order_relaxed);
    k_gather_u32<<<(n + 255) / 256, 256, 0, s>>>(src, idx, n, dst);
    return cudaGetLastError();
}

cudaError_t launch_group_cost_batch(const CostJob* jobs, int count, int rs, int dense, int chunk_len, cudaStream_t s)
{
    return each_chunk(jobs, count, [&](const JobList<CostJob>& L) {
        int gmax = 1;
        for (int i = 0; i < L.count; ++i) gmax = max(gmax, L.j[i].ngroups);
        g_launch_count.fetch_add(1, std::memory_order_relaxed);
        k_group_cost_b<<<dim3((gmax + 3) / 4, L.count), 128, 0, s>>>(L, rs, dense, chunk_len);
        return cudaGetLastError();
    });
}

cudaError_t launch_gather_batch(const GatherJob* jobs, int count, cudaStream_t s)
{
    return each_chunk(jobs, count, [&](const JobList<GatherJob>& L) {
        int nmax = 1;
        for (int i = 0; i < L.count; ++i) nmax = max(nmax, L.j[i].n);
        g_launch_count.fetch_add(1, std::memory_order_relaxed);
        k_gather_b<<<dim3((nmax + 255) / 256, L.count), 256, 0, s>>>(L);
        return cudaGetLastError();
    });
}

cudaError_t launch_write_items_batch(const ItemsJob* jobs, int count, cudaStream_t s)
{
    return each_chunk(jobs, count, [&](const JobList<ItemsJob>& L) {
        int gmax = 1;
        for (int i = 0; i < L.count; ++i) gmax = max(gmax, L.j[i].ngroups);
        g_launch_count.fetch_add(1, std::memory_order_relaxed);
        k_write_items_b<<<dim3((gmax + 127) / 128, L.count), 128, 0, s>>>(L);
        return cudaGetLastError();
    });
}

cudaError_t launch_write_items(const LevelDesc* levels, int level, const unsigned* sorted_groups, const unsigned* nch,
                               const unsigned* offsets, int ngroups, int4* items, cudaStream_t s)
{
    if (ngroups <= 0) return cudaSuccess;
    g_launch_count.fetch_add(1, std::memory_order_relaxed);
    k_write_items<<<(ngroups + 127) / 128, 128, 0, s>>>(levels, level, sorted_groups, nch, offsets, ngroups, items);
    return cudaGetLastError();
}

cudaError_t launch_sweep(const SweepArgs& a, int nblocks, cudaStream_t s)
{
    SweepLaunch li;
    cudaError_t e = sweep_launch_info(a.fc, a.rs, a.lanes, &li, a.item_rows != nullptr);
    if (e != cudaSuccess) return e;
    void* args[1] = {(void*)&a};
    g_launch_count.fetch_add(1, std::memory_order_relaxed);
    const size_t smem = li.smem + (a.item_rows != nullptr ? queue_smem(a.npairs) : 0);
    return cudaLaunchKernel(li.func, dim3(nblocks), dim3(li.threads), args, smem, s);
}

}  // namespace cvo
