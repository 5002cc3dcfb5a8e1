// The fused neighbour sweep: the hot loop of the double sum of Eq. (double_sum)
//
//   F = sum_{i,j} sigma^2 exp(-|x_i - T z_j|^2 / (2 l^2)) * c_ij
//
// evaluated in Z's frame, |x_i - T z_j| = |x'_i - z_j| with x'_i = T^-1 x_i.
//
// Work decomposition.  A warp owns one query group: up to 32 queries that lie
// in one Morton super-cell of X (so they stay spatially compact under any
// rigid motion), one query per lane.  The group's candidate stream is every Z
// point in the grid cells that overlap the group's bounding box in Z's frame,
// grown by the cutoff radius; since the grid sorts Z by cell with x fastest,
// the stream is a short list of contiguous runs (one per (y, z) cell row).
// A group's stream is split into up to kChunks chunks, each its own work item.
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
// registers.  Per work item, each lane folds its moments into 43 linear
// statistics held in shared memory (see cvo_internal.cuh), from which the
// finalize kernel assembles F, the se(3) gradient and the Hessian.
//
// Precision.  x'_i is formed in double-float (hi + lo FP32 pair) from the
// FP32 input coordinates and a double-float copy of T^-1, so the offset
// e = (z - x'_hi) - x'_lo keeps the coordinates' full precision even 80 m
// from the origin (GB300's FP64 rate, 1/72 of FP32, rules out FP64 here).
#include "cvo_internal.cuh"

namespace cvo {
namespace {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ float ex2(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e)
{
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// x' = A x + b with A, b given as hi + lo FP32 pairs; result as hi + lo.
__device__ __forceinline__ void transform_df(const float x[3], const float* Ahi, const float* Alo, const float* bhi,
                                             const float* blo, float xh[3], float xl[3])
{
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        float s = bhi[r], e = blo[r];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float a = Ahi[3 * r + c];
            const float p = __fmul_rn(a, x[c]);
            const float pe = __fmaf_rn(a, x[c], -p);   // exact error of the product
            float t, te;
            two_sum(s, p, t, te);
            s = t;
            e = __fadd_rn(e, __fadd_rn(te, __fmaf_rn(Alo[3 * r + c], x[c], pe)));
        }
        const float hi = __fadd_rn(s, e);
        xh[r] = hi;
        xl[r] = __fsub_rn(e, __fsub_rn(hi, s));
    }
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_one() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

// ---- feature kernels c_ij ---------------------------------------------------
// Records are read through generic pointers: the query from global memory,
// the candidates from the shared-memory staging buffer.

// Eq. (geometric_only): no features, c_ij = 1.
struct FeatNone {
    struct Q {};
    __device__ static void load_query(Q&, const float4*, const FeatConst&) {}
    __device__ static float pair(const Q&, const float4*, float&, const FeatConst&) { return 1.0f; }
};

// One squared-exponential block (Eq. newscalar) of DSE entries followed by
// one inner-product block (Eq. scalar) of DDOT entries; either may be empty.
template <int DSE, int DDOT, bool BF16>
struct FeatFixed {
    static constexpr int D = DSE + DDOT;
    static constexpr int kVec = BF16 ? (2 * D + 15) / 16 : (4 * D + 15) / 16;
    struct Q {
        float v[D];
    };
    __device__ static void unpack(const float4* src, float (&v)[D])
    {
        if constexpr (BF16) {
            unsigned w[kVec * 4];
#pragma unroll
            for (int k = 0; k < kVec; ++k) {
                const uint4 u = reinterpret_cast<const uint4*>(src)[k];
                w[4 * k] = u.x; w[4 * k + 1] = u.y; w[4 * k + 2] = u.z; w[4 * k + 3] = u.w;
            }
#pragma unroll
            for (int k = 0; k < D; ++k)
                v[k] = (k & 1) ? __uint_as_float(w[k >> 1] & 0xffff0000u) : __uint_as_float(w[k >> 1] << 16);
        } else {
            float f[kVec * 4];
#pragma unroll
            for (int k = 0; k < kVec; ++k) {
                const float4 u = src[k];
                f[4 * k] = u.x; f[4 * k + 1] = u.y; f[4 * k + 2] = u.z; f[4 * k + 3] = u.w;
            }
#pragma unroll
            for (int k = 0; k < D; ++k) v[k] = f[k];
        }
    }
    __device__ static void load_query(Q& q, const float4* rec, const FeatConst&) { unpack(rec + 1, q.v); }
    __device__ static float pair(const Q& q, const float4* rec, float& arg, const FeatConst& fc)
    {
        float v[D];
        unpack(rec + 1, v);
        if constexpr (DSE > 0) {
            float du2 = 0.0f;
#pragma unroll
            for (int k = 0; k < DSE; ++k) {
                const float d = q.v[k] - v[k];
                du2 = fmaf(d, d, du2);
            }
            arg = fmaf(du2, fc.s[0], arg);
        }
        if constexpr (DDOT > 0) {
            float dot = 0.0f;
#pragma unroll
            for (int k = 0; k < DDOT; ++k) dot = fmaf(q.v[DSE + k], v[DSE + k], dot);
            return dot;
        }
        return 1.0f;
    }
};

// Any block list (up to 4 blocks, 64 entries): features read per pair.
struct FeatGeneric {
    struct Q {
        const float4* rec;
    };
    __device__ static float get(const float4* rec, int k, int bf16)
    {
        if (bf16) return __uint_as_float(((unsigned)reinterpret_cast<const unsigned short*>(rec + 1)[k]) << 16);
        return reinterpret_cast<const float*>(rec + 1)[k];
    }
    __device__ static void load_query(Q& q, const float4* rec, const FeatConst&) { q.rec = rec; }
    __device__ static float pair(const Q& q, const float4* rec, float& arg, const FeatConst& fc)
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
            if (fc.kind[b] == 0) arg = fmaf(acc, fc.s[b], arg);
            else mult *= acc;
        }
        return mult;
    }
};

// ---- the sweep --------------------------------------------------------------

__device__ __forceinline__ int floor_cell(float v, float o, float inv_h)
{
    const float c = floorf((v - o) * inv_h);
    return (int)fminf(fmaxf(c, -2.0e9f), 2.0e9f);
}

struct Moments {
    float W, E0, E1, E2, Qxx, Qyy, Qzz, Qxy, Qxz, Qyz;
};

// Evaluates the cnt staged candidates of one batch for this lane's query.
template <class Feat>
__device__ __forceinline__ void eval_batch(const float4* sb, int cnt, int rs, const typename Feat::Q& qf,
                                           const float xh[3], const float xl[3], bool act, bool dense, float sg,
                                           float rc2, const FeatConst& fc, Moments& mo, unsigned& npairs)
{
#pragma unroll 2
    for (int c = 0; c < cnt; ++c) {
        const float4* zr = sb + c * rs;
        const float4 z = zr[0];
        const float dx = __fsub_rn(__fsub_rn(z.x, xh[0]), xl[0]);
        const float dy = __fsub_rn(__fsub_rn(z.y, xh[1]), xl[1]);
        const float dz = __fsub_rn(__fsub_rn(z.z, xh[2]), xl[2]);
        const float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
        const bool in = act && (dense || d2 <= rc2);
        if (__any_sync(kFull, in)) {
            float arg = d2 * sg;
            const float mult = Feat::pair(qf, zr, arg, fc);
            const float w = in ? ex2(arg) * mult : 0.0f;
            npairs += in ? 1u : 0u;
            mo.W += w;
            const float wx = w * dx, wy = w * dy, wz = w * dz;
            mo.E0 += wx; mo.E1 += wy; mo.E2 += wz;
            mo.Qxx = fmaf(wx, dx, mo.Qxx); mo.Qyy = fmaf(wy, dy, mo.Qyy); mo.Qzz = fmaf(wz, dz, mo.Qzz);
            mo.Qxy = fmaf(wx, dy, mo.Qxy); mo.Qxz = fmaf(wx, dz, mo.Qxz); mo.Qyz = fmaf(wy, dz, mo.Qyz);
        }
    }
}

template <class Feat>
__global__ void __launch_bounds__(kSweepWarps * 32) k_sweep(SweepArgs a)
{
    extern __shared__ float4 stage_mem[];   // [kSweepWarps][2][32][rs]
    __shared__ float acc_s[kSweepWarps][kStatN][32];
    __shared__ unsigned long long redc[kSweepWarps][2];
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
#pragma unroll
    for (int k = 0; k < kStatN; ++k) acc_s[warp][k][lane] = 0.0f;
    __syncthreads();
    const float* Ahi = cst;
    const float* Alo = cst + 9;
    const float* bhi = cst + 18;
    const float* blo = cst + 21;
    const float* chi = cst + 24;
    const float* clo = cst + 27;
    const LevelDesc L = P.levels[st->level];
    const int rs = a.rs;
    const bool dense = a.dense != 0;
    const float sg = st->sg, rc = st->rc, rc2 = st->rc2;
    const FeatConst fc = a.fc;
    float4* stage = stage_mem + (size_t)warp * 2 * 32 * rs;
    unsigned npairs = 0, ncand = 0;

    const int nitems = L.ngroups * kChunks;
    const int nblk = P.b1 - P.b0, bloc = (int)blockIdx.x - P.b0;
    for (int item = bloc * kSweepWarps + warp; item < nitems; item += nblk * kSweepWarps) {
        const int g = item / kChunks;
        const int k = item - g * kChunks;
        const int2 grp = L.groups[g];
        const bool act = lane < grp.y;
        const int qi = grp.x + (act ? lane : 0);
        const float4* qrec = P.xrec + (size_t)qi * rs;
        const float4 xq4 = qrec[0];
        const float xq[3] = {xq4.x, xq4.y, xq4.z};
        float xh[3], xl[3];
        transform_df(xq, Ahi, Alo, bhi, blo, xh, xl);

        // candidate stream: runs of cells (one per (y, z) cell row)
        int cx0 = 0, cx1 = 0, cy0 = 0, cz0 = 0, nry = 1, nruns = 1;
        if (!dense) {
            float mn[3], mx[3];
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                mn[r] = act ? xh[r] : 3.0e38f;
                mx[r] = act ? xh[r] : -3.0e38f;
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
                for (int r = 0; r < 3; ++r) {
                    mn[r] = fminf(mn[r], __shfl_xor_sync(kFull, mn[r], o));
                    mx[r] = fmaxf(mx[r], __shfl_xor_sync(kFull, mx[r], o));
                }
            }
            const float o3[3] = {L.ox, L.oy, L.oz};
            const int n3[3] = {L.nx, L.ny, L.nz};
            int c0[3], c1[3];
            bool empty = false;
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                const float pad = rc * 1.0001f + 4.0e-7f * fmaxf(fabsf(mn[r]), fabsf(mx[r])) + 1.0e-6f;
                c0[r] = floor_cell(mn[r] - pad, o3[r], L.inv_h);
                c1[r] = floor_cell(mx[r] + pad, o3[r], L.inv_h);
                if (c1[r] < 0 || c0[r] > n3[r] - 1) empty = true;
                c0[r] = max(c0[r], 0);
                c1[r] = min(c1[r], n3[r] - 1);
            }
            if (empty) continue;
            cx0 = c0[0]; cx1 = c1[0]; cy0 = c0[1]; cz0 = c0[2];
            nry = c1[1] - c0[1] + 1;
            nruns = nry * (c1[2] - c0[2] + 1);
        }
        // total stream length
        int total = 0;
        for (int b0 = 0; b0 < nruns; b0 += 32) {
            int len = 0;
            const int r = b0 + lane;
            if (r < nruns) {
                if (dense) {
                    len = P.m;
                } else {
                    const int cy = cy0 + r % nry, cz = cz0 + r / nry;
                    const int row = (cz * L.ny + cy) * L.nx;
                    len = __ldg(L.cell_start + row + cx1 + 1) - __ldg(L.cell_start + row + cx0);
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) len += __shfl_xor_sync(kFull, len, o);
            total += len;
        }
        if (total == 0) continue;
        const int nch = min(kChunks, (total + kChunkMin - 1) / kChunkMin);
        if (k >= nch) continue;
        const int clo_ = (int)(((long long)total * k) / nch);
        const int chi_ = (int)(((long long)total * (k + 1)) / nch);

        typename Feat::Q qf;
        Feat::load_query(qf, qrec, fc);
        Moments mo = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};

        int base = 0;
        for (int b0 = 0; b0 < nruns && base < chi_; b0 += 32) {
            int rstart = 0, rlen = 0;
            const int r = b0 + lane;
            if (r < nruns) {
                if (dense) {
                    rstart = 0;
                    rlen = P.m;
                } else {
                    const int cy = cy0 + r % nry, cz = cz0 + r / nry;
                    const int row = (cz * L.ny + cy) * L.nx;
                    rstart = __ldg(L.cell_start + row + cx0);
                    rlen = __ldg(L.cell_start + row + cx1 + 1) - rstart;
                }
            }
            int incl = rlen;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int v = __shfl_up_sync(kFull, incl, o);
                if (lane >= o) incl += v;
            }
            const int roff = incl - rlen;
            const int btotal = __shfl_sync(kFull, incl, 31);
            const int lo = max(clo_, base) - base;   // positions relative to this pass
            const int hi = min(chi_, base + btotal) - base;
            if (lo < hi) {
                const int nbat = (hi - lo + 31) >> 5;
                // stage batch bi (positions lo + 32 bi + lane) into buffer bi & 1
                auto issue = [&](int bi) {
                    const int p0 = lo + 32 * bi;
                    const int p = p0 + lane;
                    // first run that ends after p0
                    const unsigned before = __ballot_sync(kFull, (r < nruns) && (roff + rlen <= p0));
                    int j = -1;
                    for (int ri = __popc(before); ri < 32; ++ri) {
                        const int o = __shfl_sync(kFull, roff, ri);
                        const int l = __shfl_sync(kFull, rlen, ri);
                        const int s0 = __shfl_sync(kFull, rstart, ri);
                        if (o >= p0 + 32 || o >= hi) break;
                        if (p < hi && p >= o && p < o + l) j = s0 + (p - o);
                    }
                    if (j >= 0) {
                        const float4* src = L.zrec + (size_t)j * rs;
                        float4* dst = stage + ((bi & 1) * 32 + lane) * rs;
                        for (int q = 0; q < rs; ++q) cp_async16(dst + q, src + q);
                    }
                    cp_async_commit();
                };
                issue(0);
                for (int bi = 0; bi < nbat; ++bi) {
                    if (bi + 1 < nbat) {
                        issue(bi + 1);
                        cp_async_wait_one();
                    } else {
                        cp_async_wait_all();
                    }
                    __syncwarp();
                    const int cnt = min(32, hi - (lo + 32 * bi));
                    eval_batch<Feat>(stage + (bi & 1) * 32 * rs, cnt, rs, qf, xh, xl, act, dense, sg, rc2, fc, mo,
                                     npairs);
                    ncand += act ? (unsigned)cnt : 0u;
                    __syncwarp();
                }
            }
            base += btotal;
        }
        if (act) {
            // lever arm p = x' - c
            const float p0 = (xh[0] - chi[0]) + (xl[0] - clo[0]);
            const float p1 = (xh[1] - chi[1]) + (xl[1] - clo[1]);
            const float p2 = (xh[2] - chi[2]) + (xl[2] - clo[2]);
            const float Q[3][3] = {{mo.Qxx, mo.Qxy, mo.Qxz}, {mo.Qxy, mo.Qyy, mo.Qyz}, {mo.Qxz, mo.Qyz, mo.Qzz}};
            float PQ[3][3];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                PQ[0][c] = -p2 * Q[1][c] + p1 * Q[2][c];
                PQ[1][c] = p2 * Q[0][c] - p0 * Q[2][c];
                PQ[2][c] = -p1 * Q[0][c] + p0 * Q[1][c];
            }
            float* acc = &acc_s[warp][0][lane];
            auto add = [&](int s, float v) { acc[s * 32] += v; };
            add(ST_W, mo.W);
            add(ST_E + 0, mo.E0); add(ST_E + 1, mo.E1); add(ST_E + 2, mo.E2);
            add(ST_Q + 0, mo.Qxx); add(ST_Q + 1, mo.Qyy); add(ST_Q + 2, mo.Qzz);
            add(ST_Q + 3, mo.Qxy); add(ST_Q + 4, mo.Qxz); add(ST_Q + 5, mo.Qyz);
#pragma unroll
            for (int rr = 0; rr < 3; ++rr)
#pragma unroll
                for (int c = 0; c < 3; ++c) add(ST_PQ + 3 * rr + c, PQ[rr][c]);
            // [p]x Q [p]x, symmetric: (0,0) (1,1) (2,2) (0,1) (0,2) (1,2)
            add(ST_PQP + 0, PQ[0][1] * p2 - PQ[0][2] * p1);
            add(ST_PQP + 1, -PQ[1][0] * p2 + PQ[1][2] * p0);
            add(ST_PQP + 2, PQ[2][0] * p1 - PQ[2][1] * p0);
            add(ST_PQP + 3, -PQ[0][0] * p2 + PQ[0][2] * p0);
            add(ST_PQP + 4, PQ[0][0] * p1 - PQ[0][1] * p0);
            add(ST_PQP + 5, PQ[1][0] * p1 - PQ[1][1] * p0);
            const float Wp0 = mo.W * p0, Wp1 = mo.W * p1, Wp2 = mo.W * p2;
            add(ST_WP + 0, Wp0); add(ST_WP + 1, Wp1); add(ST_WP + 2, Wp2);
            add(ST_WPP + 0, Wp0 * p0); add(ST_WPP + 1, Wp1 * p1); add(ST_WPP + 2, Wp2 * p2);
            add(ST_WPP + 3, Wp0 * p1); add(ST_WPP + 4, Wp0 * p2); add(ST_WPP + 5, Wp1 * p2);
            const float Ev[3] = {mo.E0, mo.E1, mo.E2}, pv[3] = {p0, p1, p2};
#pragma unroll
            for (int rr = 0; rr < 3; ++rr)
#pragma unroll
                for (int c = 0; c < 3; ++c) add(ST_EP + 3 * rr + c, Ev[rr] * pv[c]);
        }
    }

    // warp tree (FP32, fixed order), then the block's warps in double-float
    __syncwarp();
    for (int k = 0; k < kStatN; ++k) {
        float v = acc_s[warp][k][lane];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
        if (lane == 0) acc_s[warp][k][0] = v;
    }
    unsigned long long cp = npairs, cc = ncand;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        cp += __shfl_xor_sync(kFull, cp, o);
        cc += __shfl_xor_sync(kFull, cc, o);
    }
    if (lane == 0) {
        redc[warp][0] = cp;
        redc[warp][1] = cc;
    }
    __syncthreads();
    if (threadIdx.x < kStatN) {
        float hi = 0.0f, lo = 0.0f;
        for (int w = 0; w < kSweepWarps; ++w) {
            float s, e;
            two_sum(hi, acc_s[w][threadIdx.x][0], s, e);
            e = __fadd_rn(e, lo);
            hi = __fadd_rn(s, e);
            lo = __fsub_rn(e, __fsub_rn(hi, s));
        }
        a.part_stats[(size_t)threadIdx.x * a.part_cap + blockIdx.x] = make_float2(hi, lo);
    } else if (threadIdx.x == kStatN) {
        unsigned long long t0 = 0, t1 = 0;
        for (int w = 0; w < kSweepWarps; ++w) {
            t0 += redc[w][0];
            t1 += redc[w][1];
        }
        a.part_cnt[blockIdx.x] = t0;
        a.part_cnt[(size_t)a.part_cap + blockIdx.x] = t1;
    }

    // Group reduction: the last block of each group of kGroupBlocks blocks to
    // arrive sums the group's partials in block order (deterministic; nothing
    // waits) and resets the group's arrival counter for the next launch.
    if (a.grp_arrivals == nullptr) return;   // batch: the finalize sums the block partials per pair
    __shared__ int is_last;
    const int grp = blockIdx.x / kGroupBlocks;
    const int first = grp * kGroupBlocks;
    const int members = min(kGroupBlocks, (int)gridDim.x - first);
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) is_last = (atomicAdd(&a.grp_arrivals[grp], 1u) == (unsigned)(members - 1));
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    if (threadIdx.x < kStatN) {
        const float2* row = a.part_stats + (size_t)threadIdx.x * a.part_cap + first;
        float2 v[kGroupBlocks];
#pragma unroll
        for (int b = 0; b < kGroupBlocks; ++b) v[b] = b < members ? __ldcg(row + b) : make_float2(0.0f, 0.0f);
        float hi = 0.0f, lo = 0.0f;
#pragma unroll
        for (int b = 0; b < kGroupBlocks; ++b) {
            float s, e;
            two_sum(hi, v[b].x, s, e);
            e = __fadd_rn(e, __fadd_rn(lo, v[b].y));
            hi = __fadd_rn(s, e);
            lo = __fsub_rn(e, __fsub_rn(hi, s));
        }
        a.grp_stats[(size_t)threadIdx.x * kMaxGroups + grp] = make_float2(hi, lo);
    } else if (threadIdx.x == kStatN || threadIdx.x == kStatN + 1) {
        const int c = threadIdx.x - kStatN;
        unsigned long long t = 0;
        for (int b = 0; b < members; ++b) t += __ldcg(a.part_cnt + (size_t)c * a.part_cap + first + b);
        a.grp_cnt[(size_t)c * kMaxGroups + grp] = t;
    }
    if (threadIdx.x == 0) a.grp_arrivals[grp] = 0u;
}

template <class Feat>
cudaError_t info_t(int rs, SweepLaunch* out)
{
    static bool attr_set = false;   // one-time opt-in above the 48 KB default
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(k_sweep<Feat>, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    out->func = (const void*)k_sweep<Feat>;
    out->smem = (size_t)kSweepWarps * 2 * 32 * rs * sizeof(float4);
    return cudaSuccess;
}

}  // namespace

// The sweep specialisation for a block list: kernel and dynamic shared memory.
cudaError_t sweep_launch_info(const FeatConst& f, int rs, SweepLaunch* out)
{
    if (f.n_blocks == 0) return info_t<FeatNone>(rs, out);
    const bool se3 = f.n_blocks >= 1 && f.kind[0] == 0 && f.dim[0] == 3;
    if (f.n_blocks == 1 && se3)
        return f.bf16 ? info_t<FeatFixed<3, 0, true>>(rs, out) : info_t<FeatFixed<3, 0, false>>(rs, out);
    if (f.n_blocks == 2 && se3 && f.kind[1] == 1 && f.dim[1] == 19)
        return f.bf16 ? info_t<FeatFixed<3, 19, true>>(rs, out) : info_t<FeatFixed<3, 19, false>>(rs, out);
    if (f.n_blocks == 1 && f.kind[0] == 1 && f.dim[0] == 19)
        return f.bf16 ? info_t<FeatFixed<0, 19, true>>(rs, out) : info_t<FeatFixed<0, 19, false>>(rs, out);
    return info_t<FeatGeneric>(rs, out);
}

cudaError_t launch_sweep(const SweepArgs& a, int nblocks, cudaStream_t s)
{
    SweepLaunch li;
    cudaError_t e = sweep_launch_info(a.fc, a.rs, &li);
    if (e != cudaSuccess) return e;
    void* args[1] = {(void*)&a};
    g_launch_count.fetch_add(1, std::memory_order_relaxed);
    return cudaLaunchKernel(li.func, dim3(nblocks), dim3(kSweepWarps * 32), args, li.smem, s);
}

}  // namespace cvo
