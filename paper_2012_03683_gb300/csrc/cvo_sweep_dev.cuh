// Device code of the neighbour sweep (query transform, feature kernels,
// candidate streams and their staging, the pairwise evaluation), shared by
// the sweep kernels and the persistent registration kernel.  See
// cvo_sweep.cu for the design.
#pragma once
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
// Interface of a feature policy: kScratch bytes of shared memory per warp;
// kRs, the record stride in float4 that its layout fixes (0 where only the
// launch knows it: the host checks the two agree, and a fixed stride lets
// the compiler fold the staged records' addresses); load_query once per work
// item; batch once per staged batch of candidates
// (warp-uniform); pair per candidate c of the batch, adding the feature
// exponent to arg, clearing in when the feature-space cutoff excludes the
// pair, and returning the product of the inner-product factors.
struct FeatNone {
    static constexpr int kScratch = 0;
    static constexpr int kRs = 1;
    struct Q {};
    __device__ static void load_query(Q&, const float4*, const FeatConst&, unsigned char*, int) {}
    __device__ static void batch(Q&, const float4*, int, int, int) {}
    __device__ static float pair(const Q&, const float4*, int, float&, bool&, const FeatConst&) { return 1.0f; }
};

// One squared-exponential block (Eq. newscalar) of DSE entries followed by
// one inner-product block (Eq. scalar) of DDOT entries; either may be empty.
// Cut: the feature-space cutoff is on (else its test is compiled out).
template <int DSE, int DDOT, bool BF16, bool Cut>
struct FeatFixed {
    static constexpr int kScratch = 0;
    static constexpr int D = DSE + DDOT;
    static constexpr int kVec = BF16 ? (2 * D + 15) / 16 : (4 * D + 15) / 16;
    static constexpr int kRs = 1 + kVec;
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
    __device__ static void load_query(Q& q, const float4* rec, const FeatConst&, unsigned char*, int)
    {
        unpack(rec + 1, q.v);
    }
    __device__ static void batch(Q&, const float4*, int, int, int) {}
    __device__ static float pair(const Q& q, const float4* rec, int, float& arg, bool& in, const FeatConst& fc)
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
            if constexpr (Cut) {
                if (du2 > fc.fcut2[0]) in = false;
            }
        }
        if constexpr (DDOT > 0) {
            float d4[4] = {0.0f, 0.0f, 0.0f, 0.0f};   // four independent chains
#pragma unroll
            for (int k = 0; k < DDOT; ++k) d4[k & 3] = fmaf(q.v[DSE + k], v[DSE + k], d4[k & 3]);
            return (d4[0] + d4[1]) + (d4[2] + d4[3]);
        }
        return 1.0f;
    }
};

// Any block list (up to 4 blocks, 64 entries): features read per pair.
struct FeatGeneric {
    static constexpr int kScratch = 0;
    static constexpr int kRs = 0;
    struct Q {
        const float4* rec;
    };
    __device__ static float get(const float4* rec, int k, int bf16)
    {
        if (bf16) return __uint_as_float(((unsigned)reinterpret_cast<const unsigned short*>(rec + 1)[k]) << 16);
        return reinterpret_cast<const float*>(rec + 1)[k];
    }
    __device__ static void load_query(Q& q, const float4* rec, const FeatConst&, unsigned char*, int) { q.rec = rec; }
    __device__ static void batch(Q&, const float4*, int, int, int) {}
    __device__ static float pair(const Q& q, const float4* rec, int, float& arg, bool& in, const FeatConst& fc)
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
            if (fc.kind[b] == 0) {
                arg = fmaf(acc, fc.s[b], arg);
                if (acc > fc.fcut2[b]) in = false;
            } else {
                mult *= acc;
            }
        }
        return mult;
    }
};

// One squared-exponential block of DSE entries (0 or 3) and one inner-product
// block of 19 labels, stored in bfloat16: the label inner products of a
// warp's 32 queries with a staged batch of 32 candidates form a 32 x 32 x 19
// contraction, done on the tensor cores (mma.sync m16n8k16, bfloat16 inputs,
// float32 accumulation: the products of bfloat16 values are exact, so this
// matches the scalar float32 sum up to its order).  Per warp scratch: a
// 32 x 40 bfloat16 tile (the queries' labels once per item, then each
// batch's candidate labels) and the 32 x 32 float results, candidate-major
// with a row stride of 36 floats: the accumulator fragments store without
// bank conflicts (lane (g, t) of a fragment writes bank g + 8 t) and each
// candidate's row is read by the 32 lanes from 32 consecutive words.
// With S lanes per query (S = 2, 4: groups of 32 / S queries, one row tile
// of 16) the results are stored in rows of S candidates x 32 / S queries,
// row stride 40 floats: the fragment stores stay conflict free (lane (g, t)
// writes bank 8 t + g plus a constant) and the S lanes of a query, which
// take S consecutive candidates at once, read one row's disjoint parts.
template <int DSE, bool Cut, int S = 1>
struct FeatMMA {
    static constexpr int kL = 19;
    static constexpr int D = DSE + kL;
    static constexpr int kQ = 32 / S;                         // queries per group
    static constexpr int kMt = S == 1 ? 2 : 1;                // row tiles of 16 queries
    static constexpr int kRowBytes = 80;                      // 32 labels + pad: conflict-free fragment loads
    static constexpr int kTileBytes = 32 * kRowBytes;
    static constexpr int kCsStride = 36;
    static constexpr int kCsRow = 40;
    static constexpr int kScratch = kTileBytes + 32 * kCsStride * 4;
    static constexpr int kRs = 1 + (2 * D + 15) / 16;   // xyz, then D bfloat16 features
    static_assert(S == 1 || (32 / S) * kCsRow <= 32 * kCsStride, "the grouped result rows fit the tile");
    struct Q {
        float se[DSE > 0 ? DSE : 1];
        unsigned a[kMt][2][4];      // A fragments [m tile][k step][register]
        unsigned char* tile;
        float* cs;
        int col;                    // this lane's query (its column of the results)
    };
    // where the label product of candidate c and query r is kept
    __device__ static int cs_index(int c, int r)
    {
        if constexpr (S == 1) return c * kCsStride + r;
        else return (c / S) * kCsRow + (c % S) * kQ + r;
    }
    // label pairs (l, l + 1), l = 0, 2, ..., 30 (zero past the 19th) of a
    // record's bfloat16 feature row
    __device__ static void label_pairs(const float4* feat, unsigned (&out)[16])
    {
        unsigned w[12];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const uint4 u = reinterpret_cast<const uint4*>(feat)[k];
            w[4 * k] = u.x; w[4 * k + 1] = u.y; w[4 * k + 2] = u.z; w[4 * k + 3] = u.w;
        }
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const int l = 2 * j;
            if (l >= 20) {
                out[j] = 0u;
            } else if constexpr (DSE & 1) {
                out[j] = __byte_perm(w[(DSE + l) >> 1], w[((DSE + l) >> 1) + 1], 0x5432);
            } else {
                out[j] = w[(DSE + l) >> 1];
            }
        }
        // the 20th entry of the last pair is the row's zero padding (or, with
        // an odd DSE, the next feature slot, also padding)
    }
    __device__ static void store_row(unsigned char* tile, int row, const unsigned (&v)[16])
    {
        uint4* dst = reinterpret_cast<uint4*>(tile + row * kRowBytes);
#pragma unroll
        for (int k = 0; k < 4; ++k) dst[k] = make_uint4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]);
    }
    __device__ static unsigned word(const unsigned char* tile, int row, int col)
    {
        return reinterpret_cast<const unsigned*>(tile + row * kRowBytes)[col];
    }
    __device__ static void load_query(Q& q, const float4* rec, const FeatConst&, unsigned char* scratch, int lane)
    {
        q.tile = scratch;
        q.cs = reinterpret_cast<float*>(scratch + kTileBytes);
        q.col = lane & (kQ - 1);
        if constexpr (DSE > 0) {
            const uint4 u = reinterpret_cast<const uint4*>(rec + 1)[0];
            const unsigned w[2] = {u.x, u.y};
#pragma unroll
            for (int k = 0; k < DSE; ++k)
                q.se[k] = (k & 1) ? __uint_as_float(w[k >> 1] & 0xffff0000u) : __uint_as_float(w[k >> 1] << 16);
        }
        unsigned v[16];
        label_pairs(rec + 1, v);
        __syncwarp();
        store_row(q.tile, lane, v);
        __syncwarp();
        const int g = lane >> 2, t = lane & 3;
#pragma unroll
        for (int mt = 0; mt < kMt; ++mt)
#pragma unroll
            for (int ks = 0; ks < 2; ++ks) {
                q.a[mt][ks][0] = word(q.tile, g + 16 * mt, t + 8 * ks);
                q.a[mt][ks][1] = word(q.tile, g + 8 + 16 * mt, t + 8 * ks);
                q.a[mt][ks][2] = word(q.tile, g + 16 * mt, t + 4 + 8 * ks);
                q.a[mt][ks][3] = word(q.tile, g + 8 + 16 * mt, t + 4 + 8 * ks);
            }
        __syncwarp();
    }
    // the 32 x 32 label inner products of the batch, into cs (query-major)
    __device__ static void batch(Q& q, const float4* sb, int cnt, int rs, int lane)
    {
        unsigned v[16];
        if (lane < cnt) {
            label_pairs(sb + (size_t)lane * rs + 1, v);
        } else {
#pragma unroll
            for (int j = 0; j < 16; ++j) v[j] = 0u;
        }
        store_row(q.tile, lane, v);
        __syncwarp();
        const int g = lane >> 2, t = lane & 3;
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) {
            unsigned b[2][2];
#pragma unroll
            for (int ks = 0; ks < 2; ++ks) {
                b[ks][0] = word(q.tile, g + 8 * nt, t + 8 * ks);
                b[ks][1] = word(q.tile, g + 8 * nt, t + 4 + 8 * ks);
            }
#pragma unroll
            for (int mt = 0; mt < kMt; ++mt) {
                float c0 = 0.0f, c1 = 0.0f, c2 = 0.0f, c3 = 0.0f;
#pragma unroll
                for (int ks = 0; ks < 2; ++ks)
                    asm volatile(
                        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, "
                        "{%8, %9}, {%0, %1, %2, %3};\n"
                        : "+f"(c0), "+f"(c1), "+f"(c2), "+f"(c3)
                        : "r"(q.a[mt][ks][0]), "r"(q.a[mt][ks][1]), "r"(q.a[mt][ks][2]), "r"(q.a[mt][ks][3]),
                          "r"(b[ks][0]), "r"(b[ks][1]));
                const int r0 = g + 16 * mt, col = 2 * t + 8 * nt;   // query row, candidate column
                q.cs[cs_index(col, r0)] = c0;
                q.cs[cs_index(col + 1, r0)] = c1;
                if (r0 + 8 < kQ) {   // rows past the group's queries are not kept
                    q.cs[cs_index(col, r0 + 8)] = c2;
                    q.cs[cs_index(col + 1, r0 + 8)] = c3;
                }
            }
        }
        __syncwarp();
    }
    __device__ static float pair(const Q& q, const float4* rec, int c, float& arg, bool& in, const FeatConst& fc)
    {
        if constexpr (DSE > 0) {
            const uint4 u = reinterpret_cast<const uint4*>(rec + 1)[0];
            const unsigned w[2] = {u.x, u.y};
            float du2 = 0.0f;
#pragma unroll
            for (int k = 0; k < DSE; ++k) {
                const float v = (k & 1) ? __uint_as_float(w[k >> 1] & 0xffff0000u) : __uint_as_float(w[k >> 1] << 16);
                const float d = q.se[k] - v;
                du2 = fmaf(d, d, du2);
            }
            arg = fmaf(du2, fc.s[0], arg);
            if constexpr (Cut) {
                if (du2 > fc.fcut2[0]) in = false;
            }
        }
        return q.cs[cs_index(c, q.col)];
    }
};

// ---- the sweep --------------------------------------------------------------


// The record stride a kernel of policy Feat works with: the policy's own
// where it fixes one (a compile-time constant), else the launch's.
template <class Feat>
__device__ __forceinline__ int rec_stride(int rs)
{
    return Feat::kRs > 0 ? Feat::kRs : rs;
}

__device__ __forceinline__ int floor_cell(float v, float o, float inv_h)
{
    const float c = floorf((v - o) * inv_h);
    return (int)fminf(fmaxf(c, -2.0e9f), 2.0e9f);
}

// A query group's candidate stream: for each (y, z) row of grid cells that
// overlaps the group's bounding box grown by the cutoff radius, the run of
// the row's cells whose x-range can hold a point within the radius of the
// group.  A point at (y, z) distance d from the row needs only the x-range
// within sqrt(r^2 - d^2) of it (none when d > r).  Taken for the group's
// box, the run covers the box grown by a ball, not by a cube, in whole
// cells; with the level's trim flag, runs 0-31 take it for each query and
// cover the union of the queries' ranges, the queries' balls (on the cube
// scenes 12 % fewer candidates, for a loop over the queries per row; a
// stream has rarely more runs).  r0start / r0len: this lane's run's first
// cell record and record count for runs 0-31 (the walk's first pass reads
// them instead of bounding the rows again).
struct Stream {
    int cx0, cx1, cy0, cz0, nry, nruns, total, nq, r0start, r0len;
};

// The group's box (Z frame: min xyz, max xyz) and the cutoff radius with its
// rounding margin, per warp in shared memory (read once per run, so they
// need not hold registers through the candidate loop).  Warps of up to
// 1024-thread blocks.
__device__ __forceinline__ float* stream_box()
{
    __shared__ float box[32][8];
    return box[threadIdx.x >> 5];
}

// The group's query positions (Z frame, the high parts of x'), per warp in
// shared memory: entry q is lane q's query; an inactive lane's entry lies
// out of every row's reach.  Warps of blocks of up to kStreamWarps warps
// (every kernel that forms streams is launched with at most that many).
__device__ __forceinline__ float4* stream_queries()
{
    __shared__ float4 qp[kStreamWarps][32];
    return qp[threadIdx.x >> 5];
}

__device__ __forceinline__ float sqrt_approx(float x)
{
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// The cells [a, b] of run r (row cy0 + r % nry, cz0 + r / nry) of a stream
// with a cutoff; a > b when the row is out of reach.  The gaps between the
// row's cell extent and the box (or the queries) are shrunk, and the radius
// grown, by margins above the FP32 rounding of the coordinates (and of the
// square root), so no pair within the cutoff is left out.  per_query: the
// run takes the union of the queries' ranges (else the box's range).
__device__ __forceinline__ void run_cells(const LevelDesc& L, const Stream& s, int r, bool per_query, int& a, int& b)
{
    const float* bx = stream_box();
    const float bmn[3] = {bx[0], bx[1], bx[2]}, bmx[3] = {bx[3], bx[4], bx[5]}, rad = bx[6];
    const int cy = s.cy0 + r % s.nry, cz = s.cz0 + r / s.nry;
    const float ylo = L.oy + (float)cy * L.h, zlo = L.oz + (float)cz * L.h;
    const float yhi = ylo + L.h, zhi = zlo + L.h;
    // margins: the rounding of the cell bounds (|origin| + |bound| + h) and of the box
    const float ty = 4.0e-7f * (fabsf(L.oy) + fabsf(ylo) + L.h + fmaxf(fabsf(bmn[1]), fabsf(bmx[1]))) + 1.0e-6f;
    const float tz = 4.0e-7f * (fabsf(L.oz) + fabsf(zlo) + L.h + fmaxf(fabsf(bmn[2]), fabsf(bmx[2]))) + 1.0e-6f;
    float lo = 3.0e38f, hi = -3.0e38f;
    if (per_query) {
        const float4* qp = stream_queries();
        const float rad2 = rad * rad;
        for (int q = 0; q < s.nq; ++q) {
            const float4 x = qp[q];
            const float gy = fmaxf(0.0f, fmaxf(ylo - x.y, x.y - yhi) - ty);
            const float gz = fmaxf(0.0f, fmaxf(zlo - x.z, x.z - zhi) - tz);
            const float w2 = rad2 - fmaf(gy, gy, gz * gz);
            if (w2 >= 0.0f) {
                const float w = sqrt_approx(w2) * 1.0001f;
                lo = fminf(lo, x.x - w);
                hi = fmaxf(hi, x.x + w);
            }
        }
    } else {
        const float gy = fmaxf(0.0f, fmaxf(ylo - bmx[1], bmn[1] - yhi) - ty);
        const float gz = fmaxf(0.0f, fmaxf(zlo - bmx[2], bmn[2] - zhi) - tz);
        const float w2 = rad * rad - (gy * gy + gz * gz);
        if (w2 >= 0.0f) {
            const float w = sqrtf(w2) * 1.0001f;
            lo = bmn[0] - w;
            hi = bmx[0] + w;
        }
    }
    if (lo > hi) {
        a = 1;
        b = 0;
        return;
    }
    const float tx = 4.0e-7f * fmaxf(fabsf(bmn[0]), fabsf(bmx[0])) + 1.0e-6f;
    a = max(s.cx0, floor_cell(lo - tx, L.ox, L.inv_hx));
    b = min(s.cx1, floor_cell(hi + tx, L.ox, L.inv_hx));
}

// Warp-uniform.  Returns false when the grown box misses the grid.
__device__ __forceinline__ bool stream_setup(const LevelDesc& L, int m, bool dense, bool act, const float xh[3],
                                             float rc, int lane, Stream& s)
{
    s.cx0 = s.cx1 = s.cy0 = s.cz0 = 0;
    s.nry = 1;
    s.nruns = 1;
    s.nq = 0;
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
            const float inv = r == 0 ? L.inv_hx : L.inv_h;
            c0[r] = floor_cell(mn[r] - pad, o3[r], inv);
            c1[r] = floor_cell(mx[r] + pad, o3[r], inv);
            if (c1[r] < 0 || c0[r] > n3[r] - 1) empty = true;
            c0[r] = max(c0[r], 0);
            c1[r] = min(c1[r], n3[r] - 1);
        }
        if (empty) return false;
        s.cx0 = c0[0]; s.cx1 = c1[0]; s.cy0 = c0[1]; s.cz0 = c0[2];
        s.nry = c1[1] - c0[1] + 1;
        s.nruns = s.nry * (c1[2] - c0[2] + 1);
        float* bx = stream_box();
        float4* qp = stream_queries();
        __syncwarp();   // a previous stream of this warp may still be reading the box and queries
        if (lane == 0) {
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                bx[q] = mn[q];
                bx[3 + q] = mx[q];
            }
            bx[6] = rc * 1.0001f + 1.0e-6f;
        }
        if (L.trim) {
            qp[lane] = act ? make_float4(xh[0], xh[1], xh[2], 0.0f) : make_float4(0.0f, 3.0e38f, 3.0e38f, 0.0f);
            s.nq = 32 - __clz(__ballot_sync(kFull, act));   // entries past the last active lane are not read
        }
        __syncwarp();
    }
    int total = 0;
    s.r0start = 0;
    s.r0len = 0;
    for (int b0 = 0; b0 < s.nruns; b0 += 32) {
        int start = 0, len = 0;
        const int r = b0 + lane;
        if (r < s.nruns) {
            if (dense) {
                len = m;
            } else {
                int a, b;
                run_cells(L, s, r, L.trim && b0 == 0, a, b);
                if (a <= b) {
                    const int cy = s.cy0 + r % s.nry, cz = s.cz0 + r / s.nry;
                    const int row = (cz * L.ny + cy) * L.nx;
                    start = __ldg(L.cell_start + row + a);
                    len = __ldg(L.cell_start + row + b + 1) - start;
                }
            }
        }
        if (b0 == 0) {
            s.r0start = start;
            s.r0len = len;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) len += __shfl_xor_sync(kFull, len, o);
        total += len;
    }
    s.total = total;
    return true;
}

// Stages the stream positions [clo, chi) into shared memory 32 records at a
// time (cp.async, one record per lane, double buffered) and calls
// op(batch, count) on each staged batch.  Warp-uniform.
template <class Op>
__device__ __forceinline__ void stream_walk(const LevelDesc& L, int m, bool dense, const Stream& s, int clo, int chi,
                                            int rs, float4* stage, int lane, Op&& op)
{
    int base = 0;
    for (int b0 = 0; b0 < s.nruns && base < chi; b0 += 32) {
        int rstart = 0, rlen = 0;
        const int r = b0 + lane;
        if (b0 == 0) {   // the runs the setup trimmed
            rstart = s.r0start;
            rlen = s.r0len;
        } else if (r < s.nruns) {
            if (dense) {
                rstart = 0;
                rlen = m;
            } else {
                int a, b;
                run_cells(L, s, r, false, a, b);   // runs past the first 32 take the box's range
                if (a <= b) {
                    const int cy = s.cy0 + r % s.nry, cz = s.cz0 + r / s.nry;
                    const int row = (cz * L.ny + cy) * L.nx;
                    rstart = __ldg(L.cell_start + row + a);
                    rlen = __ldg(L.cell_start + row + b + 1) - rstart;
                }
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
        const int lo = max(clo, base) - base;   // positions relative to this pass
        const int hi = min(chi, base + btotal) - base;
        if (lo < hi) {
            const int nbat = (hi - lo + 31) >> 5;
            // stage batch bi (positions lo + 32 bi + lane) into buffer bi & 1
            auto issue = [&](int bi) {
                const int p0 = lo + 32 * bi;
                const int p = p0 + lane;
                // first run that ends after p0
                const unsigned before = __ballot_sync(kFull, (r < s.nruns) && (roff + rlen <= p0));
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
                op(stage + (bi & 1) * 32 * rs, min(32, hi - (lo + 32 * bi)));
                __syncwarp();
            }
        }
        base += btotal;
    }
}

struct Moments {
    float W, E0, E1, E2, Qxx, Qyy, Qzz, Qxy, Qxz, Qyz;
};

// Offset e = z - x' (double-float query) and its squared length.
struct Offset {
    float dx, dy, dz, d2;
};
__device__ __forceinline__ Offset offset_to(const float4& z, const float xh[3], const float xl[3])
{
    Offset o;
    o.dx = __fsub_rn(__fsub_rn(z.x, xh[0]), xl[0]);
    o.dy = __fsub_rn(__fsub_rn(z.y, xh[1]), xl[1]);
    o.dz = __fsub_rn(__fsub_rn(z.z, xh[2]), xl[2]);
    o.d2 = fmaf(o.dx, o.dx, fmaf(o.dy, o.dy, o.dz * o.dz));
    return o;
}

__device__ __forceinline__ void add_moments(Moments& mo, float w, const Offset& o)
{
    mo.W += w;
    const float wx = w * o.dx, wy = w * o.dy, wz = w * o.dz;
    mo.E0 += wx; mo.E1 += wy; mo.E2 += wz;
    mo.Qxx = fmaf(wx, o.dx, mo.Qxx); mo.Qyy = fmaf(wy, o.dy, mo.Qyy); mo.Qzz = fmaf(wz, o.dz, mo.Qzz);
    mo.Qxy = fmaf(wx, o.dy, mo.Qxy); mo.Qxz = fmaf(wx, o.dz, mo.Qxz); mo.Qyz = fmaf(wy, o.dz, mo.Qyz);
}

// Evaluates the cnt staged candidates of one batch for this lane's query.
// Candidates go two at a time under one warp vote: the two evaluations are
// independent chains (staged loads, feature products, ex2), which hides
// latency at this kernel's occupancy; a pair with no lane in range is skipped.
// With S lanes per query (S > 1), lane s of a query takes candidates s, s + S,
// s + 2 S, ... of the batch, two at a time.
template <class Feat, int S = 1>
__device__ __forceinline__ void eval_batch(const float4* sb, int cnt, int rs, typename Feat::Q& qf,
                                           const float xh[3], const float xl[3], bool act, bool dense, float sg,
                                           float rc2, const FeatConst& fc, Moments& mo, unsigned& npairs, int lane)
{
    Feat::batch(qf, sb, cnt, rs, lane);
    // one comparison per candidate: an inactive lane takes no pair, the dense
    // sum every pair
    const float lim = act ? (dense ? 3.0e38f : rc2) : -1.0f;
    if constexpr (S > 1) {
        const int s = lane / (32 / S);
        for (int base = 0; base < cnt; base += 2 * S) {
            const int c0 = base + s, c1 = base + S + s;
            const bool v0 = c0 < cnt, v1 = c1 < cnt;
            const int r0 = v0 ? c0 : 0, r1 = v1 ? c1 : 0;   // past the batch: read record 0, take no pair
            const float4* zr0 = sb + r0 * rs;
            const float4* zr1 = sb + r1 * rs;
            const Offset o0 = offset_to(zr0[0], xh, xl);
            const Offset o1 = offset_to(zr1[0], xh, xl);
            bool in0 = v0 && o0.d2 <= lim;
            bool in1 = v1 && o1.d2 <= lim;
            if (__any_sync(kFull, in0 || in1)) {
                float a0 = o0.d2 * sg, a1 = o1.d2 * sg;
                const float m0 = Feat::pair(qf, zr0, r0, a0, in0, fc);
                const float m1 = Feat::pair(qf, zr1, r1, a1, in1, fc);
                const float w0 = in0 ? ex2(a0) * m0 : 0.0f;
                const float w1 = in1 ? ex2(a1) * m1 : 0.0f;
                npairs += (in0 ? 1u : 0u) + (in1 ? 1u : 0u);
                add_moments(mo, w0, o0);
                add_moments(mo, w1, o1);
            }
        }
        return;
    }
    auto two = [&](int c) {
        const float4* zr0 = sb + c * rs;
        const float4* zr1 = zr0 + rs;
        const Offset o0 = offset_to(zr0[0], xh, xl);
        const Offset o1 = offset_to(zr1[0], xh, xl);
        bool in0 = o0.d2 <= lim;
        bool in1 = o1.d2 <= lim;
        if (__any_sync(kFull, in0 || in1)) {
            float a0 = o0.d2 * sg, a1 = o1.d2 * sg;
            const float m0 = Feat::pair(qf, zr0, c, a0, in0, fc);
            const float m1 = Feat::pair(qf, zr1, c + 1, a1, in1, fc);
            const float w0 = in0 ? ex2(a0) * m0 : 0.0f;
            const float w1 = in1 ? ex2(a1) * m1 : 0.0f;
            npairs += (in0 ? 1u : 0u) + (in1 ? 1u : 0u);
            add_moments(mo, w0, o0);
            add_moments(mo, w1, o1);
        }
    };
    // a full batch: a loop of fixed trip count, not unrolled (unrolled 4 or
    // 16 times it measured slower: the loop body is long already)
    if (cnt == 32) {
#pragma unroll 1
        for (int c = 0; c < 32; c += 2) two(c);
        return;
    }
    int c = 0;
    for (; c + 1 < cnt; c += 2) two(c);
    if (c < cnt) {
        const float4* zr = sb + c * rs;
        const Offset o = offset_to(zr[0], xh, xl);
        bool in = o.d2 <= lim;
        if (__any_sync(kFull, in)) {
            float arg = o.d2 * sg;
            const float mult = Feat::pair(qf, zr, c, arg, in, fc);
            const float w = in ? ex2(arg) * mult : 0.0f;
            npairs += in ? 1u : 0u;
            add_moments(mo, w, o);
        }
    }
}

// Chunk k of n of one query group's candidate stream (grp = first query,
// count): the moments of this lane's query over the chunk, and its lever
// arm p = x' - c.  cst: the state's derived constants Ahi, Alo, bhi, blo,
// chi, clo (30 floats).  Returns false when the group's stream is empty.
template <class Feat, int S = 1>
__device__ __forceinline__ bool sweep_chunk(const PairDesc& P, const LevelDesc& L, int2 grp, int k, int nch,
                                            const float* cst, int rs, bool dense, float sg, float rc, float rc2,
                                            const FeatConst& fc, float4* stage, unsigned char* scratch, int lane,
                                            Moments& mo, float p[3], bool& act, unsigned& npairs, unsigned& ncand,
                                            int chunk_min = 0, unsigned* nch_next = nullptr, int chunk_len = 0,
                                            int group = 0)
{
    const float* Ahi = cst;
    const float* Alo = cst + 9;
    const float* bhi = cst + 18;
    const float* blo = cst + 21;
    const float* chi = cst + 24;
    const float* clo = cst + 27;
    // this lane's query: lane % (32 / S) of the group (its S lanes share its candidates)
    const int ql = lane & (32 / S - 1);
    act = ql < grp.y;
    const int qi = grp.x + (act ? ql : 0);
    const float4* qrec = P.xrec + (size_t)qi * rs;
    const float4 xq4 = qrec[0];
    const float xq[3] = {xq4.x, xq4.y, xq4.z};
    float xh[3], xl[3];
    transform_df(xq, Ahi, Alo, bhi, blo, xh, xl);

    Stream sm;
    const int total = stream_setup(L, P.m, dense, act, xh, rc, lane, sm) ? sm.total : 0;
    if (nch_next != nullptr && k == 0 && lane == 0)   // the group's items in the next sweep (one even if empty)
        nch_next[group] = total == 0 ? 1u : (unsigned)min(kMaxChunks, (total + chunk_len - 1) / chunk_len);
    if (total == 0) return false;
    if (chunk_min > 0) {   // cut at run time: no chunk shorter than chunk_min
        nch = min(nch, (total + chunk_min - 1) / chunk_min);
        if (k >= nch) return false;
    }
    const int clo_ = (int)(((long long)total * k) / nch);
    const int chi_ = (int)(((long long)total * (k + 1)) / nch);

    typename Feat::Q qf;
    Feat::load_query(qf, qrec, fc, scratch, lane);
    mo = Moments{0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    stream_walk(L, P.m, dense, sm, clo_, chi_, rs, stage, lane, [&](const float4* sb, int cnt) {
        eval_batch<Feat, S>(sb, cnt, rs, qf, xh, xl, act, dense, sg, rc2, fc, mo, npairs, lane);
        ncand += (act && lane < 32 / S) ? (unsigned)cnt : 0u;   // (query, candidate) tests
    });
    p[0] = (xh[0] - chi[0]) + (xl[0] - clo[0]);
    p[1] = (xh[1] - chi[1]) + (xl[1] - clo[1]);
    p[2] = (xh[2] - chi[2]) + (xl[2] - clo[2]);
    return true;
}

// One work item of a sweep from the level's item table.
template <class Feat, int S = 1>
__device__ __forceinline__ bool sweep_item(const PairDesc& P, const LevelDesc& L, int item, const float* cst, int rs,
                                           bool dense, float sg, float rc, float rc2, const FeatConst& fc,
                                           float4* stage, unsigned char* scratch, int lane, Moments& mo, float p[3],
                                           bool& act, unsigned& npairs, unsigned& ncand, unsigned* nch_next = nullptr,
                                           int chunk_len = 0)
{
    const int4 w = L.items[item];
    return sweep_chunk<Feat, S>(P, L, make_int2(w.x, w.y), w.z & 0xffff, w.z >> 16, cst, rs, dense, sg, rc, rc2, fc,
                                stage, scratch, lane, mo, p, act, npairs, ncand, L.chunk_min, nch_next, chunk_len,
                                w.w);
}

// The 43 linear statistics of one query's moments about the lever centre
// (indices of StatIndex), passed to f(index, value).
template <class F>
__device__ __forceinline__ void for_each_stat(const Moments& mo, const float p[3], F&& f)
{
    const float p0 = p[0], p1 = p[1], p2 = p[2];
    const float Q[3][3] = {{mo.Qxx, mo.Qxy, mo.Qxz}, {mo.Qxy, mo.Qyy, mo.Qyz}, {mo.Qxz, mo.Qyz, mo.Qzz}};
    float PQ[3][3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        PQ[0][c] = -p2 * Q[1][c] + p1 * Q[2][c];
        PQ[1][c] = p2 * Q[0][c] - p0 * Q[2][c];
        PQ[2][c] = -p1 * Q[0][c] + p0 * Q[1][c];
    }
    f(ST_W, mo.W);
    f(ST_E + 0, mo.E0); f(ST_E + 1, mo.E1); f(ST_E + 2, mo.E2);
    f(ST_Q + 0, mo.Qxx); f(ST_Q + 1, mo.Qyy); f(ST_Q + 2, mo.Qzz);
    f(ST_Q + 3, mo.Qxy); f(ST_Q + 4, mo.Qxz); f(ST_Q + 5, mo.Qyz);
#pragma unroll
    for (int rr = 0; rr < 3; ++rr)
#pragma unroll
        for (int c = 0; c < 3; ++c) f(ST_PQ + 3 * rr + c, PQ[rr][c]);
    // [p]x Q [p]x, symmetric: (0,0) (1,1) (2,2) (0,1) (0,2) (1,2)
    f(ST_PQP + 0, PQ[0][1] * p2 - PQ[0][2] * p1);
    f(ST_PQP + 1, -PQ[1][0] * p2 + PQ[1][2] * p0);
    f(ST_PQP + 2, PQ[2][0] * p1 - PQ[2][1] * p0);
    f(ST_PQP + 3, -PQ[0][0] * p2 + PQ[0][2] * p0);
    f(ST_PQP + 4, PQ[0][0] * p1 - PQ[0][1] * p0);
    f(ST_PQP + 5, PQ[1][0] * p1 - PQ[1][1] * p0);
    const float Wp0 = mo.W * p0, Wp1 = mo.W * p1, Wp2 = mo.W * p2;
    f(ST_WP + 0, Wp0); f(ST_WP + 1, Wp1); f(ST_WP + 2, Wp2);
    f(ST_WPP + 0, Wp0 * p0); f(ST_WPP + 1, Wp1 * p1); f(ST_WPP + 2, Wp2 * p2);
    f(ST_WPP + 3, Wp0 * p1); f(ST_WPP + 4, Wp0 * p2); f(ST_WPP + 5, Wp1 * p2);
    const float Ev[3] = {mo.E0, mo.E1, mo.E2};
#pragma unroll
    for (int rr = 0; rr < 3; ++rr)
#pragma unroll
        for (int c = 0; c < 3; ++c) f(ST_EP + 3 * rr + c, Ev[rr] * p[c]);
}

// ---- the 43 statistics, summed over a warp after every work item ------------
// The lanes' statistics of one item (48 slots, 43 used) are summed over the
// warp in a fixed butterfly: each step keeps half of a lane's values and adds
// the partner lane's copy of the same half.  Lane l ends with the sums of two
// statistics whose indices depend on l only, so it keeps running sums of
// those two across its work items (no per-lane table of 43 in shared memory).
constexpr int kStatPad = 48;

template <int H>
__device__ __forceinline__ void stat_butterfly(float (&v)[kStatPad], int lane, int off)
{
    const bool up = (lane & off) != 0;
#pragma unroll
    for (int j = 0; j < H; ++j) {
        const float keep = up ? v[j + H] : v[j];
        const float send = up ? v[j] : v[j + H];
        v[j] = keep + __shfl_xor_sync(kFull, send, off);
    }
}

struct StatAcc {
    float s0, s1;   // running sums of statistics i0, i1 (-1: none)
    int i0, i1;
};

__device__ __forceinline__ void stat_acc_init(StatAcc& a, int lane)
{
    // halves kept at the butterfly steps over bits 4..1: 24, 12, 6, 3 slots;
    // the last step splits the remaining 3 (padded to 4) over bit 0
    const int base = ((lane >> 4) & 1) * 24 + ((lane >> 3) & 1) * 12 + ((lane >> 2) & 1) * 6 + ((lane >> 1) & 1) * 3;
    const bool up = (lane & 1) != 0;
    a.i0 = base + (up ? 2 : 0);
    a.i1 = up ? -1 : base + 1;
    if (a.i0 >= kStatN) a.i0 = -1;
    if (a.i1 >= kStatN) a.i1 = -1;
    a.s0 = 0.0f;
    a.s1 = 0.0f;
}

// One work item's statistics summed over the warp (zero for an inactive
// lane): lane l gets the sums of the two statistics (i0, i1) that
// stat_acc_init gives it.  Warp-uniform.
__device__ __forceinline__ void stat_item_sums(const Moments& mo, const float p[3], bool act, int lane, float& s0,
                                               float& s1)
{
    float v[kStatPad];
#pragma unroll
    for (int s = 0; s < kStatPad; ++s) v[s] = 0.0f;
    if (act) for_each_stat(mo, p, [&](int s, float x) { v[s] = x; });
    stat_butterfly<24>(v, lane, 16);
    stat_butterfly<12>(v, lane, 8);
    stat_butterfly<6>(v, lane, 4);
    stat_butterfly<3>(v, lane, 2);
    const bool up = (lane & 1) != 0;
    const float a0 = up ? v[2] : v[0];
    const float a1 = up ? 0.0f : v[1];
    const float b0 = up ? v[0] : v[2];
    const float b1 = up ? v[1] : 0.0f;
    s0 = a0 + __shfl_xor_sync(kFull, b0, 1);
    s1 = a1 + __shfl_xor_sync(kFull, b1, 1);
}

// Adds one work item's statistics to the lane's running sums.  Warp-uniform.
__device__ __forceinline__ void stat_acc_add(StatAcc& a, const Moments& mo, const float p[3], bool act, int lane)
{
    float s0, s1;
    stat_item_sums(mo, p, act, lane, s0, s1);
    a.s0 += s0;
    a.s1 += s1;
}

// One work item's statistics into its row of a batch's work-queue table
// (kRowFloats floats: the 43 statistics, then the item's pair and test
// counts as 32-bit integers).  Every statistic of the row is written (zero
// for an empty item), so rows left by an earlier sweep are never read.
// idx: the lane's statistic indices (stat_acc_init).  Warp-uniform.
__device__ __forceinline__ void stat_row_write(float* row, const StatAcc& idx, const Moments& mo, const float p[3],
                                               bool act, unsigned np, unsigned nc, int lane)
{
    float s0, s1;
    stat_item_sums(mo, p, act, lane, s0, s1);
    if (idx.i0 >= 0) row[idx.i0] = s0;
    if (idx.i1 >= 0) row[idx.i1] = s1;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        np += __shfl_xor_sync(kFull, np, o);
        nc += __shfl_xor_sync(kFull, nc, o);
    }
    if (lane == 0) {
        row[kStatN] = __uint_as_float(np);
        row[kStatN + 1] = __uint_as_float(nc);
    }
}

// End of a sweep block's work: the warps' running sums added over the block's
// warps in double-float and written as the block's partials, and the group
// reduction: the last block of each group of kGroupBlocks blocks to arrive
// sums the group's partials in block order (deterministic; nothing waits)
// and resets the group's arrival counter for the next sweep.
// block / nblocks: this block's index and the number of sweep blocks.
__device__ __forceinline__ void sweep_epilogue(const StatAcc& acc, unsigned npairs, unsigned ncand,
                                               const SweepArgs& a, int block, int nblocks)
{
    __shared__ float red[kSweepWarps][kStatPad];
    __shared__ unsigned long long redc[kSweepWarps][2];
    __shared__ int is_last;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (acc.i0 >= 0) red[warp][acc.i0] = acc.s0;
    if (acc.i1 >= 0) red[warp][acc.i1] = acc.s1;
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
            two_sum(hi, red[w][threadIdx.x], s, e);
            e = __fadd_rn(e, lo);
            hi = __fadd_rn(s, e);
            lo = __fsub_rn(e, __fsub_rn(hi, s));
        }
        a.part_stats[(size_t)threadIdx.x * a.part_cap + block] = make_float2(hi, lo);
    } else if (threadIdx.x == kStatN) {
        unsigned long long t0 = 0, t1 = 0;
        for (int w = 0; w < kSweepWarps; ++w) {
            t0 += redc[w][0];
            t1 += redc[w][1];
        }
        a.part_cnt[block] = t0;
        a.part_cnt[(size_t)a.part_cap + block] = t1;
    }

    if (a.grp_arrivals == nullptr) return;   // batch: the finalize sums the block partials per pair
    const int grp = block / kGroupBlocks;
    const int first = grp * kGroupBlocks;
    const int members = min(kGroupBlocks, nblocks - first);
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

}  // namespace
}  // namespace cvo
