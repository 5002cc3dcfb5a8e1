// Setup kernels, run once per cloud pair: bounding boxes, the uniform grid of
// Z (a stable counting sort by cell key), the Hilbert order of X and its query
// groups.  The paper notes that the double sum is sparse (Sec. III-B); the
// grid is how the sweep visits only the pairs near each query.
#include <cmath>
#include <cstdint>
#include <cstring>

#include "cvo_internal.cuh"

namespace cvo {

namespace {

__device__ __forceinline__ unsigned orderable(float f)
{
    const unsigned u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

// Kernel bodies take their block index and block count (bx, nbx) or their
// element index, so that the single-pair kernels and the batched ones (one
// launch for many pairs, blockIdx.y the pair) run the same code.

__device__ __forceinline__ void bbox_body(const float* __restrict__ xyz, int n, unsigned* out6, int* bad, int bx,
                                          int nbx)
{
    float mn[3] = {3.0e38f, 3.0e38f, 3.0e38f}, mx[3] = {-3.0e38f, -3.0e38f, -3.0e38f};
    int nonfinite = 0;
    for (int i = bx * blockDim.x + threadIdx.x; i < n; i += nbx * blockDim.x) {
        for (int a = 0; a < 3; ++a) {
            const float v = xyz[3 * (size_t)i + a];
            if (!isfinite(v)) {
                nonfinite = 1;
                continue;
            }
            mn[a] = fminf(mn[a], v);
            mx[a] = fmaxf(mx[a], v);
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        for (int a = 0; a < 3; ++a) {
            mn[a] = fminf(mn[a], __shfl_xor_sync(0xffffffffu, mn[a], o));
            mx[a] = fmaxf(mx[a], __shfl_xor_sync(0xffffffffu, mx[a], o));
        }
        nonfinite |= __shfl_xor_sync(0xffffffffu, nonfinite, o);
    }
    if ((threadIdx.x & 31) == 0) {
        for (int a = 0; a < 3; ++a) {
            atomicMin(out6 + a, orderable(mn[a]));
            atomicMax(out6 + 3 + a, orderable(mx[a]));
        }
        if (nonfinite) atomicOr(bad, 1);
    }
}

__global__ void k_bbox(const float* __restrict__ xyz, int n, unsigned* out6, int* bad)
{
    bbox_body(xyz, n, out6, bad, blockIdx.x, gridDim.x);
}

// a word of two bfloat16 values, or one FP32 value: some exponent all ones
__device__ __forceinline__ bool word_nonfinite(unsigned w, int bf16)
{
    return (w & 0x7f800000u) == 0x7f800000u || (bf16 && (w & 0x7f80u) == 0x7f80u);
}

__device__ __forceinline__ void check_feat_body(const void* __restrict__ feat, long long count, int bf16, int* bad,
                                                int bx, int nbx)
{
    int nonfinite = 0;
    const long long t0 = bx * (long long)blockDim.x + threadIdx.x, stride = (long long)nbx * blockDim.x;
    long long done = 0;   // values checked 16 bytes at a time
    if ((reinterpret_cast<uintptr_t>(feat) & 15) == 0) {
        const int per = bf16 ? 8 : 4;
        const long long nv = count / per;
        const uint4* v4 = reinterpret_cast<const uint4*>(feat);
        for (long long i = t0; i < nv; i += stride) {
            const uint4 u = v4[i];
            if (word_nonfinite(u.x, bf16) || word_nonfinite(u.y, bf16) || word_nonfinite(u.z, bf16) ||
                word_nonfinite(u.w, bf16))
                nonfinite = 1;
        }
        done = nv * per;
    }
    for (long long i = done + t0; i < count; i += stride) {
        float v;
        if (bf16) v = __uint_as_float(((unsigned)((const unsigned short*)feat)[i]) << 16);
        else v = ((const float*)feat)[i];
        if (!isfinite(v)) nonfinite = 1;
    }
    if (__any_sync(0xffffffffu, nonfinite) && (threadIdx.x & 31) == 0) atomicOr(bad, 1);
}

__global__ void k_check_feat(const void* __restrict__ feat, long long count, int bf16, int* bad)
{
    check_feat_body(feat, count, bf16, bad, blockIdx.x, gridDim.x);
}

__device__ __forceinline__ int cell_of(float v, float o, float inv_h, int n)
{
    int c = (int)floorf((v - o) * inv_h);
    return min(max(c, 0), n - 1);
}

__device__ __forceinline__ void cell_keys_body(const float* __restrict__ xyz, int n, float ox, float oy, float oz,
                                               float inv_h, float inv_hx, int nx, int ny, int nz, unsigned* keys,
                                               unsigned* vals, int j)
{
    if (j >= n) return;
    const int cx = cell_of(xyz[3 * (size_t)j + 0], ox, inv_hx, nx);
    const int cy = cell_of(xyz[3 * (size_t)j + 1], oy, inv_h, ny);
    const int cz = cell_of(xyz[3 * (size_t)j + 2], oz, inv_h, nz);
    keys[j] = (unsigned)((cz * ny + cy) * nx + cx);
    vals[j] = (unsigned)j;
}

__global__ void k_cell_keys(const float* __restrict__ xyz, int n, float ox, float oy, float oz, float inv_h,
                            float inv_hx, int nx, int ny, int nz, unsigned* keys, unsigned* vals)
{
    cell_keys_body(xyz, n, ox, oy, oz, inv_h, inv_hx, nx, ny, nz, keys, vals, blockIdx.x * blockDim.x + threadIdx.x);
}

__device__ __forceinline__ unsigned spread10(unsigned v)
{
    v &= 0x3ffu;
    v = (v | (v << 16)) & 0x030000ffu;
    v = (v | (v << 8)) & 0x0300f00fu;
    v = (v | (v << 4)) & 0x030c30c3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}

// The 30-bit index along the 3-D Hilbert curve of the cell (x, y, z) of a
// 1024^3 grid, by Skilling's transform of the coordinates to the curve's
// "transposed" index (J. Skilling, Programming the Hilbert curve, AIP Conf.
// Proc. 707, 2004): for each bit from the top, invert or exchange the lower
// bits, then Gray-encode; the index interleaves the transposed words' bits,
// x's bit b at 3b + 2.  Consecutive indices are neighbouring cells, and the
// cells of an octree cell of edge 2^k are 2^3k consecutive indices (the
// key's top bits name the octree cell, as with Morton keys).
__device__ __forceinline__ unsigned hilbert_index10(unsigned x, unsigned y, unsigned z)
{
    unsigned X[3] = {x, y, z};
    for (unsigned Q = 1u << 9; Q > 1u; Q >>= 1) {
        const unsigned P = Q - 1u;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            if (X[i] & Q) {
                X[0] ^= P;   // invert
            } else {         // exchange
                const unsigned t = (X[0] ^ X[i]) & P;
                X[0] ^= t;
                X[i] ^= t;
            }
        }
    }
    X[1] ^= X[0];   // Gray encode
    X[2] ^= X[1];
    unsigned t = 0u;
    for (unsigned Q = 1u << 9; Q > 1u; Q >>= 1)
        if (X[2] & Q) t ^= Q - 1u;
#pragma unroll
    for (int i = 0; i < 3; ++i) X[i] ^= t;
    return (spread10(X[0]) << 2) | (spread10(X[1]) << 1) | spread10(X[2]);
}

// The queries' order: the Hilbert index of each point's cell (edge 1 /
// inv_cell from the origin o, 1024 cells a side), with the point indices as
// values.  Chunks of 32 consecutive queries in Hilbert order are more compact
// than in Hilbert order, which has jumps across octree cells (on the cube
// scenes about 5 % fewer candidates streamed and evaluated).
__device__ __forceinline__ void hilbert_keys_body(const float* __restrict__ xyz, int n, float ox, float oy, float oz,
                                                  float inv_cell, unsigned* keys, unsigned* vals, int j)
{
    if (j >= n) return;
    unsigned q[3];
    const float o[3] = {ox, oy, oz};
    for (int a = 0; a < 3; ++a) {
        int c = (int)floorf((xyz[3 * (size_t)j + a] - o[a]) * inv_cell);
        q[a] = (unsigned)min(max(c, 0), 1023);
    }
    keys[j] = hilbert_index10(q[0], q[1], q[2]);
    vals[j] = (unsigned)j;
}

__global__ void k_hilbert_keys(const float* __restrict__ xyz, int n, float ox, float oy, float oz, float inv_cell,
                              unsigned* keys, unsigned* vals)
{
    hilbert_keys_body(xyz, n, ox, oy, oz, inv_cell, keys, vals, blockIdx.x * blockDim.x + threadIdx.x);
}

// ---- stable LSD radix sort, 8-bit digits ------------------------------------

constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kSortTile = 1024;                  // keys per block (small tiles: the sorts here are short and latency bound)
constexpr int kSortSub = kSortTile / kSortWarps; // keys per warp

// tile bx of nb: its digit counts into hist[digit * nb + bx]
__device__ __forceinline__ void radix_hist_body(const unsigned* __restrict__ keys, int n, int shift, unsigned* hist,
                                                int nb, int bx)
{
    __shared__ unsigned cnt[256];
    cnt[threadIdx.x] = 0;
    __syncthreads();
    const int base = bx * kSortTile;
    for (int k = threadIdx.x; k < kSortTile; k += kSortThreads) {
        const int i = base + k;
        if (i < n) atomicAdd(&cnt[(keys[i] >> shift) & 255u], 1u);
    }
    __syncthreads();
    hist[threadIdx.x * nb + bx] = cnt[threadIdx.x];
}

__global__ void k_radix_hist(const unsigned* __restrict__ keys, int n, int shift, unsigned* hist, int nb)
{
    radix_hist_body(keys, n, shift, hist, nb, blockIdx.x);
}

// tile bx of nb: its keys scattered stably to their offsets (offs: the
// exclusive scan of hist)
__device__ __forceinline__ void radix_scatter_body(const unsigned* __restrict__ keys, const unsigned* __restrict__ vals,
                                                   int n, int shift, const unsigned* __restrict__ offs, int nb,
                                                   unsigned* keys_out, unsigned* vals_out, int bx)
{
    __shared__ unsigned wcnt[kSortWarps][256];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int d = threadIdx.x; d < kSortWarps * 256; d += kSortThreads) (&wcnt[0][0])[d] = 0;
    __syncthreads();
    const int base = bx * kSortTile + warp * kSortSub;
    for (int r = 0; r < kSortSub; r += 32) {
        const int i = base + r + lane;
        if (i < n) atomicAdd(&wcnt[warp][(keys[i] >> shift) & 255u], 1u);
    }
    __syncthreads();
    {   // per digit: block offset plus the counts of the earlier warps
        const int d = threadIdx.x;
        unsigned run = offs[d * nb + bx];
        for (int w = 0; w < kSortWarps; ++w) {
            const unsigned c = wcnt[w][d];
            wcnt[w][d] = run;
            run += c;
        }
    }
    __syncthreads();
    const unsigned lt = (1u << lane) - 1u;
    for (int r = 0; r < kSortSub; r += 32) {
        const int i = base + r + lane;
        const bool ok = i < n;
        const unsigned valid = __ballot_sync(0xffffffffu, ok);
        if (ok) {
            const unsigned k = keys[i];
            const unsigned d = (k >> shift) & 255u;
            const unsigned peers = __match_any_sync(valid, d);
            const unsigned pos = wcnt[warp][d] + __popc(peers & lt);
            keys_out[pos] = k;
            vals_out[pos] = vals[i];
            __syncwarp(valid);
            if ((peers & lt) == 0) wcnt[warp][d] += __popc(peers);
        }
        __syncwarp();
    }
}

__global__ void k_radix_scatter(const unsigned* __restrict__ keys, const unsigned* __restrict__ vals, int n,
                                int shift, const unsigned* __restrict__ offs, int nb, unsigned* keys_out,
                                unsigned* vals_out)
{
    radix_scatter_body(keys, vals, n, shift, offs, nb, keys_out, vals_out, blockIdx.x);
}

// Short arrays (n <= kSmallSort): the whole LSD radix sort in one block, in
// shared memory, one launch instead of three per digit.  Each warp owns a
// contiguous run of n / 32 keys; per digit pass: the warps' digit counts, the
// digit offsets (totals of smaller digits plus the counts of earlier warps),
// then a stable scatter (warps in order, lanes in order within a warp).
constexpr int kSmallSort = 8192;
constexpr int kSmallThreads = 1024;
constexpr int kSmallWarps = kSmallThreads / 32;
constexpr size_t kSmallSmem = (size_t)4 * kSmallSort * sizeof(unsigned) + (size_t)kSmallWarps * 256 * sizeof(unsigned);

__global__ void __launch_bounds__(kSmallThreads) k_sort_small(unsigned* keys, unsigned* vals, int n, int nbits)
{
    extern __shared__ unsigned sm[];
    unsigned* kb[2] = {sm, sm + kSmallSort};
    unsigned* vb[2] = {sm + 2 * kSmallSort, sm + 3 * kSmallSort};
    unsigned* wcnt = sm + 4 * kSmallSort;   // [kSmallWarps][256]
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < n; i += kSmallThreads) {
        kb[0][i] = keys[i];
        vb[0][i] = vals[i];
    }
    const int per = (n + kSmallWarps - 1) / kSmallWarps;
    const int w0 = min(n, warp * per), w1 = min(n, w0 + per);
    const unsigned lt = (1u << lane) - 1u;
    int cur = 0;
    for (int shift = 0; shift < nbits; shift += 8) {
        for (int d = threadIdx.x; d < kSmallWarps * 256; d += kSmallThreads) wcnt[d] = 0u;
        __syncthreads();
        const unsigned* kin = kb[cur];
        for (int i = w0 + lane; i < w1; i += 32) atomicAdd(&wcnt[warp * 256 + ((kin[i] >> shift) & 255u)], 1u);
        __syncthreads();
        if (threadIdx.x < 256) {   // per digit: running offsets over the warps, then over the digits
            const int d = threadIdx.x;
            unsigned run = 0;
            for (int w = 0; w < kSmallWarps; ++w) {
                const unsigned c = wcnt[w * 256 + d];
                wcnt[w * 256 + d] = run;
                run += c;
            }
            // exclusive scan of the digit totals across the 256 threads (8 warps)
            unsigned incl = run;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned t = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += t;
            }
            __shared__ unsigned wsum[8];
            if (lane == 31) wsum[warp] = incl;
            asm volatile("bar.sync 1, 256;" ::: "memory");
            unsigned before = incl - run;
            for (int w = 0; w < warp; ++w) before += wsum[w];
            for (int w = 0; w < kSmallWarps; ++w) wcnt[w * 256 + d] += before;
        }
        __syncthreads();
        unsigned* kout = kb[cur ^ 1];
        unsigned* vout = vb[cur ^ 1];
        const unsigned* vin = vb[cur];
        for (int r = w0; r < w1; r += 32) {
            const int i = r + lane;
            const bool ok = i < w1;
            const unsigned valid = __ballot_sync(0xffffffffu, ok);
            if (ok) {
                const unsigned k = kin[i];
                const unsigned d = (k >> shift) & 255u;
                const unsigned peers = __match_any_sync(valid, d);
                const unsigned pos = wcnt[warp * 256 + d] + __popc(peers & lt);
                kout[pos] = k;
                vout[pos] = vin[i];
                __syncwarp(valid);
                if ((peers & lt) == 0) wcnt[warp * 256 + d] += __popc(peers);
            }
            __syncwarp();
        }
        __syncthreads();
        cur ^= 1;
    }
    for (int i = threadIdx.x; i < n; i += kSmallThreads) {
        keys[i] = kb[cur][i];
        vals[i] = vb[cur][i];
    }
}

// single-block (1024 threads) exclusive scan; total (optional) receives the sum
__device__ __forceinline__ void scan_body(const unsigned* __restrict__ in, unsigned* out, int n, unsigned* total)
{
    __shared__ unsigned sums[1024];
    const int t = threadIdx.x;
    const int chunk = (n + 1023) / 1024;
    const int lo = min(n, t * chunk), hi = min(n, lo + chunk);
    unsigned s = 0;
    for (int i = lo; i < hi; ++i) s += in[i];
    sums[t] = s;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
        const unsigned v = t >= o ? sums[t - o] : 0u;
        __syncthreads();
        sums[t] += v;
        __syncthreads();
    }
    unsigned run = sums[t] - s;
    for (int i = lo; i < hi; ++i) {
        const unsigned v = in[i];
        out[i] = run;
        run += v;
    }
    if (t == 1023 && total) *total = sums[1023];
}

__global__ void k_scan_single(const unsigned* __restrict__ in, unsigned* out, int n, unsigned* total)
{
    scan_body(in, out, n, total);
}

__device__ __forceinline__ void cell_start_body(const unsigned* __restrict__ keys, int n, int ncells, int* cell_start,
                                                long long c)
{
    if (c > ncells) return;
    int lo = 0, hi = n;   // first index with key >= c
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if ((long long)keys[mid] < c) lo = mid + 1;
        else hi = mid;
    }
    cell_start[c] = lo;
}

__global__ void k_cell_start(const unsigned* __restrict__ keys, int n, int ncells, int* cell_start)
{
    cell_start_body(keys, n, ncells, cell_start, blockIdx.x * (long long)blockDim.x + threadIdx.x);
}

__device__ __forceinline__ unsigned short f32_to_bf16_bits(float f)
{
    const unsigned u = __float_as_uint(f);
    return (unsigned short)((u + 0x7fffu + ((u >> 16) & 1u)) >> 16);
}

__device__ __forceinline__ void pack_body(const float* __restrict__ xyz, const void* __restrict__ feat, int feat_bf16,
                                          int D, const unsigned* __restrict__ order, int n, float4* rec, int rs,
                                          int rec_bf16, int s)
{
    if (s >= n) return;
    const int j = order ? (int)order[s] : s;
    float4* r = rec + (size_t)s * rs;
    // w carries the point's index in the caller's order (for per-point outputs)
    r[0] = make_float4(xyz[3 * (size_t)j], xyz[3 * (size_t)j + 1], xyz[3 * (size_t)j + 2], __int_as_float(j));
    if (rs <= 1) return;
    // the feature part of the record, 16 bytes at a time (zero past D)
    uint4* dst = reinterpret_cast<uint4*>(r + 1);
    const unsigned short* f16 = (const unsigned short*)feat + (size_t)j * D;
    const float* f32 = (const float*)feat + (size_t)j * D;
    if (rec_bf16) {
        auto half = [&](int k) -> unsigned {
            if (k >= D) return 0u;
            return feat_bf16 ? (unsigned)f16[k] : (unsigned)f32_to_bf16_bits(f32[k]);
        };
        // an even D (and a 4-byte aligned array) keeps every row's bfloat16
        // pairs 4-byte aligned
        const bool words = feat_bf16 && (D & 1) == 0 && (reinterpret_cast<uintptr_t>(feat) & 3) == 0;
        for (int q = 0; q < rs - 1; ++q) {
            unsigned v[4];
            for (int t = 0; t < 4; ++t) {
                const int k = 8 * q + 2 * t;
                v[t] = (words && k + 1 < D) ? reinterpret_cast<const unsigned*>(f16)[k >> 1]
                                            : (half(k) | (half(k + 1) << 16));
            }
            dst[q] = make_uint4(v[0], v[1], v[2], v[3]);
        }
    } else {
        auto val = [&](int k) -> float {
            if (k >= D) return 0.0f;
            return feat_bf16 ? __uint_as_float(((unsigned)f16[k]) << 16) : f32[k];
        };
        for (int q = 0; q < rs - 1; ++q)
            reinterpret_cast<float4*>(dst)[q] = make_float4(val(4 * q), val(4 * q + 1), val(4 * q + 2), val(4 * q + 3));
    }
}

__global__ void k_pack(const float* __restrict__ xyz, const void* __restrict__ feat, int feat_bf16, int D,
                       const unsigned* __restrict__ order, int n, float4* rec, int rs, int rec_bf16)
{
    pack_body(xyz, feat, feat_bf16, D, order, n, rec, rs, rec_bf16, blockIdx.x * blockDim.x + threadIdx.x);
}

__device__ __forceinline__ int lower_bound_u32(const unsigned* a, int n, unsigned long long v)
{
    int lo = 0, hi = n;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if ((unsigned long long)a[mid] < v) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// groups of up to gsize consecutive queries of one octree super-cell
__device__ __forceinline__ void group_flags_body(const unsigned* __restrict__ hkeys, int n, int shift, int gsize,
                                                 unsigned* flags, int i)
{
    if (i >= n) return;
    const unsigned long long seg = (unsigned long long)(hkeys[i] >> shift);
    const int start = lower_bound_u32(hkeys, n, seg << shift);
    flags[i] = ((i - start) % gsize == 0) ? 1u : 0u;
}

__global__ void k_group_flags(const unsigned* __restrict__ hkeys, int n, int shift, int gsize, unsigned* flags)
{
    group_flags_body(hkeys, n, shift, gsize, flags, blockIdx.x * blockDim.x + threadIdx.x);
}

__device__ __forceinline__ void group_write_body(const unsigned* __restrict__ hkeys,
                                                 const unsigned* __restrict__ flags,
                                                 const unsigned* __restrict__ gidx, int n, int shift, int gsize,
                                                 int2* groups, int i)
{
    if (i >= n || !flags[i]) return;
    const unsigned long long seg = (unsigned long long)(hkeys[i] >> shift);
    const int end = lower_bound_u32(hkeys, n, (seg + 1ull) << shift);
    groups[gidx[i]] = make_int2(i, min(gsize, end - i));
}

__global__ void k_group_write(const unsigned* __restrict__ hkeys, const unsigned* __restrict__ flags,
                              const unsigned* __restrict__ gidx, int n, int shift, int gsize, int2* groups)
{
    group_write_body(hkeys, flags, gidx, n, shift, gsize, groups, blockIdx.x * blockDim.x + threadIdx.x);
}

// Deterministic sum of n floats: per-thread double-float partials in a fixed
// stride, then a fixed-order block reduction.  One block.
__global__ void k_sum_f32(const float* __restrict__ v, int n, double* out)
{
    __shared__ float sh[1024], sl[1024];
    float hi = 0.0f, lo = 0.0f;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const float s = __fadd_rn(hi, v[i]);
        const float bb = __fsub_rn(s, hi);
        const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(v[i], bb));
        const float t = __fadd_rn(lo, e);
        hi = __fadd_rn(s, t);
        lo = __fsub_rn(t, __fsub_rn(hi, s));
    }
    sh[threadIdx.x] = hi;
    sl[threadIdx.x] = lo;
    __syncthreads();
    if (threadIdx.x == 0) {
        double acc = 0.0;
        for (int t = 0; t < (int)blockDim.x; ++t) acc += (double)sh[t] + (double)sl[t];
        *out = acc;
    }
}

// Z's centroid, mean squared distance from it and largest such distance,
// for the metric and the trust region of the registration step, in two
// passes over many blocks.  Sums are kept in 64-bit fixed point (integer
// additions do not depend on their order, so the result is the same run to
// run whatever the blocks' timing): coordinates in units of 2^-32 m,
// squared distances in units of 2^-24 m^2.  Each block adds its points' sum
// (a warp butterfly, then the warps in order) into the output with one
// atomic add per word; the largest squared distance by an atomic max on its
// (non-negative) FP32 bit pattern.  out (zeroed before the launch): [0..2]
// coordinate sums, [3] squared-distance sum (long long), then word 8 the
// largest squared distance's bits.
constexpr int kZStatsThreads = 256;
constexpr float kCoordScale = 4294967296.0f;   // 2^32
constexpr float kSqScale = 16777216.0f;        // 2^24

__device__ __forceinline__ long long warp_sum_ll(long long v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ void zsum_body(const float* __restrict__ xyz, int n, long long* out, int bx, int nbx)
{
    __shared__ long long part[kZStatsThreads / 32][3];
    long long s[3] = {0, 0, 0};
    for (int i = bx * kZStatsThreads + threadIdx.x; i < n; i += nbx * kZStatsThreads)
        for (int a = 0; a < 3; ++a) s[a] += __float2ll_rn(xyz[3 * (size_t)i + a] * kCoordScale);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int a = 0; a < 3; ++a) {
        const long long w = warp_sum_ll(s[a]);
        if (lane == 0) part[warp][a] = w;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        long long t = 0;
        for (int k = 0; k < kZStatsThreads / 32; ++k) t += part[k][threadIdx.x];
        atomicAdd(reinterpret_cast<unsigned long long*>(out + threadIdx.x), (unsigned long long)t);
    }
}

__global__ void __launch_bounds__(kZStatsThreads) k_zsum(const float* __restrict__ xyz, int n, long long* out)
{
    zsum_body(xyz, n, out, blockIdx.x, gridDim.x);
}

__device__ __forceinline__ void zspread_body(const float* __restrict__ xyz, int n, long long* out, int bx, int nbx)
{
    __shared__ long long part[kZStatsThreads / 32];
    __shared__ float mx_part[kZStatsThreads / 32];
    __shared__ float m_hl[6];
    if (threadIdx.x < 3) {   // the centroid as a double-float pair
        const double mean = (double)out[threadIdx.x] / (double)kCoordScale / (double)n;
        m_hl[threadIdx.x] = (float)mean;
        m_hl[3 + threadIdx.x] = (float)(mean - (double)m_hl[threadIdx.x]);
    }
    __syncthreads();
    const float mhi[3] = {m_hl[0], m_hl[1], m_hl[2]}, mlo[3] = {m_hl[3], m_hl[4], m_hl[5]};
    long long s = 0;
    float mx = 0.0f;
    for (int i = bx * kZStatsThreads + threadIdx.x; i < n; i += nbx * kZStatsThreads) {
        float q = 0.0f;
        for (int a = 0; a < 3; ++a) {
            const float e = __fsub_rn(__fsub_rn(xyz[3 * (size_t)i + a], mhi[a]), mlo[a]);
            q = fmaf(e, e, q);
        }
        s += __float2ll_rn(q * kSqScale);
        mx = fmaxf(mx, q);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    s = warp_sum_ll(s);
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) {
        part[warp] = s;
        mx_part[warp] = mx;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        long long t = 0;
        float m = 0.0f;
        for (int k = 0; k < kZStatsThreads / 32; ++k) {
            t += part[k];
            m = fmaxf(m, mx_part[k]);
        }
        atomicAdd(reinterpret_cast<unsigned long long*>(out + 3), (unsigned long long)t);
        atomicMax(reinterpret_cast<unsigned*>(out + 4), __float_as_uint(m));
    }
}

__global__ void __launch_bounds__(kZStatsThreads) k_zspread(const float* __restrict__ xyz, int n, long long* out)
{
    zspread_body(xyz, n, out, blockIdx.x, gridDim.x);
}

// ---- batched kernels: blockIdx.y is the job ---------------------------------

__global__ void k_boxes_init_b(JobList<BoxJob> J)
{
    const BoxJob& b = J.j[blockIdx.y];
    const int t = threadIdx.x;
    if (t < 6) {   // minima start at the largest orderable value, maxima at 0
        b.box_x[t] = t < 3 ? 0xffffffffu : 0u;
        b.box_z[t] = t < 3 ? 0xffffffffu : 0u;
    }
    if (t == 6) *b.bad = 0;
    if (t >= 8 && t < 13) b.zstats[t - 8] = 0;
}

__global__ void k_bbox_b(JobList<BoxJob> J)
{
    const BoxJob& b = J.j[blockIdx.y];
    if (blockIdx.z == 0) bbox_body(b.xyz_x, b.n, b.box_x, b.bad, blockIdx.x, gridDim.x);
    else bbox_body(b.xyz_z, b.m, b.box_z, b.bad, blockIdx.x, gridDim.x);
}

__global__ void k_check_feat_b(JobList<BoxJob> J)
{
    const BoxJob& b = J.j[blockIdx.y];
    if (blockIdx.z == 0) {
        if (b.nfx > 0) check_feat_body(b.feat_x, b.nfx, b.fx_bf16, b.bad, blockIdx.x, gridDim.x);
    } else if (b.nfz > 0) {
        check_feat_body(b.feat_z, b.nfz, b.fz_bf16, b.bad, blockIdx.x, gridDim.x);
    }
}

__global__ void __launch_bounds__(kZStatsThreads) k_zsum_b(JobList<BoxJob> J)
{
    const BoxJob& b = J.j[blockIdx.y];
    if (b.m > 0) zsum_body(b.xyz_z, b.m, b.zstats, blockIdx.x, gridDim.x);
}

__global__ void __launch_bounds__(kZStatsThreads) k_zspread_b(JobList<BoxJob> J)
{
    const BoxJob& b = J.j[blockIdx.y];
    if (b.m > 0) zspread_body(b.xyz_z, b.m, b.zstats, blockIdx.x, gridDim.x);
}

__global__ void k_cell_keys_b(JobList<KeyJob> J)
{
    const KeyJob& k = J.j[blockIdx.y];
    cell_keys_body(k.xyz, k.n, k.ox, k.oy, k.oz, k.inv, k.invx, k.nx, k.ny, k.nz, k.keys, k.vals,
                   blockIdx.x * blockDim.x + threadIdx.x);
}

__global__ void k_hilbert_keys_b(JobList<KeyJob> J)
{
    const KeyJob& k = J.j[blockIdx.y];
    hilbert_keys_body(k.xyz, k.n, k.ox, k.oy, k.oz, k.inv, k.keys, k.vals, blockIdx.x * blockDim.x + threadIdx.x);
}

__device__ __forceinline__ int sort_tiles(int n) { return (n + kSortTile - 1) / kSortTile; }

// parity 0: (keys, vals) -> (keys2, vals2); 1: the other way
__global__ void k_radix_hist_b(JobList<SortJob> J, int shift, int parity)
{
    const SortJob& q = J.j[blockIdx.y];
    const int nb = sort_tiles(q.n);
    if ((int)blockIdx.x >= nb) return;
    radix_hist_body(parity ? q.keys2 : q.keys, q.n, shift, q.temp, nb, blockIdx.x);
}

__global__ void k_radix_scan_b(JobList<SortJob> J)
{
    const SortJob& q = J.j[blockIdx.y];
    const int nb = sort_tiles(q.n);
    scan_body(q.temp, q.temp + 256 * nb, 256 * nb, nullptr);
}

__global__ void k_radix_scatter_b(JobList<SortJob> J, int shift, int parity)
{
    const SortJob& q = J.j[blockIdx.y];
    const int nb = sort_tiles(q.n);
    if ((int)blockIdx.x >= nb) return;
    if (parity)
        radix_scatter_body(q.keys2, q.vals2, q.n, shift, q.temp + 256 * nb, nb, q.keys, q.vals, blockIdx.x);
    else
        radix_scatter_body(q.keys, q.vals, q.n, shift, q.temp + 256 * nb, nb, q.keys2, q.vals2, blockIdx.x);
}

__global__ void k_cell_start_b(JobList<CellStartJob> J)
{
    const CellStartJob& c = J.j[blockIdx.y];
    cell_start_body(c.keys, c.n, c.ncells, c.cell_start, blockIdx.x * (long long)blockDim.x + threadIdx.x);
}

__global__ void k_pack_b(JobList<PackJob> J, int D, int rs, int rec_bf16)
{
    const PackJob& q = J.j[blockIdx.y];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    pack_body(q.xyz, q.feat, q.feat_bf16, D, q.order, q.n, q.rec, rs, rec_bf16, i);
    if (q.keys_out != nullptr && i < q.n) q.keys_out[i] = q.keys[i];
}

__global__ void k_scan_b(JobList<ScanJob> J)
{
    const ScanJob& q = J.j[blockIdx.y];
    scan_body(q.in, q.out, q.n, q.total);
}

__global__ void k_group_flags_b(JobList<GroupJob> J)
{
    const GroupJob& q = J.j[blockIdx.y];
    group_flags_body(q.hkeys, q.n, q.shift, q.gsize, q.flags, blockIdx.x * blockDim.x + threadIdx.x);
}

__global__ void k_copy_b(JobList<CopyJob> J)
{
    const CopyJob& c = J.j[blockIdx.y];
    const unsigned* src = static_cast<const unsigned*>(c.src);
    unsigned* dst = static_cast<unsigned*>(c.dst);
    for (int i = threadIdx.x; i < c.bytes / 4; i += blockDim.x) dst[i] = src[i];
}

// Job blockIdx.y copied by gridDim.x blocks, each a slice of a multiple of 16
// bytes: 16-byte loads and stores where both ends are 16-byte aligned, else
// single bytes.  Reading page-locked host memory this way runs at the
// host link's rate in one launch for many arrays (on GB300 about 210 GB/s,
// against 138 GB/s for 256 copy-engine copies of the same bytes).
__global__ void k_pull_b(JobList<PullJob> J)
{
    const PullJob& c = J.j[blockIdx.y];
    const unsigned char* src = static_cast<const unsigned char*>(c.src);
    unsigned char* dst = static_cast<unsigned char*>(c.dst);
    const long long nb = c.bytes;
    const long long per = ((nb + gridDim.x - 1) / gridDim.x + 15) & ~15ll;
    const long long lo = min(nb, per * (long long)blockIdx.x), hi = min(nb, lo + per);
    long long done = lo;
    if (((reinterpret_cast<unsigned long long>(src) | reinterpret_cast<unsigned long long>(dst)) & 15ull) == 0) {
        const long long n16 = (hi - lo) >> 4;
        const uint4* s4 = reinterpret_cast<const uint4*>(src + lo);
        uint4* d4 = reinterpret_cast<uint4*>(dst + lo);
        for (long long i = threadIdx.x; i < n16; i += blockDim.x) d4[i] = s4[i];
        done = lo + (n16 << 4);
    }
    for (long long i = done + threadIdx.x; i < hi; i += blockDim.x) dst[i] = src[i];
}

__global__ void k_group_write_b(JobList<GroupJob> J)
{
    const GroupJob& q = J.j[blockIdx.y];
    group_write_body(q.hkeys, q.flags, q.gidx, q.n, q.shift, q.gsize, q.groups,
                     blockIdx.x * blockDim.x + threadIdx.x);
}

inline int blocks_for(long long n, int t) { return (int)((n + t - 1) / t); }

}  // namespace

cudaError_t launch_zstats(const float* xyz, int n, long long* out, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    const int nb = min(blocks_for(n, 4 * kZStatsThreads), 64);
    g_launch_count.fetch_add(2, std::memory_order_relaxed);
    k_zsum<<<nb, kZStatsThreads, 0, s>>>(xyz, n, out);
    k_zspread<<<nb, kZStatsThreads, 0, s>>>(xyz, n, out);
    return cudaGetLastError();
}

void decode_zstats(const long long* raw, int n, double out5[5])
{
    for (int a = 0; a < 3; ++a) out5[a] = n > 0 ? (double)raw[a] / (double)kCoordScale / (double)n : 0.0;
    out5[3] = n > 0 ? (double)raw[3] / (double)kSqScale / (double)n : 0.0;
    unsigned bits;
    std::memcpy(&bits, raw + 4, sizeof(bits));
    float mx;
    std::memcpy(&mx, &bits, sizeof(mx));
    out5[4] = std::sqrt((double)mx);
}

cudaError_t launch_sum_f32(const float* v, int n, double* out, cudaStream_t s)
{
    g_launch_count.fetch_add(1, std::memory_order_relaxed);
    k_sum_f32<<<1, 1024, 0, s>>>(v, n, out);
    return cudaGetLastError();
}

cudaError_t launch_bbox(const float* xyz, int n, unsigned* out6, int* bad, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    const int nb = min(blocks_for(n, 256), 1024);
    g_launch_count.fetch_add(1, std::memory_order_relaxed);
    k_bbox<<<nb, 256, 0, s>>>(xyz, n, out6, bad);
    return cudaGetLastError();
}

cudaError_t launch_check_feat(const void* feat, long long count, int bf16, int* bad, cudaStream_t s)
{
    if (count <= 0) return cudaSuccess;
    const int nb = (int)min((long long)blocks_for(count, 256), 2048LL);
    g_launch_count.fetch_add(1, std::memory_order_relaxed);
    k_check_feat<<<nb, 256, 0, s>>>(feat, count, bf16, bad);
    return cudaGetLastError();
}

cudaError_t launch_cell_keys(const float* xyz, int n, float ox, float oy, float oz, float inv_h, float inv_hx, int nx,
                             int ny, int nz, unsigned* keys, unsigned* vals, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    g_launch_count.fetch_add(1, std::memory_order_relaxed);
    k_cell_keys<<<blocks_for(n, 256), 256, 0, s>>>(xyz, n, ox, oy, oz, inv_h, inv_hx, nx, ny, nz, keys, vals);
    return cudaGetLastError();
}

cudaError_t launch_hilbert_keys(const float* xyz, int n, float ox, float oy, float oz, float inv_cell,
                               unsigned* keys, unsigned* vals, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    g_launch_count.fetch_add(1, std::memory_order_relaxed);
    k_hilbert_keys<<<blocks_for(n, 256), 256, 0, s>>>(xyz, n, ox, oy, oz, inv_cell, keys, vals);
    return cudaGetLastError();
}

size_t radix_sort_temp_bytes(int n)
{
    const int nb = (n + kSortTile - 1) / kSortTile;
    return (size_t)2 * 256 * (nb > 0 ? nb : 1) * sizeof(unsigned) + 16;
}

cudaError_t radix_sort_pairs(unsigned* keys, unsigned* vals, unsigned* keys_alt, unsigned* vals_alt, int n,
                             int nbits, void* temp, int* result_in_alt, cudaStream_t s)
{
    *result_in_alt = 0;
    if (n <= 1) return cudaSuccess;
    if (n <= kSmallSort) {
        static bool attr_set = false;   // one-time opt-in above the 48 KB default
        if (!attr_set) {
            const cudaError_t e = cudaFuncSetAttribute(k_sort_small, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                       (int)kSmallSmem);
            if (e != cudaSuccess) return e;
            attr_set = true;
        }
        g_launch_count.fetch_add(1, std::memory_order_relaxed);
        k_sort_small<<<1, kSmallThreads, kSmallSmem, s>>>(keys, vals, n, nbits);
        return cudaGetLastError();
    }
    const int nb = (n + kSortTile - 1) / kSortTile;
    unsigned* hist = (unsigned*)temp;
    unsigned* offs = hist + 256 * nb;
    unsigned *kin = keys, *vin = vals, *kout = keys_alt, *vout = vals_alt;
    int alt = 0;
    for (int shift = 0; shift < nbits; shift += 8) {
        g_launch_count.fetch_add(1, std::memory_order_relaxed);
        k_radix_hist<<<nb, kSortThreads, 0, s>>>(kin, n, shift, hist, nb);
        g_launch_count.fetch_add(1, std::memory_order_relaxed);
        k_scan_single<<<1, 1024, 0, s>>>(hist, offs, 256 * nb, nullptr);
        g_launch_count.fetch_add(1, std::memory_order_relaxed);
        k_radix_scatter<<<nb, kSortThreads, 0, s>>>(kin, vin, n, shift, offs, nb, kout, vout);
        unsigned* t = kin; kin = kout; kout = t;
        t = vin; vin = vout; vout = t;
        alt ^= 1;
    }
    *result_in_alt = alt;
    return cudaGetLastError();
}

cudaError_t launch_cell_start(const unsigned* sorted_keys, int n, int ncells, int* cell_start, cudaStream_t s)
{
    g_launch_count.fetch_add(1, std::memory_order_relaxed);
    k_cell_start<<<blocks_for((long long)ncells + 1, 256), 256, 0, s>>>(sorted_keys, n, ncells, cell_start);
    return cudaGetLastError();
}

cudaError_t launch_pack(const float* xyz, const void* feat, int feat_bf16, int D, const unsigned* order, int n,
                        float4* rec, int rs, int rec_bf16, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    g_launch_count.fetch_add(1, std::memory_order_relaxed);
    k_pack<<<blocks_for(n, 128), 128, 0, s>>>(xyz, feat, feat_bf16, D, order, n, rec, rs, rec_bf16);
    return cudaGetLastError();
}

cudaError_t launch_group_flags(const unsigned* sorted_keys, int n, int shift, int gsize, unsigned* flags,
                               cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    g_launch_count.fetch_add(1, std::memory_order_relaxed);
    k_group_flags<<<blocks_for(n, 256), 256, 0, s>>>(sorted_keys, n, shift, gsize, flags);
    return cudaGetLastError();
}

cudaError_t exclusive_scan_u32(const unsigned* in, unsigned* out, int n, unsigned* total, cudaStream_t s)
{
    g_launch_count.fetch_add(1, std::memory_order_relaxed);
    k_scan_single<<<1, 1024, 0, s>>>(in, out, n, total);
    return cudaGetLastError();
}

cudaError_t launch_group_write(const unsigned* sorted_keys, const unsigned* flags, const unsigned* gidx, int n,
                               int shift, int gsize, int2* groups, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    g_launch_count.fetch_add(1, std::memory_order_relaxed);
    k_group_write<<<blocks_for(n, 256), 256, 0, s>>>(sorted_keys, flags, gidx, n, shift, gsize, groups);
    return cudaGetLastError();
}

// ---- batched launchers ----------------------------------------------------------

namespace {

// f(list) for each run of up to kJobsPerLaunch jobs
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

}  // namespace

size_t sort_batch_temp_words(int n)
{
    const int nb = (n + kSortTile - 1) / kSortTile;
    return (size_t)2 * 256 * (nb > 0 ? nb : 1);
}

cudaError_t launch_boxes_batch(const BoxJob* jobs, int count, cudaStream_t s)
{
    return each_chunk(jobs, count, [&](const JobList<BoxJob>& L) {
        int nmax = 1, mmax = 1;
        long long fmax = 1;
        for (int i = 0; i < L.count; ++i) {
            nmax = max(nmax, max(L.j[i].n, L.j[i].m));
            mmax = max(mmax, L.j[i].m);
            fmax = max(fmax, max(L.j[i].nfx, L.j[i].nfz));
        }
        g_launch_count.fetch_add(5, std::memory_order_relaxed);
        k_boxes_init_b<<<dim3(1, L.count), 32, 0, s>>>(L);
        k_bbox_b<<<dim3(min(blocks_for(nmax, 256), 64), L.count, 2), 256, 0, s>>>(L);
        const int nz = min(blocks_for(mmax, 4 * kZStatsThreads), 64);
        k_zsum_b<<<dim3(nz, L.count), kZStatsThreads, 0, s>>>(L);
        k_zspread_b<<<dim3(nz, L.count), kZStatsThreads, 0, s>>>(L);
        k_check_feat_b<<<dim3((int)min((long long)blocks_for(fmax, 256), 256LL), L.count, 2), 256, 0, s>>>(L);
        return cudaGetLastError();
    });
}

cudaError_t launch_cell_keys_batch(const KeyJob* jobs, int count, cudaStream_t s)
{
    return each_chunk(jobs, count, [&](const JobList<KeyJob>& L) {
        int nmax = 1;
        for (int i = 0; i < L.count; ++i) nmax = max(nmax, L.j[i].n);
        g_launch_count.fetch_add(1, std::memory_order_relaxed);
        k_cell_keys_b<<<dim3(blocks_for(nmax, 256), L.count), 256, 0, s>>>(L);
        return cudaGetLastError();
    });
}

cudaError_t launch_hilbert_keys_batch(const KeyJob* jobs, int count, cudaStream_t s)
{
    return each_chunk(jobs, count, [&](const JobList<KeyJob>& L) {
        int nmax = 1;
        for (int i = 0; i < L.count; ++i) nmax = max(nmax, L.j[i].n);
        g_launch_count.fetch_add(1, std::memory_order_relaxed);
        k_hilbert_keys_b<<<dim3(blocks_for(nmax, 256), L.count), 256, 0, s>>>(L);
        return cudaGetLastError();
    });
}

cudaError_t radix_sort_batch(const SortJob* jobs, int count, int nbits, int* result_in_alt, cudaStream_t s)
{
    int passes = 0;
    for (int shift = 0; shift < nbits; shift += 8) ++passes;
    *result_in_alt = passes & 1;
    return each_chunk(jobs, count, [&](const JobList<SortJob>& L) {
        int nbmax = 1;
        for (int i = 0; i < L.count; ++i) nbmax = max(nbmax, (L.j[i].n + kSortTile - 1) / kSortTile);
        int parity = 0;
        for (int shift = 0; shift < nbits; shift += 8) {
            g_launch_count.fetch_add(3, std::memory_order_relaxed);
            k_radix_hist_b<<<dim3(nbmax, L.count), kSortThreads, 0, s>>>(L, shift, parity);
            k_radix_scan_b<<<dim3(1, L.count), 1024, 0, s>>>(L);
            k_radix_scatter_b<<<dim3(nbmax, L.count), kSortThreads, 0, s>>>(L, shift, parity);
            parity ^= 1;
        }
        return cudaGetLastError();
    });
}

cudaError_t launch_cell_start_batch(const CellStartJob* jobs, int count, cudaStream_t s)
{
    return each_chunk(jobs, count, [&](const JobList<CellStartJob>& L) {
        long long cmax = 1;
        for (int i = 0; i < L.count; ++i) cmax = max(cmax, (long long)L.j[i].ncells + 1);
        g_launch_count.fetch_add(1, std::memory_order_relaxed);
        k_cell_start_b<<<dim3(blocks_for(cmax, 256), L.count), 256, 0, s>>>(L);
        return cudaGetLastError();
    });
}

cudaError_t launch_pack_batch(const PackJob* jobs, int count, int D, int rs, int rec_bf16, cudaStream_t s)
{
    return each_chunk(jobs, count, [&](const JobList<PackJob>& L) {
        int nmax = 1;
        for (int i = 0; i < L.count; ++i) nmax = max(nmax, L.j[i].n);
        g_launch_count.fetch_add(1, std::memory_order_relaxed);
        k_pack_b<<<dim3(blocks_for(nmax, 128), L.count), 128, 0, s>>>(L, D, rs, rec_bf16);
        return cudaGetLastError();
    });
}

cudaError_t launch_scan_batch(const ScanJob* jobs, int count, cudaStream_t s)
{
    return each_chunk(jobs, count, [&](const JobList<ScanJob>& L) {
        g_launch_count.fetch_add(1, std::memory_order_relaxed);
        k_scan_b<<<dim3(1, L.count), 1024, 0, s>>>(L);
        return cudaGetLastError();
    });
}

cudaError_t launch_group_flags_batch(const GroupJob* jobs, int count, cudaStream_t s)
{
    return each_chunk(jobs, count, [&](const JobList<GroupJob>& L) {
        int nmax = 1;
        for (int i = 0; i < L.count; ++i) nmax = max(nmax, L.j[i].n);
        g_launch_count.fetch_add(1, std::memory_order_relaxed);
        k_group_flags_b<<<dim3(blocks_for(nmax, 256), L.count), 256, 0, s>>>(L);
        return cudaGetLastError();
    });
}

cudaError_t launch_group_write_batch(const GroupJob* jobs, int count, cudaStream_t s)
{
    return each_chunk(jobs, count, [&](const JobList<GroupJob>& L) {
        int nmax = 1;
        for (int i = 0; i < L.count; ++i) nmax = max(nmax, L.j[i].n);
        g_launch_count.fetch_add(1, std::memory_order_relaxed);
        k_group_write_b<<<dim3(blocks_for(nmax, 256), L.count), 256, 0, s>>>(L);
        return cudaGetLastError();
    });
}

cudaError_t launch_pull_batch(const PullJob* jobs, int count, cudaStream_t s)
{
    return each_chunk(jobs, count, [&](const JobList<PullJob>& L) {
        long long nmax = 1;
        for (int i = 0; i < L.count; ++i) nmax = max(nmax, L.j[i].bytes);
        // about 64 KB per block, at most 64 blocks per job
        const int bx = (int)min(64ll, (nmax + 65535) / 65536);
        g_launch_count.fetch_add(1, std::memory_order_relaxed);
        k_pull_b<<<dim3(bx, L.count), 256, 0, s>>>(L);
        return cudaGetLastError();
    });
}

cudaError_t launch_copy_batch(const CopyJob* jobs, int count, cudaStream_t s)
{
    return each_chunk(jobs, count, [&](const JobList<CopyJob>& L) {
        g_launch_count.fetch_add(1, std::memory_order_relaxed);
        k_copy_b<<<dim3(1, L.count), 256, 0, s>>>(L);
        return cudaGetLastError();
    });
}

}  // namespace cvo
