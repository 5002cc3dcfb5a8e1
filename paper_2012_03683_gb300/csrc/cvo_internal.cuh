// Internal declarations shared by the CUDA translation units of libcvo.
//
// Data layout in device memory (one handle, one pair):
//   zrec[level]   M records sorted by grid cell (x fastest), RS float4 each:
//                 rec[0] = (x, y, z, index) float32 as given, the w lane
//                 holding the point's index bits; rec[1..] = the point's
//                 feature row (float32 or bfloat16, blocks concatenated,
//                 zero padded to 16 bytes)
//   cell_start    per level, ncells + 1 ints: records of cell c are
//                 [cell_start[c], cell_start[c+1])
//   xrec          N query records in the same layout, in Hilbert order of X's
//                 own frame (spatially compact runs)
//   groups        per level, (first query, count <= 32) of each query group:
//                 consecutive queries inside one octree super-cell whose edge
//                 does not exceed that level's cell edge
//   items         per level, the work items of a sweep: (first query, count,
//                 chunk k | chunks n << 16, group index) -- chunk k of n of one
//                 group's candidate stream.  Planned (evaluations, batches,
//                 dense registrations): n from the stream's length at the
//                 pose of the call (about chunk_len candidates per item),
//                 groups with the longest streams first.  A registration with
//                 a cutoff, whose pose moves: the first sweep of a level takes
//                 uniform items (8 chunks per group in Hilbert order, cut at
//                 run time to min(8, length / 64)); every sweep records each
//                 group's stream length and k_layout lays out the next sweep's
//                 items from them (n = ceil(length / chunk_len), group order)
//   IterState     pose, lengthscale, annealing state and the derived
//                 per-iteration constants, written by the finalize kernel and
//                 read by the sweep kernel (no host round trip per iteration)
//   partials      per sweep block: 43 linear statistics as (hi, lo) float
//                 pairs plus the pair and candidate counts; a single pair's
//                 blocks are also summed in groups of kGroupBlocks by each
//                 group's last block (the group sums the step kernel adds)
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

namespace cvo {

constexpr int kStatN = 43;       // linear statistics of the per-query moments
constexpr int kSweepWarps = 4;   // warps per sweep block
constexpr int kSweepBlocksPerSm = 8;   // most sweep blocks launched per SM (two waves of four resident blocks)
constexpr int kMaxLevels = 24;   // grid levels of one registration
constexpr int kMaxChunks = 64;   // most work items (chunks) one query group's stream splits into
constexpr int kChunkLen = 128;   // default candidates per planned work item
constexpr int kChunks = 8;       // chunks per group of the uniform items
constexpr int kChunkMin = 64;    // shortest run-time chunk of the uniform items
constexpr int kTrimChunkLen = 768;   // planned items at least this long trim the stream rows by each query
constexpr int kFinalizeThreads = 256;  // threads of a batched step block
constexpr int kStepCluster = 4;        // blocks per pair of the batched step with a work queue (a cluster)
constexpr int kStepThreads = 384;      // threads of the single-pair step block (its registers allow 12 warps)
constexpr int kGroupBlocks = 8;    // sweep blocks per reduction group (the group's last block sums them)
constexpr int kMaxGroups = 256;    // reduction groups per sweep launch (so at most kGroupBlocks * kMaxGroups sweep blocks)
constexpr int kTraceStride = 22;  // doubles per iteration in the trace (CVO_TRACE_STRIDE)

// Offsets of the 43 statistics (see the finalize kernel for their use).
enum StatIndex {
    ST_W = 0,     // sum W
    ST_E = 1,     // sum E (3)
    ST_Q = 4,     // sum Q (xx, yy, zz, xy, xz, yz)
    ST_PQ = 10,   // sum [p]x Q (3x3 row major)
    ST_PQP = 19,  // sum [p]x Q [p]x (xx, yy, zz, xy, xz, yz)
    ST_WP = 25,   // sum W p (3)
    ST_WPP = 28,  // sum W p p^T (xx, yy, zz, xy, xz, yz)
    ST_EP = 34    // sum E p^T (3x3 row major)
};

struct LevelDesc {
    float h, inv_h;          // cell edge and its inverse (y and z)
    float inv_hx;            // inverse cell edge along x (the cells' rows; a fraction of h trims the rows' runs)
    float ox, oy, oz;        // grid origin (minimum corner), Z frame
    int nx, ny, nz;          // cells per axis
    const int* cell_start;   // nx*ny*nz + 1
    const float4* zrec;      // M records sorted by cell
    const int2* groups;      // query groups (first, count)
    const int4* items;       // work items (first query, count, chunk | chunks << 16, group index)
    int ngroups;
    int nitems;
    int chunk_min;           // > 0: a group's stream is cut into min(chunks, length / chunk_min) chunks at
                             // run time (the rest of its items are empty); 0: into the planned chunks
    int trim;                // 1: the stream rows' runs cover the queries' balls; 0: the group's box grown by a ball
};

// Feature-kernel constants (exponent in log2 units).
struct FeatConst {
    int n_blocks;
    int dim[4];
    int kind[4];             // 0 squared exponential, 1 inner product
    int off[4];              // column offset of each block
    float s[4];              // -log2(e) / (2 l_b^2) for squared-exponential blocks
    float fcut2[4];          // feature-space cutoff of squared-exponential blocks: |u - v|^2 <= fcut2 (3e38: off)
    int D;                   // total feature dim
    int bf16;                // storage of the records' features
};

struct IterState {
    double T[16];            // current pose, row major
    double ell;              // current lengthscale
    double ell_last;         // lengthscale of the last completed iteration
    // derived constants for the sweep: x' = A x + b with A = R^T, b = -R^T t
    float Ahi[9], Alo[9], bhi[3], blo[3];
    float chi[3], clo[3];    // lever centre c (Z frame)
    float sg;                // -log2(e) / (2 l^2)
    float rc;                // cutoff radius (m); < 0: dense
    float rc2;               // rc^2
    int level;               // grid level for this iteration
    int done;                // 1: no more iterations
    int iter;                // iterations completed
    int mode;                // 0 eval, 1 register
    int have_ref;
    double i_ref;
    // results of the last sweep / step
    double F, i_theta, gnorm, Fpp, t, srot, strans;
    double grad[6];
    double hess[36];
    long long pairs, cands, pairs_total, cands_total;
    int status;              // 0 converged, 1 not converged
    int decayed;
    // constants of the registration
    double kappa;            // sigma^2 * prod sigma_b^2 over squared-exponential blocks
    double norm;             // 1 / sqrt(N M) (0 if empty)
    double cutoff_mult, ell_min, decay, indicator_tol;
    double step_tol_rot, step_tol_trans, max_step_rot, max_step_trans;
    double c[3];             // lever centre (double): the centroid of Z
    double rho2;             // mean squared distance of Z's points from c (the step's rotation weight, plus l^2)
    double rmax;             // largest distance of a point of Z from c (the step's trust region)
    int max_iters, anneal;
    int nlevels;
    float level_h[kMaxLevels];
};

// One registration pair as the sweep sees it.  Sweep blocks [b0, b1) work on
// this pair (a batch splits the grid among its pairs in proportion to their
// work); each block's partial sums belong to one pair.
struct PairDesc {
    const LevelDesc* levels;   // device array [nlevels]
    const float4* xrec;        // N query records
    IterState* st;
    int n, m;
    int b0, b1;
    int bmax;                  // most sweep blocks a batch may give this pair when it re-splits the grid
};

struct SweepArgs {
    const PairDesc* pairs;     // device array [npairs], ordered by b0
    int npairs;
    int rs;                    // record stride (float4)
    int dense;
    float2* part_stats;        // [kStatN][part_cap] per-block sums
    unsigned long long* part_cnt; // [2][part_cap]
    int part_cap;
    float2* grp_stats;         // [kStatN][kMaxGroups] per-group sums (read by the finalize)
    unsigned long long* grp_cnt;  // [2][kMaxGroups]
    unsigned* grp_arrivals;    // [kMaxGroups] arrival counters, zero between launches;
                               // NULL in a batch (its finalize sums the block partials)
    FeatConst fc;
    unsigned* nch_next;        // registration with a cutoff: each group's chunk count for the next sweep,
                               // ceil(stream length / chunk_len), written by the group's item with chunk 0
                               // (NULL: not recorded)
    int chunk_len;
    int lanes;                 // lanes per query (query groups of 32 / lanes queries)
    int* swept_level;          // with nch_next: the level the sweep covered (written by block 0)
    // a batch's work queue (item_rows non-NULL): one resident wave of blocks
    // whose warps take the batch's work items from a counter, largest pair
    // first; item i (pair p's item i - ibase[p]) leaves its statistics in
    // row i, and the batched step sums each pair's rows in item order
    float* item_rows;          // [items][kRowFloats]: the 43 statistics, then the pair and test counts (as bits)
    unsigned* queue;           // [0] the next item to take, [1] the items of this sweep
    const int* ibase;          // [npairs + 1] first item of each pair (a stopped pair has none)
};

constexpr int kRowFloats = 48;   // floats per work item's statistics row (43 + 2 counts, padded)
constexpr int kQueueWarps = 4;        // warps per work-queue sweep block (six, three blocks per SM, measured slower)
constexpr int kStreamWarps = kQueueWarps > kSweepWarps ? kQueueWarps : kSweepWarps;   // most warps per block that form streams

// The batched step's view of the work queue (rows NULL: the per-block partials).
struct BatchQueue {
    const float* rows;
    int* ibase;                // rewritten for the next sweep by the last block
    unsigned* queue;
};

// ---- launchers (host) ------------------------------------------------------

// Kernels launched by this library in this process (every launcher adds its own).
extern std::atomic<long long> g_launch_count;

cudaError_t launch_sweep(const SweepArgs& a, int nblocks, cudaStream_t s);

// Batched step: one block per pair sums that pair's block partials and takes
// its step, and records the work the pair has left (its work items at its
// grid level, 0 once it has stopped) in work[pair]; the last block to finish
// writes the number of pairs still running to counters[2], re-splits the
// sweep grid of part_cap blocks among the running pairs in proportion to
// their work (at least one block each, at most bmax; stopped pairs get none)
// by rewriting the pairs' b0 / b1 for the next sweep, and, inside a graph,
// sets the loop's condition.  traces: npairs x trace_stride doubles (NULL: no
// trace).
// With a work queue (bq.rows non-NULL) each pair's statistics are the sum
// of its items' rows, in item order, and the last block writes the next
// sweep's ibase (the running pairs' work items, in pair order) and resets
// the queue instead of re-splitting the grid.
cudaError_t launch_finalize_batch(PairDesc* pairs, int npairs, const float2* part_stats,
                                  const unsigned long long* part_cnt, int part_cap, double* traces,
                                  long long trace_stride, unsigned* counters, unsigned* work, BatchQueue bq,
                                  cudaStream_t s);
// k_finalize_batch(PairDesc*, int npairs, const float2*, const unsigned long long*, int cap,
//                  double* traces, long long trace_stride, unsigned* counters, unsigned* work,
//                  BatchQueue bq, cudaGraphConditionalHandle cond, int use_cond); counters[0] arrivals,
//                  counters[1] active pairs being counted, counters[2] the last count
const void* finalize_batch_kernel();
// The same step with a work queue: a cluster of kStepCluster blocks per pair
// (grid npairs * kStepCluster), k_finalize_batch_q(PairDesc*, int npairs,
// double* traces, long long trace_stride, unsigned* counters, unsigned* work,
// BatchQueue bq, cudaGraphConditionalHandle cond, int use_cond).
const void* finalize_batch_queue_kernel();
// The first sweep's work queue of a batch (work: npairs scratch words; ibase
// npairs + 1 ints; queue 2 words), from the pairs' initial states.
cudaError_t launch_queue_init(const PairDesc* pairs, int npairs, unsigned* work, int* ibase, unsigned* queue,
                              cudaStream_t s);

// Kernel handles for CUDA-graph kernel nodes.
struct SweepLaunch {
    const void* func;   // k_sweep (or k_sweep_q) specialisation
    size_t smem;        // dynamic shared memory
    int threads;        // threads per block
};
// lanes: lanes per query of the sweep (1, 2, 4; the query groups hold 32 / lanes queries);
// queue: the work-queue form of a batch (k_sweep_q)
cudaError_t sweep_launch_info(const FeatConst& fc, int rs, int lanes, SweepLaunch* out, bool queue = false);
// Dynamic shared memory a work-queue sweep adds to SweepLaunch::smem: its
// copy of ibase (npairs + 1 ints).
inline size_t queue_smem(int npairs) { return ((size_t)(npairs + 1) * sizeof(int) + 15) & ~(size_t)15; }
// k_finalize(IterState*, const float2* grp_stats, const unsigned long long* grp_cnt, int ngroups,
//            double* trace, cudaGraphConditionalHandle cond, int use_cond), kStepThreads threads
const void* finalize_kernel();
cudaError_t launch_init_state(IterState* st, cudaStream_t s);
// Reduces the ceil(nblocks / kGroupBlocks) group sums of a sweep and takes the step.
cudaError_t launch_finalize(IterState* st, const float2* grp_stats, const unsigned long long* grp_cnt, int nblocks,
                            double* trace, cudaStream_t s);
// X-row shards of one registration: the statistics of a sweep as
// kShardStats doubles (43 statistics, pair count, candidate count), and the
// step from such statistics summed over the shards.
constexpr int kShardStats = kStatN + 2;
cudaError_t launch_stats_out(const float2* grp_stats, const unsigned long long* grp_cnt, int nblocks, double* out,
                             cudaStream_t s);
cudaError_t launch_finalize_stats(IterState* st, const double* stats, double* trace, cudaStream_t s);
// Lays out the swept level's work items for the next sweep from the chunk
// counts the sweep recorded (registration with a cutoff; one block, run
// beside the step).  k_layout(LevelDesc* levels, const int* swept_level,
// const unsigned* nch_next), kLayoutThreads threads.
constexpr int kLayoutThreads = 256;
cudaError_t launch_layout(LevelDesc* levels, const int* swept_level, const unsigned* nch_next, cudaStream_t s);
const void* layout_kernel();

// Gradients of F with respect to one cloud's points and features: a sweep with
// that cloud as the queries (see cvo_sweep.cu, k_grad).
struct GradArgs {
    const LevelDesc* levels;   // grid of the other cloud
    const float4* xrec;        // queries; record w = the point's index in the caller's order
    const IterState* st;       // query transform, lengthscale, cutoff, level
    int m;                     // points in the other cloud
    int rs, dense;
    FeatConst fc;
    float Rout[9];             // rotation from the sweep frame to the queries' frame (row major)
    float scale_pos;           // dF * kappa / l^2
    float scale_ell;           // dF * kappa / l^3
    float feat_scale[64];      // per feature column: -dF kappa / l_b^2 (squared exponential), dF kappa (inner product)
    float* part;               // per work item and lane: E (3), sum w d^2, feature sums (D)
    float* out_pos;            // N x 3, or NULL
    float* out_feat;           // N x D, or NULL
    float* out_tq;             // N per-query terms of dF/dl, or NULL
};
// The gradient sweep over the level's planned work items (raw sums per item
// and lane into g.part, nitems x 32 x (4 + D) floats), then the per-group
// reduction in chunk order; every query's outputs are written (zero when it
// has no pair in range).
cudaError_t launch_grad(const GradArgs& g, int nblocks, cudaStream_t s);
// Deterministic sum of n floats into *out (one block).
cudaError_t launch_sum_f32(const float* v, int n, double* out, cudaStream_t s);

// Persistent registration loop of one pair (cvo_persist.cu): the blocks a
// cooperative launch of it may have (one resident wave), and the launch.
// sw is set up for at least nblocks sweep blocks; ctl: 6 unsigned, zero
// before the launch (ctl[4] != 0 afterwards: a grid barrier gave up); nch:
// one unsigned per query group of the largest level.
cudaError_t persistent_grid(const SweepArgs& sw, int* nblocks);
// leave_at >= 0: the last block leaves at that grid barrier instead of
// arriving (failure injection); spin_limit: polls before a barrier gives up
// (0: the default of seconds).
cudaError_t launch_register_persistent(const SweepArgs& sw, unsigned* ctl, unsigned* nch, int chunk_len, double* trace,
                                       int nblocks, int leave_at, unsigned spin_limit, cudaStream_t s);

// Work-item planning of one grid level (cvo_sweep.cu): per query group the
// length of its candidate stream at the state's pose for cutoff radius rc,
// as a descending sort key (keys), the group index (vals) and its chunk count
// ceil(length / chunk_len) clamped to [1, kMaxChunks] (nch); chunk_len <= 0:
// no lengths, vals = the group index and nch = kChunks (uniform items).
// Then, with the groups sorted and the chunk counts scanned, the item table.
cudaError_t launch_group_cost(const LevelDesc* levels, int level, int ngroups, const float4* xrec, int m, int rs,
                              int dense, const IterState* st, float rc, int chunk_len, unsigned* keys, unsigned* vals,
                              unsigned* nch, cudaStream_t s);
cudaError_t launch_gather_u32(const unsigned* src, const unsigned* idx, int n, unsigned* dst, cudaStream_t s);
cudaError_t launch_write_items(const LevelDesc* levels, int level, const unsigned* sorted_groups, const unsigned* nch,
                               const unsigned* offsets, int ngroups, int4* items, cudaStream_t s);

// ---- batched setup: one launch for the pairs of a batch ---------------------
// The per-pair stages of the set-up (boxes, grids, Hilbert order, groups,
// work items) for many pairs at once: each launch takes up to
// kJobsPerLaunch pairs' jobs by value as a kernel parameter, blockIdx.y
// selects the job, and the kernels run the single-pair kernels' bodies, so
// the results are the same.  The launchers take a host array of any length
// and launch once per kJobsPerLaunch jobs.  Every pointer is the pair's own
// buffer (or its segment of a shared scratch buffer) with room for the
// counts given.
constexpr int kJobsPerLaunch = 64;

template <class J>
struct JobList {
    int count;
    J j[kJobsPerLaunch];
};

// boxes of X and Z (6 words each: min bits x3, max bits x3), the
// non-finite flag, Z's moments (5 words of 8 bytes) and the features' check
struct BoxJob {
    const float* xyz_x;
    const float* xyz_z;
    const void* feat_x;
    const void* feat_z;
    long long nfx, nfz;   // feature values to check (n D, m D)
    int n, m, fx_bf16, fz_bf16;
    unsigned* box_x;
    unsigned* box_z;
    int* bad;
    long long* zstats;
};

// grid-cell keys (nx, ny, nz, inv = 1 / cell edge) or Hilbert keys (inv = 1 /
// the edge of the curve's cells) of one cloud, with the point indices as values
struct KeyJob {
    const float* xyz;
    unsigned* keys;
    unsigned* vals;
    float ox, oy, oz, inv, invx;   // invx: along x (grid cells)
    int n, nx, ny, nz;
};

// a stable sort of n (key, value) pairs; temp holds 2 * 256 * ceil(n /
// 1024) words; the result is in (keys, vals) after an even number of
// passes, else in (keys2, vals2)
struct SortJob {
    unsigned* keys;
    unsigned* vals;
    unsigned* keys2;
    unsigned* vals2;
    unsigned* temp;
    int n;
};

struct CellStartJob {
    const unsigned* keys;   // sorted cell keys
    int* cell_start;        // ncells + 1
    int n, ncells;
};

// records of one cloud in the order given (order NULL: as stored); keys_out
// (optional) receives the sorted keys
struct PackJob {
    const float* xyz;
    const void* feat;
    const unsigned* order;
    const unsigned* keys;
    unsigned* keys_out;
    float4* rec;
    int n, feat_bf16;
};

// exclusive scan of n words; total (optional) receives the sum
struct ScanJob {
    const unsigned* in;
    unsigned* out;
    unsigned* total;
    int n;
};

// query groups of one level from the Hilbert-sorted keys: flags (first query
// of each group), then (with gidx, the flags' scan) the group table
struct GroupJob {
    const unsigned* hkeys;
    unsigned* flags;
    const unsigned* gidx;
    int2* groups;
    int n, shift, gsize;
};

size_t sort_batch_temp_words(int n);
cudaError_t launch_boxes_batch(const BoxJob* jobs, int count, cudaStream_t s);   // zeroes its outputs first
cudaError_t launch_cell_keys_batch(const KeyJob* jobs, int count, cudaStream_t s);
cudaError_t launch_hilbert_keys_batch(const KeyJob* jobs, int count, cudaStream_t s);
cudaError_t radix_sort_batch(const SortJob* jobs, int count, int nbits, int* result_in_alt, cudaStream_t s);
cudaError_t launch_cell_start_batch(const CellStartJob* jobs, int count, cudaStream_t s);
cudaError_t launch_pack_batch(const PackJob* jobs, int count, int D, int rs, int rec_bf16, cudaStream_t s);
cudaError_t launch_scan_batch(const ScanJob* jobs, int count, cudaStream_t s);
cudaError_t launch_group_flags_batch(const GroupJob* jobs, int count, cudaStream_t s);
cudaError_t launch_group_write_batch(const GroupJob* jobs, int count, cudaStream_t s);

// work items of one level of many pairs (cvo_sweep.cu), as launch_group_cost,
// launch_gather_u32 and launch_write_items
struct CostJob {
    const LevelDesc* levels;
    const float4* xrec;
    const IterState* st;
    unsigned* keys;
    unsigned* vals;
    unsigned* nch;
    int level, ngroups, m;
    float rc;
};
struct GatherJob {
    const unsigned* src;
    const unsigned* idx;
    unsigned* dst;
    int n;
};
struct ItemsJob {
    const LevelDesc* levels;
    const unsigned* sorted_groups;
    const unsigned* nch;
    const unsigned* offsets;
    int4* items;
    int level, ngroups;
};
cudaError_t launch_group_cost_batch(const CostJob* jobs, int count, int rs, int dense, int chunk_len, cudaStream_t s);
cudaError_t launch_gather_batch(const GatherJob* jobs, int count, cudaStream_t s);
cudaError_t launch_write_items_batch(const ItemsJob* jobs, int count, cudaStream_t s);

// blocks of bytes (multiples of 4) copied between device buffers, one block
// per job (cvo_setup.cu)
struct CopyJob {
    const void* src;
    void* dst;
    int bytes;
};
cudaError_t launch_copy_batch(const CopyJob* jobs, int count, cudaStream_t s);
// a host-resident input pulled into device memory by the SMs (src: the
// device-side address of page-locked, mapped host memory)
struct PullJob {
    const void* src;
    void* dst;
    long long bytes;
};
cudaError_t launch_pull_batch(const PullJob* jobs, int count, cudaStream_t s);

// k_init_state of many pairs (cvo_finalize.cu)
struct StateJob {
    IterState* st;
};
cudaError_t launch_init_state_batch(const StateJob* jobs, int count, cudaStream_t s);

// setup (cvo_setup.cu)
cudaError_t launch_bbox(const float* xyz, int n, unsigned* out6, int* bad, cudaStream_t s);
cudaError_t launch_check_feat(const void* feat, long long count, int bf16, int* bad, cudaStream_t s);
// a cloud's centroid, mean squared distance from it and largest such
// distance: raw sums into out (5 words of 8 bytes, zeroed before), which
// decode_zstats turns into (cx, cy, cz, mean r^2, max r) on the host
cudaError_t launch_zstats(const float* xyz, int n, long long* out, cudaStream_t s);
void decode_zstats(const long long* raw, int n, double out5[5]);
cudaError_t launch_cell_keys(const float* xyz, int n, float ox, float oy, float oz, float inv_h, float inv_hx, int nx,
                             int ny, int nz, unsigned* keys, unsigned* vals, cudaStream_t s);
cudaError_t launch_hilbert_keys(const float* xyz, int n, float ox, float oy, float oz, float inv_cell,
                               unsigned* keys, unsigned* vals, cudaStream_t s);
size_t radix_sort_temp_bytes(int n);
cudaError_t radix_sort_pairs(unsigned* keys, unsigned* vals, unsigned* keys_alt, unsigned* vals_alt, int n,
                             int nbits, void* temp, int* result_in_alt, cudaStream_t s);
cudaError_t launch_cell_start(const unsigned* sorted_keys, int n, int ncells, int* cell_start, cudaStream_t s);
cudaError_t launch_pack(const float* xyz, const void* feat, int feat_bf16, int D, const unsigned* order, int n,
                        float4* rec, int rs, int rec_bf16, cudaStream_t s);
// query groups: up to gsize consecutive Hilbert-sorted queries of one super-cell
// (2^shift key units: an octree cell) each
cudaError_t launch_group_flags(const unsigned* sorted_keys, int n, int shift, int gsize, unsigned* flags,
                               cudaStream_t s);
cudaError_t exclusive_scan_u32(const unsigned* in, unsigned* out, int n, unsigned* total, cudaStream_t s);
cudaError_t launch_group_write(const unsigned* sorted_keys, const unsigned* flags, const unsigned* gidx, int n,
                               int shift, int gsize, int2* groups, cudaStream_t s);

}  // namespace cvo
