/*
 * cvo.h -- C ABI of the GB300 (sm_103a) library for the RKHS point-cloud
 * registration of "A New Framework for Registration of Semantic Point Clouds
 * from Stereo and RGB-D Cameras" (arXiv:2012.03683).
 *
 * Two clouds X = {x_i} (N points) and Z = {z_j} (M points) with per-point
 * feature vectors are aligned by maximising the RKHS inner product of
 * Problem 1 (Sec. III, Eq. max) over SE(3):
 *
 *   F(T) = sum_{i,j} k(x_i, T z_j) * c_ij                    Eq. (double_sum)
 *   k(x, y) = sigma^2 exp(-|x - y|^2 / (2 l^2))              Eq. (k)
 *   c_ij = prod_b k_b(u_bi, v_bj)                            Eq. (tensor_product)
 *     k_b = sigma_b^2 exp(-|u - v|^2 / (2 l_b^2))  (CVO_FEAT_SE,  Eq. newscalar)
 *     k_b = <u, v>                                 (CVO_FEAT_DOT, Eq. scalar)
 *
 * The pose T (row-major 4x4, double) maps Z into X's frame, y_j = R z_j + t;
 * it is the inverse of the h of Problem 1.  A pair enters the sum when
 * |x_i - y_j| <= cutoff_mult * l (inclusive; the paper calls the sum sparse,
 * Sec. III-B, but gives no threshold) or, with cutoff_mult <= 0, always.
 *
 * Conventions shared by every entry point:
 *  - Return value: a cvo_status.  On an error the thread-local message of
 *    cvo_last_error() says what went wrong; outputs are then unspecified.
 *  - Clouds: cvo_cloud.xyz is N x 3 float32, row major (x, y, z per point).
 *    cvo_cloud.feat is N x D row major, D = sum of the handle's block dims,
 *    blocks concatenated in the order of cvo_params.blocks, stored as float32
 *    or bfloat16 (cvo_cloud.feat_dtype); NULL when D == 0.  With on_device
 *    = 1 both pointers are device pointers valid on the handle's stream, and
 *    with on_device = 0 host pointers (the library copies them).  The caller
 *    owns all input and output buffers; the library keeps no pointer to them
 *    after the call returns.
 *  - Empty clouds (N = 0 or M = 0) are not an error: F = 0, gradient 0,
 *    indicator 0, and a registration returns T_init with status CVO_OK.
 *  - T: the last row must be (0, 0, 0, 1) and R orthonormal within 1e-6,
 *    otherwise CVO_ERR_INVALID_ARG.  Non-finite coordinates or features give
 *    CVO_ERR_INVALID_ARG.
 *  - Every call is synchronous: it returns after the results are on the host.
 *  - A handle is not thread safe; use one handle per host thread.  The handle
 *    owns its device scratch (grids, sorted copies of the clouds, partial
 *    sums), allocated with cudaMalloc on first use and grown on demand.
 */
#ifndef CVO_H
#define CVO_H

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    CVO_OK = 0,
    CVO_NOT_CONVERGED = 1,     /* registration hit max_iters (not an error) */
    CVO_ERR_INVALID_ARG = -1,
    CVO_ERR_CUDA = -2,
    CVO_ERR_OOM = -3,
    CVO_ERR_TIMEOUT = -4
} cvo_status;

typedef enum {
    CVO_FEAT_SE = 0,   /* sigma_b^2 exp(-|u - v|^2 / (2 scale^2)), Eq. (newscalar) */
    CVO_FEAT_DOT = 1   /* <u, v>, Eq. (scalar); scale and sigma unused */
} cvo_feat_kind;

typedef enum { CVO_F32 = 0, CVO_BF16 = 1 } cvo_dtype;

#define CVO_MAX_BLOCKS 4
#define CVO_MAX_FEAT_DIM 64
#define CVO_TRACE_STRIDE 22

typedef struct {
    int dim;        /* entries of this block in each feature row (>= 1) */
    int kind;       /* cvo_feat_kind */
    double scale;   /* l_b of a CVO_FEAT_SE block (> 0) */
    double sigma;   /* sigma_b of a CVO_FEAT_SE block */
} cvo_feat_block;

typedef struct {
    const float* xyz;  /* n x 3 float32 */
    int n;             /* number of points (>= 0) */
    const void* feat;  /* n x D, float32 or bfloat16 (see feat_dtype); NULL if D == 0 */
    int feat_dtype;    /* cvo_dtype */
    int on_device;     /* 1: device pointers, 0: host pointers */
} cvo_cloud;

typedef struct {
    double ell;            /* geometric lengthscale l of Eq. (k) (> 0); the first l of a registration */
    double ell_min;        /* annealing floor (0 < ell_min <= ell) */
    double sigma;          /* sigma of Eq. (k) */
    double cutoff_mult;    /* r_c = cutoff_mult * l; <= 0 means every pair (dense) */
    int n_blocks;          /* 0..CVO_MAX_BLOCKS feature blocks; total dim <= CVO_MAX_FEAT_DIM */
    cvo_feat_block blocks[CVO_MAX_BLOCKS];
    int max_iters;         /* iteration cap of a registration (>= 0) */
    int anneal;            /* 1: lengthscale annealing of Sec. IV */
    double decay;          /* l <- max(decay * l, ell_min) when the indicator stabilises (0.98: 2 %) */
    double indicator_tol;  /* "stabilised": |i_k - i_ref| < indicator_tol * |i_ref| at the same l */
    double step_tol_rot;   /* converged when the step's rotation |t omega| < step_tol_rot ... */
    double step_tol_trans; /* ... and the motion of Z's centroid < step_tol_trans, with l at its floor */
    double max_step_rot;   /* bound on the step's rotation |t omega| per iteration (rad) */
    double max_step_trans; /* bound on any point of Z's motion per iteration (m); <= 0: 0.5 * current l */
    double feat_cutoff_mult; /* > 0: a pair also needs |u_b - v_b| <= feat_cutoff_mult * scale_b for every
                                CVO_FEAT_SE block b (the feature-space sparsity of Sec. III-B; changes F);
                                <= 0: off (default) */
} cvo_params;

typedef struct {
    int iters;              /* iterations run */
    int status;             /* CVO_OK (converged) or CVO_NOT_CONVERGED */
    double ell_final;       /* lengthscale of the last iteration */
    double F;               /* F at the last iteration's pose (before its step) */
    double i_theta;         /* Eq. (indicator_actual) at that pose: F / sqrt(N M) */
    double last_step_rot;   /* |t omega| of the last step */
    double last_step_trans; /* |t v| of the last step */
    long long pairs;        /* pairs inside the cutoff, summed over iterations */
    long long candidates;   /* point pairs the sweep examined (>= pairs) */
} cvo_info;

typedef struct {
    double F;          /* Eq. (double_sum) */
    double grad[6];    /* (omega; v): d/dxi F(exp(xi^) T) at xi = 0 */
    double hess[36];   /* row-major Hessian of xi -> F(exp(xi^) T) at 0 (symmetric) */
    double i_theta;    /* F / sqrt(N M), Eq. (indicator_actual) */
    long long pairs;   /* pairs inside the cutoff */
    long long candidates;
} cvo_eval;

typedef struct cvo_handle_s* cvo_handle;

/* Creates a handle bound to a CUDA stream (a cudaStream_t; NULL = the legacy
 * default stream) on the current device.  Validates *params (copied).
 * Allocates nothing on the device until the first computation. */
cvo_status cvo_create(const cvo_params* params, void* cuda_stream, cvo_handle* out);

/* Releases the handle and its device scratch.  NULL is accepted. */
cvo_status cvo_destroy(cvo_handle h);

/* Replaces the handle's parameters (validated, copied). */
cvo_status cvo_set_params(cvo_handle h, const cvo_params* params);

/* F(T) of Eq. (double_sum) at lengthscale params.ell. */
cvo_status cvo_inner_product(cvo_handle h, const cvo_cloud* X, const cvo_cloud* Z, const double T[16], double* F);

/* Gradient (omega; v) of xi -> F(exp(xi^) T) at xi = 0 (left perturbation),
 * the ascent direction of the Lie-group gradient method the paper cites
 * (Sec. I).  F may be NULL. */
cvo_status cvo_gradient(cvo_handle h, const cvo_cloud* X, const cvo_cloud* Z, const double T[16], double grad[6],
                        double* F);

/* The alignment indicator of Eq. (indicator_actual), i_theta = F / sqrt(N M),
 * at pose T and lengthscale params.ell. */
cvo_status cvo_metric(cvo_handle h, const cvo_cloud* X, const cvo_cloud* Z, const double T[16], double* i_theta);

/* The exact alignment indicator of Eq. (indicator): the cosine of the angle
 * between f_X and the moved f_Z in the RKHS,
 *   cos_theta = F(X, Z, T) / sqrt(F(X, X, I) F(Z, Z, I)),
 * of which cvo_metric is the approximation of Eq. (indicator_actual).  The
 * squared norms F(X, X, I) and F(Z, Z, I) do not depend on T: with
 * norms2_in = NULL they are computed (two extra sweeps, each cloud against
 * itself with the same kernel and cutoff) and, when norms2_out is not NULL,
 * returned there so that later calls for other poses can pass them back in
 * through norms2_in.  An empty cloud gives cos_theta = 0.  With every pair
 * (cutoff_mult <= 0) the kernel is positive definite and |cos_theta| <= 1;
 * with a cutoff the same truncated sums are used throughout, for which the
 * bound is not guaranteed. */
cvo_status cvo_cosine(cvo_handle h, const cvo_cloud* X, const cvo_cloud* Z, const double T[16],
                      const double* norms2_in, double* cos_theta, double* norms2_out);

/* The exact indicator cos_theta of Eq. (indicator) at lengthscale params.ell
 * (as cvo_cosine computes it, the norms recomputed) and its derivative with
 * respect to the lengthscale, for callers that treat l as a variable of
 * their own objective (the paper mentions an adaptive lengthscale, Sec. VI):
 *   dcos/dl = cos (F'_XZ / F_XZ - (F'_XX / F_XX + F'_ZZ / F_ZZ) / 2),
 * F' = dF/dl of each of the three double sums (the pair set held fixed, as
 * in cvo_backward).  Empty clouds, or a zero numerator, give dcos/dl = 0.
 * The cosine itself rises towards its l -> infinity limit on typical clouds
 * (every geometric kernel value tends to 1), so it does not fix l on its own.
 * Cost: three evaluations and three gradient sweeps. */
cvo_status cvo_cosine_dell(cvo_handle h, const cvo_cloud* X, const cvo_cloud* Z, const double T[16], double* cos_theta,
                           double* dcos_dell);

/* F, gradient, Hessian, indicator and pair counts in one sweep. */
cvo_status cvo_evaluate(cvo_handle h, const cvo_cloud* X, const cvo_cloud* Z, const double T[16], cvo_eval* out);

/* Gradients of dF * F(T) (Eq. double_sum at lengthscale params.ell) with
 * respect to the inputs, for using F or the indicator as a differentiable
 * loss (the learning use the paper proposes as future work, Sec. VI).  The
 * set of pairs inside the cutoff is held fixed, so these are the derivatives
 * almost everywhere.  With w_ij the pair's weight, y_j = R z_j + t and
 * d_ij = x_i - y_j:
 *   dX[i]  = dF/dx_i = -(1/l^2) sum_j w_ij d_ij                    (N x 3)
 *   dZ[j]  = dF/dz_j = (1/l^2) R^T sum_i w_ij d_ij                 (M x 3)
 *   dFX[i] = dF/du_i: for a CVO_FEAT_SE block -(1/l_b^2) sum_j w_ij (u_bi - v_bj),
 *            for a CVO_FEAT_DOT block sum_j w_ij^(b) v_bj, w_ij^(b) being
 *            the weight without that block's factor                (N x D)
 *   dFZ[j] = dF/dv_j, the same with the clouds' roles exchanged    (M x D)
 *   *dell  = dF/dl = (1/l^3) sum_ij w_ij |d_ij|^2
 * all multiplied by dF (the upstream gradient).  Outputs are float32, row
 * major, in the clouds' own point order; features give float32 gradients
 * whatever their storage type (with bfloat16 features, the gradient at the
 * bfloat16 values).  Any output may be NULL and is then neither computed nor
 * written.  outputs_on_device = 1: dX, dFX, dZ, dFZ are device pointers
 * (written on the handle's stream); 0: host pointers.  dell is a host
 * pointer either way.  The gradient with respect to the pose is the se(3)
 * gradient of cvo_gradient.  Precision: float32 accumulation per point
 * (relative error about 1e-6 of the largest term); dF/dl summed in
 * double-float.  Cost: one sweep per requested side, each about the cost of
 * one cvo_evaluate. */
cvo_status cvo_backward(cvo_handle h, const cvo_cloud* X, const cvo_cloud* Z, const double T[16], double dF,
                        float* dX, float* dFX, float* dZ, float* dFZ, double* dell, int outputs_on_device);

/* Gradients of di * i_theta, the indicator of Eq. (indicator_actual)
 * i_theta = F / sqrt(N M) at lengthscale params.ell, with respect to the
 * same inputs as cvo_backward (and with its conventions for the outputs,
 * their layout and the pair set): the paper proposes the indicator as a loss
 * for learning (Sec. III-C, Sec. VI).  Equivalent to cvo_backward with
 * dF = di / sqrt(N M); an empty cloud gives zero gradients. */
cvo_status cvo_metric_backward(cvo_handle h, const cvo_cloud* X, const cvo_cloud* Z, const double T[16], double di,
                               float* dX, float* dFX, float* dZ, float* dFZ, double* dell, int outputs_on_device);

/* Registration (Problem 1): gradient ascent on SE(3) from T_init (Sec. I).
 * Each iteration takes the ascent direction in a metric that names no
 * coordinate origin (rotation and translation about Z's moved centroid,
 * the rotation weighted by Z's mean squared radius plus l^2), a
 * line-Newton step along it (F' / -F'' when F'' < 0, else the edge of the
 * trust region) inside a trust region on the motion of Z's points (none
 * moves more than max_step_trans, or half a lengthscale when that is <= 0,
 * and the rotation is at most max_step_rot), and T <- exp(t xi^) T; the
 * lengthscale anneals as in Sec. IV when params.anneal = 1.  T_out
 * receives the final pose; info (nullable) the summary.  Returns CVO_OK
 * when converged, CVO_NOT_CONVERGED at max_iters. */
cvo_status cvo_register_pair(cvo_handle h, const cvo_cloud* X, const cvo_cloud* Z, const double T_init[16],
                             double T_out[16], cvo_info* info);

/* Registers npairs independent pairs (X[k], Z[k]) from T_init[16k..16k+15];
 * T_out and infos (nullable) are indexed the same way.  Returns the worst
 * status (an error, else CVO_NOT_CONVERGED if any pair hit max_iters).
 * All pairs share one sweep per iteration (one CUDA graph for the loop),
 * whose blocks go to the pairs in order of Z's size, largest first; a pair
 * stops on its own (a per-pair mask) and its blocks pass to the pairs
 * still running.  CVO_BATCH_QUEUE=1 in the environment selects a work-queue
 * sweep instead (warps take the pairs' work items from a counter; results
 * independent of the device's SM count, about 1 % slower on 64 pairs). */
cvo_status cvo_register_batch(cvo_handle h, int npairs, const cvo_cloud* X, const cvo_cloud* Z,
                              const double* T_init, double* T_out, cvo_info* infos);

/* Frame-to-frame odometry (Sec. IV and V-A): registers frame k+1 onto frame
 * k for k = 0 .. nframes - 2.  The first registration starts from T_first
 * (NULL: identity) with lengthscale ell_first (the paper starts the first
 * frame of a sequence at a larger lengthscale); every later one starts from
 * the previous relative estimate with params.ell, the other parameters as
 * set on the handle.  T_rel (nframes - 1 poses of 16 doubles) receives the
 * motion mapping frame k+1 into frame k; T_abs (nullable, nframes poses)
 * the poses of every frame in frame 0 (T_abs[0] = I, T_abs[k+1] =
 * T_abs[k] T_rel[k]); infos (nullable, nframes - 1) the registrations'
 * summaries.  Returns the worst status (an error stops the sequence). */
cvo_status cvo_register_sequence(cvo_handle h, int nframes, const cvo_cloud* frames, double ell_first,
                                 const double T_first[16], double* T_rel, double* T_abs, cvo_info* infos);

/* X-row shards of one registration, for running a single pair on several
 * GPUs.  The paper uses one GPU; this follows the data-parallel structure of
 * Eq. (double_sum): F and its derivatives are sums over the rows x_i of X,
 * so the rows can be split into disjoint shards, each swept against all of Z
 * on its own GPU, and the per-iteration statistics added before the step.
 *
 * One handle per shard (on that shard's GPU), all created with the same
 * parameters.  Each shard calls
 *   cvo_shard_begin(h, X_rows, Z, n_total, T_init)   once: its rows of X, all
 *       of Z, the number of rows of all shards together (n_total, the N of
 *       the indicator i_theta = F / sqrt(N M), Eq. indicator_actual) and the
 *       common start pose;
 * then for each iteration
 *   cvo_shard_sweep(h, stats)  queues the shard's sweep and writes
 *       CVO_SHARD_STATS doubles to the DEVICE buffer stats on the handle's
 *       stream: the 43 linear statistics of the per-point moments (about the
 *       centre of Z's bounding box, which every shard computes alike), the
 *       pair count and the candidate count;
 *   (the caller sums stats over the shards, elementwise, e.g. an all-reduce
 *       on the handle's stream, so that every shard holds the same sum);
 *   cvo_shard_step(h, stats, done)  queues the step of cvo_register_pair
 *       (step rule, SE(3) update, annealing, stopping test) from the summed
 *       statistics; done (nullable, host): with a non-NULL pointer the call
 *       waits for the step and sets *done = 1 once the registration has
 *       stopped (later sweeps and steps then do nothing);
 * and finally
 *   cvo_shard_end(h, T_out, info)  the final pose and summary, as
 *       cvo_register_pair returns them (the trace through cvo_get_trace).
 * Every shard takes the same steps as long as the summed statistics are the
 * same bits on every shard.  A shard needs at least one row of X and one
 * point of Z, and max_iters >= 1.  The handle's stream orders the calls;
 * stats must stay valid until the step that reads it has run. */
#define CVO_SHARD_STATS 45
cvo_status cvo_shard_begin(cvo_handle h, const cvo_cloud* X_rows, const cvo_cloud* Z, long long n_total,
                           const double T_init[16]);
cvo_status cvo_shard_sweep(cvo_handle h, double* stats_device);
cvo_status cvo_shard_step(cvo_handle h, const double* stats_device, int* done);
cvo_status cvo_shard_end(cvo_handle h, double T_out[16], cvo_info* info);

/* Copies the per-iteration trace of the handle's last registration into out
 * (capacity cap iterations, CVO_TRACE_STRIDE doubles each: l, F, i_theta,
 * |g|, F'' along g, t, |t omega|, |t v|, decayed (0/1), pairs, then the first
 * three rows of the pose the iteration started from) and returns the number
 * of iterations, or a negative cvo_status. */
int cvo_get_trace(cvo_handle h, double* out, int cap);

/* Tuning of the neighbour sweep (performance only; results do not depend on
 * it beyond rounding): grid cell edge = cell_factor * cutoff radius
 * (0.25..4), query groups drawn from octree super-cells about
 * 2^super_delta cutoff radii wide (-2..6).  Defaults 0.5 and 2. */
cvo_status cvo_set_tuning(cvo_handle h, double cell_factor, int super_delta);

/* Tuning of the neighbour sweep: grid cell edge (cell_factor x cutoff
 * radius), query-group extent (octree super-cells about 2^super_delta
 * cutoff radii wide) and the work split (each query group's candidate
 * stream is cut into work items of about chunk_len candidates, so up to
 * length / chunk_len warps serve one query group: evaluations, batches and
 * dense registrations measure the streams at the call's pose, longest
 * first; a single registration with a cutoff measures them again in every
 * sweep and lays out the next sweep's items from them, since its streams
 * follow the moving pose), and the lanes per query of the sweep (1, 2 or 4,
 * default 1: query groups of 32 / query_lanes queries, each query's
 * candidates shared among that many lanes; a block list other than RGB + 19
 * labels, or the feature-space cutoff, keeps one lane per query and leaves
 * the group's other lanes idle).  measured_ms: the time cvo_autotune
 * measured for the tuning it kept, else 0. */
typedef struct {
    double cell_factor;
    int super_delta;
    int chunk_len;
    double measured_ms;
    int query_lanes;   /* 0 is read as 1 */
} cvo_tuning;

/* Autotuner: registers (X, Z) from pose T with the handle's parameters
 * under each tuning of a small grid (cell_factor 0.35 / 0.5 / 0.7 / 1.0 and
 * super_delta 1 / 2 / 3 at the current chunk_len; with cutoff_mult <= 0 there
 * is no grid and these stay as they are), then, for the fastest, query_lanes
 * 1 / 2 / 4, then chunk_len 64 / 96 / 128 / 192 / 384 / 768 / 1536; each
 * timed on the host clock as a
 * caller sees it (setup, iterations, result copies; best of two runs).
 * Keeps the fastest tuning on the handle and returns it in *out
 * (measured_ms: its time).  Results do not depend on the tuning beyond
 * rounding; every tuning's F at the start pose is checked against the first
 * (CVO_ERR_CUDA if they differ by more than 1e-4 relative).  Costs up to 38
 * registrations. */
cvo_status cvo_autotune(cvo_handle h, const cvo_cloud* X, const cvo_cloud* Z, const double T[16], cvo_tuning* out);

/* The same search timed on a batched registration (cvo_register_batch) of
 * the npairs pairs (arguments as there; the results are not returned): a
 * batch fills the device with many pairs' work items, so its best tuning
 * (typically longer items) differs from one pair's.  The check value is the
 * sum over the pairs of F at their start poses.  Costs up to 38 batched
 * registrations. */
cvo_status cvo_autotune_batch(cvo_handle h, int npairs, const cvo_cloud* X, const cvo_cloud* Z, const double* T_init,
                              cvo_tuning* out);

/* The handle's current tuning (measured_ms = 0), and setting it (validated as
 * cvo_set_tuning, chunk_len in [16, 4096], query_lanes 1, 2 or 4). */
cvo_status cvo_get_tuning(cvo_handle h, cvo_tuning* out);
cvo_status cvo_apply_tuning(cvo_handle h, const cvo_tuning* t);

/* How a single-pair registration runs its iterations (batches always use
 * the graph, or the host queue in CVO_LOOP_HOST):
 *   CVO_LOOP_GRAPH (default)  a CUDA graph whose WHILE node repeats
 *       (sweep, step);
 *   CVO_LOOP_PERSISTENT  one cooperative kernel for the whole loop, which
 *       re-plans the work split every iteration, with grid barriers between
 *       plan, sweep and step (bounded waits: CVO_ERR_TIMEOUT if one gives
 *       up);
 *   CVO_LOOP_HOST   the same two kernels queued from the host (what a
 *       profiler can attribute per kernel).
 * Results are deterministic in every mode; GRAPH and HOST are bitwise
 * equal, PERSISTENT sums in another fixed order (same tolerances).  The
 * environment variable CVO_LOOP=graph|persistent|host sets the default of
 * new handles (CVO_GRAPH=0 means host). */
enum { CVO_LOOP_HOST = 0, CVO_LOOP_GRAPH = 1, CVO_LOOP_PERSISTENT = 2 };
cvo_status cvo_set_loop(cvo_handle h, int mode);

/* Failure injection for the persistent loop (CVO_LOOP_PERSISTENT), so that
 * its error path can be tested without a fault: for the handle's next
 * registration only, the last block of the persistent kernel leaves at grid
 * barrier number `barrier` (counted from 0 over the whole loop; three per
 * iteration) instead of arriving, and every grid barrier gives up after
 * poll_limit polls (> 0; about 1 us each) instead of the default of
 * seconds.  The blocks still waiting give up, the kernel returns and the
 * registration reports CVO_ERR_TIMEOUT; the handle stays usable.  No other
 * loop mode is affected; barrier < 0 clears a pending injection.  The paper
 * has no counterpart. */
cvo_status cvo_inject_barrier_stall(cvo_handle h, int barrier, unsigned poll_limit);

/* Device time (ms) of the handle's last registration's sweeps when timing
 * is on (cvo_set_timing): in the graph and host modes CUDA events around
 * each sweep launch (the loop is then queued from the host), average per
 * launch, and the number of launches; in the persistent mode events around
 * the one kernel, i.e. sweep and step together, per iteration, and the
 * number of iterations.  After cvo_backward (or cvo_metric_backward): events
 * around each gradient sweep (one per cloud whose gradients were asked for). */
cvo_status cvo_set_timing(cvo_handle h, int on);
cvo_status cvo_sweep_time(cvo_handle h, double* avg_ms, int* launches);

/* Message of the last error on the calling thread ("" if none). */
const char* cvo_last_error(void);

/* Library version string. */
const char* cvo_version(void);

/* CUDA kernels this library has launched in the calling process (all
 * handles, all threads), for launch accounting by benchmarks. */
long long cvo_kernel_launches(void);

/* Measured throughput of the units the sweep runs on, for roofline
 * denominators.  An addition of this library: the paper has no counterpart.
 * The sweep is bound by FP32 arithmetic and by one ex2 per pair; counting
 * units (SMs x 128 FP32 lanes x 2 x clock) gives a ceiling the hardware may
 * not reach, so this call measures the rates the current device reaches:
 * kernels of independent fma.rn.f32 chains and of ex2.approx.ftz.f32 chains
 * on 8 blocks of 256 threads per SM, each timed with CUDA events on
 * cuda_stream (NULL: legacy default stream), best of 5 launches after one
 * untimed launch; about 20 ms in all.  Synchronous.  out receives the FP32
 * rate in FLOP/s (an FMA counts 2), the ex2 rate in evaluations per second,
 * the best launch times and the SM count.  CVO_ERR_INVALID_ARG for a NULL
 * out, CVO_ERR_CUDA when a launch fails.  Allocates nothing; the figures
 * hold for the clocks the GPU ran at while measured. */
typedef struct {
    double ffma_flops;   /* FP32 FLOP/s of fused multiply-adds */
    double ex2_per_s;    /* ex2.approx.ftz.f32 evaluations per second */
    double ms_ffma, ms_ex2;   /* best launch times */
    int sms;
} cvo_throughput;
cvo_status cvo_measure_throughput(void* cuda_stream, cvo_throughput* out);

/* Dense evaluation that allocates nothing.  This entry point is an addition
 * of this library: the paper has no counterpart.
 *
 * Who needs it: callers that must not allocate device memory once they are
 * running -- a real-time odometry loop that fixed its memory budget at
 * start-up (cudaMalloc / cudaFree can synchronise the device and stall the
 * loop, or fail half way through a run), or a plugin inside a host
 * application whose memory pool owns the GPU.  The handle-based calls above
 * allocate scratch on demand, so they cannot serve these callers.
 *
 * What it computes: the same F, gradient, Hessian, indicator and pair counts
 * as cvo_evaluate with cutoff_mult <= 0 (every pair), with the same kernels.
 * It needs no handle and calls no cudaMalloc, cudaFree or other allocating
 * routine: all scratch lives in one fixed 4.5 MiB array inside the library,
 * which every GPU that loads the library holds until the process exits.
 *
 * Arguments: params as for cvo_create (cutoff_mult must be <= 0); cuda_stream
 * a cudaStream_t (NULL: legacy default stream); X and Z with on_device = 1
 * (device pointers, float32 or bfloat16 features); T a host row-major pose;
 * out_device a DEVICE pointer to one cvo_eval that receives the results.
 *
 * Limits: at most 16384 points per cloud and 24 feature entries per point;
 * larger requests return CVO_ERR_INVALID_ARG with a message naming the limit.
 *
 * Behaviour: asynchronous -- the work is queued on cuda_stream and
 * *out_device is valid once the stream has reached it.  Because the call does
 * not wait for the GPU, non-finite coordinates or features are reported as
 * NaN results, not as an error code.  The first call on each device looks up
 * the array's device address (cudaGetSymbolAddress) and the SM count with
 * that device current; make that first call before any stream capture.
 * Under CUDA's lazy module loading (the default), the library's device code
 * and with it the array may be loaded on a device only at that first call, so
 * the 4.5 MiB are committed then: make one call per device at start-up, while
 * allocating is still allowed, and later calls commit nothing.  Every call reuses the same
 * array, which keeps the previous call's contents (each call rewrites all it
 * reads): calls that overlap on the GPU -- on two streams, or from two host
 * threads on one device -- race and must be serialised by the caller. */
cvo_status cvo_evaluate_dense_noalloc(const cvo_params* params, void* cuda_stream, const cvo_cloud* X,
                                      const cvo_cloud* Z, const double T[16], cvo_eval* out_device);

#ifdef __cplusplus
}
#endif
#endif /* CVO_H */
