/*
 * FP64 CPU oracle for the RKHS registration of "A New Framework for Registration
 * of Semantic Point Clouds from Stereo and RGB-D Cameras" (arXiv:2012.03683).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain, obviously correct
 * reference that the CUDA library is compared against.  Only the tests, the
 * package smoke check and the benchmark's CPU-baseline leg may load it.  It
 * shares no code, header or constant with the CUDA library.
 *
 * Every quantity is computed by brute force over all N x M point pairs in
 * double precision, in the order the definitions state them:
 *
 *   y_j   = R z_j + t                      the pose T = (R, t) maps Z into X's
 *                                          frame; T is the inverse of the h of
 *                                          Problem 1 (Sec. III, Eq. max)
 *   k     = sigma^2 exp(-|x_i - y_j|^2 / (2 l^2))           Eq. (k)
 *   c_ij  = prod_k k_Vk(u_ki, v_kj)        Eq. (tensor_product) / (double_sum)
 *           k_Vk = sigma_k^2 exp(-|u-v|^2/(2 l_k^2))        Eq. (newscalar)
 *                  or <u, v>                                Eq. (scalar)
 *   F     = sum_{pairs} k * c_ij                            Eq. (double_sum)
 *   i_th  = F / sqrt(N M)                                   Eq. (indicator_actual)
 *
 * A pair enters the sum when the cutoff is off (cutoff_mult <= 0) or when
 * |x_i - y_j|^2 <= (cutoff_mult * l)^2 (inclusive, in double precision).  The
 * paper says the sum is sparse (Sec. III-B) but fixes no threshold.  The same
 * passage names pairs far apart in feature space as the other source of
 * sparsity: with feat_cutoff_mult > 0 a pair also needs, for every
 * squared-exponential block k, |u_k - v_k|^2 <= (feat_cutoff_mult * l_k)^2
 * (off by default: it changes F).
 *
 * The gradient, the second derivative, the step rule and the stopping rules
 * are not printed in the paper (it cites gradient ascent on the Lie group,
 * Sec. I).  They are derived here from Eq. (double_sum) for the left
 * perturbation T(xi) = exp(xi^) T, xi = (omega, v):
 *
 *   dF/dv     = (1/l^2) sum w (x_i - y_j)
 *   dF/domega = (1/l^2) sum w (y_j x x_i)
 *   d^2/dt^2 F(exp(t xi^) T) at t=0, with d = omega x y_j + v, e = y_j - x_i:
 *             = sum w [ (e.d)^2 / l^4 - (|d|^2 + e.(omega x d)) / l^2 ]
 *
 * The gradient and the second derivative are pinned by central finite
 * differences of F (tests).  The step rule is a reading (the paper names a
 * step size without a rule, and cites gradient ascent on the Lie group): a
 * line-Newton step along the ascent direction of an origin-free metric,
 * inside a trust region on the motion of Z's points (orc_register).  It, its
 * trust region, its step to the region's edge where F'' >= 0 and the
 * left-composed update are pinned by closed-form Newton iterates on problems
 * whose objective along the ascent direction has one variable, and by the
 * equivariance of the whole registration under a common rigid motion of the
 * inputs.  The annealing
 * trigger and the convergence test (readings of Sec. IV) are pinned on the
 * same problems: there every iteration's indicator, step and decision follow
 * from a scalar formula, and the tests compare the decay iterations, the
 * lengthscales and the stop iteration with that closed form.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_MAX_BLOCKS 4

typedef struct {
    double ell;          /* geometric lengthscale l, Eq. (k) */
    double sigma;        /* sigma of Eq. (k) */
    double cutoff_mult;  /* pairs with |x-y| <= cutoff_mult*l enter; <= 0: all pairs */
    int n_blocks;        /* feature blocks, concatenated per point */
    int dim[ORC_MAX_BLOCKS];
    int kind[ORC_MAX_BLOCKS];     /* 0: squared exponential, Eq. (newscalar); 1: inner product, Eq. (scalar) */
    double scale[ORC_MAX_BLOCKS]; /* l_k of a squared-exponential block */
    double sigk[ORC_MAX_BLOCKS];  /* sigma_k of a squared-exponential block */
    double feat_cutoff_mult;      /* > 0: squared-exponential blocks need |u-v| <= feat_cutoff_mult*l_k */
} orc_kernel;

typedef struct {
    int n;               /* points */
    const double* xyz;   /* n x 3, row major */
    const double* feat;  /* n x D, row major, blocks concatenated (NULL if D == 0) */
} orc_cloud;

static int feat_dim(const orc_kernel* k)
{
    int d = 0;
    for (int b = 0; b < k->n_blocks; ++b) d += k->dim[b];
    return d;
}

/* c_ij of Eq. (double_sum): the product over blocks of each block's kernel. */
static double feature_kernel(const orc_kernel* k, const double* u, const double* v)
{
    double c = 1.0;
    int off = 0;
    for (int b = 0; b < k->n_blocks; ++b) {
        const int d = k->dim[b];
        if (k->kind[b] == 0) {
            double s = 0.0;
            for (int a = 0; a < d; ++a) {
                const double diff = u[off + a] - v[off + a];
                s += diff * diff;
            }
            c *= k->sigk[b] * k->sigk[b] * exp(-s / (2.0 * k->scale[b] * k->scale[b]));
        } else {
            double s = 0.0;
            for (int a = 0; a < d; ++a) s += u[off + a] * v[off + a];
            c *= s;
        }
        off += d;
    }
    return c;
}

/* Whether a pair passes the feature-space cutoff (always when it is off). */
static int feature_in(const orc_kernel* k, const double* u, const double* v)
{
    if (!(k->feat_cutoff_mult > 0.0)) return 1;
    int off = 0;
    for (int b = 0; b < k->n_blocks; ++b) {
        const int d = k->dim[b];
        if (k->kind[b] == 0) {
            double s = 0.0;
            for (int a = 0; a < d; ++a) {
                const double diff = u[off + a] - v[off + a];
                s += diff * diff;
            }
            const double r = k->feat_cutoff_mult * k->scale[b];
            if (!(s <= r * r)) return 0;
        }
        off += d;
    }
    return 1;
}

static void cross3(const double a[3], const double b[3], double out[3])
{
    out[0] = a[1] * b[2] - a[2] * b[1];
    out[1] = a[2] * b[0] - a[0] * b[2];
    out[2] = a[0] * b[1] - a[1] * b[0];
}

static double dot3(const double a[3], const double b[3])
{
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

/*
 * Brute-force evaluation at pose T (row-major 4x4).
 *   out[0]   F                      Eq. (double_sum)
 *   out[1:4] dF/domega              left perturbation
 *   out[4:7] dF/dv
 *   out[7]   d^2F along dir (0 if dir == NULL)
 *   out[8]   sum over pairs of |w (y x x)| + |w (x - y)|, divided by l^2: the
 *            scale of the gradient's terms (for rounding-error bounds)
 * npairs receives the number of pairs inside the cutoff.
 * Returns 0, or -1 on an invalid argument.
 */
int orc_eval(const orc_kernel* k, const orc_cloud* X, const orc_cloud* Z, const double T[16],
             const double* dir, double out[9], long long* npairs, int nthreads)
{
    if (!k || !X || !Z || !T || !out || k->ell <= 0.0 || k->n_blocks < 0 || k->n_blocks > ORC_MAX_BLOCKS)
        return -1;
    const int D = feat_dim(k);
    const double l2 = k->ell * k->ell;
    const double l4 = l2 * l2;
    const double rc2 = k->cutoff_mult > 0.0 ? (k->cutoff_mult * k->ell) * (k->cutoff_mult * k->ell) : -1.0;
    const double s2 = k->sigma * k->sigma;
    double F = 0.0, gw[3] = {0, 0, 0}, gv[3] = {0, 0, 0}, Fpp = 0.0, gab = 0.0;
    long long cnt = 0;
    double om[3] = {0, 0, 0}, vv[3] = {0, 0, 0};
    if (dir) {
        om[0] = dir[0]; om[1] = dir[1]; om[2] = dir[2];
        vv[0] = dir[3]; vv[1] = dir[4]; vv[2] = dir[5];
    }
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
    /* Per-point partial sums, then one ordered sum: the result does not depend
       on the thread count or schedule. */
    double* part = (double*)calloc((size_t)(X->n > 0 ? X->n : 1) * 9, sizeof(double));
    long long* pcnt = (long long*)calloc((size_t)(X->n > 0 ? X->n : 1), sizeof(long long));
    if (!part || !pcnt) {
        free(part);
        free(pcnt);
        return -1;
    }
#pragma omp parallel for schedule(dynamic, 16)
    for (int i = 0; i < X->n; ++i) {
        const double* x = X->xyz + 3 * (size_t)i;
        double Fi = 0.0, gwi[3] = {0, 0, 0}, gvi[3] = {0, 0, 0}, Fppi = 0.0, gabi = 0.0;
        long long ci = 0;
        for (int j = 0; j < Z->n; ++j) {
            const double* z = Z->xyz + 3 * (size_t)j;
            double y[3];
            for (int r = 0; r < 3; ++r) y[r] = T[4 * r + 0] * z[0] + T[4 * r + 1] * z[1] + T[4 * r + 2] * z[2] + T[4 * r + 3];
            const double e[3] = {y[0] - x[0], y[1] - x[1], y[2] - x[2]};
            const double d2 = dot3(e, e);
            if (rc2 >= 0.0 && !(d2 <= rc2)) continue;
            if (D > 0 && !feature_in(k, X->feat + (size_t)D * i, Z->feat + (size_t)D * j)) continue;
            double c = 1.0;
            if (D > 0) c = feature_kernel(k, X->feat + (size_t)D * i, Z->feat + (size_t)D * j);
            const double w = s2 * exp(-d2 / (2.0 * l2)) * c;
            ci += 1;
            Fi += w;
            double yx[3];
            cross3(y, x, yx);
            for (int r = 0; r < 3; ++r) {
                gwi[r] += w * yx[r] / l2;
                gvi[r] += -w * e[r] / l2;
            }
            gabi += fabs(w) * (sqrt(dot3(yx, yx)) + sqrt(d2)) / l2;
            if (dir) {
                double d[3], od[3];
                cross3(om, y, d);
                d[0] += vv[0]; d[1] += vv[1]; d[2] += vv[2];
                cross3(om, d, od);
                const double ed = dot3(e, d);
                Fppi += w * (ed * ed / l4 - (dot3(d, d) + dot3(e, od)) / l2);
            }
        }
        double* p = part + 9 * (size_t)i;
        p[0] = Fi;
        p[1] = gwi[0]; p[2] = gwi[1]; p[3] = gwi[2];
        p[4] = gvi[0]; p[5] = gvi[1]; p[6] = gvi[2];
        p[7] = Fppi;
        p[8] = gabi;
        pcnt[i] = ci;
    }
    for (int i = 0; i < X->n; ++i) {
        const double* p = part + 9 * (size_t)i;
        F += p[0];
        gw[0] += p[1]; gw[1] += p[2]; gw[2] += p[3];
        gv[0] += p[4]; gv[1] += p[5]; gv[2] += p[6];
        Fpp += p[7];
        gab += p[8];
        cnt += pcnt[i];
    }
    free(part);
    free(pcnt);
    out[0] = F;
    out[1] = gw[0]; out[2] = gw[1]; out[3] = gw[2];
    out[4] = gv[0]; out[5] = gv[1]; out[6] = gv[2];
    out[7] = Fpp;
    out[8] = gab;
    if (npairs) *npairs = cnt;
    return 0;
}

/* Number of pairs whose squared distance lies within [lo, hi] (cutoff-boundary census). */
long long orc_count_band(const orc_cloud* X, const orc_cloud* Z, const double T[16], double lo, double hi)
{
    long long cnt = 0;
#pragma omp parallel for schedule(static) reduction(+ : cnt)
    for (int i = 0; i < X->n; ++i) {
        const double* x = X->xyz + 3 * (size_t)i;
        for (int j = 0; j < Z->n; ++j) {
            const double* z = Z->xyz + 3 * (size_t)j;
            double d2 = 0.0;
            for (int r = 0; r < 3; ++r) {
                const double y = T[4 * r + 0] * z[0] + T[4 * r + 1] * z[1] + T[4 * r + 2] * z[2] + T[4 * r + 3];
                d2 += (y - x[r]) * (y - x[r]);
            }
            if (d2 >= lo && d2 <= hi) cnt += 1;
        }
    }
    return cnt;
}

/* ------------------------------------------------------------------------ */
/* SE(3): closed-form exponential and logarithm (textbook, e.g. Murray, Li  */
/* and Sastry), xi = (omega, v), hat(xi) = [[omega]x, v; 0, 0].             */
/* ------------------------------------------------------------------------ */

/* A = sin(th)/th, B = (1-cos th)/th^2, C = (th - sin th)/th^3.
 * A and B take their Taylor series below 1e-3; above it B is written as
 * 2 sin^2(th/2)/th^2, the same quantity without the cancellation of 1 - cos.
 * The difference th - sin th cancels for small th (about 7 digits at 1e-3),
 * so C takes its Taylor series below 0.1, to the th^8 term (the first term
 * left out is below 1e-19 there). */
static void se3_coeffs(double th, double* A, double* B, double* C)
{
    const double t2 = th * th;
    if (th < 1e-3) {
        *A = 1.0 - t2 / 6.0 + t2 * t2 / 120.0;
        *B = 0.5 - t2 / 24.0 + t2 * t2 / 720.0;
    } else {
        const double h = sin(0.5 * th);
        *A = sin(th) / th;
        *B = 2.0 * h * h / t2;
    }
    if (th < 0.1)
        *C = 1.0 / 6.0 - t2 / 120.0 + t2 * t2 / 5040.0 - t2 * t2 * t2 / 362880.0 + t2 * t2 * t2 * t2 / 39916800.0;
    else
        *C = (th - sin(th)) / (t2 * th);
}

void orc_se3_exp(const double xi[6], double T[16])
{
    const double* w = xi;
    const double* v = xi + 3;
    const double th = sqrt(dot3(w, w));
    double A, B, C;
    se3_coeffs(th, &A, &B, &C);
    const double W[9] = {0, -w[2], w[1], w[2], 0, -w[0], -w[1], w[0], 0};
    double W2[9];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
            double s = 0.0;
            for (int q = 0; q < 3; ++q) s += W[3 * r + q] * W[3 * q + c];
            W2[3 * r + c] = s;
        }
    for (int r = 0; r < 3; ++r) {
        double tr = 0.0;
        for (int c = 0; c < 3; ++c) {
            const double I = (r == c) ? 1.0 : 0.0;
            T[4 * r + c] = I + A * W[3 * r + c] + B * W2[3 * r + c];
            tr += (I + B * W[3 * r + c] + C * W2[3 * r + c]) * v[c];
        }
        T[4 * r + 3] = tr;
    }
    T[12] = 0.0; T[13] = 0.0; T[14] = 0.0; T[15] = 1.0;
}

/* Logarithm for rotation angles below pi.  Returns 0, or -1 near pi. */
int orc_se3_log(const double T[16], double xi[6])
{
    const double tr = T[0] + T[5] + T[10];
    double c = 0.5 * (tr - 1.0);
    if (c > 1.0) c = 1.0;
    if (c < -1.0) c = -1.0;
    const double th = acos(c);
    if (th > M_PI - 1e-6) return -1;
    const double vee[3] = {T[9] - T[6], T[2] - T[8], T[4] - T[1]};
    double f; /* omega = f * vee, f = th / (2 sin th) */
    if (th < 1e-4) f = 0.5 + th * th / 12.0;
    else f = th / (2.0 * sin(th));
    const double w[3] = {f * vee[0], f * vee[1], f * vee[2]};
    double A, B, C;
    se3_coeffs(th, &A, &B, &C);
    /* V^{-1} = I - W/2 + (1/th^2)(1 - A/(2B)) W^2 */
    double k2;
    if (th < 1e-3) k2 = 1.0 / 12.0 + th * th / 720.0;
    else k2 = (1.0 - A / (2.0 * B)) / (th * th);
    const double W[9] = {0, -w[2], w[1], w[2], 0, -w[0], -w[1], w[0], 0};
    const double t[3] = {T[3], T[7], T[11]};
    for (int r = 0; r < 3; ++r) {
        double s = 0.0;
        for (int q = 0; q < 3; ++q) {
            double W2rq = 0.0;
            for (int p = 0; p < 3; ++p) W2rq += W[3 * r + p] * W[3 * p + q];
            const double I = (r == q) ? 1.0 : 0.0;
            s += (I - 0.5 * W[3 * r + q] + k2 * W2rq) * t[q];
        }
        xi[3 + r] = s;
    }
    xi[0] = w[0]; xi[1] = w[1]; xi[2] = w[2];
    return 0;
}

static void mat4_mul(const double A[16], const double B[16], double C[16])
{
    double tmp[16];
    for (int r = 0; r < 4; ++r)
        for (int c = 0; c < 4; ++c) {
            double s = 0.0;
            for (int q = 0; q < 4; ++q) s += A[4 * r + q] * B[4 * q + c];
            tmp[4 * r + c] = s;
        }
    memcpy(C, tmp, sizeof(tmp));
}

/* Gram-Schmidt on the columns of R (keeps det R = +1). */
static void reorthonormalize(double T[16])
{
    double c0[3] = {T[0], T[4], T[8]}, c1[3] = {T[1], T[5], T[9]}, c2[3];
    double n0 = sqrt(dot3(c0, c0));
    for (int r = 0; r < 3; ++r) c0[r] /= n0;
    const double p = dot3(c0, c1);
    for (int r = 0; r < 3; ++r) c1[r] -= p * c0[r];
    double n1 = sqrt(dot3(c1, c1));
    for (int r = 0; r < 3; ++r) c1[r] /= n1;
    cross3(c0, c1, c2);
    for (int r = 0; r < 3; ++r) {
        T[4 * r + 0] = c0[r];
        T[4 * r + 1] = c1[r];
        T[4 * r + 2] = c2[r];
    }
}

/* ------------------------------------------------------------------------ */
/* Registration loop                                                        */
/* ------------------------------------------------------------------------ */

typedef struct {
    double ell_init, ell_min;     /* lengthscale schedule */
    double decay;                 /* l <- max(decay*l, ell_min) when the indicator stabilises (Sec. IV: 2 %) */
    double indicator_tol;         /* |i_k - i_ref| < tol * |i_ref| counts as "stabilised" */
    int max_iters;
    int anneal;
    double step_tol_rot, step_tol_trans;   /* convergence: |t omega| and |t v| below these */
    double max_step_rot;                   /* clamp |t omega| (rad) */
    double max_step_trans;                 /* clamp |t v| (m); <= 0: 0.5 * current l */
} orc_reg;

typedef struct {
    int iters;
    int status;          /* 0 converged, 1 iteration cap */
    double ell_final, F, i_theta, last_step_rot, last_step_trans;
    long long pairs_total;
} orc_info;

#define ORC_TRACE_STRIDE 22 /* ell, F, i_theta, sqrt(F'), Fpp, t, |t omega|, |t u|, decayed, pairs, rows 0-2 of T_k */

/*
 * Gradient ascent on SE(3), one line-Newton step along the ascent direction
 * per iteration inside a trust region, with the lengthscale annealing of
 * Sec. IV.
 *
 * The ascent direction is the gradient in a metric on se(3) that does not
 * depend on where the origin of the coordinates lies: perturbations are
 * written about the moved centroid p = R zbar + t of Z, eta = (omega, u) with
 * u the velocity of p (xi = (omega, u + p x omega)), and measured by
 * |eta|^2 = rho^2 |omega|^2 + |u|^2 with rho^2 the mean squared distance of
 * Z's points from zbar plus l^2 (finite for a cloud of one point).  In these
 * coordinates the gradient is h = (g_omega + g_v x p, g_v), the ascent
 * direction d = (h_omega / rho^2, h_u), and F' = h.d.
 * The trust region bounds how far any point of Z moves in one step,
 * t (|omega| R + |u|) <= delta, R the largest distance of a point of Z from
 * zbar, delta = max_step_trans (> 0) or half the lengthscale; and the
 * rotation, t |omega| <= max_step_rot.
 *
 * Iteration k at pose T_k and lengthscale l_k:
 *   1. F, g, the ascent direction d, and the second derivative F'' along d
 *      (brute force).
 *   2. i_k = F / sqrt(N M), Eq. (indicator_actual).
 *   3. Step: t = F' / (-F'') if F'' < 0, else the trust region's edge; in
 *      both cases at most the trust region's edge.
 *   4. T_{k+1} = exp(t d^) T_k (d as xi); Gram-Schmidt on R every 16 iterations.
 *   5. Stop (converged) if annealing is off or l_k == ell_min, and
 *      |t omega| < step_tol_rot and |t u| < step_tol_trans.
 *   6. Annealing: if a reference indicator i_ref at l_k exists and
 *      |i_k - i_ref| < tol |i_ref|, then l_{k+1} = max(decay l_k, ell_min) and
 *      the reference is cleared; otherwise i_ref = i_k.
 * replay (optional, max_iters entries): when given, replay[k] in {0,1} forces
 * the decay decision of step 6 instead of the indicator test.
 * trace (optional, max_iters x ORC_TRACE_STRIDE doubles) records each iteration,
 * including the first three rows of the pose T_k the iteration started from.
 */
int orc_register(const orc_kernel* kin, const orc_reg* r, const orc_cloud* X, const orc_cloud* Z,
                 const double T_init[16], double T_out[16], orc_info* info, double* trace,
                 const int* replay, int nthreads)
{
    if (!kin || !r || !X || !Z || !T_init || !T_out || r->max_iters < 0) return -1;
    orc_kernel k = *kin;
    double T[16];
    memcpy(T, T_init, sizeof(T));
    double ell = r->ell_init;
    int have_ref = 0;
    double i_ref = 0.0;
    const double norm = (X->n > 0 && Z->n > 0) ? 1.0 / sqrt((double)X->n * (double)Z->n) : 0.0;
    /* centroid of Z, mean squared and largest distance of its points from it */
    double zbar[3] = {0.0, 0.0, 0.0}, r2 = 0.0, rmax = 0.0;
    for (int j = 0; j < Z->n; ++j)
        for (int a = 0; a < 3; ++a) zbar[a] += Z->xyz[3 * (size_t)j + a];
    for (int a = 0; a < 3; ++a) zbar[a] = Z->n > 0 ? zbar[a] / Z->n : 0.0;
    for (int j = 0; j < Z->n; ++j) {
        const double* z = Z->xyz + 3 * (size_t)j;
        const double e[3] = {z[0] - zbar[0], z[1] - zbar[1], z[2] - zbar[2]};
        const double q = dot3(e, e);
        r2 += q;
        if (sqrt(q) > rmax) rmax = sqrt(q);
    }
    if (Z->n > 0) r2 /= Z->n;
    orc_info inf;
    memset(&inf, 0, sizeof(inf));
    inf.status = 1;
    int it;
    for (it = 0; it < r->max_iters; ++it) {
        k.ell = ell;
        double out[9];
        double T_k[16];
        memcpy(T_k, T, sizeof(T_k));
        long long np = 0;
        orc_eval(&k, X, Z, T, NULL, out, &np, nthreads);
        double g[6];
        memcpy(g, out + 1, sizeof(g));
        /* the gradient about the moved centroid p, and the ascent direction
           d in the origin's coordinates xi = (omega, u + p x omega) */
        double p[3];
        for (int a = 0; a < 3; ++a) p[a] = T[4 * a] * zbar[0] + T[4 * a + 1] * zbar[1] + T[4 * a + 2] * zbar[2] + T[4 * a + 3];
        double hw[3], hu[3], gvxp[3];
        cross3(g + 3, p, gvxp);
        for (int a = 0; a < 3; ++a) {
            hw[a] = g[a] + gvxp[a];
            hu[a] = g[3 + a];
        }
        const double rho2 = r2 + ell * ell;
        double dw[3], pxw[3], d[6];
        for (int a = 0; a < 3; ++a) dw[a] = hw[a] / rho2;
        cross3(p, dw, pxw);
        for (int a = 0; a < 3; ++a) {
            d[a] = dw[a];
            d[3 + a] = hu[a] + pxw[a];
        }
        const double Fp = dot3(hw, dw) + dot3(hu, hu);   /* F' along d */
        /* second derivative along d */
        orc_eval(&k, X, Z, T, d, out, NULL, nthreads);
        const double F = out[0], Fpp = out[7];
        const double ith = F * norm;
        const double wn = sqrt(dot3(dw, dw)), un = sqrt(dot3(hu, hu));
        double t = 0.0;
        if (Fp > 0.0) {
            const double delta = r->max_step_trans > 0.0 ? r->max_step_trans : 0.5 * ell;
            const double m = wn * rmax + un;   /* bound on the speed of Z's points along d */
            double tmax = m > 0.0 ? delta / m : HUGE_VAL;
            if (wn > 0.0 && tmax * wn > r->max_step_rot) tmax = r->max_step_rot / wn;
            t = (Fpp < 0.0) ? Fp / (-Fpp) : tmax;
            if (t > tmax) t = tmax;
        }
        double xi[6], E[16];
        for (int q = 0; q < 6; ++q) xi[q] = t * d[q];
        orc_se3_exp(xi, E);
        mat4_mul(E, T, T);
        if ((it + 1) % 16 == 0) reorthonormalize(T);
        const double srot = t * wn;
        const double strans = t * un;
        const double gn = sqrt(Fp);
        inf.pairs_total += np;
        inf.F = F;
        inf.i_theta = ith;
        inf.last_step_rot = srot;
        inf.last_step_trans = strans;
        inf.ell_final = ell;
        int decayed = 0;
        const int at_floor = !r->anneal || ell <= r->ell_min;
        const int converged = at_floor && srot < r->step_tol_rot && strans < r->step_tol_trans;
        if (!converged && r->anneal && ell > r->ell_min) {
            int fire;
            if (replay) fire = replay[it] != 0;
            else fire = have_ref && fabs(ith - i_ref) < r->indicator_tol * fabs(i_ref);
            if (fire) {
                ell = r->decay * ell;
                if (ell < r->ell_min) ell = r->ell_min;
                have_ref = 0;
                decayed = 1;
            } else {
                i_ref = ith;
                have_ref = 1;
            }
        }
        if (trace) {
            double* tr = trace + (size_t)ORC_TRACE_STRIDE * it;
            tr[0] = k.ell; tr[1] = F; tr[2] = ith; tr[3] = gn; tr[4] = Fpp;
            tr[5] = t; tr[6] = srot; tr[7] = strans; tr[8] = decayed; tr[9] = (double)np;
            for (int q = 0; q < 12; ++q) tr[10 + q] = T_k[q];
        }
        if (converged) {
            inf.status = 0;
            ++it;
            break;
        }
    }
    inf.iters = it;
    memcpy(T_out, T, sizeof(T));
    if (info) *info = inf;
    return 0;
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Gradients of F with respect to the inputs (derived from Eq. double_sum   */
/* for the pairs inside the cutoff; the pair set is held fixed, i.e. the    */
/* derivative almost everywhere).  With w = sigma^2 exp(-d^2/(2 l^2)) c_ij,  */
/* y_j = R z_j + t, d = |x_i - y_j|:                                        */
/*   dF/dx_i = sum_j w (y_j - x_i) / l^2                                    */
/*   dF/dz_j = R^T sum_i w (x_i - y_j) / l^2                                */
/*   dF/dl   = sum w d^2 / l^3                                              */
/*   squared-exponential block b:  dF/du_bi = -sum_j w (u_bi - v_bj) / l_b^2 */
/*   inner-product block b:        dF/du_bi = sum_j w_(b) v_bj, with w_(b)  */
/*     the weight with block b's factor left out (the other blocks' product) */
/* and the same with the roles of (x, u) and (z, v) exchanged.              */
/* Pinned by central finite differences of F (tests).                       */
/* ------------------------------------------------------------------------ */

/* weight of pair (i, j) with block `skip` left out (skip < 0: full weight) */
static double pair_weight(const orc_kernel* k, double d2, const double* u, const double* v, int skip)
{
    double c = k->sigma * k->sigma * exp(-d2 / (2.0 * k->ell * k->ell));
    int off = 0;
    for (int b = 0; b < k->n_blocks; ++b) {
        const int d = k->dim[b];
        if (b != skip) {
            if (k->kind[b] == 0) {
                double s = 0.0;
                for (int a = 0; a < d; ++a) s += (u[off + a] - v[off + a]) * (u[off + a] - v[off + a]);
                c *= k->sigk[b] * k->sigk[b] * exp(-s / (2.0 * k->scale[b] * k->scale[b]));
            } else {
                double s = 0.0;
                for (int a = 0; a < d; ++a) s += u[off + a] * v[off + a];
                c *= s;
            }
        }
        off += d;
    }
    return c;
}

/* gradient of the pair's weight with respect to the first point's features */
static void feature_grad(const orc_kernel* k, double d2, const double* u, const double* v, double w, double* g)
{
    int off = 0;
    for (int b = 0; b < k->n_blocks; ++b) {
        const int d = k->dim[b];
        if (k->kind[b] == 0) {
            for (int a = 0; a < d; ++a) g[off + a] += -w * (u[off + a] - v[off + a]) / (k->scale[b] * k->scale[b]);
        } else {
            const double wb = pair_weight(k, d2, u, v, b);
            for (int a = 0; a < d; ++a) g[off + a] += wb * v[off + a];
        }
        off += d;
    }
}

int orc_backward(const orc_kernel* k, const orc_cloud* X, const orc_cloud* Z, const double T[16], double* dX,
                 double* dFX, double* dZ, double* dFZ, double* dell, int nthreads)
{
    if (!k || !X || !Z || !T || k->ell <= 0.0) return -1;
    const int D = feat_dim(k);
    const double l2 = k->ell * k->ell, l3 = l2 * k->ell;
    const double rc2 = k->cutoff_mult > 0.0 ? (k->cutoff_mult * k->ell) * (k->cutoff_mult * k->ell) : -1.0;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
    double* dl_part = (double*)calloc((size_t)(X->n > 0 ? X->n : 1), sizeof(double));
    if (!dl_part) return -1;
    /* X side: loop i outer */
#pragma omp parallel for schedule(dynamic, 16)
    for (int i = 0; i < X->n; ++i) {
        const double* x = X->xyz + 3 * (size_t)i;
        const double* u = D > 0 ? X->feat + (size_t)D * i : NULL;
        double gx[3] = {0, 0, 0}, dl = 0.0;
        double* gu = dFX ? dFX + (size_t)D * i : NULL;
        if (gu) for (int a = 0; a < D; ++a) gu[a] = 0.0;
        for (int j = 0; j < Z->n; ++j) {
            const double* z = Z->xyz + 3 * (size_t)j;
            double y[3], e[3];
            for (int r = 0; r < 3; ++r) {
                y[r] = T[4 * r + 0] * z[0] + T[4 * r + 1] * z[1] + T[4 * r + 2] * z[2] + T[4 * r + 3];
                e[r] = y[r] - x[r];
            }
            const double d2 = dot3(e, e);
            if (rc2 >= 0.0 && !(d2 <= rc2)) continue;
            const double* v = D > 0 ? Z->feat + (size_t)D * j : NULL;
            if (D > 0 && !feature_in(k, u, v)) continue;
            const double w = pair_weight(k, d2, u, v, -1);
            for (int r = 0; r < 3; ++r) gx[r] += w * e[r] / l2;
            dl += w * d2 / l3;
            if (gu) feature_grad(k, d2, u, v, w, gu);
        }
        if (dX) for (int r = 0; r < 3; ++r) dX[3 * (size_t)i + r] = gx[r];
        dl_part[i] = dl;
    }
    double dls = 0.0;
    for (int i = 0; i < X->n; ++i) dls += dl_part[i];
    free(dl_part);
    if (dell) *dell = dls;
    /* Z side: loop j outer */
#pragma omp parallel for schedule(dynamic, 16)
    for (int j = 0; j < Z->n; ++j) {
        const double* z = Z->xyz + 3 * (size_t)j;
        const double* v = D > 0 ? Z->feat + (size_t)D * j : NULL;
        double y[3];
        for (int r = 0; r < 3; ++r) y[r] = T[4 * r + 0] * z[0] + T[4 * r + 1] * z[1] + T[4 * r + 2] * z[2] + T[4 * r + 3];
        double gy[3] = {0, 0, 0};
        double* gv = dFZ ? dFZ + (size_t)D * j : NULL;
        if (gv) for (int a = 0; a < D; ++a) gv[a] = 0.0;
        for (int i = 0; i < X->n; ++i) {
            const double* x = X->xyz + 3 * (size_t)i;
            const double e[3] = {y[0] - x[0], y[1] - x[1], y[2] - x[2]};
            const double d2 = dot3(e, e);
            if (rc2 >= 0.0 && !(d2 <= rc2)) continue;
            const double* u = D > 0 ? X->feat + (size_t)D * i : NULL;
            if (D > 0 && !feature_in(k, u, v)) continue;
            const double w = pair_weight(k, d2, u, v, -1);
            for (int r = 0; r < 3; ++r) gy[r] += -w * e[r] / l2;
            if (gv) feature_grad(k, d2, v, u, w, gv);
        }
        if (dZ) /* dF/dz = R^T dF/dy */
            for (int c = 0; c < 3; ++c) dZ[3 * (size_t)j + c] = T[c] * gy[0] + T[4 + c] * gy[1] + T[8 + c] * gy[2];
    }
    return 0;
}
