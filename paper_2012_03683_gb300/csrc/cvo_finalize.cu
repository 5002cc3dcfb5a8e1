// One block per iteration: reduces the sweep's per-block statistics and takes
// the step on the device, so a registration never waits on the host.
//
// 1. Sums the 43 statistics over the sweep blocks in double-float (hi + lo
//    FP32 pairs, error-free two-sum), one warp per statistic, in block order:
//    deterministic, and as accurate as FP64 accumulation at FP32 speed.
// 2. In FP64 (one thread): F = kappa S_W; the gradient of
//    eta -> F(T exp(eta^)) about the lever centre c in Z's frame, mapped to
//    the left perturbation exp(xi^) T.  With gc = (gc_w, gc_v) the centred
//    gradient, R, t the pose:  g_v = R gc_v,  g_w = R (gc_w + c x gc_v) + t x g_v.
//    The indicator of Eq. (indicator_actual) is F / sqrt(N M).
// 3. Registration: the step along the gradient (the method is gradient ascent
//    on SE(3), Sec. I), t = |g|^2 / -F'' with F'' = g^T H g when negative,
//    else 1e-3 / |g|; the clamps; T <- exp(t g^) T (closed-form SE(3)
//    exponential, Rodrigues + left Jacobian); Gram-Schmidt on R every 16
//    iterations; the stopping test; the lengthscale annealing of Sec. IV
//    (l <- max(decay l, l_min) once the indicator at the current l changes by
//    less than indicator_tol relative).  F'' is the quadratic form of the
//    centred Hessian at (w~, v~) = (R^T g_w, -c x w~ + R^T (g_v - t x g_w)).
// 4. Writes the derived constants of the next sweep (double-float T^-1,
//    exponent scale, cutoff, grid level).
// An evaluation (no step) also assembles the full 6x6 Hessian.
//
// GB300 runs FP64 at 1/72 of the FP32 rate, so this serial code is kept to
// closed forms (no 6x6 products on the registration path).
#include <math.h>

#include "cvo_internal.cuh"

namespace cvo {
namespace {

__device__ __forceinline__ void df_add(float& hi, float& lo, float bh, float bl)
{
    const float s = __fadd_rn(hi, bh);
    const float bb = __fsub_rn(s, hi);
    float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(bh, bb));
    e = __fadd_rn(e, __fadd_rn(lo, bl));
    hi = __fadd_rn(s, e);
    lo = __fsub_rn(e, __fsub_rn(hi, s));
}

__device__ __forceinline__ void split_df(double v, float& hi, float& lo)
{
    hi = (float)v;
    lo = (float)(v - (double)hi);
}

struct V3 {
    double x, y, z;
};
__device__ __forceinline__ V3 v3(double x, double y, double z) { return {x, y, z}; }
__device__ __forceinline__ V3 cross(V3 a, V3 b) { return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x}; }
__device__ __forceinline__ double dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ V3 add(V3 a, V3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
__device__ __forceinline__ V3 sub(V3 a, V3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ V3 scale(V3 a, double s) { return {a.x * s, a.y * s, a.z * s}; }
// R a and R^T a with R the rotation block of a row-major 4x4 pose
__device__ __forceinline__ V3 rmul(const double* T, V3 a)
{
    return {T[0] * a.x + T[1] * a.y + T[2] * a.z, T[4] * a.x + T[5] * a.y + T[6] * a.z,
            T[8] * a.x + T[9] * a.y + T[10] * a.z};
}
__device__ __forceinline__ V3 rtmul(const double* T, V3 a)
{
    return {T[0] * a.x + T[4] * a.y + T[8] * a.z, T[1] * a.x + T[5] * a.y + T[9] * a.z,
            T[2] * a.x + T[6] * a.y + T[10] * a.z};
}
// a^T M b with M symmetric from (xx, yy, zz, xy, xz, yz)
__device__ __forceinline__ double symq(const double* m, V3 a, V3 b)
{
    return m[0] * a.x * b.x + m[1] * a.y * b.y + m[2] * a.z * b.z + m[3] * (a.x * b.y + a.y * b.x) +
           m[4] * (a.x * b.z + a.z * b.x) + m[5] * (a.y * b.z + a.z * b.y);
}
// a^T M b with M full 3x3 row major
__device__ __forceinline__ double fullq(const double* m, V3 a, V3 b)
{
    return a.x * (m[0] * b.x + m[1] * b.y + m[2] * b.z) + a.y * (m[3] * b.x + m[4] * b.y + m[5] * b.z) +
           a.z * (m[6] * b.x + m[7] * b.y + m[8] * b.z);
}

// sin(th)/th, (1 - cos th)/th^2, (th - sin th)/th^3: Taylor series in th^2
// (alternating series, truncation below 1e-19 for th < 0.5), else sincos.
__device__ void se3_coeffs(double th2, double& a, double& b, double& c)
{
    if (th2 < 0.25) {
        // Horner in th^2 over 1/(2k+1)!, 1/(2k+2)!, 1/(2k+3)!, k = 8 .. 0
        double pa = 1.0 / 355687428096000.0, pb = 1.0 / 6402373705728000.0, pc = 1.0 / 121645100408832000.0;
        const double fa[8] = {1.0 / 1307674368000.0, 1.0 / 6227020800.0, 1.0 / 39916800.0, 1.0 / 362880.0,
                              1.0 / 5040.0, 1.0 / 120.0, 1.0 / 6.0, 1.0};
        const double fb[8] = {1.0 / 20922789888000.0, 1.0 / 87178291200.0, 1.0 / 479001600.0, 1.0 / 3628800.0,
                              1.0 / 40320.0, 1.0 / 720.0, 1.0 / 24.0, 1.0 / 2.0};
        const double fc[8] = {1.0 / 355687428096000.0, 1.0 / 1307674368000.0, 1.0 / 6227020800.0,
                              1.0 / 39916800.0, 1.0 / 362880.0, 1.0 / 5040.0, 1.0 / 120.0, 1.0 / 6.0};
        for (int k = 0; k < 8; ++k) {
            pa = fa[k] - th2 * pa;
            pb = fb[k] - th2 * pb;
            pc = fc[k] - th2 * pc;
        }
        a = pa;
        b = pb;
        c = pc;
    } else {
        const double th = sqrt(th2);
        double s, co;
        sincos(th, &s, &co);
        a = s / th;
        b = (1.0 - co) / th2;
        c = (th - s) / (th2 * th);
    }
}

// exp of xi = (omega, v) in SE(3), row-major 4x4
__device__ void se3_exp_dev(const double xi[6], double E[16])
{
    const V3 w = v3(xi[0], xi[1], xi[2]);
    const V3 v = v3(xi[3], xi[4], xi[5]);
    double a, b, c;
    se3_coeffs(dot(w, w), a, b, c);
    // R = I + a W + b W^2, V v = v + b (w x v) + c (w x (w x v)); W^2 = w w^T - |w|^2 I
    const double ww = dot(w, w);
    const double W[9] = {0.0, -w.z, w.y, w.z, 0.0, -w.x, -w.y, w.x, 0.0};
    const double wv[3] = {w.x, w.y, w.z};
    for (int r = 0; r < 3; ++r)
        for (int q = 0; q < 3; ++q) {
            const double w2 = wv[r] * wv[q] - (r == q ? ww : 0.0);
            E[4 * r + q] = (r == q ? 1.0 : 0.0) + a * W[3 * r + q] + b * w2;
        }
    const V3 wxv = cross(w, v);
    const V3 wxwxv = cross(w, wxv);
    E[3] = v.x + b * wxv.x + c * wxwxv.x;
    E[7] = v.y + b * wxv.y + c * wxwxv.y;
    E[11] = v.z + b * wxv.z + c * wxwxv.z;
    E[12] = 0.0; E[13] = 0.0; E[14] = 0.0; E[15] = 1.0;
}

// T <- E T for rigid motions (last rows (0, 0, 0, 1))
__device__ void compose(const double E[16], double T[16])
{
    double t[12];
    for (int r = 0; r < 3; ++r)
        for (int q = 0; q < 4; ++q)
            t[4 * r + q] = E[4 * r] * T[q] + E[4 * r + 1] * T[4 + q] + E[4 * r + 2] * T[8 + q] + (q == 3 ? E[4 * r + 3] : 0.0);
    for (int k = 0; k < 12; ++k) T[k] = t[k];
}

__device__ void orthonormalize(double T[16])
{
    V3 c0 = v3(T[0], T[4], T[8]), c1 = v3(T[1], T[5], T[9]);
    c0 = scale(c0, 1.0 / sqrt(dot(c0, c0)));
    c1 = sub(c1, scale(c0, dot(c0, c1)));
    c1 = scale(c1, 1.0 / sqrt(dot(c1, c1)));
    const V3 c2 = cross(c0, c1);
    T[0] = c0.x; T[4] = c0.y; T[8] = c0.z;
    T[1] = c1.x; T[5] = c1.y; T[9] = c1.z;
    T[2] = c2.x; T[6] = c2.y; T[10] = c2.z;
}

// Constants the next sweep reads.
__device__ void update_derived(IterState* st)
{
    const double* T = st->T;
    // A = R^T, b = -R^T t
    for (int r = 0; r < 3; ++r) {
        double bv = 0.0;
        for (int q = 0; q < 3; ++q) {
            const double a = T[4 * q + r];
            split_df(a, st->Ahi[3 * r + q], st->Alo[3 * r + q]);
            bv -= a * T[4 * q + 3];
        }
        split_df(bv, st->bhi[r], st->blo[r]);
    }
    const double ell = st->ell;
    st->sg = -1.44269504f / (2.0f * (float)(ell * ell));   // FP32: the sweep uses it in FP32
    if (st->cutoff_mult > 0.0) {
        const double rc = st->cutoff_mult * ell;
        st->rc = (float)rc;
        st->rc2 = (float)(rc * rc);
        int lv = 0;
        for (int k = 1; k < st->nlevels; ++k)
            if ((double)st->level_h[k] >= rc * 1.0001) lv = k;
        st->level = lv;
    } else {
        st->rc = -1.0f;
        st->rc2 = -1.0f;
        st->level = 0;
    }
}

__global__ void k_init_state(IterState* st)
{
    for (int r = 0; r < 3; ++r) split_df(st->c[r], st->chi[r], st->clo[r]);
    update_derived(st);
}

// Full Hessian of xi -> F(exp(xi^) T) (evaluation only): H = B^T Hc B with
// B = [[R^T, 0], [-[c]x R^T - R^T [t]x, R^T]].
__device__ void full_hessian(const double* s, double iL2, double iL4, const double* T, const double* c, double* H)
{
    double Hc[36];
    const double* Q = s + ST_Q;
    const double* PQP = s + ST_PQP;
    const double* Wpp = s + ST_WPP;
    const double* PQ = s + ST_PQ;
    const double* Ep = s + ST_EP;
    const double* E = s + ST_E;
    const double* Wp = s + ST_WP;
    const double W = s[ST_W];
    auto symv = [](const double* m, int r, int q) {
        if (r == q) return m[r];
        const int a = r < q ? r : q, b = r < q ? q : r;
        return a == 0 ? (b == 1 ? m[3] : m[4]) : m[5];
    };
    auto skew = [](const double* a, int r, int q) {
        const double M[9] = {0.0, -a[2], a[1], a[2], 0.0, -a[0], -a[1], a[0], 0.0};
        return M[3 * r + q];
    };
    const double trWpp = Wpp[0] + Wpp[1] + Wpp[2];
    const double trEp = Ep[0] + Ep[4] + Ep[8];
    for (int r = 0; r < 3; ++r)
        for (int q = 0; q < 3; ++q) {
            const double id = (r == q) ? 1.0 : 0.0;
            Hc[6 * r + q] = -symv(PQP, r, q) * iL4 - (trWpp * id - symv(Wpp, r, q)) * iL2 +
                            0.5 * (Ep[3 * r + q] + Ep[3 * q + r] - 2.0 * trEp * id) * iL2;
            const double hwv = PQ[3 * r + q] * iL4 - skew(Wp, r, q) * iL2 - 0.5 * skew(E, r, q) * iL2;
            Hc[6 * r + 3 + q] = hwv;
            Hc[6 * (3 + q) + r] = hwv;
            Hc[6 * (3 + r) + 3 + q] = symv(Q, r, q) * iL4 - W * id * iL2;
        }
    double B[36];
    for (int k = 0; k < 36; ++k) B[k] = 0.0;
    const double tv[3] = {T[3], T[7], T[11]};
    for (int r = 0; r < 3; ++r)
        for (int q = 0; q < 3; ++q) {
            const double rt = T[4 * q + r];
            B[6 * r + q] = rt;
            B[6 * (3 + r) + 3 + q] = rt;
            double a1 = 0.0, a2 = 0.0;
            for (int k = 0; k < 3; ++k) {
                a1 += skew(c, r, k) * T[4 * q + k];
                a2 += T[4 * k + r] * skew(tv, k, q);
            }
            B[6 * (3 + r) + q] = -a1 - a2;
        }
    double HB[36];
    for (int r = 0; r < 6; ++r)
        for (int q = 0; q < 6; ++q) {
            double acc = 0.0;
            for (int k = 0; k < 6; ++k) acc += Hc[6 * r + k] * B[6 * k + q];
            HB[6 * r + q] = acc;
        }
    for (int r = 0; r < 6; ++r)
        for (int q = 0; q < 6; ++q) {
            double acc = 0.0;
            for (int k = 0; k < 6; ++k) acc += B[6 * k + r] * HB[6 * k + q];
            H[6 * r + q] = acc;
        }
}

__global__ void __launch_bounds__(kFinalizeThreads)
k_finalize(IterState* st, const float2* __restrict__ ps, const unsigned long long* __restrict__ pc, int cap, int nb,
           double* trace, cudaGraphConditionalHandle cond, int use_cond)
{
    __shared__ double S[kStatN];
    __shared__ unsigned long long cs[2][kFinalizeThreads / 32];
    if (st->done) {
        // inside a graph's loop: stop it
        if (use_cond && threadIdx.x == 0) cudaGraphSetConditional(cond, 0u);
        return;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int v = warp; v < kStatN; v += kFinalizeThreads / 32) {
        float hi = 0.0f, lo = 0.0f;
        const float2* row = ps + (size_t)v * cap;
        int b = lane;
        for (; b + 96 < nb; b += 128) {   // four loads in flight per lane
            const float2 x0 = row[b], x1 = row[b + 32], x2 = row[b + 64], x3 = row[b + 96];
            df_add(hi, lo, x0.x, x0.y);
            df_add(hi, lo, x1.x, x1.y);
            df_add(hi, lo, x2.x, x2.y);
            df_add(hi, lo, x3.x, x3.y);
        }
        for (; b < nb; b += 32) {
            const float2 x = row[b];
            df_add(hi, lo, x.x, x.y);
        }
        for (int o = 16; o > 0; o >>= 1) {
            const float oh = __shfl_xor_sync(0xffffffffu, hi, o);
            const float ol = __shfl_xor_sync(0xffffffffu, lo, o);
            df_add(hi, lo, oh, ol);
        }
        if (lane == 0) S[v] = (double)hi + (double)lo;
    }
    unsigned long long c0 = 0, c1 = 0;
    for (int b = threadIdx.x; b < nb; b += kFinalizeThreads) {
        c0 += pc[b];
        c1 += pc[(size_t)cap + b];
    }
    for (int o = 16; o > 0; o >>= 1) {
        c0 += __shfl_xor_sync(0xffffffffu, c0, o);
        c1 += __shfl_xor_sync(0xffffffffu, c1, o);
    }
    if (lane == 0) {
        cs[0][warp] = c0;
        cs[1][warp] = c1;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;

    unsigned long long pairs = 0, cands = 0;
    for (int w = 0; w < kFinalizeThreads / 32; ++w) {
        pairs += cs[0][w];
        cands += cs[1][w];
    }
    const double kap = st->kappa;
    const double ell = st->ell, L2 = ell * ell;
    const double iL2 = 1.0 / L2, iL4 = iL2 * iL2;   // one FP64 division (about 660 cycles on GB300)
    const double F = kap * S[ST_W];
    const double* Ep = S + ST_EP;
    // centred gradient (kappa applied here)
    const V3 gcw = scale(v3(Ep[5] - Ep[7], Ep[6] - Ep[2], Ep[1] - Ep[3]), kap * iL2);
    const V3 gcv = scale(v3(S[ST_E], S[ST_E + 1], S[ST_E + 2]), -kap * iL2);
    double* T = st->T;
    const V3 c = v3(st->c[0], st->c[1], st->c[2]);
    const V3 tt = v3(T[3], T[7], T[11]);
    const V3 gv = rmul(T, gcv);
    const V3 gw = add(rmul(T, add(gcw, cross(c, gcv))), cross(tt, gv));
    const double g[6] = {gw.x, gw.y, gw.z, gv.x, gv.y, gv.z};
    const double ith = F * st->norm;
    st->F = F;
    st->i_theta = ith;
    st->pairs = (long long)pairs;
    st->cands = (long long)cands;
    for (int q = 0; q < 6; ++q) st->grad[q] = g[q];

    if (st->mode == 0) {
        double s[kStatN];
        for (int k = 0; k < kStatN; ++k) s[k] = kap * S[k];
        full_hessian(s, iL2, iL4, T, st->c, st->hess);
        st->done = 1;
        if (use_cond) cudaGraphSetConditional(cond, 0u);
        return;
    }

    // ---- registration step --------------------------------------------------
    const int it = st->iter;
    // the gradient direction in the centred coordinates
    const V3 wt = rtmul(T, gw);
    const V3 vt = add(scale(cross(c, wt), -1.0), rtmul(T, sub(gv, cross(tt, gw))));
    // F'' = w~^T Hww w~ + 2 w~^T Hwv v~ + v~^T Hvv v~ (centred Hessian blocks)
    const double trWpp = S[ST_WPP] + S[ST_WPP + 1] + S[ST_WPP + 2];
    const double trEp = Ep[0] + Ep[4] + Ep[8];
    const double ww = dot(wt, wt), vv = dot(vt, vt);
    const double hww = -symq(S + ST_PQP, wt, wt) * iL4 - (trWpp * ww - symq(S + ST_WPP, wt, wt)) * iL2 +
                       (fullq(Ep, wt, wt) - trEp * ww) * iL2;
    const V3 Ev = v3(S[ST_E], S[ST_E + 1], S[ST_E + 2]);
    const V3 Wpv = v3(S[ST_WP], S[ST_WP + 1], S[ST_WP + 2]);
    const double hwv = fullq(S + ST_PQ, wt, vt) * iL4 - (dot(wt, cross(Wpv, vt)) + 0.5 * dot(wt, cross(Ev, vt))) * iL2;
    const double hvv = symq(S + ST_Q, vt, vt) * iL4 - S[ST_W] * vv * iL2;
    const double Fpp = kap * (hww + 2.0 * hwv + hvv);
    double gn2 = 0.0;
    for (int q = 0; q < 6; ++q) gn2 += g[q] * g[q];
    // Norms and clamp ratios only feed thresholds and the step length: FP32
    // square roots and divisions (FP64 ones cost ~700 cycles each here).
    const double wn = (double)sqrtf((float)dot(gw, gw));
    const double vn = (double)sqrtf((float)dot(gv, gv));
    double t = 0.0;
    if (gn2 > 0.0) {
        t = (Fpp < 0.0) ? gn2 / (-Fpp) : 1e-3 / (double)sqrtf((float)gn2);
        const double max_tr = st->max_step_trans > 0.0 ? st->max_step_trans : 0.5 * ell;
        if (t * wn > st->max_step_rot) t = (double)((float)st->max_step_rot / (float)wn);
        if (t * vn > max_tr) t = (double)((float)max_tr / (float)vn);
    }
    double T_k[12];
    for (int q = 0; q < 12; ++q) T_k[q] = T[q];
    double xi[6], Ex[16];
    for (int q = 0; q < 6; ++q) xi[q] = t * g[q];
    se3_exp_dev(xi, Ex);
    compose(Ex, T);
    if ((it + 1) % 16 == 0) orthonormalize(T);
    const double srot = t * wn;
    const double strans = t * vn;
    st->pairs_total += (long long)pairs;
    st->cands_total += (long long)cands;
    st->Fpp = Fpp;
    st->gnorm = (double)sqrtf((float)gn2);
    st->t = t;
    st->srot = srot;
    st->strans = strans;
    const double ell_used = ell;
    const int at_floor = !st->anneal || ell <= st->ell_min;
    const int converged = at_floor && srot < st->step_tol_rot && strans < st->step_tol_trans;
    int decayed = 0;
    if (!converged && st->anneal && ell > st->ell_min) {
        const int fire = st->have_ref && fabs(ith - st->i_ref) < st->indicator_tol * fabs(st->i_ref);
        if (fire) {
            double nl = st->decay * ell;
            if (nl < st->ell_min) nl = st->ell_min;
            st->ell = nl;
            st->have_ref = 0;
            decayed = 1;
        } else {
            st->i_ref = ith;
            st->have_ref = 1;
        }
    }
    st->decayed = decayed;
    if (trace) {
        double* tr = trace + (size_t)kTraceStride * it;
        tr[0] = ell_used; tr[1] = F; tr[2] = ith; tr[3] = st->gnorm; tr[4] = Fpp;
        tr[5] = t; tr[6] = srot; tr[7] = strans; tr[8] = decayed; tr[9] = (double)pairs;
        for (int q = 0; q < 12; ++q) tr[10 + q] = T_k[q];
    }
    st->ell_last = ell_used;
    st->iter = it + 1;
    if (converged) {
        st->status = 0;
        st->done = 1;
    } else if (it + 1 >= st->max_iters) {
        st->status = 1;
        st->done = 1;
    }
    update_derived(st);
    if (use_cond) cudaGraphSetConditional(cond, st->done ? 0u : 1u);
}

}  // namespace

const void* finalize_kernel() { return (const void*)k_finalize; }

cudaError_t launch_init_state(IterState* st, cudaStream_t s)
{
    g_launch_count.fetch_add(1, std::memory_order_relaxed);
    k_init_state<<<1, 1, 0, s>>>(st);
    return cudaGetLastError();
}

cudaError_t launch_finalize(IterState* st, const float2* part_stats, const unsigned long long* part_cnt, int part_cap,
                            int nblocks, double* trace, cudaStream_t s)
{
    g_launch_count.fetch_add(1, std::memory_order_relaxed);
    k_finalize<<<1, kFinalizeThreads, 0, s>>>(st, part_stats, part_cnt, part_cap, nblocks, trace,
                                               cudaGraphConditionalHandle{}, 0);
    return cudaGetLastError();
}

}  // namespace cvo
