// Device code of the registration step (the FP64 pose update, the
// Hessian assembly, the derived constants of the next sweep), shared by the
// finalize kernels and the persistent registration kernel.  See
// cvo_finalize.cu for the method.
#pragma once
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

// An evaluation (no step): F, the gradient, the full Hessian and the
// indicator, by one thread on a shared-memory copy of the state (global
// loads after global stores to the same struct would each wait a full L2
// round trip).
__device__ void take_step(IterState* st, const double* S, unsigned long long pairs, unsigned long long cands)
{
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

    double s[kStatN];
    for (int k = 0; k < kStatN; ++k) s[k] = kap * S[k];
    full_hessian(s, iL2, iL4, T, st->c, st->hess);
    st->done = 1;
}

// Horner coefficients (highest order first) of sin(th)/th, (1 - cos th)/th^2
// and (th - sin th)/th^3 in th^2: 1/(2k+1)!, 1/(2k+2)!, 1/(2k+3)!, k = 8 .. 0.
__constant__ double c_se3_series[3][9] = {
    {1.0 / 355687428096000.0, 1.0 / 1307674368000.0, 1.0 / 6227020800.0, 1.0 / 39916800.0, 1.0 / 362880.0,
     1.0 / 5040.0, 1.0 / 120.0, 1.0 / 6.0, 1.0},
    {1.0 / 6402373705728000.0, 1.0 / 20922789888000.0, 1.0 / 87178291200.0, 1.0 / 479001600.0, 1.0 / 3628800.0,
     1.0 / 40320.0, 1.0 / 720.0, 1.0 / 24.0, 1.0 / 2.0},
    {1.0 / 121645100408832000.0, 1.0 / 355687428096000.0, 1.0 / 1307674368000.0, 1.0 / 6227020800.0,
     1.0 / 39916800.0, 1.0 / 362880.0, 1.0 / 5040.0, 1.0 / 120.0, 1.0 / 6.0}};

// The registration step, run by one warp on the shared-memory state.
// Gradient ascent on SE(3) (Sec. I) with a step size (Sec. III-B), neither
// given by the paper as a formula; the rule taken:
//   direction: the gradient in a metric that names no coordinate origin.
//     Perturbations are written about the moved centroid p = T c of Z,
//     eta = (omega, u) with u the velocity of p, and measured by
//     rho^2 |omega|^2 + |u|^2 (rho^2 = mean squared radius of Z + l^2).  In
//     the centred coordinates of Z's frame this is (w~, v~) = (gc_w / rho^2,
//     gc_v), gc the centred gradient the statistics give directly, and
//     F' = |gc_w|^2 / rho^2 + |gc_v|^2;
//   length: the Newton step F' / -F'' where F'' < 0, else the trust
//     region's edge, and never beyond it: no point of Z moves more than
//     delta = max_step_trans (or l / 2), t (|w~| r_max + |v~|) <= delta, and
//     t |w~| <= max_step_rot;
//   update: T <- exp(t xi^) T with xi = (R w~, R v~ + p x R w~);
//   stop: |t w~| < step_tol_rot and |t v~| < step_tol_trans at the floor.
// GB300 issues an FP64 warp instruction in about 80 cycles whether one lane
// or all 32 are active, so the pose arithmetic (FP64) is spread over lanes:
// the three exponential coefficients on lanes 0-2, the exponential's and the
// new pose's 12 entries on lanes 0-11, the 12 derived constants on lanes
// 0-11.  The direction, F'' along it and the step length come from the
// double-float sums in FP32: they set a direction and a length, while the
// pose they update stays in FP64.
__device__ void step_warp(IterState* st, const double* S, const float* Shi, const float* Slo,
                          unsigned long long pairs, unsigned long long cands, double* trace)
{
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    auto sf = [&](int k) { return Shi[k] + Slo[k]; };
    const int it = st->iter;
    const float ellf = (float)st->ell;
    const float il2 = 1.0f / (ellf * ellf), il4 = il2 * il2;
    const float kapf = (float)st->kappa;
    const float kl = kapf * il2;
    // centred gradient: antisymmetric part of sum E p^T, and -sum E
    const float gcw[3] = {((Shi[ST_EP + 5] - Shi[ST_EP + 7]) + (Slo[ST_EP + 5] - Slo[ST_EP + 7])) * kl,
                          ((Shi[ST_EP + 6] - Shi[ST_EP + 2]) + (Slo[ST_EP + 6] - Slo[ST_EP + 2])) * kl,
                          ((Shi[ST_EP + 1] - Shi[ST_EP + 3]) + (Slo[ST_EP + 1] - Slo[ST_EP + 3])) * kl};
    const float gcv[3] = {-sf(ST_E) * kl, -sf(ST_E + 1) * kl, -sf(ST_E + 2) * kl};
    // R = A^T, t = -R b, and the lever centre c, from the FP32 derived constants
    float R[9], tt[3], cc[3], bv[3];
    for (int r = 0; r < 3; ++r)
        for (int q = 0; q < 3; ++q) R[3 * r + q] = st->Ahi[3 * q + r] + st->Alo[3 * q + r];
    for (int r = 0; r < 3; ++r) {
        bv[r] = st->bhi[r] + st->blo[r];
        cc[r] = st->chi[r] + st->clo[r];
    }
    for (int r = 0; r < 3; ++r) tt[r] = -(R[3 * r] * bv[0] + R[3 * r + 1] * bv[1] + R[3 * r + 2] * bv[2]);
    auto rm = [&](const float* a, float* o) {
        for (int r = 0; r < 3; ++r) o[r] = R[3 * r] * a[0] + R[3 * r + 1] * a[1] + R[3 * r + 2] * a[2];
    };
    auto cr = [](const float* a, const float* b, float* o) {
        o[0] = a[1] * b[2] - a[2] * b[1];
        o[1] = a[2] * b[0] - a[0] * b[2];
        o[2] = a[0] * b[1] - a[1] * b[0];
    };
    float gv[3], gw[3], tmp[3], tmp2[3];
    rm(gcv, gv);
    cr(cc, gcv, tmp);
    for (int r = 0; r < 3; ++r) tmp[r] += gcw[r];
    rm(tmp, gw);
    cr(tt, gv, tmp);
    for (int r = 0; r < 3; ++r) gw[r] += tmp[r];
    // the ascent direction in the centred coordinates of Z's frame
    const float rho2 = (float)st->rho2 + ellf * ellf;
    float wt[3], vt[3];
    for (int r = 0; r < 3; ++r) {
        wt[r] = gcw[r] / rho2;
        vt[r] = gcv[r];
    }
    auto symqf = [&](int base, const float* a, const float* b) {
        return sf(base) * a[0] * b[0] + sf(base + 1) * a[1] * b[1] + sf(base + 2) * a[2] * b[2] +
               sf(base + 3) * (a[0] * b[1] + a[1] * b[0]) + sf(base + 4) * (a[0] * b[2] + a[2] * b[0]) +
               sf(base + 5) * (a[1] * b[2] + a[2] * b[1]);
    };
    auto fullqf = [&](int base, const float* a, const float* b) {
        float s = 0.0f;
        for (int r = 0; r < 3; ++r)
            s += a[r] * (sf(base + 3 * r) * b[0] + sf(base + 3 * r + 1) * b[1] + sf(base + 3 * r + 2) * b[2]);
        return s;
    };
    const float ww = wt[0] * wt[0] + wt[1] * wt[1] + wt[2] * wt[2];
    const float vv = vt[0] * vt[0] + vt[1] * vt[1] + vt[2] * vt[2];
    const float trWpp = sf(ST_WPP) + sf(ST_WPP + 1) + sf(ST_WPP + 2);
    const float trEp = sf(ST_EP) + sf(ST_EP + 4) + sf(ST_EP + 8);
    const float hww = -symqf(ST_PQP, wt, wt) * il4 - (trWpp * ww - symqf(ST_WPP, wt, wt)) * il2 +
                      (fullqf(ST_EP, wt, wt) - trEp * ww) * il2;
    const float Ev[3] = {sf(ST_E), sf(ST_E + 1), sf(ST_E + 2)};
    const float Wpv[3] = {sf(ST_WP), sf(ST_WP + 1), sf(ST_WP + 2)};
    cr(Wpv, vt, tmp);
    cr(Ev, vt, tmp2);
    const float hwv = fullqf(ST_PQ, wt, vt) * il4 -
                      ((wt[0] * tmp[0] + wt[1] * tmp[1] + wt[2] * tmp[2]) +
                       0.5f * (wt[0] * tmp2[0] + wt[1] * tmp2[1] + wt[2] * tmp2[2])) * il2;
    const float hvv = symqf(ST_Q, vt, vt) * il4 - sf(ST_W) * vv * il2;
    const float Fpp = kapf * (hww + 2.0f * hwv + hvv);
    const float g[6] = {gw[0], gw[1], gw[2], gv[0], gv[1], gv[2]};
    const float Fp = (gcw[0] * wt[0] + gcw[1] * wt[1] + gcw[2] * wt[2]) + vv;   // F' along the direction
    const float wn = sqrtf(ww);
    const float vn = sqrtf(vv);
    float t = 0.0f;
    if (Fp > 0.0f) {
        const float delta = st->max_step_trans > 0.0 ? (float)st->max_step_trans : 0.5f * ellf;
        const float speed = wn * (float)st->rmax + vn;   // bound on the speed of Z's points
        float tmax = speed > 0.0f ? delta / speed : 3.0e38f;
        if (wn > 0.0f && tmax * wn > (float)st->max_step_rot) tmax = (float)st->max_step_rot / wn;
        t = (Fpp < 0.0f) ? fminf(Fp / (-Fpp), tmax) : tmax;
    }
    // the step in the origin's coordinates: xi = t (R w~, R v~ + p x R w~), p = R c + t
    float om[3], uo[3], pc[3], pxo[3];
    rm(wt, om);
    rm(vt, uo);
    rm(cc, pc);
    for (int r = 0; r < 3; ++r) pc[r] += tt[r];
    cr(pc, om, pxo);
    // ---- FP64: exp(xi^) and T <- exp(xi^) T, across lanes ------------------
    double xd[6];
    for (int q = 0; q < 3; ++q) {
        xd[q] = (double)(t * om[q]);
        xd[3 + q] = (double)(t * (uo[q] + pxo[q]));
    }
    const double th2 = xd[0] * xd[0] + xd[1] * xd[1] + xd[2] * xd[2];
    double coef = 0.0;
    if (th2 < 0.25) {
        const int s = lane < 3 ? lane : 0;
        double p = c_se3_series[s][0];
#pragma unroll
        for (int k = 1; k < 9; ++k) p = c_se3_series[s][k] - th2 * p;
        coef = p;
    } else {
        const double th = sqrt(th2);
        double sn, cs;
        sincos(th, &sn, &cs);
        coef = lane == 0 ? sn / th : (lane == 1 ? (1.0 - cs) / th2 : (th - sn) / (th2 * th));
    }
    const double ca = __shfl_sync(full, coef, 0), cb = __shfl_sync(full, coef, 1), ccf = __shfl_sync(full, coef, 2);
    const int r = (lane < 12) ? (lane >> 2) : 0;
    const int q = lane & 3;
    double e = 0.0;
    {
        const double w[3] = {xd[0], xd[1], xd[2]}, v[3] = {xd[3], xd[4], xd[5]};
        if (q < 3) {
            const double Wrq = (r == q) ? 0.0 : ((r == 0) ? (q == 1 ? -w[2] : w[1]) : (r == 1) ? (q == 0 ? w[2] : -w[0]) : (q == 0 ? -w[1] : w[0]));
            const double w2 = w[r] * w[q] - (r == q ? th2 : 0.0);
            e = (r == q ? 1.0 : 0.0) + ca * Wrq + cb * w2;
        } else {
            const double wxv[3] = {w[1] * v[2] - w[2] * v[1], w[2] * v[0] - w[0] * v[2], w[0] * v[1] - w[1] * v[0]};
            const double wwv[3] = {w[1] * wxv[2] - w[2] * wxv[1], w[2] * wxv[0] - w[0] * wxv[2], w[0] * wxv[1] - w[1] * wxv[0]};
            e = v[r] + cb * wxv[r] + ccf * wwv[r];
        }
    }
    const double Er0 = __shfl_sync(full, e, 4 * r), Er1 = __shfl_sync(full, e, 4 * r + 1);
    const double Er2 = __shfl_sync(full, e, 4 * r + 2), Er3 = __shfl_sync(full, e, 4 * r + 3);
    double* T = st->T;
    const double told = (lane < 12) ? T[lane] : 0.0;
    const double tn = Er0 * T[q] + Er1 * T[4 + q] + Er2 * T[8 + q] + (q == 3 ? Er3 : 0.0);
    if (trace && lane < 12) trace[(size_t)kTraceStride * it + 10 + lane] = told;
    __syncwarp();
    if (lane < 12) T[lane] = tn;
    __syncwarp();
    if (lane == 0) {
        if ((it + 1) % 16 == 0) orthonormalize(T);
        const double F = st->kappa * S[ST_W];
        const double ith = F * st->norm;
        const double srot = (double)(t * wn), strans = (double)(t * vn);
        st->F = F;
        st->i_theta = ith;
        st->pairs = (long long)pairs;
        st->cands = (long long)cands;
        for (int k = 0; k < 6; ++k) st->grad[k] = (double)g[k];
        st->pairs_total += (long long)pairs;
        st->cands_total += (long long)cands;
        st->Fpp = (double)Fpp;
        st->gnorm = (double)sqrtf(fmaxf(Fp, 0.0f));
        st->t = (double)t;
        st->srot = srot;
        st->strans = strans;
        const double ell = st->ell;
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
            tr[0] = ell; tr[1] = F; tr[2] = ith; tr[3] = st->gnorm; tr[4] = (double)Fpp;
            tr[5] = (double)t; tr[6] = srot; tr[7] = strans; tr[8] = decayed; tr[9] = (double)pairs;
        }
        st->ell_last = ell;
        st->iter = it + 1;
        if (converged) {
            st->status = 0;
            st->done = 1;
        } else if (it + 1 >= st->max_iters) {
            st->status = 1;
            st->done = 1;
        }
        // scalar derived constants
        const float ln = (float)st->ell;
        st->sg = -1.44269504f / (2.0f * ln * ln);
        if (st->cutoff_mult > 0.0) {
            const float rc = (float)st->cutoff_mult * ln;
            st->rc = rc;
            st->rc2 = rc * rc;
            int lv = 0;
            for (int k = 1; k < st->nlevels; ++k)
                if (st->level_h[k] >= rc * 1.0001f) lv = k;
            st->level = lv;
        } else {
            st->rc = -1.0f;
            st->rc2 = -1.0f;
            st->level = 0;
        }
    }
    __syncwarp();
    // derived T^-1 = (R^T, -R^T t) as double-float pairs, one entry per lane
    if (lane < 9) {
        const int rr = lane / 3, qq = lane % 3;
        split_df(T[4 * qq + rr], st->Ahi[lane], st->Alo[lane]);
    } else if (lane < 12) {
        const int rr = lane - 9;
        const double bvd = -(T[rr] * T[3] + T[4 + rr] * T[7] + T[8 + rr] * T[11]);
        split_df(bvd, st->bhi[rr], st->blo[rr]);
    }
    __syncwarp();
}

}  // namespace
}  // namespace cvo
