// One block per iteration: reduces the sweep's per-block statistics and takes
// the step on the device, so a registration never waits on the host.
//
// 1. Sums the 43 statistics over the sweep blocks in double-float (hi + lo
//    FP32 pairs, error-free two-sum), one warp per statistic, in block order:
//    deterministic, and as accurate as FP64 accumulation at FP32 speed.
// 2. In FP64 (one thread): F = kappa S_W; the gradient and Hessian of
//    eta -> F(T exp(eta^)) about the lever centre c in Z's frame; mapped to the
//    left perturbation exp(xi^) T by xi_c = A Ad_{T^-1} xi,
//    A = [[I, 0], [-[c]x, I]].  The indicator of Eq. (indicator_actual) is
//    F / sqrt(N M).
// 3. Registration: the step along the gradient (the method is gradient ascent
//    on SE(3), Sec. I), t = |g|^2 / -F'' with F'' = g^T H g when negative,
//    else 1e-3 / |g|; the clamps; T <- exp(t g^) T (closed-form SE(3)
//    exponential, Rodrigues + left Jacobian); Gram-Schmidt on R every 16
//    iterations; the stopping test; the lengthscale annealing of Sec. IV
//    (l <- max(decay l, l_min) once the indicator at the current l changes by
//    less than indicator_tol relative).
// 4. Writes the derived constants of the next sweep (double-float T^-1,
//    exponent scale, cutoff, grid level).
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

__device__ void skew3(const double a[3], double M[9])
{
    M[0] = 0.0;   M[1] = -a[2]; M[2] = a[1];
    M[3] = a[2];  M[4] = 0.0;   M[5] = -a[0];
    M[6] = -a[1]; M[7] = a[0];  M[8] = 0.0;
}

// exp of xi = (omega, v) in SE(3), row-major 4x4
__device__ void se3_exp_dev(const double xi[6], double E[16])
{
    const double wx = xi[0], wy = xi[1], wz = xi[2];
    const double th2 = wx * wx + wy * wy + wz * wz;
    const double th = sqrt(th2);
    double a, b, c;   // sin(th)/th, (1-cos th)/th^2, (th - sin th)/th^3
    if (th < 1e-3) {
        a = 1.0 - th2 / 6.0 + th2 * th2 / 120.0;
        b = 0.5 - th2 / 24.0 + th2 * th2 / 720.0;
        c = 1.0 / 6.0 - th2 / 120.0 + th2 * th2 / 5040.0;
    } else {
        double s, co;
        sincos(th, &s, &co);
        a = s / th;
        b = (1.0 - co) / th2;
        c = (th - s) / (th2 * th);
    }
    double K[9], K2[9];
    const double w[3] = {wx, wy, wz};
    skew3(w, K);
    for (int r = 0; r < 3; ++r)
        for (int q = 0; q < 3; ++q) K2[3 * r + q] = K[3 * r] * K[q] + K[3 * r + 1] * K[3 + q] + K[3 * r + 2] * K[6 + q];
    for (int r = 0; r < 3; ++r) {
        double tv = 0.0;
        for (int q = 0; q < 3; ++q) {
            const double id = (r == q) ? 1.0 : 0.0;
            E[4 * r + q] = id + a * K[3 * r + q] + b * K2[3 * r + q];
            tv += (id + b * K[3 * r + q] + c * K2[3 * r + q]) * xi[3 + q];
        }
        E[4 * r + 3] = tv;
    }
    E[12] = 0.0; E[13] = 0.0; E[14] = 0.0; E[15] = 1.0;
}

__device__ void mul44(const double A[16], const double B[16], double C[16])
{
    double t[16];
    for (int r = 0; r < 4; ++r)
        for (int q = 0; q < 4; ++q)
            t[4 * r + q] = A[4 * r] * B[q] + A[4 * r + 1] * B[4 + q] + A[4 * r + 2] * B[8 + q] + A[4 * r + 3] * B[12 + q];
    for (int k = 0; k < 16; ++k) C[k] = t[k];
}

__device__ void orthonormalize(double T[16])
{
    double c0[3] = {T[0], T[4], T[8]}, c1[3] = {T[1], T[5], T[9]};
    const double n0 = sqrt(c0[0] * c0[0] + c0[1] * c0[1] + c0[2] * c0[2]);
    for (int r = 0; r < 3; ++r) c0[r] /= n0;
    const double d = c0[0] * c1[0] + c0[1] * c1[1] + c0[2] * c1[2];
    for (int r = 0; r < 3; ++r) c1[r] -= d * c0[r];
    const double n1 = sqrt(c1[0] * c1[0] + c1[1] * c1[1] + c1[2] * c1[2]);
    for (int r = 0; r < 3; ++r) c1[r] /= n1;
    const double c2[3] = {c0[1] * c1[2] - c0[2] * c1[1], c0[2] * c1[0] - c0[0] * c1[2], c0[0] * c1[1] - c0[1] * c1[0]};
    for (int r = 0; r < 3; ++r) {
        T[4 * r] = c0[r];
        T[4 * r + 1] = c1[r];
        T[4 * r + 2] = c2[r];
    }
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
    st->sg = (float)(-1.4426950408889634 / (2.0 * ell * ell));
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

__global__ void __launch_bounds__(kFinalizeThreads)
k_finalize(IterState* st, const float2* __restrict__ ps, const unsigned long long* __restrict__ pc, int cap, int nb,
           double* trace)
{
    __shared__ double S[kStatN];
    __shared__ unsigned long long cs[2][kFinalizeThreads / 32];
    if (st->done) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int v = warp; v < kStatN; v += kFinalizeThreads / 32) {
        float hi = 0.0f, lo = 0.0f;
        for (int b = lane; b < nb; b += 32) {
            const float2 x = ps[(size_t)v * cap + b];
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
    const double ell = st->ell, L2 = ell * ell, L4 = L2 * L2;
    double s[kStatN];
    for (int k = 0; k < kStatN; ++k) s[k] = kap * S[k];
    const double F = s[ST_W];

    // symmetric 3x3 from (xx, yy, zz, xy, xz, yz)
    auto sym = [](const double* v, double M[9]) {
        M[0] = v[0]; M[4] = v[1]; M[8] = v[2];
        M[1] = M[3] = v[3]; M[2] = M[6] = v[4]; M[5] = M[7] = v[5];
    };
    double Q[9], PQP[9], Wpp[9];
    sym(s + ST_Q, Q);
    sym(s + ST_PQP, PQP);
    sym(s + ST_WPP, Wpp);
    const double* PQ = s + ST_PQ;
    const double* Ep = s + ST_EP;
    const double* E = s + ST_E;
    const double* Wp = s + ST_WP;
    const double W = s[ST_W];
    // gradient in the centred Z-frame coordinates
    double gc[6];
    gc[0] = (Ep[5] - Ep[7]) / L2;   // (E x p)_0 = Ep[1][2] - Ep[2][1]
    gc[1] = (Ep[6] - Ep[2]) / L2;   // (E x p)_1 = Ep[2][0] - Ep[0][2]
    gc[2] = (Ep[1] - Ep[3]) / L2;   // (E x p)_2 = Ep[0][1] - Ep[1][0]
    gc[3] = -E[0] / L2;
    gc[4] = -E[1] / L2;
    gc[5] = -E[2] / L2;
    // Hessian blocks in the same coordinates
    double Hc[36];
    const double trWpp = Wpp[0] + Wpp[4] + Wpp[8];
    const double trEp = Ep[0] + Ep[4] + Ep[8];
    double KWp[9], KE[9];
    skew3(Wp, KWp);
    skew3(E, KE);
    for (int r = 0; r < 3; ++r)
        for (int q = 0; q < 3; ++q) {
            const double id = (r == q) ? 1.0 : 0.0;
            const double hww = -PQP[3 * r + q] / L4 - (trWpp * id - Wpp[3 * r + q]) / L2 +
                               0.5 * (Ep[3 * r + q] + Ep[3 * q + r] - 2.0 * trEp * id) / L2;
            const double hwv = PQ[3 * r + q] / L4 - KWp[3 * r + q] / L2 - 0.5 * KE[3 * r + q] / L2;
            const double hvv = Q[3 * r + q] / L4 - W * id / L2;
            Hc[6 * r + q] = hww;
            Hc[6 * r + 3 + q] = hwv;
            Hc[6 * (3 + q) + r] = hwv;
            Hc[6 * (3 + r) + 3 + q] = hvv;
        }
    // B = A Ad_{T^-1} = [[R^T, 0], [B21, R^T]],  B21 = -[c]x R^T - R^T [t]x
    const double* T = st->T;
    double Rt[9], Kc[9], Kt[9], B21[9];
    for (int r = 0; r < 3; ++r)
        for (int q = 0; q < 3; ++q) Rt[3 * r + q] = T[4 * q + r];
    const double tv[3] = {T[3], T[7], T[11]};
    skew3(st->c, Kc);
    skew3(tv, Kt);
    for (int r = 0; r < 3; ++r)
        for (int q = 0; q < 3; ++q) {
            double a1 = 0.0, a2 = 0.0;
            for (int k = 0; k < 3; ++k) {
                a1 += Kc[3 * r + k] * Rt[3 * k + q];
                a2 += Rt[3 * r + k] * Kt[3 * k + q];
            }
            B21[3 * r + q] = -a1 - a2;
        }
    double B[36];
    for (int k = 0; k < 36; ++k) B[k] = 0.0;
    for (int r = 0; r < 3; ++r)
        for (int q = 0; q < 3; ++q) {
            B[6 * r + q] = Rt[3 * r + q];
            B[6 * (3 + r) + 3 + q] = Rt[3 * r + q];
            B[6 * (3 + r) + q] = B21[3 * r + q];
        }
    double g[6];
    for (int q = 0; q < 6; ++q) {
        double acc = 0.0;
        for (int r = 0; r < 6; ++r) acc += B[6 * r + q] * gc[r];
        g[q] = acc;
    }
    const double ith = F * st->norm;
    st->F = F;
    st->i_theta = ith;
    st->pairs = (long long)pairs;
    st->cands = (long long)cands;
    for (int q = 0; q < 6; ++q) st->grad[q] = g[q];

    if (st->mode == 0) {
        // full Hessian H = B^T Hc B
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
                st->hess[6 * r + q] = acc;
            }
        st->done = 1;
        return;
    }

    // ---- registration step --------------------------------------------------
    const int it = st->iter;
    double xc[6];   // B g: the gradient direction in the centred coordinates
    for (int r = 0; r < 6; ++r) {
        double acc = 0.0;
        for (int q = 0; q < 6; ++q) acc += B[6 * r + q] * g[q];
        xc[r] = acc;
    }
    double Fpp = 0.0;
    for (int r = 0; r < 6; ++r) {
        double acc = 0.0;
        for (int q = 0; q < 6; ++q) acc += Hc[6 * r + q] * xc[q];
        Fpp += xc[r] * acc;
    }
    double gn2 = 0.0;
    for (int q = 0; q < 6; ++q) gn2 += g[q] * g[q];
    double t = 0.0;
    if (gn2 > 0.0) {
        t = (Fpp < 0.0) ? gn2 / (-Fpp) : 1e-3 / sqrt(gn2);
        const double wn = sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
        const double vn = sqrt(g[3] * g[3] + g[4] * g[4] + g[5] * g[5]);
        const double max_tr = st->max_step_trans > 0.0 ? st->max_step_trans : 0.5 * ell;
        if (t * wn > st->max_step_rot) t = st->max_step_rot / wn;
        if (t * vn > max_tr) t = max_tr / vn;
    }
    double T_k[12];
    for (int q = 0; q < 12; ++q) T_k[q] = st->T[q];
    double xi[6], Ex[16];
    for (int q = 0; q < 6; ++q) xi[q] = t * g[q];
    se3_exp_dev(xi, Ex);
    mul44(Ex, st->T, st->T);
    if ((it + 1) % 16 == 0) orthonormalize(st->T);
    const double srot = sqrt(xi[0] * xi[0] + xi[1] * xi[1] + xi[2] * xi[2]);
    const double strans = sqrt(xi[3] * xi[3] + xi[4] * xi[4] + xi[5] * xi[5]);
    st->pairs_total += (long long)pairs;
    st->cands_total += (long long)cands;
    st->Fpp = Fpp;
    st->gnorm = sqrt(gn2);
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
        tr[0] = ell_used; tr[1] = F; tr[2] = ith; tr[3] = sqrt(gn2); tr[4] = Fpp;
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
}

}  // namespace

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
    k_finalize<<<1, kFinalizeThreads, 0, s>>>(st, part_stats, part_cnt, part_cap, nblocks, trace);
    return cudaGetLastError();
}

}  // namespace cvo
