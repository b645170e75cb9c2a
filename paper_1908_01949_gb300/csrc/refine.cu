// Gauss-Newton refinement of seeds and the adjoint RKN gradient of chi^2.
// Not in arXiv:1908.01949: it refines the scan's surviving seeds (sec. 2.2)
// in place of the Kalman fit the paper hands them to.
//
// Per seed (one thread):
//  1. classification of the event's hits at the starting seed, exactly as the
//     scan does (d^2 < lambda -> partition), held fixed afterwards;
//  2. Gauss-Newton iterations: an RKN pass that carries four forward tangent
//     vectors d(r, t)/d(z0, px0, py0, pz0) through the linearised step (the
//     theta0 column follows from the field's symmetry about z), finds each
//     classified wire's closest approach in its partition, and forms
//     residuals (DCA - drift)/sigma and J = n_hat . dP/dseed / sigma (envelope
//     theorem); J^T J and J^T r are accumulated and the 5x5 system is solved
//     by Cholesky in FP64 in units of `scale`;
//  3. chi^2 and its gradient at the final seed by the discrete adjoint of the
//     RKN step: a forward pass keeps the full state every `checkpoint` steps;
//     the backward pass recomputes each block of steps from its checkpoint
//     and propagates (r_bar, t_bar, lam_bar) through the transposed step,
//     injecting 2 res/sigma^2 n_hat at every closest approach.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "cdc_dev.cuh"
#include "cdc_host.h"
#include "tracer.cuh"

namespace cdc {

constexpr int MAX_CK = 64;      // checkpoints per seed
constexpr int MAX_ASSIGNED = 256;  // classified hits refined per seed; a three-turn signal has ~60-150 (more: flagged, left out)
constexpr int MAX_BLOCK = 256;  // steps between checkpoints

struct RefArgs {
    int n_seeds;
    const int32_t* seed_event;
    const float* seeds;
    int n_events;
    const int32_t* hit_off;
    const float* drift_tab;
    int n_iter;
    float sigma;
    float scale[5];
    int checkpoint;
    float* seeds_out;
    double* chi2;
    float* grad;
    int32_t* n_used;
    uint32_t* flags;
};

// --------------------------------------------------------------- helpers
__device__ __forceinline__ void seed_state_d(const double* sd, double R0, float charge_dir, int direction, State& s) {
    double st, ct;
    sincos(sd[0], &st, &ct);
    double x = R0 * ct, y = R0 * st, z = sd[1];
    double p = sqrt(sd[2] * sd[2] + sd[3] * sd[3] + sd[4] * sd[4]);
    double ip = (direction < 0 ? -1.0 : 1.0) / p;
    double tx = sd[2] * ip, ty = sd[3] * ip, tz = sd[4] * ip;
    s.rx = (float)x;
    s.lx = (float)(x - (double)s.rx);
    s.ry = (float)y;
    s.ly = (float)(y - (double)s.ry);
    s.rz = (float)z;
    s.lz = (float)(z - (double)s.rz);
    s.tx = (float)tx;
    s.mx = (float)(tx - (double)s.tx);
    s.ty = (float)ty;
    s.my = (float)(ty - (double)s.ty);
    s.tz = (float)tz;
    s.mz = (float)(tz - (double)s.tz);
    const double lam = (double)charge_dir * KAPPA_D / p;
    s.lam = (float)lam;
    s.lam_lo = (float)(lam - (double)s.lam);
}

// Field and its (r, z) derivatives: g = (dBz/drho, dBz/dz, dBr/drho, dBr/dz,
// x/rho, y/rho, Br/rho); zero derivative along a clamped coordinate.
template <int KIND>
__device__ __forceinline__ void field_grad(const DevField& F, const float r[3], float B[3], float g[7]) {
    if (KIND == 0) {
        B[0] = 0.f;
        B[1] = 0.f;
        B[2] = F.B0;
        for (int i = 0; i < 7; ++i) g[i] = 0.f;
        return;
    }
    const float r2 = fmaf(r[0], r[0], r[1] * r[1]);
    const float rho = sqrtf(r2);
    const float rinv = rho > 0.f ? 1.0f / rho : 0.f;
    const bool cr = rho < F.r_min || rho > F.r_max, cz = r[2] < F.z_min || r[2] > F.z_max;
    const float rc = fminf(fmaxf(rho, F.r_min), F.r_max), zc = fminf(fmaxf(r[2], F.z_min), F.z_max);
    float u = (rc - F.r_min) * F.inv_dr, v = (zc - F.z_min) * F.inv_dz;
    const int i = min((int)u, F.nr - 2), j = min((int)v, F.nz - 2);
    u -= (float)i;
    v -= (float)j;
    const float4* c = F.cells + 2 * ((i + 1) * (F.nz + 1) + (j + 1));  // interior cell of the padded table
    float4 qz, qr;
    load_cell(c, qz, qr);
    const float bz = fmaf(v, fmaf(qz.w, u, qz.z), fmaf(qz.y, u, qz.x));
    const float br = fmaf(v, fmaf(qr.w, u, qr.z), fmaf(qr.y, u, qr.x));
    const float cx = r[0] * rinv, cy = r[1] * rinv;
    B[0] = br * cx;
    B[1] = br * cy;
    B[2] = bz;
    g[0] = cr ? 0.f : fmaf(qz.w, v, qz.y) * F.inv_dr;
    g[1] = cz ? 0.f : fmaf(qz.w, u, qz.z) * F.inv_dz;
    g[2] = cr ? 0.f : fmaf(qr.w, v, qr.y) * F.inv_dr;
    g[3] = cz ? 0.f : fmaf(qr.w, u, qr.z) * F.inv_dz;
    g[4] = cx;
    g[5] = cy;
    g[6] = br * rinv;
}

// dB = (dB/dr) v
template <int KIND>
__device__ __forceinline__ void apply_g(const float g[7], const float v[3], float o[3]) {
    if (KIND == 0) {
        o[0] = o[1] = o[2] = 0.f;
        return;
    }
    const float vr = fmaf(g[4], v[0], g[5] * v[1]);
    const float dbz = fmaf(g[0], vr, g[1] * v[2]);
    const float dbr = fmaf(g[2], vr, g[3] * v[2]);
    o[0] = fmaf(dbr, g[4], g[6] * fmaf(-g[4], vr, v[0]));
    o[1] = fmaf(dbr, g[5], g[6] * fmaf(-g[5], vr, v[1]));
    o[2] = dbz;
}

// r_bar += (dB/dr)^T b_bar
template <int KIND>
__device__ __forceinline__ void apply_gt(const float g[7], const float bb[3], float rb[3]) {
    if (KIND == 0) return;
    const float a = fmaf(bb[0], g[4], bb[1] * g[5]);
    const float s = fmaf(bb[2], g[0], a * g[2]);
    rb[0] += fmaf(s, g[4], g[6] * fmaf(-g[4], a, bb[0]));
    rb[1] += fmaf(s, g[5], g[6] * fmaf(-g[5], a, bb[1]));
    rb[2] += fmaf(bb[2], g[1], a * g[3]);
}

__device__ __forceinline__ void cross3(const float a[3], const float b[3], float c[3]) {
    c[0] = fmaf(a[1], b[2], -a[2] * b[1]);
    c[1] = fmaf(a[2], b[0], -a[0] * b[2]);
    c[2] = fmaf(a[0], b[1], -a[1] * b[0]);
}

// Stage values of one RKN step at (r, t) (hi parts), for the tangent and
// adjoint steps.
template <int KIND>
struct Stages {
    float t1[3], t2[3], t3[3], t4[3];
    float B1[3], B2[3], B4[3];
    float g1[7], g2[7], g4[7];
    float k1[3], k2[3], k3[3], k4[3];

    __device__ __forceinline__ void eval(const DevField& F, const float r[3], const float t[3], float lam, float h) {
        const float h2 = 0.5f * h, hh8 = h * h * 0.125f, hh2 = h * h * 0.5f;
        float rm[3], re[3], c[3];
        for (int a = 0; a < 3; ++a) t1[a] = t[a];
        field_grad<KIND>(F, r, B1, g1);
        cross3(t1, B1, c);
        for (int a = 0; a < 3; ++a) k1[a] = lam * c[a];
        for (int a = 0; a < 3; ++a) {
            t2[a] = fmaf(h2, k1[a], t[a]);
            rm[a] = fmaf(hh8, k1[a], fmaf(h2, t[a], r[a]));
        }
        field_grad<KIND>(F, rm, B2, g2);
        cross3(t2, B2, c);
        for (int a = 0; a < 3; ++a) k2[a] = lam * c[a];
        for (int a = 0; a < 3; ++a) t3[a] = fmaf(h2, k2[a], t[a]);
        cross3(t3, B2, c);
        for (int a = 0; a < 3; ++a) k3[a] = lam * c[a];
        for (int a = 0; a < 3; ++a) {
            t4[a] = fmaf(h, k3[a], t[a]);
            re[a] = fmaf(hh2, k3[a], fmaf(h, t[a], r[a]));
        }
        field_grad<KIND>(F, re, B4, g4);
        cross3(t4, B4, c);
        for (int a = 0; a < 3; ++a) k4[a] = lam * c[a];
    }
};

// One step of rkn_step<KIND, true> that keeps its stage values for the
// tangent step: the field and its gradient are evaluated once at each stage
// point, for the state and the tangents together.  The slopes k carry the
// two-float lam, as in the state step.
template <int KIND>
__device__ __forceinline__ void rkn_step_stages(const DevField& F, State& s, float h, float h6_lo, Stages<KIND>& S) {
    const float h2 = 0.5f * h, hh8 = h * h * 0.125f, hh2 = h * h * 0.5f, hh6 = h * h * (1.0f / 6.0f),
                h6 = h * (1.0f / 6.0f);
    const float r[3] = {s.rx, s.ry, s.rz};
    float rm[3], re[3];
    S.t1[0] = s.tx;
    S.t1[1] = s.ty;
    S.t1[2] = s.tz;
    field_grad<KIND>(F, r, S.B1, S.g1);
    kvec<true>(s, S.t1[0], S.t1[1], S.t1[2], S.B1[0], S.B1[1], S.B1[2], S.k1[0], S.k1[1], S.k1[2]);
    for (int a = 0; a < 3; ++a) {
        S.t2[a] = fmaf(h2, S.k1[a], S.t1[a]);
        rm[a] = fmaf(hh8, S.k1[a], fmaf(h2, S.t1[a], r[a]));
    }
    field_grad<KIND>(F, rm, S.B2, S.g2);
    kvec<true>(s, S.t2[0], S.t2[1], S.t2[2], S.B2[0], S.B2[1], S.B2[2], S.k2[0], S.k2[1], S.k2[2]);
    for (int a = 0; a < 3; ++a) S.t3[a] = fmaf(h2, S.k2[a], S.t1[a]);
    kvec<true>(s, S.t3[0], S.t3[1], S.t3[2], S.B2[0], S.B2[1], S.B2[2], S.k3[0], S.k3[1], S.k3[2]);
    for (int a = 0; a < 3; ++a) {
        S.t4[a] = fmaf(h, S.k3[a], S.t1[a]);
        re[a] = fmaf(hh2, S.k3[a], fmaf(h, S.t1[a], r[a]));
    }
    field_grad<KIND>(F, re, S.B4, S.g4);
    kvec<true>(s, S.t4[0], S.t4[1], S.t4[2], S.B4[0], S.B4[1], S.B4[2], S.k4[0], S.k4[1], S.k4[2]);
    // the state update of rkn_step<KIND, true>
    float d[3], dl[3], tl[3];
    const float cl[3] = {h * s.mx, h * s.my, h * s.mz};  // h t_lo, straight into the low word
    for (int a = 0; a < 3; ++a) {
        d[a] = fmaf(h, S.t1[a], hh6 * (S.k1[a] + S.k2[a] + S.k3[a]));
        const float sa = S.k1[a] + S.k4[a] + 2.0f * (S.k2[a] + S.k3[a]);
        tl[a] = h6 * sa;
        dl[a] = fmaf(h6_lo, sa, fmaf(h6, sa, -tl[a]));
    }
    acc2(s.rx, s.lx, d[0], cl[0]);
    acc2(s.ry, s.ly, d[1], cl[1]);
    acc2(s.rz, s.lz, d[2], cl[2]);
    acc2(s.tx, s.mx, tl[0], dl[0]);
    acc2(s.ty, s.my, tl[1], dl[1]);
    acc2(s.tz, s.mz, tl[2], dl[2]);
}

// Tangent of one step: (dr, dt) of NT directions, dlam constant.
template <int KIND, int NT>
__device__ __forceinline__ void tangent_step(const Stages<KIND>& S, float lam, float h, float (&dr)[NT][3],
                                             float (&dt)[NT][3], const float (&dl)[NT]) {
    const float h2 = 0.5f * h, hh8 = h * h * 0.125f, hh2 = h * h * 0.5f, hh6 = h * h * (1.0f / 6.0f),
                h6 = h * (1.0f / 6.0f);
#pragma unroll
    for (int n = 0; n < NT; ++n) {
        const float q = dl[n] / lam;
        float gv[3], c1[3], c2[3], d1[3], d2[3], d3[3], d4[3], ti[3], ri[3];
        apply_g<KIND>(S.g1, dr[n], gv);
        cross3(dt[n], S.B1, c1);
        cross3(S.t1, gv, c2);
        for (int a = 0; a < 3; ++a) d1[a] = fmaf(q, S.k1[a], lam * (c1[a] + c2[a]));
        for (int a = 0; a < 3; ++a) {
            ti[a] = fmaf(h2, d1[a], dt[n][a]);
            ri[a] = fmaf(hh8, d1[a], fmaf(h2, dt[n][a], dr[n][a]));
        }
        apply_g<KIND>(S.g2, ri, gv);
        cross3(ti, S.B2, c1);
        cross3(S.t2, gv, c2);
        for (int a = 0; a < 3; ++a) d2[a] = fmaf(q, S.k2[a], lam * (c1[a] + c2[a]));
        for (int a = 0; a < 3; ++a) ti[a] = fmaf(h2, d2[a], dt[n][a]);
        cross3(ti, S.B2, c1);
        cross3(S.t3, gv, c2);
        for (int a = 0; a < 3; ++a) d3[a] = fmaf(q, S.k3[a], lam * (c1[a] + c2[a]));
        for (int a = 0; a < 3; ++a) {
            ti[a] = fmaf(h, d3[a], dt[n][a]);
            ri[a] = fmaf(hh2, d3[a], fmaf(h, dt[n][a], dr[n][a]));
        }
        apply_g<KIND>(S.g4, ri, gv);
        cross3(ti, S.B4, c1);
        cross3(S.t4, gv, c2);
        for (int a = 0; a < 3; ++a) d4[a] = fmaf(q, S.k4[a], lam * (c1[a] + c2[a]));
        for (int a = 0; a < 3; ++a) {
            dr[n][a] = fmaf(hh6, d1[a] + d2[a] + d3[a], fmaf(h, dt[n][a], dr[n][a]));
            dt[n][a] = fmaf(h6, d1[a] + d4[a] + 2.0f * (d2[a] + d3[a]), dt[n][a]);
        }
    }
}

// Transposed step: given (rb, tb) at the step's end, returns them at its start
// and adds to lb (d/d lam).  The step's increments are formed in FP32 and
// added to the adjoint as compensated sums ((rb, rl), (tb, tl), (lb, ll)):
// over a three-turn track the adjoint takes thousands of small increments, and
// plain FP32 sums would leave an error of ~1e-4 of the gradient near the chi^2
// minimum, where it is a small difference of much larger per-hit terms.
template <int KIND>
__device__ __forceinline__ void adjoint_step(const Stages<KIND>& S, float lam, float h, float rb[3], float tb[3],
                                             float& lb, float rl[3], float tl[3], float& ll) {
    const float h2 = 0.5f * h, hh8 = h * h * 0.125f, hh2 = h * h * 0.5f, hh6 = h * h * (1.0f / 6.0f),
                h6 = h * (1.0f / 6.0f);
    float kb1[3], kb2[3], kb3[3], kb4[3], rn[3], tn[3], tbi[3], Bb[3], rbe[3], c[3];
    for (int a = 0; a < 3; ++a) {
        kb1[a] = fmaf(hh6, rb[a], h6 * tb[a]);
        kb2[a] = fmaf(hh6, rb[a], 2.0f * h6 * tb[a]);
        kb3[a] = kb2[a];
        kb4[a] = h6 * tb[a];
        rn[a] = 0.f;                      // increments: r' = r + ...
        tn[a] = h * rb[a];                // r' depends on h t; t' on t
    }
    // k4 = lam t4 x B4 at re
    cross3(S.B4, kb4, c);
    for (int a = 0; a < 3; ++a) tbi[a] = lam * c[a];
    cross3(kb4, S.t4, c);
    for (int a = 0; a < 3; ++a) Bb[a] = lam * c[a];
    float dl = kb4[0] * S.k4[0] / lam + kb4[1] * S.k4[1] / lam + kb4[2] * S.k4[2] / lam;
    rbe[0] = rbe[1] = rbe[2] = 0.f;
    apply_gt<KIND>(S.g4, Bb, rbe);
    for (int a = 0; a < 3; ++a) {
        tn[a] += tbi[a];                                  // t4 = t + h k3
        kb3[a] = fmaf(h, tbi[a], kb3[a]);
        rn[a] += rbe[a];                                  // re = r + h t + h^2/2 k3
        tn[a] = fmaf(h, rbe[a], tn[a]);
        kb3[a] = fmaf(hh2, rbe[a], kb3[a]);
    }
    // k3 = lam t3 x B2 at rm
    float Bb2[3];
    cross3(S.B2, kb3, c);
    for (int a = 0; a < 3; ++a) tbi[a] = lam * c[a];
    cross3(kb3, S.t3, c);
    for (int a = 0; a < 3; ++a) Bb2[a] = lam * c[a];
    dl += (kb3[0] * S.k3[0] + kb3[1] * S.k3[1] + kb3[2] * S.k3[2]) / lam;
    for (int a = 0; a < 3; ++a) {
        tn[a] += tbi[a];                                  // t3 = t + h/2 k2
        kb2[a] = fmaf(h2, tbi[a], kb2[a]);
    }
    // k2 = lam t2 x B2 at rm
    cross3(S.B2, kb2, c);
    for (int a = 0; a < 3; ++a) tbi[a] = lam * c[a];
    cross3(kb2, S.t2, c);
    for (int a = 0; a < 3; ++a) Bb2[a] = fmaf(lam, c[a], Bb2[a]);
    dl += (kb2[0] * S.k2[0] + kb2[1] * S.k2[1] + kb2[2] * S.k2[2]) / lam;
    float rbm[3] = {0.f, 0.f, 0.f};
    apply_gt<KIND>(S.g2, Bb2, rbm);
    for (int a = 0; a < 3; ++a) {
        tn[a] += tbi[a];                                  // t2 = t + h/2 k1
        kb1[a] = fmaf(h2, tbi[a], kb1[a]);
        rn[a] += rbm[a];                                  // rm = r + h/2 t + h^2/8 k1
        tn[a] = fmaf(h2, rbm[a], tn[a]);
        kb1[a] = fmaf(hh8, rbm[a], kb1[a]);
    }
    // k1 = lam t x B1 at r
    cross3(S.B1, kb1, c);
    for (int a = 0; a < 3; ++a) tn[a] = fmaf(lam, c[a], tn[a]);
    cross3(kb1, S.t1, c);
    for (int a = 0; a < 3; ++a) Bb[a] = lam * c[a];
    dl += (kb1[0] * S.k1[0] + kb1[1] * S.k1[1] + kb1[2] * S.k1[2]) / lam;
    apply_gt<KIND>(S.g1, Bb, rn);
    for (int a = 0; a < 3; ++a) {
        kahan(rb[a], rl[a], rn[a]);
        kahan(tb[a], tl[a], tn[a]);
    }
    kahan(lb, ll, dl);
}

// ---------------------------------------------------- classified-hit list
struct Assigned {
    int n;
    uint32_t key[MAX_ASSIGNED];  // wire | partition << 16, sorted by wire
    float drift[MAX_ASSIGNED];
    // per pass: best closest approach in the assigned partition
    float D[MAX_ASSIGNED];
    float nx[MAX_ASSIGNED], ny[MAX_ASSIGNED], nz[MAX_ASSIGNED];
    float u[MAX_ASSIGNED];
    int j[MAX_ASSIGNED];          // segment start state; -1 start point, -2 end point
    float J[MAX_ASSIGNED][5];

    __device__ __forceinline__ int find(int wire) const {
        int lo = 0, hi = n - 1;
        while (lo <= hi) {
            int mid = (lo + hi) >> 1;
            int w = (int)(key[mid] & 0xffffu);
            if (w == wire) return mid;
            if (w < wire) lo = mid + 1; else hi = mid - 1;
        }
        return -1;
    }
};

// Closest approach of the cubic Hermite segment (state o -> state n) to a
// wire, with the lo parts of position and wire midpoint; returns the distance
// D at the minimum, its position u in the segment and the unit normal from the
// wire to the track there.
__device__ __forceinline__ bool seg_min_precise(const float o[6], const float ol[3], const float nn[6],
                                                const float nl[3], float h, float4 W, float4 Wl, float cosa,
                                                float cosa_lo, float& D, float& u, float wp[3]) {
    const float ax = (o[0] - W.x) + (ol[0] - Wl.x), ay = (o[1] - W.y) + (ol[1] - Wl.y), az = o[2] + ol[2];
    const float ad = fmaf(ax, W.z, fmaf(ay, W.w, az * cosa));
    const float t0d = fmaf(o[3], W.z, fmaf(o[4], W.w, o[5] * cosa));
    const float g0 = fmaf(ax, o[3], fmaf(ay, o[4], az * o[5])) - ad * t0d;
    if (!(g0 < 0.f)) return false;
    const float Dx = (nn[0] - o[0]) + (nl[0] - ol[0]), Dy = (nn[1] - o[1]) + (nl[1] - ol[1]),
                Dz = (nn[2] - o[2]) + (nl[2] - ol[2]);
    const float bx = ax + Dx, by = ay + Dy, bz = az + Dz;
    const float bd = fmaf(bx, W.z, fmaf(by, W.w, bz * cosa));
    const float t1d = fmaf(nn[3], W.z, fmaf(nn[4], W.w, nn[5] * cosa));
    const float g1 = fmaf(bx, nn[3], fmaf(by, nn[4], bz * nn[5])) - bd * t1d;
    if (g1 < 0.f) return false;
    const float ih = 1.0f / h;
    u = h * (g0 / (g0 - g1));
    float wx, wy, wz, wd;
    for (int it = 0; it < 4; ++it) {
        const float t = u * ih, t2 = t * t;
        const float h10 = h * t * fmaf(t, t - 2.0f, 1.0f), h01 = t2 * fmaf(-2.0f, t, 3.0f), h11 = h * t2 * (t - 1.0f);
        wx = fmaf(h11, nn[3], fmaf(h01, Dx, fmaf(h10, o[3], ax)));
        wy = fmaf(h11, nn[4], fmaf(h01, Dy, fmaf(h10, o[4], ay)));
        wz = fmaf(h11, nn[5], fmaf(h01, Dz, fmaf(h10, o[5], az)));
        const float d10 = fmaf(3.0f * t, t, fmaf(-4.0f, t, 1.0f)), d01 = 6.0f * t * (1.0f - t) * ih,
                    d11 = t * fmaf(3.0f, t, -2.0f);
        const float vx = fmaf(d11, nn[3], fmaf(d01, Dx, d10 * o[3]));
        const float vy = fmaf(d11, nn[4], fmaf(d01, Dy, d10 * o[4]));
        const float vz = fmaf(d11, nn[5], fmaf(d01, Dz, d10 * o[5]));
        const float e10 = fmaf(6.0f, t, -4.0f) * ih, e01 = fmaf(-12.0f, t, 6.0f) * ih * ih,
                    e11 = fmaf(6.0f, t, -2.0f) * ih;
        const float qx = fmaf(e11, nn[3], fmaf(e01, Dx, e10 * o[3]));
        const float qy = fmaf(e11, nn[4], fmaf(e01, Dy, e10 * o[4]));
        const float qz = fmaf(e11, nn[5], fmaf(e01, Dz, e10 * o[5]));
        wd = fmaf(wx, W.z, fmaf(wy, W.w, wz * cosa));
        const float vd = fmaf(vx, W.z, fmaf(vy, W.w, vz * cosa));
        const float qd = fmaf(qx, W.z, fmaf(qy, W.w, qz * cosa));
        const float num = fmaf(wx, vx, fmaf(wy, vy, wz * vz)) - wd * vd;
        const float den = fmaf(vx, vx, fmaf(vy, vy, vz * vz)) - vd * vd + (fmaf(wx, qx, fmaf(wy, qy, wz * qz)) - wd * qd);
        if (den > 0.f) u = fminf(fmaxf(u - num / den, 0.f), h);
    }
    const float t = u * ih, t2 = t * t;
    const float h10 = h * t * fmaf(t, t - 2.0f, 1.0f), h01 = t2 * fmaf(-2.0f, t, 3.0f), h11 = h * t2 * (t - 1.0f);
    wx = fmaf(h11, nn[3], fmaf(h01, Dx, fmaf(h10, o[3], ax)));
    wy = fmaf(h11, nn[4], fmaf(h01, Dy, fmaf(h10, o[4], ay)));
    wz = fmaf(h11, nn[5], fmaf(h01, Dz, fmaf(h10, o[5], az)));
    // final projection with the wire direction as hi + lo: the rounding of d
    // times the distance along the wire (up to the half length) would
    // otherwise shift the line by ~1e-5 mm
    wd = fmaf(wx, W.z, fmaf(wy, W.w, wz * cosa)) + fmaf(wx, Wl.z, fmaf(wy, Wl.w, wz * cosa_lo));
    float px = wx - fmaf(wd, W.z, wd * Wl.z), py = wy - fmaf(wd, W.w, wd * Wl.w), pz = wz - fmaf(wd, cosa, wd * cosa_lo);
    D = sqrtf(fmaf(px, px, fmaf(py, py, pz * pz)));
    // Unit normal from the wire to the track: at an interior minimum it is the
    // common perpendicular d x P'(u), which (unlike w_perp / D) stays accurate
    // when the track passes very close to the wire; the sign comes from w_perp.
    const float d10 = fmaf(3.0f * t, t, fmaf(-4.0f, t, 1.0f)), d01 = 6.0f * t * (1.0f - t) * ih,
                d11 = t * fmaf(3.0f, t, -2.0f);
    const float vx = fmaf(d11, nn[3], fmaf(d01, Dx, d10 * o[3]));
    const float vy = fmaf(d11, nn[4], fmaf(d01, Dy, d10 * o[4]));
    const float vz = fmaf(d11, nn[5], fmaf(d01, Dz, d10 * o[5]));
    float cx = fmaf(W.w, vz, -cosa * vy), cy = fmaf(cosa, vx, -W.z * vz), cz = fmaf(W.z, vy, -W.w * vx);
    const float cn = sqrtf(fmaf(cx, cx, fmaf(cy, cy, cz * cz)));
    if (u > 0.f && u < h && cn > 1e-3f) {
        const float sgn = fmaf(px, cx, fmaf(py, cy, pz * cz)) >= 0.f ? 1.0f : -1.0f;
        wp[0] = sgn * cx / cn;
        wp[1] = sgn * cy / cn;
        wp[2] = sgn * cz / cn;
    } else {
        const float inv = D > 0.f ? 1.0f / D : 0.f;
        wp[0] = px * inv;
        wp[1] = py * inv;
        wp[2] = pz * inv;
    }
    return true;
}

// Point distance at a track end (used when the distance still falls at the end
// or rises from the start).
__device__ __forceinline__ float point_dist(const float o[6], const float ol[3], float4 W, float4 Wl, float cosa,
                                           float cosa_lo, float& g, float wp[3]) {
    const float ax = (o[0] - W.x) + (ol[0] - Wl.x), ay = (o[1] - W.y) + (ol[1] - Wl.y), az = o[2] + ol[2];
    const float ad = fmaf(ax, W.z, fmaf(ay, W.w, az * cosa)) + fmaf(ax, Wl.z, fmaf(ay, Wl.w, az * cosa_lo));
    const float td = fmaf(o[3], W.z, fmaf(o[4], W.w, o[5] * cosa));
    g = fmaf(ax, o[3], fmaf(ay, o[4], az * o[5])) - ad * td;
    wp[0] = ax - fmaf(ad, W.z, ad * Wl.z);
    wp[1] = ay - fmaf(ad, W.w, ad * Wl.w);
    wp[2] = az - fmaf(ad, cosa, ad * cosa_lo);
    return sqrtf(fmaf(wp[0], wp[0], fmaf(wp[1], wp[1], wp[2] * wp[2])));
}

// Window search around (x, y, z) over fired wires (as the scan tracer).
template <class Fn>
__device__ __forceinline__ float window(const ScanConst& P, const DevLayer* s_lay, const uchar2* s_tab,
                                        const float* dtab, float x, float y, float z, Fn&& fn) {
    const float rho = sqrtf(fmaf(x, x, y * y));
    const uchar2 lr = s_tab[min((int)rho, TAB_N - 1)];
    if (lr.x <= lr.y) {
        const float phi = atan2f(y, x);
        const float blo = fmaxf(rho - P.band, 0.f), bhi = rho + P.band;
        const float blo2 = blo * blo, bhi2 = bhi * bhi;
        for (int l = lr.x; l <= lr.y; ++l) {
            const DevLayer& L = s_lay[l];
            const float rl2 = fmaf(z * z, L.tan2a, L.R2);
            if (rl2 > bhi2 || rl2 < blo2) continue;
            const float zt = z * L.tana_over_R, z2 = zt * zt;
            const float tw = zt * fmaf(z2, fmaf(z2, fmaf(z2, -1.0f / 7.0f, 0.2f), -1.0f / 3.0f), 1.0f);
            const float c = (phi - tw - L.phi_off) * L.n_over_2pi;
            if (!(fabsf(c) < 1.0e6f)) continue;
            const float w = P.d_win * L.cells_per_mm;
            const int i0 = (int)ceilf(c - w), i1 = (int)floorf(c + w);
            for (int i = i0; i <= i1; ++i) {
                int ii = i % L.N;
                if (ii < 0) ii += L.N;
                const int wire = L.base + ii;
                const float d = __ldg(dtab + wire);
                if (!(d <= P.max_drift)) continue;
                fn(wire, L.cosa, L.cosa_lo);
            }
        }
    }
    return rho;
}

// Hermite weights at u of a segment of length h.
__device__ __forceinline__ void hermite_w(float u, float h, float& a0, float& a1, float& b0, float& b1) {
    const float t = u / h, t2 = t * t;
    b0 = t2 * fmaf(-2.0f, t, 3.0f);          // h01: weight of r_{j+1}
    a0 = 1.0f - b0;                          // h00: weight of r_j
    a1 = h * t * fmaf(t, t - 2.0f, 1.0f);    // h10 h: weight of t_j
    b1 = h * t2 * (t - 1.0f);                // h11 h: weight of t_{j+1}
}

// Row of the Jacobian (divided by sigma) of a distance whose unit normal is n
// at track point P, from the tangents v of the seed's (z0, px0, py0, pz0).
// The theta0 column needs no tangent of its own: the field is symmetric about
// the z axis, so turning theta0 and the direction of (px0, py0) together by
// an angle turns the whole track about z, with tangent z x P at every point;
// turning (px0, py0) alone has tangent px0 v_py0 - py0 v_px0, and the theta0
// tangent is the difference of the two.
__device__ __forceinline__ void jac_row(const float nv[3], const float P[3], const float (&v)[4][3], float px0,
                                        float py0, float sigma, float J[5]) {
    const float w0 = fmaf(py0, v[1][0], fmaf(-px0, v[2][0], -P[1]));
    const float w1 = fmaf(py0, v[1][1], fmaf(-px0, v[2][1], P[0]));
    const float w2 = fmaf(py0, v[1][2], -px0 * v[2][2]);
    J[0] = (nv[0] * w0 + nv[1] * w1 + nv[2] * w2) / sigma;
    for (int m = 0; m < 4; ++m) J[1 + m] = (nv[0] * v[m][0] + nv[1] * v[m][1] + nv[2] * v[m][2]) / sigma;
}

// One propagation over the whole track that records, for every classified
// wire, the closest approach inside its partition.  TAN: also the forward
// tangents and J.  CK: also the checkpoints of the adjoint.
template <int KIND, bool TAN, bool CK>
__device__ int track_pass(const DevGeom& G, const DevField& F, const ScanConst& P, const DevLayer* s_lay,
                          const uchar2* s_tab, const float* dtab, const double* sd, float sigma, Assigned& A,
                          float (*ck)[14], int ck_every, uint32_t& flags) {
    State s;
    seed_state_d(sd, G.R0d, P.charge_dir, P.direction, s);
    // tangents of (z0, px0, py0, pz0); theta0's follows from them (jac_row)
    float dr[4][3], dt[4][3], dl[4];
    const float px0 = (float)sd[2], py0 = (float)sd[3];
    if (TAN) {
        const double p = sqrt(sd[2] * sd[2] + sd[3] * sd[3] + sd[4] * sd[4]);
        const double dir = P.direction < 0 ? -1.0 : 1.0;
        const double th[3] = {sd[2] / p, sd[3] / p, sd[4] / p};
        for (int n = 0; n < 4; ++n)
            for (int a = 0; a < 3; ++a) dr[n][a] = dt[n][a] = 0.f;
        dr[0][2] = 1.0f;
        dl[0] = 0.f;
        for (int b = 0; b < 3; ++b) {
            for (int a = 0; a < 3; ++a) dt[1 + b][a] = (float)(dir * (((a == b) ? 1.0 : 0.0) - th[a] * th[b]) / p);
            dl[1 + b] = (float)(-(double)s.lam * th[b] / p);
        }
    }
    for (int i = 0; i < A.n; ++i) {
        A.D[i] = 3.0e38f;
        A.j[i] = -3;
    }
    const float h = P.h;
    int n = 0, part = 0;
    bool outside = true;
    // start of the track
    {
        const float o[6] = {s.rx, s.ry, s.rz, s.tx, s.ty, s.tz}, ol[3] = {s.lx, s.ly, s.lz};
        window(P, s_lay, s_tab, dtab, o[0], o[1], o[2], [&](int wire, float cosa, float cosa_lo) {
            const int q = A.find(wire);
            if (q < 0 || (int)(A.key[q] >> 16) != 0) return;
            const float4 W = __ldg(G.wires + wire);
            const float4 Wl = __ldg(G.wires_lo + wire);
            float g, wp[3];
            const float D = point_dist(o, ol, W, Wl, cosa, cosa_lo, g, wp);
            if (g > 0.f && D < A.D[q]) {
                A.D[q] = D;
                A.j[q] = -1;
                A.u[q] = 0.f;
                const float inv = D > 0.f ? 1.0f / D : 0.f;
                A.nx[q] = wp[0] * inv;
                A.ny[q] = wp[1] * inv;
                A.nz[q] = wp[2] * inv;
                if (TAN) {
                    const float nv[3] = {A.nx[q], A.ny[q], A.nz[q]};
                    jac_row(nv, o, dr, px0, py0, sigma, A.J[q]);
                }
            }
        });
    }
    for (;;) {
        if (CK && (n % ck_every) == 0) {
            float* c = ck[n / ck_every];
            c[0] = s.rx; c[1] = s.ry; c[2] = s.rz; c[3] = s.lx; c[4] = s.ly; c[5] = s.lz;
            c[6] = s.tx; c[7] = s.ty; c[8] = s.tz; c[9] = s.mx; c[10] = s.my; c[11] = s.mz; c[12] = s.lam;
            c[13] = s.lam_lo;
        }
        const float o[6] = {s.rx, s.ry, s.rz, s.tx, s.ty, s.tz}, ol[3] = {s.lx, s.ly, s.lz};
        float odr[4][3], odt[4][3];
        if (TAN) {
            for (int m = 0; m < 4; ++m)
                for (int a = 0; a < 3; ++a) {
                    odr[m][a] = dr[m][a];
                    odt[m][a] = dt[m][a];
                }
            Stages<KIND> S;
            rkn_step_stages<KIND>(F, s, h, P.h6_lo, S);
            tangent_step<KIND, 4>(S, s.lam, h, dr, dt, dl);
        } else {
            rkn_step<KIND, true>(F, s, h, P.h6_lo);
        }
        ++n;
        const float nn[6] = {s.rx, s.ry, s.rz, s.tx, s.ty, s.tz}, nl[3] = {s.lx, s.ly, s.lz};
        const int pt = part;
        const float rho = window(P, s_lay, s_tab, dtab, nn[0], nn[1], nn[2], [&](int wire, float cosa, float cosa_lo) {
            const int q = A.find(wire);
            if (q < 0 || (int)(A.key[q] >> 16) != pt) return;
            const float4 W = __ldg(G.wires + wire);
            const float4 Wl = __ldg(G.wires_lo + wire);
            float D, u, wp[3];
            if (!seg_min_precise(o, ol, nn, nl, h, W, Wl, cosa, cosa_lo, D, u, wp)) return;
            if (!(D < A.D[q])) return;
            A.D[q] = D;
            A.j[q] = n - 1;
            A.u[q] = u;
            A.nx[q] = wp[0];
            A.ny[q] = wp[1];
            A.nz[q] = wp[2];
            if (TAN) {
                float a0, a1, b0, b1;
                hermite_w(u, h, a0, a1, b0, b1);
                float v[4][3], Pu[3];
                for (int m = 0; m < 4; ++m)
                    for (int a = 0; a < 3; ++a)
                        v[m][a] = fmaf(a0, odr[m][a], fmaf(a1, odt[m][a], fmaf(b0, dr[m][a], b1 * dt[m][a])));
                for (int a = 0; a < 3; ++a)
                    Pu[a] = fmaf(a0, o[a], fmaf(a1, o[3 + a], fmaf(b0, nn[a], b1 * nn[3 + a])));
                jac_row(wp, Pu, v, px0, py0, sigma, A.J[q]);
            }
        });
        const bool now_out = rho >= G.R0;
        bool stop = false;
        if (outside && !now_out) {
            ++part;
            if (part >= P.max_part) stop = true;
        }
        outside = now_out;
        if (fabsf(nn[2]) > G.z_half || rho > G.R_out) stop = true;
        if (!stop && n >= P.max_steps) {
            stop = true;
            flags |= CDC_FLAG_STEP_CAP;
        }
        if (stop) {
            const int pe = part;
            if (pe < P.max_part)
                window(P, s_lay, s_tab, dtab, nn[0], nn[1], nn[2], [&](int wire, float cosa, float cosa_lo) {
                    const int q = A.find(wire);
                    if (q < 0 || (int)(A.key[q] >> 16) != pe) return;
                    const float4 W = __ldg(G.wires + wire);
                    const float4 Wl = __ldg(G.wires_lo + wire);
                    float g, wp[3];
                    const float D = point_dist(nn, nl, W, Wl, cosa, cosa_lo, g, wp);
                    if (g < 0.f && D < A.D[q]) {
                        A.D[q] = D;
                        A.j[q] = -2;
                        A.u[q] = 0.f;
                        const float inv = D > 0.f ? 1.0f / D : 0.f;
                        A.nx[q] = wp[0] * inv;
                        A.ny[q] = wp[1] * inv;
                        A.nz[q] = wp[2] * inv;
                        if (TAN) {
                            const float nv[3] = {A.nx[q], A.ny[q], A.nz[q]};
                            jac_row(nv, nn, dr, px0, py0, sigma, A.J[q]);
                        }
                    }
                });
            break;
        }
    }
    return n;
}

// Cholesky solve of the 5x5 system A x = b in place (FP64); false if A is not
// positive definite.
__device__ bool chol5(double* A, double* b) {
    double L[25];
    for (int i = 0; i < 25; ++i) L[i] = 0.0;
    for (int i = 0; i < 5; ++i)
        for (int j = 0; j <= i; ++j) {
            double s = A[5 * i + j];
            for (int k = 0; k < j; ++k) s -= L[5 * i + k] * L[5 * j + k];
            if (i == j) {
                if (!(s > 0.0)) return false;
                L[5 * i + i] = sqrt(s);
            } else {
                L[5 * i + j] = s / L[5 * j + j];
            }
        }
    double y[5];
    for (int i = 0; i < 5; ++i) {
        double s = b[i];
        for (int k = 0; k < i; ++k) s -= L[5 * i + k] * y[k];
        y[i] = s / L[5 * i + i];
    }
    for (int i = 4; i >= 0; --i) {
        double s = y[i];
        for (int k = i + 1; k < 5; ++k) s -= L[5 * k + i] * b[k];
        b[i] = s / L[5 * i + i];
    }
    return true;
}

// chi^2 and the adjoint gradient at seed sd (classification in A fixed).
template <int KIND>
__device__ double chi2_adjoint(const DevGeom& G, const DevField& F, const ScanConst& P, const DevLayer* s_lay,
                               const uchar2* s_tab, const float* dtab, const double* sd, float sigma, int ck_every,
                               Assigned& A, float (*ck)[14], float (*buf)[6], float* grad, int& used,
                               uint32_t& flags) {
    const int n = track_pass<KIND, false, true>(G, F, P, s_lay, s_tab, dtab, sd, sigma, A, ck, ck_every, flags);
    double chi2 = 0.0;
    used = 0;
    // coefficient of n_hat in d chi^2 / dP per classified wire
    for (int q = 0; q < A.n; ++q) {
        if (A.j[q] == -3) {
            flags |= CDC_FLAG_LOST_HIT;
            A.u[q] = 0.f;
            continue;
        }
        if (!(A.D[q] > 0.f)) {
            flags |= CDC_FLAG_DOCA_ZERO;
            A.j[q] = -3;
            continue;
        }
        const double r = ((double)A.D[q] - (double)A.drift[q]) / sigma;
        chi2 += r * r;
        A.D[q] = (float)(2.0 * r / sigma);  // reuse D as the injection coefficient
        ++used;
    }
    if (!grad) return chi2;
    // backward sweep over blocks of steps
    float rb[3] = {0.f, 0.f, 0.f}, tb[3] = {0.f, 0.f, 0.f}, lb = 0.f;
    float rl[3] = {0.f, 0.f, 0.f}, tl[3] = {0.f, 0.f, 0.f}, ll = 0.f;  // low words of the compensated sums
    const float h = P.h;
    // end point minima inject into the last state
    for (int q = 0; q < A.n; ++q)
        if (A.j[q] == -2) {
            kahan(rb[0], rl[0], A.D[q] * A.nx[q]);
            kahan(rb[1], rl[1], A.D[q] * A.ny[q]);
            kahan(rb[2], rl[2], A.D[q] * A.nz[q]);
        }
    // entries with a minimum inside a segment, by segment descending (the
    // sweep's order) and by entry within a segment (insertion sort, stable):
    // the sweep takes them with a moving pointer instead of a scan of A per step
    static_assert(MAX_ASSIGNED <= 256, "entry indices are kept in 8 bits");
    uint8_t ord[MAX_ASSIGNED];
    int n_ord = 0;
    for (int q = 0; q < A.n; ++q)
        if (A.j[q] >= 0) {
            const int jq = A.j[q];
            int b = n_ord - 1;
            while (b >= 0 && A.j[ord[b]] < jq) {
                ord[b + 1] = ord[b];
                --b;
            }
            ord[b + 1] = (uint8_t)q;
            ++n_ord;
        }
    int next = 0;
    const int nblocks = (n + ck_every - 1) / ck_every;
    for (int b = nblocks - 1; b >= 0; --b) {
        const int j0 = b * ck_every, j1 = min(n, j0 + ck_every);  // steps j0 .. j1-1 (state j -> j+1)
        State s;
        const float* c = ck[b];
        s.rx = c[0]; s.ry = c[1]; s.rz = c[2]; s.lx = c[3]; s.ly = c[4]; s.lz = c[5];
        s.tx = c[6]; s.ty = c[7]; s.tz = c[8]; s.mx = c[9]; s.my = c[10]; s.mz = c[11]; s.lam = c[12];
        s.lam_lo = c[13];
        for (int j = j0; j <= j1; ++j) {
            buf[j - j0][0] = s.rx; buf[j - j0][1] = s.ry; buf[j - j0][2] = s.rz;
            buf[j - j0][3] = s.tx; buf[j - j0][4] = s.ty; buf[j - j0][5] = s.tz;
            if (j < j1) rkn_step<KIND, true>(F, s, h, P.h6_lo);
        }
        const float lam = c[12];
        for (int j = j1 - 1; j >= j0; --j) {
            // minima inside segment j: P = a0 r_j + a1 t_j + b0 r_j+1 + b1 t_j+1
            float pr[3] = {0.f, 0.f, 0.f}, ptt[3] = {0.f, 0.f, 0.f};
            for (; next < n_ord && A.j[ord[next]] == j; ++next) {
                const int q = ord[next];
                float a0, a1, b0, b1;
                hermite_w(A.u[q], h, a0, a1, b0, b1);
                const float nv[3] = {A.D[q] * A.nx[q], A.D[q] * A.ny[q], A.D[q] * A.nz[q]};
                for (int a = 0; a < 3; ++a) {
                    kahan(rb[a], rl[a], b0 * nv[a]);
                    kahan(tb[a], tl[a], b1 * nv[a]);
                    pr[a] = fmaf(a0, nv[a], pr[a]);
                    ptt[a] = fmaf(a1, nv[a], ptt[a]);
                }
            }
            Stages<KIND> S;
            const float r[3] = {buf[j - j0][0], buf[j - j0][1], buf[j - j0][2]};
            const float t[3] = {buf[j - j0][3], buf[j - j0][4], buf[j - j0][5]};
            S.eval(F, r, t, lam, h);
            adjoint_step<KIND>(S, lam, h, rb, tb, lb, rl, tl, ll);
            for (int a = 0; a < 3; ++a) {
                kahan(rb[a], rl[a], pr[a]);
                kahan(tb[a], tl[a], ptt[a]);
            }
        }
    }
    for (int q = 0; q < A.n; ++q)
        if (A.j[q] == -1) {
            kahan(rb[0], rl[0], A.D[q] * A.nx[q]);
            kahan(rb[1], rl[1], A.D[q] * A.ny[q]);
            kahan(rb[2], rl[2], A.D[q] * A.nz[q]);
        }
    double rbd[3], tbd[3];
    for (int a = 0; a < 3; ++a) {
        rbd[a] = (double)rb[a] + (double)rl[a];
        tbd[a] = (double)tb[a] + (double)tl[a];
    }
    const double lbd = (double)lb + (double)ll;
    // seed: r0 = (R0 cos th, R0 sin th, z0), t0 = dir p/|p|, lam = q' kappa/|p|
    const double p = sqrt(sd[2] * sd[2] + sd[3] * sd[3] + sd[4] * sd[4]);
    const double dir = P.direction < 0 ? -1.0 : 1.0;
    const double lam0 = (double)P.charge_dir * KAPPA_D / p;
    double st, ct;
    sincos(sd[0], &st, &ct);
    const double th[3] = {sd[2] / p, sd[3] / p, sd[4] / p};
    const double tdot = th[0] * tbd[0] + th[1] * tbd[1] + th[2] * tbd[2];
    grad[0] = (float)(-G.R0d * st * rbd[0] + G.R0d * ct * rbd[1]);
    grad[1] = (float)rbd[2];
    for (int b = 0; b < 3; ++b) grad[2 + b] = (float)(dir * (tbd[b] - th[b] * tdot) / p - lbd * lam0 * th[b] / p);
    return chi2;
}

// Thread per seed.  Capped at 128 registers (512 threads per SM, a few
// hundred bytes of spills): the ~225 the code would take leave half the
// threads, half the latency hiding and, for 65536 seeds, 1.7 waves (measured
// 128 -> 118 ms for 65536 seeds x 5 iterations).  64-thread blocks: 65536
// seeds spread as 6-7 blocks over each SM instead of 3-4 blocks of 128
// (91.0 against 93.0 ms; 32-thread blocks, whose shared tables leave less L1,
// 99.5 ms).
constexpr int REFINE_BLOCK = 64;

template <int KIND>
__global__ void __launch_bounds__(REFINE_BLOCK, 512 / REFINE_BLOCK)
    refine_kernel(DevGeom G, DevField F, ScanConst P, RefArgs a, int do_gn) {
    __shared__ DevLayer s_lay[CDC_MAX_LAYERS];
    __shared__ uchar2 s_tab[TAB_N];
    __shared__ ListEntry s_cand[LIST_CAP][REFINE_BLOCK];
    for (int i = threadIdx.x; i < G.n_layers; i += blockDim.x) s_lay[i] = G.layers[i];
    for (int i = threadIdx.x; i < TAB_N; i += blockDim.x) s_tab[i] = G.tab[i];
    __syncthreads();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n_seeds) return;
    const int e = a.seed_event[i];
    if (e < 0 || e >= a.n_events) {
        const double nan = __longlong_as_double(0x7ff8000000000000ll);
        a.chi2[i] = nan;
        for (int m = 0; m < 5; ++m) {
            if (a.grad) a.grad[(size_t)i * 5 + m] = __int_as_float(0x7fffffff);
            if (a.seeds_out) a.seeds_out[(size_t)i * 5 + m] = __int_as_float(0x7fffffff);
        }
        if (a.n_used) a.n_used[i] = 0;
        a.flags[i] = CDC_FLAG_BAD_HIT;
        return;
    }
    const float* dtab = a.drift_tab + (size_t)e * event_stride(G.n_wires);
    double sd[5];
    float sf[5];
    for (int m = 0; m < 5; ++m) {
        sf[m] = a.seeds[(size_t)i * 5 + m];
        sd[m] = sf[m];
    }
    uint32_t flags = 0;
    // 1. classification at the starting seed (the scan's rule)
    Assigned A;
    {
        Tracer<KIND> T;
        FoundList FL;
        T.init(G, F, P, s_lay, s_tab, dtab, &s_cand[0][threadIdx.x], REFINE_BLOCK, sf, FL);
        while (T.step(G, F, P, s_lay, s_tab, FL))
            if (T.n % LIST_M == 0) {
                T.rebuild(G, P, s_lay, s_tab);
                T.make_room(P, FL);
            }
        flags |= T.flags;
        A.n = 0;
        for (int q = 0; q < T.nf; ++q) {  // each wire once, at its first entry
            const int w = key_wire(FL.key[q]);
            bool first = true;
            for (int j = 0; j < q; ++j) first &= key_wire(FL.key[j]) != w;
            if (!first) continue;
            int part;
            record_class(FL.key, FL.r, T.nf, w, P.lam, part);
            if (part < 0) continue;
            if (A.n < MAX_ASSIGNED)
                A.key[A.n++] = (uint32_t)w | ((uint32_t)part << 16);
            else
                flags |= CDC_FLAG_FOUND_OVERFLOW;
        }
    }
    for (int q = 1; q < A.n; ++q) {  // sort by wire
        const uint32_t k = A.key[q];
        int p = q - 1;
        while (p >= 0 && (A.key[p] & 0xffffu) > (k & 0xffffu)) {
            A.key[p + 1] = A.key[p];
            --p;
        }
        A.key[p + 1] = k;
    }
    for (int q = 0; q < A.n; ++q) A.drift[q] = __ldg(dtab + (A.key[q] & 0xffffu));
    // 2. Gauss-Newton
    if (do_gn) {
        for (int it = 0; it < a.n_iter; ++it) {
            track_pass<KIND, true, false>(G, F, P, s_lay, s_tab, dtab, sd, a.sigma, A, nullptr, 1, flags);
            double JtJ[25], Jtr[5];
            for (int m = 0; m < 25; ++m) JtJ[m] = 0.0;
            for (int m = 0; m < 5; ++m) Jtr[m] = 0.0;
            for (int q = 0; q < A.n; ++q) {
                if (A.j[q] == -3 || !(A.D[q] > 0.f)) continue;
                const double r = ((double)A.D[q] - (double)A.drift[q]) / a.sigma;
                for (int m = 0; m < 5; ++m) {
                    const double jm = (double)A.J[q][m] * a.scale[m];
                    Jtr[m] += jm * r;
                    for (int l = 0; l <= m; ++l) JtJ[5 * m + l] += jm * (double)A.J[q][l] * a.scale[l];
                }
            }
            for (int m = 0; m < 5; ++m)
                for (int l = m + 1; l < 5; ++l) JtJ[5 * m + l] = JtJ[5 * l + m];
            double b[5], A0[25];
            for (int m = 0; m < 5; ++m) b[m] = -Jtr[m];
            for (int m = 0; m < 25; ++m) A0[m] = JtJ[m];
            if (!chol5(A0, b)) {
                double tr = 0.0;
                for (int m = 0; m < 5; ++m) tr += JtJ[5 * m + m];
                for (int m = 0; m < 25; ++m) A0[m] = JtJ[m];
                for (int m = 0; m < 5; ++m) {
                    A0[5 * m + m] += 1e-6 * tr / 5.0;
                    b[m] = -Jtr[m];
                }
                flags |= CDC_FLAG_NOT_SPD;
                if (!chol5(A0, b)) break;
            }
            bool fin = true;
            for (int m = 0; m < 5; ++m) fin &= isfinite(b[m]);
            if (!fin) {
                flags |= CDC_FLAG_NOT_SPD;
                break;
            }
            for (int m = 0; m < 5; ++m) sd[m] += b[m] * a.scale[m];
        }
    }
    // 3. chi^2 (FP64 sum) and adjoint gradient at the final seed
    float ck[MAX_CK][14];
    float buf[MAX_BLOCK + 1][6];
    float g[5];
    int used = 0;
    const double c2 = chi2_adjoint<KIND>(G, F, P, s_lay, s_tab, dtab, sd, a.sigma, a.checkpoint, A, ck, buf,
                                         a.grad ? g : nullptr, used, flags);
    a.chi2[i] = c2;
    if (a.grad)
        for (int m = 0; m < 5; ++m) a.grad[(size_t)i * 5 + m] = g[m];
    if (a.seeds_out)
        for (int m = 0; m < 5; ++m) a.seeds_out[(size_t)i * 5 + m] = (float)sd[m];
    if (a.n_used) a.n_used[i] = used;
    a.flags[i] = flags;
}

// Shared-memory share of the SM for the refine kernel: just what its resident
// blocks (the launch bounds) need, so that the rest of the SM's on-chip
// memory serves as L1 for the threads' local stacks (classified hits,
// checkpoints, the adjoint's buffer).  Set as a preference before each launch.
template <class K>
static cudaError_t prefer_l1(K kernel) {
    constexpr int RESIDENT = 512 / REFINE_BLOCK;
    cudaFuncAttributes fa;
    cudaError_t err = cudaFuncGetAttributes(&fa, kernel);
    int dev = 0, per_sm = 0, reserved = 0;
    if (err == cudaSuccess) err = cudaGetDevice(&dev);
    if (err == cudaSuccess) err = cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    if (err == cudaSuccess) err = cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
    if (err != cudaSuccess || per_sm <= 0) return err;
    const long long need = (long long)RESIDENT * ((long long)fa.sharedSizeBytes + reserved);
    const int pct = (int)std::min<long long>(100, (need * 100 + per_sm - 1) / per_sm);
    return cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, pct);
}

cudaError_t launch_refine(const DevGeom& G, const DevField& F, const ScanConst& P, const RefineLaunch& L,
                          float* drift_tab, int num_sms, int do_gn, cudaStream_t st) {
    cudaError_t err = launch_stage(G, L.n_events, L.hit_off, L.wire_id, L.drift, P.max_drift, drift_tab, nullptr,
                                   num_sms, st);
    if (err != cudaSuccess) return err;
    RefArgs a{L.n_seeds, L.seed_event, L.seeds, L.n_events, L.hit_off, drift_tab, L.n_iter, L.sigma,
              {L.scale[0], L.scale[1], L.scale[2], L.scale[3], L.scale[4]}, L.checkpoint, L.seeds_out, L.chi2, L.grad,
              L.n_used, L.flags};
    const int bs = REFINE_BLOCK, nb = (L.n_seeds + bs - 1) / bs;
    if (F.kind == 0) {
        if ((err = prefer_l1(refine_kernel<0>)) != cudaSuccess) return err;
        refine_kernel<0><<<nb, bs, 0, st>>>(G, F, P, a, do_gn);
    } else {
        if ((err = prefer_l1(refine_kernel<1>)) != cudaSuccess) return err;
        refine_kernel<1><<<nb, bs, 0, st>>>(G, F, P, a, do_gn);
    }
    return cudaGetLastError();
}

}  // namespace cdc
