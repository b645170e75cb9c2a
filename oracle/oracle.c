/*
 * FP64 CPU oracle for the seed-scanning track finder of
 * "GPU Tracking in the COMET Phase-I Cylindrical Drift Chamber" (arXiv:1908.01949).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg and reference arm may load this file's library.  It shares no
 * code, header or table with the CUDA library: it rebuilds the wire table, the
 * Hough offsets and every formula from the definitions below, plainly, in
 * double precision, with no blocking or reordering beyond what the definitions
 * state.
 *
 * What it computes (paper section / equation cited per function):
 *   - classical Runge-Kutta-Nystrom propagation (sec. 2.2, [STEP]) of a seed
 *     (sec. 2.1: R0, theta0, z0, px0, py0, pz0) through a uniform field or a
 *     bilinear (r,z) field map;
 *   - the distance of closest approach (DCA) of the continuous track to each
 *     fired wire line, per turn partition, by brute force over all steps;
 *   - the score E = sum_wires min(d_L^2, d_R^2, lambda) (Eq. 1) and the hit-to-
 *     turn classification d^2 < lambda (sec. 2.2);
 *   - the integer circle Hough transform and its peaks (sec. 2.1, Fig. 4);
 *   - a Gauss-Newton refinement of a seed with FP64 forward tangents (not in
 *     the paper; it replaces the Kalman fit of sec. 2.2 for seed refinement).
 * Readings where the paper is silent are listed in the design notes of the
 * repository; the key ones are restated next to the code that uses them.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_KAPPA 0.299792458 /* MeV/c per (T mm) */
#define ORC_PI 3.14159265358979323846
#define ORC_MAX_LAYERS 64

enum { ORC_FLAG_STEP_CAP = 1, ORC_FLAG_NOT_SPD = 8, ORC_FLAG_DOCA_ZERO = 16, ORC_FLAG_LOST_HIT = 32 };

typedef struct {
    int n_layers;
    const double* R;       /* waist radius at z = 0 [mm] */
    const double* alpha;   /* stereo angle [rad] */
    const int* N;          /* wires per layer */
    const double* phi_off; /* azimuth of wire 0 [rad] */
    double z_half, R0, R_out;
} orc_geometry;

typedef struct {
    int kind;              /* 0 uniform Bz = B0, 1 bilinear (r,z) map */
    double B0;
    int nr, nz;
    double r_min, z_min, dr, dz;
    const float* bz;       /* [nr][nz] */
    const float* br;
} orc_field;

typedef struct {
    double h;              /* RKN step [mm] */
    int max_steps;
    double lam;            /* cutoff lambda of Eq. 1 [mm^2] */
    int max_partitions;
    int direction;         /* +1 seed propagated along p, -1 against p */
    double charge;         /* particle charge in units of e */
} orc_scan_params;

/* ------------------------------------------------------------- geometry */
/* Wire line of global wire index w: midpoint m (z = 0) and unit direction d.
 * Wire i of layer l sits at phi = phi_off + 2 pi i / N_l, tilted by alpha_l
 * along the azimuthal direction (sec. 1: stereo layers). */
static int orc_wire_line(const orc_geometry* g, int w, double m[3], double d[3]) {
    int base = 0;
    for (int l = 0; l < g->n_layers; ++l) {
        if (w < base + g->N[l]) {
            int i = w - base;
            double phi = g->phi_off[l] + 2.0 * ORC_PI * (double)i / (double)g->N[l];
            double sa = sin(g->alpha[l]), ca = cos(g->alpha[l]);
            m[0] = g->R[l] * cos(phi);
            m[1] = g->R[l] * sin(phi);
            m[2] = 0.0;
            d[0] = -sa * sin(phi);
            d[1] = sa * cos(phi);
            d[2] = ca;
            return l;
        }
        base += g->N[l];
    }
    return -1;
}

static int orc_n_wires(const orc_geometry* g) {
    int n = 0;
    for (int l = 0; l < g->n_layers; ++l) n += g->N[l];
    return n;
}

/* ---------------------------------------------------------------- field */
/* B(r): uniform (0,0,B0), or bilinear interpolation in (rho, z) of the map
 * samples with coordinates clamped to the grid; Bx = Br x/rho, By = Br y/rho.
 * If grad != NULL also returns dB_i/dx_j (row i, column j) of that same
 * piecewise-bilinear function (zero along a clamped coordinate). */
static void orc_field_eval(const orc_field* f, const double r[3], double B[3], double grad[9]) {
    if (grad) memset(grad, 0, 9 * sizeof(double));
    if (f->kind == 0) {
        B[0] = 0.0; B[1] = 0.0; B[2] = f->B0;
        return;
    }
    double rho = sqrt(r[0] * r[0] + r[1] * r[1]);
    double rmax = f->r_min + f->dr * (f->nr - 1), zmax = f->z_min + f->dz * (f->nz - 1);
    int clamp_r = (rho < f->r_min) || (rho > rmax);
    int clamp_z = (r[2] < f->z_min) || (r[2] > zmax);
    double rc = rho < f->r_min ? f->r_min : (rho > rmax ? rmax : rho);
    double zc = r[2] < f->z_min ? f->z_min : (r[2] > zmax ? zmax : r[2]);
    double u = (rc - f->r_min) / f->dr, v = (zc - f->z_min) / f->dz;
    int i = (int)floor(u), j = (int)floor(v);
    if (i > f->nr - 2) i = f->nr - 2;
    if (j > f->nz - 2) j = f->nz - 2;
    if (i < 0) i = 0;
    if (j < 0) j = 0;
    u -= i;
    v -= j;
    double z00 = f->bz[i * f->nz + j], z10 = f->bz[(i + 1) * f->nz + j];
    double z01 = f->bz[i * f->nz + j + 1], z11 = f->bz[(i + 1) * f->nz + j + 1];
    double r00 = f->br[i * f->nz + j], r10 = f->br[(i + 1) * f->nz + j];
    double r01 = f->br[i * f->nz + j + 1], r11 = f->br[(i + 1) * f->nz + j + 1];
    double bz = (1 - u) * (1 - v) * z00 + u * (1 - v) * z10 + (1 - u) * v * z01 + u * v * z11;
    double br = (1 - u) * (1 - v) * r00 + u * (1 - v) * r10 + (1 - u) * v * r01 + u * v * r11;
    if (rho > 0.0) {
        B[0] = br * r[0] / rho;
        B[1] = br * r[1] / rho;
    } else {
        B[0] = 0.0;
        B[1] = 0.0;
    }
    B[2] = bz;
    if (grad && rho > 0.0) {
        double dbz_drho = clamp_r ? 0.0 : ((1 - v) * (z10 - z00) + v * (z11 - z01)) / f->dr;
        double dbr_drho = clamp_r ? 0.0 : ((1 - v) * (r10 - r00) + v * (r11 - r01)) / f->dr;
        double dbz_dz = clamp_z ? 0.0 : ((1 - u) * (z01 - z00) + u * (z11 - z10)) / f->dz;
        double dbr_dz = clamp_z ? 0.0 : ((1 - u) * (r01 - r00) + u * (r11 - r10)) / f->dz;
        double cx = r[0] / rho, cy = r[1] / rho;
        /* Bx = br cx: d/dx = dbr_drho cx cx + br (1 - cx cx)/rho */
        grad[0] = dbr_drho * cx * cx + br * (1.0 - cx * cx) / rho;
        grad[1] = dbr_drho * cx * cy - br * cx * cy / rho;
        grad[2] = dbr_dz * cx;
        grad[3] = dbr_drho * cy * cx - br * cx * cy / rho;
        grad[4] = dbr_drho * cy * cy + br * (1.0 - cy * cy) / rho;
        grad[5] = dbr_dz * cy;
        grad[6] = dbz_drho * cx;
        grad[7] = dbz_drho * cy;
        grad[8] = dbz_dz;
    }
}

/* ------------------------------------------------------------ RKN step */
static void cross3(const double a[3], const double b[3], double c[3]) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

/* One classical Runge-Kutta-Nystrom step (Abramowitz & Stegun 25.5.20) of
 * length u (any sign) for r'' = f(r', r) = lam * (r' x B(r)), arclength as the
 * independent variable, t = r' the unit direction, lam = q kappa / p.
 * Field at the start, at the midpoint r + u/2 t + u^2/8 k1 (shared by k2, k3)
 * and at the end estimate r + u t + u^2/2 k3. */
static void orc_rkn_step(const orc_field* f, double lam, double u, const double r[3], const double t[3],
                         double r_out[3], double t_out[3]) {
    double B[3], k1[3], k2[3], k3[3], k4[3], tt[3], rm[3], re[3], c[3];
    orc_field_eval(f, r, B, NULL);
    cross3(t, B, c);
    for (int a = 0; a < 3; ++a) k1[a] = lam * c[a];
    for (int a = 0; a < 3; ++a) {
        rm[a] = r[a] + 0.5 * u * t[a] + u * u / 8.0 * k1[a];
        tt[a] = t[a] + 0.5 * u * k1[a];
    }
    orc_field_eval(f, rm, B, NULL);
    cross3(tt, B, c);
    for (int a = 0; a < 3; ++a) k2[a] = lam * c[a];
    for (int a = 0; a < 3; ++a) tt[a] = t[a] + 0.5 * u * k2[a];
    cross3(tt, B, c);
    for (int a = 0; a < 3; ++a) k3[a] = lam * c[a];
    for (int a = 0; a < 3; ++a) {
        re[a] = r[a] + u * t[a] + 0.5 * u * u * k3[a];
        tt[a] = t[a] + u * k3[a];
    }
    orc_field_eval(f, re, B, NULL);
    cross3(tt, B, c);
    for (int a = 0; a < 3; ++a) k4[a] = lam * c[a];
    for (int a = 0; a < 3; ++a) {
        r_out[a] = r[a] + u * t[a] + u * u / 6.0 * (k1[a] + k2[a] + k3[a]);
        t_out[a] = t[a] + u / 6.0 * (k1[a] + 2.0 * k2[a] + 2.0 * k3[a] + k4[a]);
    }
}

/* The same step for state + NT tangent vectors (dr, dt, dlam) — the exact
 * linearisation of orc_rkn_step, used for the Jacobian of refine. */
#define NT 5
typedef struct { double r[3], t[3], lam; } orc_tan;

static void lin_stage(const orc_field* f, double lam, const double tt[3], const double rr[3],
                      const orc_tan* d_in /*dt in .t, dr in .r*/, double k[3], double dk[NT][3],
                      const double* dlam) {
    double B[3], G[9], c[3];
    orc_field_eval(f, rr, B, G);
    cross3(tt, B, c);
    for (int a = 0; a < 3; ++a) k[a] = lam * c[a];
    for (int n = 0; n < NT; ++n) {
        double dB[3], c1[3], c2[3];
        for (int a = 0; a < 3; ++a)
            dB[a] = G[3 * a + 0] * d_in[n].r[0] + G[3 * a + 1] * d_in[n].r[1] + G[3 * a + 2] * d_in[n].r[2];
        cross3(d_in[n].t, B, c1);
        cross3(tt, dB, c2);
        for (int a = 0; a < 3; ++a) dk[n][a] = dlam[n] * c[a] + lam * (c1[a] + c2[a]);
    }
}

static void orc_rkn_step_tan(const orc_field* f, double lam, double u, const double r[3], const double t[3],
                             const orc_tan* T, double r_out[3], double t_out[3], orc_tan* T_out) {
    double k1[3], k2[3], k3[3], k4[3], tt[3], rm[3], re[3];
    double dk1[NT][3], dk2[NT][3], dk3[NT][3], dk4[NT][3];
    double dlam[NT];
    orc_tan S[NT];
    for (int n = 0; n < NT; ++n) dlam[n] = T[n].lam;
    /* stage 1 at (t, r) */
    for (int n = 0; n < NT; ++n) S[n] = T[n];
    lin_stage(f, lam, t, r, S, k1, dk1, dlam);
    /* stage 2 at (t + u/2 k1, r + u/2 t + u^2/8 k1) */
    for (int a = 0; a < 3; ++a) {
        tt[a] = t[a] + 0.5 * u * k1[a];
        rm[a] = r[a] + 0.5 * u * t[a] + u * u / 8.0 * k1[a];
    }
    for (int n = 0; n < NT; ++n)
        for (int a = 0; a < 3; ++a) {
            S[n].t[a] = T[n].t[a] + 0.5 * u * dk1[n][a];
            S[n].r[a] = T[n].r[a] + 0.5 * u * T[n].t[a] + u * u / 8.0 * dk1[n][a];
        }
    lin_stage(f, lam, tt, rm, S, k2, dk2, dlam);
    /* stage 3 at (t + u/2 k2, r_m) */
    for (int a = 0; a < 3; ++a) tt[a] = t[a] + 0.5 * u * k2[a];
    for (int n = 0; n < NT; ++n)
        for (int a = 0; a < 3; ++a) S[n].t[a] = T[n].t[a] + 0.5 * u * dk2[n][a];
    lin_stage(f, lam, tt, rm, S, k3, dk3, dlam);
    /* stage 4 at (t + u k3, r + u t + u^2/2 k3) */
    for (int a = 0; a < 3; ++a) {
        tt[a] = t[a] + u * k3[a];
        re[a] = r[a] + u * t[a] + 0.5 * u * u * k3[a];
    }
    for (int n = 0; n < NT; ++n)
        for (int a = 0; a < 3; ++a) {
            S[n].t[a] = T[n].t[a] + u * dk3[n][a];
            S[n].r[a] = T[n].r[a] + u * T[n].t[a] + 0.5 * u * u * dk3[n][a];
        }
    lin_stage(f, lam, tt, re, S, k4, dk4, dlam);
    for (int a = 0; a < 3; ++a) {
        r_out[a] = r[a] + u * t[a] + u * u / 6.0 * (k1[a] + k2[a] + k3[a]);
        t_out[a] = t[a] + u / 6.0 * (k1[a] + 2.0 * k2[a] + 2.0 * k3[a] + k4[a]);
    }
    for (int n = 0; n < NT; ++n) {
        for (int a = 0; a < 3; ++a) {
            T_out[n].r[a] = T[n].r[a] + u * T[n].t[a] + u * u / 6.0 * (dk1[n][a] + dk2[n][a] + dk3[n][a]);
            T_out[n].t[a] = T[n].t[a] + u / 6.0 * (dk1[n][a] + 2.0 * dk2[n][a] + 2.0 * dk3[n][a] + dk4[n][a]);
        }
        T_out[n].lam = T[n].lam;
    }
}

/* ------------------------------------------------------------ the seed */
/* Seed (theta0, z0, px0, py0, pz0) at cylinder radius R0 (sec. 2.1) -> state.
 * direction = -1 reverses the track: t -> -t and q -> -q. */
static void orc_seed_state(const orc_geometry* g, const orc_scan_params* P, const double s[5],
                           double r[3], double t[3], double* lam, orc_tan* T) {
    double p = sqrt(s[2] * s[2] + s[3] * s[3] + s[4] * s[4]);
    double dir = P->direction < 0 ? -1.0 : 1.0;
    r[0] = g->R0 * cos(s[0]);
    r[1] = g->R0 * sin(s[0]);
    r[2] = s[1];
    double th[3] = {s[2] / p, s[3] / p, s[4] / p};
    for (int a = 0; a < 3; ++a) t[a] = dir * th[a];
    *lam = dir * P->charge * ORC_KAPPA / p;
    if (T) {
        memset(T, 0, NT * sizeof(orc_tan));
        T[0].r[0] = -g->R0 * sin(s[0]);
        T[0].r[1] = g->R0 * cos(s[0]);
        T[1].r[2] = 1.0;
        for (int b = 0; b < 3; ++b) {
            for (int a = 0; a < 3; ++a) T[2 + b].t[a] = dir * (((a == b) ? 1.0 : 0.0) - th[a] * th[b]) / p;
            T[2 + b].lam = -(*lam) * th[b] / p;
        }
    }
}

/* ------------------------------------------------------------ the trace */
/* Propagate one seed with fixed step h.  States j = 0..n are written to
 * st[7*j] = (x, y, z, tx, ty, tz, partition).  Turn partitions (reading of
 * sec. 2.2/4.2 "turn partition"): partition 0 starts at the seed; each inward
 * crossing of the R0 cylinder (previous state at rho >= R0, this one below;
 * the seed counts as outside) starts the next one; propagation stops after
 * the state that ends partition max_partitions-1, after the first state with
 * |z| > z_half or rho > R_out, or after max_steps steps (flag STEP_CAP).
 * *margin = smallest distance of any state j >= 1 to one of these decision
 * boundaries (|rho-R0|, |rho-R_out|, ||z|-z_half|).  Returns n + 1. */
static int orc_trace(const orc_geometry* g, const orc_field* f, const orc_scan_params* P, const double s[5],
                     int cap, double* st, orc_tan* tan_st, int* flags, double* margin) {
    double r[3], t[3], lam, rn[3], tn[3];
    orc_tan T[NT], Tn[NT];
    orc_seed_state(g, P, s, r, t, &lam, tan_st ? T : NULL);
    int part = 0, outside = 1, n = 0;
    double mg = INFINITY;
    *flags = 0;
    for (;;) {
        if (n < cap) {
            for (int a = 0; a < 3; ++a) {
                st[7 * n + a] = r[a];
                st[7 * n + 3 + a] = t[a];
            }
            st[7 * n + 6] = part;
            if (tan_st) memcpy(&tan_st[NT * n], T, sizeof(T));
        }
        if (n >= P->max_steps) {
            *flags |= ORC_FLAG_STEP_CAP;
            break;
        }
        if (tan_st)
            orc_rkn_step_tan(f, lam, P->h, r, t, T, rn, tn, Tn);
        else
            orc_rkn_step(f, lam, P->h, r, t, rn, tn);
        memcpy(r, rn, sizeof r);
        memcpy(t, tn, sizeof t);
        if (tan_st) memcpy(T, Tn, sizeof T);
        ++n;
        double rho = sqrt(r[0] * r[0] + r[1] * r[1]);
        double m1 = fabs(rho - g->R0), m2 = fabs(rho - g->R_out), m3 = fabs(fabs(r[2]) - g->z_half);
        if (m1 < mg) mg = m1;
        if (m2 < mg) mg = m2;
        if (m3 < mg) mg = m3;
        int now_out = rho >= g->R0;
        int stop = 0;
        if (outside && !now_out) {
            part += 1;
            if (part >= P->max_partitions) stop = 1;
        }
        outside = now_out;
        if (fabs(r[2]) > g->z_half || rho > g->R_out) stop = 1;
        if (stop) {
            if (n < cap) {
                for (int a = 0; a < 3; ++a) {
                    st[7 * n + a] = r[a];
                    st[7 * n + 3 + a] = t[a];
                }
                st[7 * n + 6] = part;
                if (tan_st) memcpy(&tan_st[NT * n], T, sizeof(T));
            }
            break;
        }
    }
    *margin = mg;
    return n + 1;
}

/* ------------------------------------------------------------- the DCA */
static double line_dist(const double p[3], const double m[3], const double d[3]) {
    double w[3] = {p[0] - m[0], p[1] - m[1], p[2] - m[2]};
    double wd = w[0] * d[0] + w[1] * d[1] + w[2] * d[2];
    double q0 = w[0] - wd * d[0], q1 = w[1] - wd * d[1], q2 = w[2] - wd * d[2];
    return sqrt(q0 * q0 + q1 * q1 + q2 * q2);
}

/* Distance from the wire of the point reached by one RKN step of length u
 * from state j (the continuous track between recorded states, cf. sec. 4.2:
 * propagation restarted from the recorded state closest to the wire). */
static double sub_dist(const orc_field* f, double lam, const double* sj, double u, const double m[3],
                       const double d[3]) {
    double ro[3], to[3];
    orc_rkn_step(f, lam, u, sj, sj + 3, ro, to);
    return line_dist(ro, m, d);
}

/* Golden-section minimisation of sub_dist over [lo, hi] to |hi-lo| < 1e-11 mm. */
static double golden_min(const orc_field* f, double lam, const double* sj, double lo, double hi,
                         const double m[3], const double d[3], double* u_best) {
    const double gr = 0.6180339887498949;
    double a = lo, b = hi;
    double c = b - gr * (b - a), e = a + gr * (b - a);
    double fc = sub_dist(f, lam, sj, c, m, d), fe = sub_dist(f, lam, sj, e, m, d);
    while (b - a > 1e-11) {
        if (fc < fe) {
            b = e;
            e = c;
            fe = fc;
            c = b - gr * (b - a);
            fc = sub_dist(f, lam, sj, c, m, d);
        } else {
            a = c;
            c = e;
            fc = fe;
            e = a + gr * (b - a);
            fe = sub_dist(f, lam, sj, e, m, d);
        }
    }
    double ub = 0.5 * (a + b);
    double fb = sub_dist(f, lam, sj, ub, m, d);
    /* the interval ends are candidates too (minimum at a trajectory end) */
    double flo = sub_dist(f, lam, sj, lo, m, d), fhi = sub_dist(f, lam, sj, hi, m, d);
    if (flo < fb) { fb = flo; ub = lo; }
    if (fhi < fb) { fb = fhi; ub = hi; }
    *u_best = ub;
    return fb;
}

typedef struct {
    double doca;  /* per-partition DCA (INFINITY if no local minimum) */
    int j;        /* state index of the minimum */
    double u;     /* sub-step length from state j */
} orc_min;

/* DCA_k(w) for every partition k < max_partitions of a recorded trace:
 * every discrete local minimum j of D_j = dist(r_j, line) (ends included,
 * D_j <= D_{j-1} and D_j < D_{j+1}) is refined over one RKN sub-step
 * u in [-h, h] (clipped at the trace ends); the smallest refined value of each
 * partition is kept.  Minima whose D_j - h exceeds `prune` are skipped: the
 * distance is 1-Lipschitz in arclength, so their refined value stays above
 * prune (callers pass drift + sqrt(lambda), where the score term is lambda). */
static void orc_wire_doca(const orc_field* f, double lam, double h, const double* st, int ns,
                          const double m[3], const double d[3], double prune, int max_part, orc_min* out) {
    for (int k = 0; k < max_part; ++k) {
        out[k].doca = INFINITY;
        out[k].j = -1;
        out[k].u = 0.0;
    }
    double Dprev = INFINITY, Dcur = line_dist(st, m, d);
    for (int j = 0; j < ns; ++j) {
        double Dnext = (j + 1 < ns) ? line_dist(st + 7 * (j + 1), m, d) : INFINITY;
        int is_min = (j == 0 || Dcur <= Dprev) && (j == ns - 1 || Dcur < Dnext);
        int k = (int)st[7 * j + 6];
        if (is_min && k < max_part && Dcur - h <= prune) {
            double lo = (j > 0) ? -h : 0.0, hi = (j < ns - 1) ? h : 0.0, ub;
            double v = golden_min(f, lam, st + 7 * j, lo, hi, m, d, &ub);
            if (v < out[k].doca) {
                out[k].doca = v;
                out[k].j = j;
                out[k].u = ub;
            }
        }
        Dprev = Dcur;
        Dcur = Dnext;
    }
}

/* ------------------------------------------------------------- the scan */
/* Eq. 1 for a list of seeds.  Per seed: E = sum over fired wires of
 * min( min_k (|DCA_k| - drift)^2, lambda ) — d_L, d_R are the distances to the
 * two mirror points at +-drift across the track, so min(d_L^2, d_R^2) =
 * (|DCA| - drift)^2.  Optional per (seed, hit) outputs: best squared residual,
 * its partition (argmin k, ties to the lower k; -1 when >= lambda: the hit
 * classification of sec. 2.2) and the distance in mm of |res| to the nearest
 * classification cut (lambda or another partition's |res|). */
int orc_scan(const orc_geometry* g, const orc_field* f, const orc_scan_params* P, int n_hits,
             const int* wire_id, const double* drift, int n_seeds, const double* seeds, double* E,
             int* n_steps, int* flags, double* margin, double* hit_res2, int* hit_part, double* hit_margin) {
    int cap = P->max_steps + 1;
    double* st = (double*)malloc(sizeof(double) * 7 * (size_t)cap);
    orc_min* mins = (orc_min*)malloc(sizeof(orc_min) * (size_t)(P->max_partitions > 0 ? P->max_partitions : 1));
    if (!st || !mins) {
        free(st);
        free(mins);
        return -1;
    }
    double sl = sqrt(P->lam);
    int nw = orc_n_wires(g);
    for (int s = 0; s < n_seeds; ++s) {
        double r[3], t[3], lam;
        orc_seed_state(g, P, seeds + 5 * s, r, t, &lam, NULL);
        int fl;
        double mg;
        int ns = orc_trace(g, f, P, seeds + 5 * s, cap, st, NULL, &fl, &mg);
        double e = 0.0;
        for (int i = 0; i < n_hits; ++i) {
            double m[3], d[3];
            if (wire_id[i] < 0 || wire_id[i] >= nw) continue;
            orc_wire_line(g, wire_id[i], m, d);
            orc_wire_doca(f, lam, P->h, st, ns, m, d, drift[i] + sl, P->max_partitions, mins);
            double best = INFINITY, second = INFINITY;
            int bk = -1;
            for (int k = 0; k < P->max_partitions; ++k) {
                if (!isfinite(mins[k].doca)) continue;
                double res = fabs(mins[k].doca - drift[i]);
                if (res < best) {
                    second = best;
                    best = res;
                    bk = k;
                } else if (res < second) {
                    second = res;
                }
            }
            double r2 = best * best;
            e += (r2 < P->lam) ? r2 : P->lam;
            if (hit_res2) hit_res2[(size_t)s * n_hits + i] = r2;
            if (hit_part) hit_part[(size_t)s * n_hits + i] = (r2 < P->lam) ? bk : -1;
            if (hit_margin) {
                double mgn = fabs(best - sl);
                if (isfinite(second) && second - best < mgn) mgn = second - best;
                hit_margin[(size_t)s * n_hits + i] = mgn;
            }
        }
        E[s] = e;
        if (n_steps) n_steps[s] = ns - 1;
        if (flags) flags[s] = fl;
        if (margin) margin[s] = mg;
    }
    free(st);
    free(mins);
    return 0;
}

/* Recorded states of one seed (propagation tests, precision sweep). */
int orc_propagate(const orc_geometry* g, const orc_field* f, const orc_scan_params* P, const double seed[5],
                  int cap, double* states, int* flags, double* margin) {
    return orc_trace(g, f, P, seed, cap, states, NULL, flags, margin);
}

/* One raw RKN step (pins: closed-form helix, order of accuracy). */
void orc_step(const orc_field* f, double lam, double h, const double r[3], const double t[3], double r_out[3],
              double t_out[3]) {
    orc_rkn_step(f, lam, h, r, t, r_out, t_out);
}

/* Field value (pins). */
void orc_field_at(const orc_field* f, const double r[3], double B[3], double grad[9]) {
    orc_field_eval(f, r, B, grad);
}

/* ------------------------------------------------------------ the Hough */
typedef struct {
    int n_bins;     /* accumulator is n_bins x n_bins over the centre (x0, y0) */
    int bin_um;     /* bin width [um], even */
    int origin_um;  /* coordinate of the lower edge of bin 0 [um] */
    int n_r;        /* radii R_j = r_min_um + j r_step_um */
    int r_min_um, r_step_um;
    int n_phi;      /* angles phi_k = 2 pi k / n_phi */
    int target_um;  /* the circle must pass within this distance of the axis */
    int min_peak;   /* absolute threshold of a peak */
    int max_cand;
    int r_hist_half_um;
    double b_nominal, charge, R0;
} orc_hough_params;

/* Wire midpoint of global wire w at z = 0, rounded to integer micrometres. */
static void orc_wire_xy_um(const orc_geometry* g, int w, int64_t* X, int64_t* Y) {
    double m[3], d[3];
    orc_wire_line(g, w, m, d);
    *X = llround(1000.0 * m[0]);
    *Y = llround(1000.0 * m[1]);
}

/* Circle Hough vote (sec. 2.1, Fig. 4): each hit votes, for every radius R_j
 * and angle phi_k, for the circle centre C = X + round(1000 R_j (cos, sin)
 * phi_k) [um], binned by floor((C - origin)/bin); a vote counts only if the
 * circle passes within target of the axis: (R_j - T)^2 <= |C|^2 <= (R_j + T)^2.
 * All arithmetic is integer, so the accumulator is exact in any vote order. */
int orc_hough_vote(const orc_geometry* g, const orc_hough_params* H, int n_hits, const int* wire_id, int32_t* acc) {
    int nb = H->n_bins;
    memset(acc, 0, sizeof(int32_t) * (size_t)nb * nb);
    int nw = orc_n_wires(g);
    for (int i = 0; i < n_hits; ++i) {
        if (wire_id[i] < 0 || wire_id[i] >= nw) continue;
        int64_t X, Y;
        orc_wire_xy_um(g, wire_id[i], &X, &Y);
        for (int j = 0; j < H->n_r; ++j) {
            int64_t R = (int64_t)H->r_min_um + (int64_t)j * H->r_step_um;
            int64_t lo = R - H->target_um, hi = R + H->target_um;
            for (int k = 0; k < H->n_phi; ++k) {
                double ph = 2.0 * ORC_PI * (double)k / (double)H->n_phi;
                int64_t cx = X + llround((double)R * cos(ph));
                int64_t cy = Y + llround((double)R * sin(ph));
                int64_t c2 = cx * cx + cy * cy;
                if (c2 < (lo > 0 ? lo * lo : 0) || c2 > hi * hi) continue;
                int64_t dx = cx - H->origin_um, dy = cy - H->origin_um;
                if (dx < 0 || dy < 0) continue;
                int64_t bx = dx / H->bin_um, by = dy / H->bin_um;
                if (bx >= nb || by >= nb) continue;
                acc[by * nb + bx] += 1;
            }
        }
    }
    return 0;
}

/* Peaks of the accumulator: count >= max(min_peak, ceil(max/2)); strict local
 * maximum over the 3x3 neighbourhood with equal counts resolved toward the
 * lower linear index; ordered by (count desc, index asc); at most max_cand.
 * Per peak: the radius bin with the most hits at |X - C| in
 * [R_j - half, R_j + half) (ties to lower j), and the seed centre where the
 * circle meets r = R0 moving outward: theta0 = atan2(P), (px0, py0) = kappa
 * |B| R t_hat (sec. 2.1: transverse seeds read off the found circle).
 * cand[4*c] = (ix, iy, count, r_bin); centre[3*c] = (theta0, px0, py0) (NaN if
 * the circle does not reach R0). Returns the number of candidates. */
int orc_hough_peaks(const orc_geometry* g, const orc_hough_params* H, int n_hits, const int* wire_id,
                    const int32_t* acc, int32_t* cand, double* centre) {
    int nb = H->n_bins;
    int32_t mx = 0;
    for (int64_t c = 0; c < (int64_t)nb * nb; ++c)
        if (acc[c] > mx) mx = acc[c];
    int32_t thr = (mx + 1) / 2;
    if (thr < H->min_peak) thr = H->min_peak;
    int nc = 0;
    for (int iy = 0; iy < nb; ++iy)
        for (int ix = 0; ix < nb; ++ix) {
            int64_t c = (int64_t)iy * nb + ix;
            int32_t v = acc[c];
            if (v < thr) continue;
            int peak = 1;
            for (int dy = -1; dy <= 1 && peak; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    if (!dx && !dy) continue;
                    int x = ix + dx, y = iy + dy;
                    if (x < 0 || y < 0 || x >= nb || y >= nb) continue;
                    int64_t n = (int64_t)y * nb + x;
                    if (acc[n] > v || (acc[n] == v && n < c)) {
                        peak = 0;
                        break;
                    }
                }
            if (!peak) continue;
            /* insertion into the ordered list, keep max_cand */
            int pos = nc;
            while (pos > 0) {
                int32_t pv = cand[4 * (pos - 1) + 2];
                int64_t pi = (int64_t)cand[4 * (pos - 1) + 1] * nb + cand[4 * (pos - 1)];
                if (pv > v || (pv == v && pi < c)) break;
                --pos;
            }
            if (pos >= H->max_cand) continue;
            int last = nc < H->max_cand ? nc : H->max_cand - 1;
            for (int q = last; q > pos; --q) memcpy(&cand[4 * q], &cand[4 * (q - 1)], 4 * sizeof(int32_t));
            cand[4 * pos] = ix;
            cand[4 * pos + 1] = iy;
            cand[4 * pos + 2] = v;
            cand[4 * pos + 3] = -1;
            if (nc < H->max_cand) ++nc;
        }
    int nw = orc_n_wires(g);
    int* hist = (int*)calloc((size_t)H->n_r, sizeof(int));
    for (int c = 0; c < nc; ++c) {
        int64_t cx = H->origin_um + (int64_t)cand[4 * c] * H->bin_um + H->bin_um / 2;
        int64_t cy = H->origin_um + (int64_t)cand[4 * c + 1] * H->bin_um + H->bin_um / 2;
        memset(hist, 0, sizeof(int) * (size_t)H->n_r);
        for (int i = 0; i < n_hits; ++i) {
            if (wire_id[i] < 0 || wire_id[i] >= nw) continue;
            int64_t X, Y;
            orc_wire_xy_um(g, wire_id[i], &X, &Y);
            int64_t d2 = (X - cx) * (X - cx) + (Y - cy) * (Y - cy);
            for (int j = 0; j < H->n_r; ++j) {
                int64_t R = (int64_t)H->r_min_um + (int64_t)j * H->r_step_um;
                int64_t lo = R - H->r_hist_half_um, hi = R + H->r_hist_half_um;
                if (d2 >= lo * lo && d2 < hi * hi) hist[j]++;
            }
        }
        int bj = -1, bc = 0;
        for (int j = 0; j < H->n_r; ++j)
            if (hist[j] > bc) {
                bc = hist[j];
                bj = j;
            }
        cand[4 * c + 3] = bj;
        double th = NAN, px = NAN, py = NAN;
        if (bj >= 0) {
            double Cx = cx / 1000.0, Cy = cy / 1000.0;
            double R = (H->r_min_um + (double)bj * H->r_step_um) / 1000.0;
            double dd = sqrt(Cx * Cx + Cy * Cy), R0 = H->R0;
            if (dd > 0.0 && R0 <= dd + R && R0 >= fabs(dd - R)) {
                double a = (R0 * R0 - R * R + dd * dd) / (2.0 * dd);
                double hp = sqrt(fmax(R0 * R0 - a * a, 0.0));
                double ccw = (H->charge * H->b_nominal < 0.0) ? 1.0 : -1.0;
                for (int sgn = 1; sgn >= -1; sgn -= 2) {
                    double Px = a * Cx / dd - sgn * hp * Cy / dd;
                    double Py = a * Cy / dd + sgn * hp * Cx / dd;
                    double tx = -ccw * (Py - Cy) / R, ty = ccw * (Px - Cx) / R;
                    if (tx * Px + ty * Py > 0.0) { /* the outward crossing */
                        double pt = ORC_KAPPA * fabs(H->b_nominal) * R;
                        th = atan2(Py, Px);
                        px = pt * tx;
                        py = pt * ty;
                        break;
                    }
                }
            }
        }
        centre[3 * c] = th;
        centre[3 * c + 1] = px;
        centre[3 * c + 2] = py;
    }
    free(hist);
    return nc;
}

/* ----------------------------------------------------------- the refine */
/* Gauss-Newton refinement of one seed (not in the paper: it stands in for the
 * Kalman fit of sec. 2.2).  chi^2 = sum over hits with part[i] >= 0 of
 * ((DCA_{part[i]}(w_i) - drift_i) / sigma)^2 with the hit-to-partition
 * classification held fixed.  J from FP64 forward tangents: dDCA/dseed =
 * n_hat . d r(s*)/dseed at the minimising point (envelope theorem).  Each
 * iteration solves (Js^T Js) delta = -Js^T res in the scaled parameters
 * seed/scale by Cholesky (mu = 1e-6 tr/5 added if not positive definite).
 * Outputs: refined seed, chi^2 and gradient d chi^2/d seed at the refined
 * seed, number of hits used. */
static int orc_chi2_grad(const orc_geometry* g, const orc_field* f, const orc_scan_params* P, const double seed[5],
                         int n_hits, const int* wire_id, const double* drift, const int* part, double sigma,
                         double* st, orc_tan* tst, int cap, double* chi2, double grad[5], double JtJ[25],
                         double Jtr[5], int* flags, int* n_used) {
    double r[3], t[3], lam, mg;
    int fl;
    orc_seed_state(g, P, seed, r, t, &lam, NULL);
    int ns = orc_trace(g, f, P, seed, cap, st, tst, &fl, &mg);
    *flags |= fl;
    int nw = orc_n_wires(g);
    orc_min* mins = (orc_min*)malloc(sizeof(orc_min) * (size_t)(P->max_partitions > 0 ? P->max_partitions : 1));
    *chi2 = 0.0;
    memset(grad, 0, 5 * sizeof(double));
    memset(JtJ, 0, 25 * sizeof(double));
    memset(Jtr, 0, 5 * sizeof(double));
    *n_used = 0;
    for (int i = 0; i < n_hits; ++i) {
        int k = part[i];
        if (k < 0 || k >= P->max_partitions || wire_id[i] < 0 || wire_id[i] >= nw) continue;
        double m[3], d[3];
        orc_wire_line(g, wire_id[i], m, d);
        orc_wire_doca(f, lam, P->h, st, ns, m, d, INFINITY, P->max_partitions, mins);
        if (mins[k].j < 0) {
            *flags |= ORC_FLAG_LOST_HIT;
            continue;
        }
        int j = mins[k].j;
        double u = mins[k].u;
        double ro[3], to[3];
        orc_tan To[NT];
        orc_rkn_step_tan(f, lam, u, st + 7 * j, st + 7 * j + 3, &tst[NT * j], ro, to, To);
        double w[3] = {ro[0] - m[0], ro[1] - m[1], ro[2] - m[2]};
        double wd = w[0] * d[0] + w[1] * d[1] + w[2] * d[2];
        double q[3] = {w[0] - wd * d[0], w[1] - wd * d[1], w[2] - wd * d[2]};
        double D = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2]);
        if (D == 0.0) {
            *flags |= ORC_FLAG_DOCA_ZERO;
            continue;
        }
        double res = (D - drift[i]) / sigma;
        double J[5];
        for (int n = 0; n < NT; ++n)
            J[n] = (q[0] * To[n].r[0] + q[1] * To[n].r[1] + q[2] * To[n].r[2]) / (D * sigma);
        *chi2 += res * res;
        for (int a = 0; a < 5; ++a) {
            grad[a] += 2.0 * res * J[a];
            Jtr[a] += J[a] * res;
            for (int b = 0; b < 5; ++b) JtJ[5 * a + b] += J[a] * J[b];
        }
        ++*n_used;
    }
    free(mins);
    return 0;
}

static int chol5(double A[25], double b[5]) {
    /* in-place Cholesky A = L L^T and solve A x = b; returns 0 if not SPD */
    double L[25] = {0};
    for (int i = 0; i < 5; ++i)
        for (int j = 0; j <= i; ++j) {
            double s = A[5 * i + j];
            for (int k = 0; k < j; ++k) s -= L[5 * i + k] * L[5 * j + k];
            if (i == j) {
                if (!(s > 0.0)) return 0;
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
    return 1;
}

int orc_refine(const orc_geometry* g, const orc_field* f, const orc_scan_params* P, int n_iter, double sigma,
               const double* scale, int n_hits, const int* wire_id, const double* drift, const int* part,
               const double seed_in[5], double seed_out[5], double* chi2, double grad[5], int* n_used, int* flags) {
    int cap = P->max_steps + 1;
    double* st = (double*)malloc(sizeof(double) * 7 * (size_t)cap);
    orc_tan* tst = (orc_tan*)malloc(sizeof(orc_tan) * NT * (size_t)cap);
    if (!st || !tst) {
        free(st);
        free(tst);
        return -1;
    }
    double s[5], JtJ[25], Jtr[5], c2, gr[5];
    memcpy(s, seed_in, sizeof s);
    *flags = 0;
    for (int it = 0; it < n_iter; ++it) {
        int nu;
        orc_chi2_grad(g, f, P, s, n_hits, wire_id, drift, part, sigma, st, tst, cap, &c2, gr, JtJ, Jtr, flags, &nu);
        double A[25], b[5];
        for (int a = 0; a < 5; ++a) {
            b[a] = -Jtr[a] * scale[a];
            for (int c = 0; c < 5; ++c) A[5 * a + c] = JtJ[5 * a + c] * scale[a] * scale[c];
        }
        double A0[25], b0[5];
        memcpy(A0, A, sizeof A);
        memcpy(b0, b, sizeof b);
        if (!chol5(A, b)) {
            double tr = 0.0;
            for (int a = 0; a < 5; ++a) tr += A0[5 * a + a];
            for (int a = 0; a < 5; ++a) A0[5 * a + a] += 1e-6 * tr / 5.0;
            memcpy(b, b0, sizeof b);
            *flags |= ORC_FLAG_NOT_SPD;
            if (!chol5(A0, b)) break;
        }
        int finite = 1;
        for (int a = 0; a < 5; ++a) finite &= isfinite(b[a]);
        if (!finite) {
            *flags |= ORC_FLAG_NOT_SPD;
            break;
        }
        for (int a = 0; a < 5; ++a) s[a] += b[a] * scale[a];
    }
    orc_chi2_grad(g, f, P, s, n_hits, wire_id, drift, part, sigma, st, tst, cap, chi2, grad, JtJ, Jtr, flags, n_used);
    memcpy(seed_out, s, sizeof s);
    free(st);
    free(tst);
    return 0;
}

/* chi^2 and its gradient at a fixed seed (gradient pins). */
int orc_chi2(const orc_geometry* g, const orc_field* f, const orc_scan_params* P, double sigma, int n_hits,
             const int* wire_id, const double* drift, const int* part, const double seed[5], double* chi2,
             double grad[5], double JtJ[25], int* n_used, int* flags) {
    int cap = P->max_steps + 1;
    double* st = (double*)malloc(sizeof(double) * 7 * (size_t)cap);
    orc_tan* tst = (orc_tan*)malloc(sizeof(orc_tan) * NT * (size_t)cap);
    if (!st || !tst) {
        free(st);
        free(tst);
        return -1;
    }
    double Jtr[5];
    *flags = 0;
    orc_chi2_grad(g, f, P, seed, n_hits, wire_id, drift, part, sigma, st, tst, cap, chi2, grad, JtJ, Jtr, flags, n_used);
    free(st);
    free(tst);
    return 0;
}

/* ------------------------------------------- the neighbouring turn (sec. 2.3) */
/* Seed of the neighbouring turn partition, for the event loop of sec. 2.3 (the
 * seeds of the previous partition are predicted by extrapolating the fitted
 * track backwards).  From the seed s of a turn (its state at the outward R0
 * crossing), the track is propagated with steps of h in `direction` (-1: back
 * in time, +1: forward).  Its side of the R0 cylinder starts as inside for -1
 * (the reversed track moves inwards) and outside for +1; at the second change
 * of side the crossing point and direction are interpolated linearly between
 * the two states around it (in rho), the point is projected onto the cylinder,
 * and out = (theta0, z0, p t) with t along the forward motion and |p| kept.
 * Returns 0, 1 if the track first leaves |z| <= z_half or rho <= R_out, 2 if
 * max_steps steps pass. */
int orc_extrapolate_turn(const orc_geometry* g, const orc_field* f, const orc_scan_params* P0, const double s[5],
                         int direction, double out[5]) {
    orc_scan_params P = *P0;
    P.direction = direction < 0 ? -1 : 1;
    double r[3], t[3], lam, rn[3], tn[3];
    orc_seed_state(g, &P, s, r, t, &lam, NULL);
    const double p = sqrt(s[2] * s[2] + s[3] * s[3] + s[4] * s[4]);
    int outside = P.direction > 0, changes = 0;
    for (int n = 0; n < P.max_steps; ++n) {
        orc_rkn_step(f, lam, P.h, r, t, rn, tn);
        const double rho0 = hypot(r[0], r[1]), rho1 = hypot(rn[0], rn[1]);
        const int now_out = rho1 >= g->R0;
        if (now_out != outside) {
            outside = now_out;
            if (++changes == 2) {
                const double w = (g->R0 - rho0) / (rho1 - rho0);
                double q[3], d[3];
                for (int a = 0; a < 3; ++a) {
                    q[a] = r[a] + w * (rn[a] - r[a]);
                    d[a] = t[a] + w * (tn[a] - t[a]);
                }
                const double dn = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
                const double sc = g->R0 / hypot(q[0], q[1]);
                const double sign = P.direction < 0 ? -1.0 : 1.0;
                out[0] = atan2(q[1] * sc, q[0] * sc);
                out[1] = q[2];
                for (int a = 0; a < 3; ++a) out[2 + a] = sign * p * d[a] / dn;
                return 0;
            }
        }
        if (fabs(rn[2]) > g->z_half || rho1 > g->R_out) return 1;
        for (int a = 0; a < 3; ++a) {
            r[a] = rn[a];
            t[a] = tn[a];
        }
    }
    return 2;
}
