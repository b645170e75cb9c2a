// Device-side data layout and helpers shared by the CUDA translation units of
// the seed-scanning track finder (arXiv:1908.01949).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/cdc.h"

namespace cdc {

constexpr float KAPPA = 0.299792458f;      // MeV/c per (T mm)
constexpr double KAPPA_D = 0.299792458;
constexpr int TAB_N = 1024;                // radial candidate-layer table, 1 mm bins
constexpr float TAB_BAND = 32.0f;          // widest layer band the table supports [mm]
constexpr int LIST_M = 8;                  // steps between rebuilds of a candidate wire list
// Per-event hit table: the drift of every wire ([n_wires] floats; a sentinel
// above any drift where the wire did not fire) followed by FIRED_WORDS words
// of fired-wire bits, layer by layer: layer l starts at word bword, bit i is
// wire i, and bits N..N+31 repeat bits 0..31 so that a window of up to 32
// cells reads two consecutive words without wrapping.
constexpr int FIRED_WORDS = CDC_MAX_WIRES / 32 + 3 * CDC_MAX_LAYERS;
__host__ __device__ __forceinline__ size_t event_stride(int n_wires) { return (size_t)n_wires + FIRED_WORDS; }
constexpr int SEG = 4096;                  // seeds per top-K segment
constexpr uint64_t KEY_NONE = ~0ull;       // empty top-K slot
constexpr unsigned FULL = 0xffffffffu;     // all lanes of a warp
constexpr int ZOOM_GRID = 243;             // 3^5 seeds per zoom grid
constexpr int ROUND_SHIFT = 27;            // best-list key: (round << 27) | index

// One sense layer, as the kernels read it from shared memory.
struct DevLayer {
    float R2;            // waist radius squared [mm^2]
    float tan2a;         // tan^2(alpha)
    float tana_over_R;   // tan(alpha) / R: tangent of the stereo twist per mm of z
    float phi_off;       // azimuth of wire 0 [rad]
    float n_over_2pi;    // N / (2 pi): cells per radian
    float cells_per_mm;  // N / (2 pi (R - TAB_BAND)): conservative cells per mm of arc
    float cosa;          // cos(alpha): z component of the wire direction
    float cosa_lo;       // cos(alpha) - cosa, the rounding residual
    int N;               // wires in the layer
    int base;            // global id of wire 0
    int bword;           // first word of the layer's fired bits in the event table
    int pad3;
};

// Geometry tables owned by the context (device memory).
struct DevGeom {
    const DevLayer* layers;  // [n_layers]
    const float4* wires;     // [n_wires]: (mx, my, dx, dy) of the wire line (m at z = 0; dz = layer cosa)
    const uchar2* tab;       // [TAB_N]: (first, last) layer whose band may contain rho in [b, b+1) mm
    const int2* wire_um;     // [n_wires]: wire (x, y) at z = 0 rounded to um (Hough input)
    const float4* wires_lo;  // [n_wires]: rounding residuals of (mx, my, dx, dy) in `wires`
    int n_layers, n_wires;
    float z_half, R0, R_out;
    double R0d;
};

// Field: uniform Bz or bilinear (r, z) map stored as per-cell coefficients.
struct DevField {
    int kind;                // 0 uniform, 1 map
    float B0;
    const float4* cells;     // [(nr+1)(nz+1)][2]: Bz and Br as a + b u + c v + d u v per cell; cell (i, j)
                             // covers map cell (i-1, j-1), the outer ring holds the edge values
    int nr, nz;
    float r_min, z_min, inv_dr, inv_dz, r_max, z_max;
    float u_off, v_off;      // 1 - r_min / dr, 1 - z_min / dz: padded cell coordinates
    double dr, dz;
};

// Scan-call parameters, resolved on the host.
struct ScanConst {
    float h, h6_lo, lam, charge_dir, band, d_win, max_drift;  // h6_lo = h/6 - float(h/6)
    float b_max;    // largest |B| of the field [T] (bounds the track curvature)
    float sqrt_lam; // sqrt(lambda): the residual cut of Eq. 1 as a distance [mm]
    int max_steps, max_part, direction, k;
};

// ------------------------------------------------------------------ field
// Padded-table cell holding (x, y, z), the in-cell coordinates (u, v) and
// 1/rho.  Only the cell index is clamped: beyond the grid it lands in the
// table's border, whose coefficients do not depend on the clamped coordinate.
// At rho = 0 the tiny floor of rho^2 makes Br x / rho vanish, as Br := 0 there.
__device__ __forceinline__ int field_cell(const DevField& F, float x, float y, float z, float& u, float& v,
                                          float& rinv) {
    const float r2 = fmaf(x, x, y * y);
    rinv = rsqrtf(fmaxf(r2, 1e-30f));
    const float rho = r2 * rinv;
    u = fmaf(rho, F.inv_dr, F.u_off);
    v = fmaf(z, F.inv_dz, F.v_off);
    const int i = min(max((int)u, 0), F.nr);
    const int j = min(max((int)v, 0), F.nz);
    u -= (float)i;
    v -= (float)j;
    return i * (F.nz + 1) + j;
}

// Bilinear (Bz, Br) of one cell at (u, v), then Bx = Br x / rho, By = Br y / rho.
__device__ __forceinline__ void field_apply(float4 cz, float4 cr, float u, float v, float rinv, float x, float y,
                                            float& bx, float& by, float& bz) {
    bz = fmaf(v, fmaf(cz.w, u, cz.z), fmaf(cz.y, u, cz.x));
    const float br = fmaf(v, fmaf(cr.w, u, cr.z), fmaf(cr.y, u, cr.x));
    const float s = br * rinv;
    bx = s * x;
    by = s * y;
}

// The two coefficient sets of one cell: 32 contiguous bytes on a 32-byte
// boundary (the table is one allocation of 32-byte records), read by one
// 256-bit load through the read-only path.  Each lane of a warp usually reads
// a different cell, so one load instead of two halves the cache wavefronts.
__device__ __forceinline__ void load_cell(const float4* c, float4& cz, float4& cr) {
    asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=f"(cz.x), "=f"(cz.y), "=f"(cz.z), "=f"(cz.w), "=f"(cr.x), "=f"(cr.y), "=f"(cr.z), "=f"(cr.w)
        : "l"(c));
}

template <int KIND>
__device__ __forceinline__ void field_eval(const DevField& F, float x, float y, float z, float& bx, float& by,
                                           float& bz) {
    if (KIND == 0) {
        bx = 0.f;
        by = 0.f;
        bz = F.B0;
    } else {
        float u, v, rinv;
        float4 cz, cr;
        load_cell(F.cells + 2 * field_cell(F, x, y, z, u, v, rinv), cz, cr);
        field_apply(cz, cr, u, v, rinv, x, y, bx, by, bz);
    }
}

// --------------------------------------------------------- FP32 stepper
// Track state: position and unit direction as unevaluated float sums
// (hi + lo, Kahan-compensated updates) and lam = q kappa / p.
struct State {
    float rx, ry, rz, lx, ly, lz;  // position hi / lo
    float tx, ty, tz, mx, my, mz;  // direction hi / lo
    float lam, lam_lo;             // q kappa / p as hi + lo (lo used by the refine path only)
};

__device__ __forceinline__ void kahan(float& hi, float& lo, float inc) {
    float y = inc + lo;
    float s = hi + y;
    lo = y - (s - hi);
    hi = s;
}

// (hi, lo) += inc + inc_lo as a two-float sum: the error of hi + inc (Fast2Sum)
// and inc_lo accumulate in the low word, which then renormalises.  Unlike the
// Kahan form above, a low word far below an ulp of the increment is kept.
__device__ __forceinline__ void acc2(float& hi, float& lo, float inc, float inc_lo) {
    const float s = hi + inc;
    const float e = inc - (s - hi);
    const float l = lo + (e + inc_lo);
    hi = s + l;
    lo = l - (hi - s);
}

__device__ __forceinline__ void cross_lam(float lam, float ax, float ay, float az, float bx, float by, float bz,
                                          float& cx, float& cy, float& cz) {
    cx = lam * fmaf(ay, bz, -az * by);
    cy = lam * fmaf(az, bx, -ax * bz);
    cz = lam * fmaf(ax, by, -ay * bx);
}

// (lam + lam_lo) (a x b): the curvature with a two-float lam, rounded once
// (fma(lam, x, lam_lo x)); rounding lam x first would leave a bias of up to
// half an ulp that acts like a scaled curvature at every step
__device__ __forceinline__ void cross_lam2(float lam, float lo, float ax, float ay, float az, float bx, float by,
                                           float bz, float& cx, float& cy, float& cz) {
    const float x = fmaf(ay, bz, -az * by), y = fmaf(az, bx, -ax * bz), z = fmaf(ax, by, -ay * bx);
    cx = fmaf(lam, x, lo * x);
    cy = fmaf(lam, y, lo * y);
    cz = fmaf(lam, z, lo * z);
}

// k = lam (a x b) with lam in one float (scan) or two (refine: PRECISE)
template <bool PRECISE>
__device__ __forceinline__ void kvec(const State& s, float ax, float ay, float az, float bx, float by, float bz,
                                     float& cx, float& cy, float& cz) {
    if (PRECISE)
        cross_lam2(s.lam, s.lam_lo, ax, ay, az, bx, by, bz, cx, cy, cz);
    else
        cross_lam(s.lam, ax, ay, az, bx, by, bz, cx, cy, cz);
}

// One Runge-Kutta-Nystrom step of length h (Abramowitz & Stegun 25.5.20) for
// r'' = lam (r' x B(r)) from the field (bx, by, bz) of its first stage, with
// the field at the midpoint r + h/2 t + h^2/8 k1 (shared by k2 and k3) and at
// the end estimate r + h t + h^2/2 k3; on return (bx, by, bz) holds the field
// of the end estimate.  The increments are formed in FP32 and added to the
// compensated state (PRECISE: two-float q/p and two-float sums, for the
// refine path).
template <int KIND, bool PRECISE = false>
__device__ __forceinline__ void rkn_step_b(const DevField& F, State& s, float& bx, float& by, float& bz, float h,
                                           float h6_lo) {
    const float h2 = 0.5f * h, hh8 = h * h * 0.125f, hh2 = h * h * 0.5f, hh6 = h * h * (1.0f / 6.0f),
                h6 = h * (1.0f / 6.0f);
    float k1x, k1y, k1z, k2x, k2y, k2z, k3x, k3y, k3z, k4x, k4y, k4z;
    kvec<PRECISE>(s, s.tx, s.ty, s.tz, bx, by, bz, k1x, k1y, k1z);
    float px = fmaf(hh8, k1x, fmaf(h2, s.tx, s.rx));
    float py = fmaf(hh8, k1y, fmaf(h2, s.ty, s.ry));
    float pz = fmaf(hh8, k1z, fmaf(h2, s.tz, s.rz));
    if (KIND != 0) field_eval<KIND>(F, px, py, pz, bx, by, bz);
    kvec<PRECISE>(s, fmaf(h2, k1x, s.tx), fmaf(h2, k1y, s.ty), fmaf(h2, k1z, s.tz), bx, by, bz, k2x, k2y, k2z);
    kvec<PRECISE>(s, fmaf(h2, k2x, s.tx), fmaf(h2, k2y, s.ty), fmaf(h2, k2z, s.tz), bx, by, bz, k3x, k3y, k3z);
    if (KIND != 0) {
        px = fmaf(hh2, k3x, fmaf(h, s.tx, s.rx));
        py = fmaf(hh2, k3y, fmaf(h, s.ty, s.ry));
        pz = fmaf(hh2, k3z, fmaf(h, s.tz, s.rz));
        field_eval<KIND>(F, px, py, pz, bx, by, bz);
    }
    kvec<PRECISE>(s, fmaf(h, k3x, s.tx), fmaf(h, k3y, s.ty), fmaf(h, k3z, s.tz), bx, by, bz, k4x, k4y, k4z);
    // position: h (t_hi + t_lo) + h^2/6 (k1 + k2 + k3); h t_lo lies below half
    // an ulp of the increment, so it goes straight into the low word (folding it
    // into the rounded increment would drop it at every step)
    float drx = fmaf(h, s.tx, hh6 * (k1x + k2x + k3x));
    float dry = fmaf(h, s.ty, hh6 * (k1y + k2y + k3y));
    float drz = fmaf(h, s.tz, hh6 * (k1z + k2z + k3z));
    const float clx = h * s.mx, cly = h * s.my, clz = h * s.mz;
    // direction: h/6 (k1 + 2 k2 + 2 k3 + k4) as a two-float increment: the
    // rounding of the product and of the constant h/6 (which alone would scale
    // the curvature by up to 3e-8 at every step) go to the low word
    const float sx = k1x + k4x + 2.0f * (k2x + k3x), sy = k1y + k4y + 2.0f * (k2y + k3y),
                sz = k1z + k4z + 2.0f * (k2z + k3z);
    const float dtx = h6 * sx, dty = h6 * sy, dtz = h6 * sz;
    const float dlx = fmaf(h6_lo, sx, fmaf(h6, sx, -dtx)), dly = fmaf(h6_lo, sy, fmaf(h6, sy, -dty)),
                dlz = fmaf(h6_lo, sz, fmaf(h6, sz, -dtz));
    if (PRECISE) {  // refine: two-float sums (gradients to 1e-4 need ~1e-6 mm)
        acc2(s.rx, s.lx, drx, clx);
        acc2(s.ry, s.ly, dry, cly);
        acc2(s.rz, s.lz, drz, clz);
        acc2(s.tx, s.mx, dtx, dlx);
        acc2(s.ty, s.my, dty, dly);
        acc2(s.tz, s.mz, dtz, dlz);
    } else {        // scan: compensated sums, ~5e-5 mm per metre
        kahan(s.rx, s.lx, drx);
        kahan(s.ry, s.ly, dry);
        kahan(s.rz, s.lz, drz);
        s.lx += clx;
        s.ly += cly;
        s.lz += clz;
        kahan(s.tx, s.mx, dtx);
        kahan(s.ty, s.my, dty);
        kahan(s.tz, s.mz, dtz);
        s.mx += dlx;
        s.my += dly;
        s.mz += dlz;
    }
}

// The classical step: field at the start, the midpoint and the end estimate.
template <int KIND, bool PRECISE = false>
__device__ __forceinline__ void rkn_step(const DevField& F, State& s, float h, float h6_lo) {
    float bx, by, bz;
    field_eval<KIND>(F, s.rx, s.ry, s.rz, bx, by, bz);
    rkn_step_b<KIND, PRECISE>(F, s, bx, by, bz, h, h6_lo);
}

// The scan's step: the field of the previous step's end estimate stands in for
// the field at the start (the two points differ by h^2/6 (2 k3 - k1 - k2), of
// order h^3 / rho^2), so each step evaluates the map twice and the first
// stage waits for no load.  Over 6 m of a 105 MeV/c track in the solenoid map
// the positions stay within 1e-6 mm of the classical step's in FP64.
// (bx, by, bz): the field at the end estimate of the last step (at the seed
// for the first step); updated in place.
template <int KIND>
__device__ __forceinline__ void rkn_step_fsal(const DevField& F, State& s, float& bx, float& by, float& bz, float h,
                                              float h6_lo) {
    rkn_step_b<KIND, false>(F, s, bx, by, bz, h, h6_lo);
}

// Seed (theta0, z0, px0, py0, pz0) at r = R0 -> state, formed in FP64 and
// split into hi/lo floats.  direction -1 reverses t and the charge.
__device__ __forceinline__ void seed_state(const float* sd, double R0, float charge_dir, int direction, State& s) {
    double st, ct;
    sincos((double)sd[0], &st, &ct);
    double x = R0 * ct, y = R0 * st, z = (double)sd[1];
    double px = sd[2], py = sd[3], pz = sd[4];
    double p = sqrt(px * px + py * py + pz * pz);
    double ip = (direction < 0 ? -1.0 : 1.0) / p;
    double tx = px * ip, ty = py * ip, tz = pz * ip;
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

// Mixed-radix decode of seed `idx` of one grid (row-major over theta0, z0,
// px0, py0, pz0); each value is the float32 nearest centre + k step.
__device__ __forceinline__ void grid_seed(const cdc_grid& g, long long idx, float* out) {
    long long q = idx;
    int ia[5];
#pragma unroll
    for (int a = 4; a >= 0; --a) {
        int n = g.n[a];
        ia[a] = (int)(q % n);
        q /= n;
    }
#pragma unroll
    for (int a = 0; a < 5; ++a) out[a] = fmaf((float)ia[a] - 0.5f * (float)(g.n[a] - 1), g.step[a], g.centre[a]);
}

constexpr int PERM_CAP = 4096;  // (z0, pz0) blocks of a coarse grid that can be reordered
constexpr int REC_SLOTS = 64;   // per event: records of zoom-round seeds that reached the event's best score

// The record of one zoom-round seed (the entries of the tracer's FoundList,
// from which its hits are classified), kept when the seed's score was at most
// the best of its event so far: the final best seed of a zoom round is then
// among them.
struct SeedRecord {
    int round, index, nf, pad;
    uint32_t key[CDC_MAX_FOUND];
    float r[CDC_MAX_FOUND];
};

// Row-major index of the q-th seed of a grid in scan order: (z0, pz0)
// outermost, then theta0, px0, py0, so that consecutive seeds (the lanes of a
// warp) differ by a step of a transverse parameter, follow nearly the same
// path and visit nearly the same wires.  The (z0, pz0) blocks come in the
// order perm gives (perm[b] = iz * n_pz0 + ip of the b-th block), or in their
// natural order for perm == nullptr or grids of more than PERM_CAP blocks.
__device__ __forceinline__ long long scan_order_index(const cdc_grid& g, long long q, const uint16_t* perm) {
    const int nt = g.n[0], nz = g.n[1], nx = g.n[2], ny = g.n[3], np = g.n[4];
    const long long iy = q % ny;
    q /= ny;
    const long long ix = q % nx;
    q /= nx;
    const long long it = q % nt;
    q /= nt;
    if (perm && (long long)nz * np <= PERM_CAP) q = perm[q];
    const long long ip = q % np;
    const long long iz = q / np;
    return (((it * nz + iz) * nx + ix) * ny + iy) * np + ip;
}

__device__ __forceinline__ long long grid_count(const cdc_grid& g) {
    long long c = 1;
#pragma unroll
    for (int a = 0; a < 5; ++a) c *= (long long)max(g.n[a], 0);
    return c;
}

// ------------------------------------------------- events and seed grids
__device__ __forceinline__ int find_event_i32(const int32_t* off, int n, int i) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= i) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ int find_event(const long long* off, int n, long long i) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= i) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// The q-th seed of event e in scan order (scan_order_index within each of the
// event's grids; perm: the block order of a single grid, or nullptr): its
// values, and its row-major index among the event's seeds.
__device__ __forceinline__ long long event_seed_ordered(const cdc_grid* grids, int gpe, int e, long long q,
                                                       float* sd, const uint16_t* perm) {
    long long base = 0;
    for (int g = 0; g < gpe; ++g) {
        const cdc_grid& gr = grids[(size_t)e * gpe + g];
        const long long c = grid_count(gr);
        if (q < c || g == gpe - 1) {
            const long long li = scan_order_index(gr, q, gpe == 1 ? perm : nullptr);
            grid_seed(gr, li, sd);
            return base + li;
        }
        q -= c;
        base += c;
    }
    return base;
}

__device__ __forceinline__ void event_seed(const cdc_grid* grids, int gpe, int e, long long local, float* sd) {
    for (int g = 0; g < gpe; ++g) {
        const cdc_grid& gr = grids[(size_t)e * gpe + g];
        long long c = grid_count(gr);
        if (local < c || g == gpe - 1) {
            grid_seed(gr, local, sd);
            return;
        }
        local -= c;
    }
}

__device__ __forceinline__ uint64_t make_key(float e, uint32_t idx) {
    uint32_t b = __float_as_uint(e);
    if (!(e >= 0.f)) b = 0x7f800000u;  // NaN or negative cannot occur; order them last
    return ((uint64_t)b << 32) | idx;
}

// Warp-resident ascending list of the K <= 64 smallest keys seen: lane l
// holds entries l and 32 + l; every lane of the warp calls with its own key
// (cand: whether it competes).
__device__ __forceinline__ uint64_t list_at(uint64_t a, uint64_t b, int i) {
    uint64_t va = __shfl_sync(FULL, a, i & 31);
    uint64_t vb = __shfl_sync(FULL, b, i & 31);
    return i < 32 ? va : vb;
}

__device__ __forceinline__ void list_insert(uint64_t& a, uint64_t& b, uint64_t key, bool cand, int K) {
    const int lane = threadIdx.x & 31;
    uint64_t thr = list_at(a, b, K - 1);
    unsigned m = __ballot_sync(FULL, cand && key < thr);
    while (m) {
        int src = __ffs(m) - 1;
        uint64_t k = __shfl_sync(FULL, key, src);
        int p = __popc(__ballot_sync(FULL, a < k)) + __popc(__ballot_sync(FULL, b < k));
        uint64_t pa = __shfl_up_sync(FULL, a, 1);
        uint64_t pb = __shfl_up_sync(FULL, b, 1);
        uint64_t a31 = __shfl_sync(FULL, a, 31);
        if (lane == 0) pb = a31;
        int ia = lane, ib = 32 + lane;
        uint64_t na = ia < p ? a : (ia == p ? k : pa);
        uint64_t nb = ib < p ? b : (ib == p ? k : pb);
        a = na;
        b = nb;
        thr = list_at(a, b, K - 1);
        m &= ~(1u << src);
        m &= __ballot_sync(FULL, cand && key < thr);
    }
}

}  // namespace cdc
