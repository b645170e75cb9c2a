// Per-seed track tracer of the scan (arXiv:1908.01949 sec. 2.2, Eq. 1):
// RKN propagation with turn-partition bookkeeping and track-centric scoring.
//
// Wire search.  Every LIST_M steps the tracer looks up the fired wires near
// the current point: the sense layers whose band contains the point (a
// per-millimetre table of candidate layers plus an exact test against the
// stereo hyperboloid r_l(z)^2 = R_l^2 + z^2 tan^2 a_l), and in each such layer
// the cells whose stereo-corrected azimuth lies within the search window.  The
// window is widened by LIST_M h so that it also covers the next LIST_M
// segments.  Of these wires only the ones the track approaches are kept (a
// short per-seed list in shared memory): near a wire the squared distance
// along the track is convex (its second derivative 2(|t_perp|^2 + w_perp .
// t'_perp) stays positive while |t_perp|^2 exceeds the window radius over the
// radius of curvature), so a receding wire cannot pass a minimum before the
// next rebuild; for tracks nearly parallel to the wires receding wires are kept
// too.  Approaching wires whose minimum provably lies beyond the list's
// lifetime (the slope of g is bounded by |t_perp|^2 plus a curvature term)
// wait for a later list, so lists hold only imminent minima.  Each step then
// evaluates, for the listed wires only, the derivative of
// the squared distance to the wire line, g = (r - m)_perp . t, at the new
// state; a sign change from - to + brackets a local minimum of the distance,
// which a Newton step on the cubic Hermite interpolant of the segment
// locates.  The window and band (host-computed) cover every wire whose distance
// of closest approach can enter Eq. 1 below the cutoff, so the result equals
// the brute-force definition.  Track ends count as minima when the distance is
// still decreasing there.  If a list overflows, the tracer searches the window
// at every step until the next rebuild.
//
// Eq. 1 per wire: the DCA of a turn partition is the smallest distance over
// all minima inside that partition, and the wire's term is the smallest
// min((|DCA_k| - drift)^2, lambda) over the partitions k.  A minimum closer than
// drift - sqrt(lambda) therefore removes its partition from the wire's term,
// and a minimum farther than drift + sqrt(lambda) never matters.  While it
// steps, the tracer only appends each minimum that can matter to the seed's
// record (a few instructions, however divergent); the terms and their sum
// are formed from the record once the seed has ended (record_score).
//
// Layout: every scalar of the tracer lives in registers; the list lives in
// shared memory ([LIST_CAP][block] layout), the per-seed record (written a few
// times per seed) in local memory.
#pragma once

#include "cdc_dev.cuh"

namespace cdc {

constexpr int LIST_CAP = 8;            // candidate wires per seed
constexpr float PARALLEL_T2 = 0.25f;   // |t_perp|^2 below which receding wires are kept

// One wire of a per-seed candidate list: wire | layer << 16 and the slope g
// of the squared distance at the last state (the drift is read again from the
// event table when a minimum is found; 8 bytes per entry keep the lists small
// beside the L1 cache that holds the field map).
struct __align__(8) ListEntry {
    uint32_t key;
    float g;
};

// Record of one seed: every distance minimum closer than drift + sqrt(lambda),
// in track order (so the partitions of one wire never decrease along it), as
// key = wire | partition << 16 and r = D - drift (-inf where cheap bounds put
// D below drift - sqrt(lambda)); when it is nearly full it is compacted
// (record_compact) before it overflows.
struct FoundList {
    uint32_t key[CDC_MAX_FOUND];
    float r[CDC_MAX_FOUND];
};

__device__ __forceinline__ int key_wire(uint32_t k) { return (int)(k & 0xffffu); }
__device__ __forceinline__ int key_part(uint32_t k) { return (int)(k >> 16); }

// Eq. 1 term of one partition's signed residual.
__device__ __forceinline__ float part_term(float r, float lam) { return fminf(r * r, lam); }

// Term of `wire` from entries i0.. of a record (i0: its first entry): per
// partition the nearest minimum (smallest residual), then the smallest term
// over the partitions, ties to the lower partition; part = its partition, or
// -1 when the term is lambda.
__device__ __forceinline__ float wire_term(const uint32_t* key, const float* r, int n, int i0, int wire, float lam,
                                           int& part) {
    float best = lam, cm = r[i0];
    int cp = key_part(key[i0]);
    part = -1;
    for (int j = i0 + 1; j < n; ++j) {
        if (key_wire(key[j]) != wire) continue;
        const int pj = key_part(key[j]);
        if (pj == cp) {
            cm = fminf(cm, r[j]);
        } else {
            const float t = part_term(cm, lam);
            if (t < best) {
                best = t;
                part = cp;
            }
            cp = pj;
            cm = r[j];
        }
    }
    const float t = part_term(cm, lam);
    if (t < best) {
        best = t;
        part = cp;
    }
    return best;
}

// Eq. 1 of a seed from its record: H lambda plus, per wire, its term minus
// lambda, summed in the order of the wires' first entries.
__device__ __forceinline__ float record_score(const uint32_t* key, const float* r, int n, float lam, int H) {
    float e = 0.f;
    for (int i = 0; i < n; ++i) {
        const int w = key_wire(key[i]);
        bool first = true;
        for (int j = 0; j < i; ++j) first &= key_wire(key[j]) != w;
        if (!first) continue;
        int part;
        e += wire_term(key, r, n, i, w, lam, part) - lam;
    }
    return fmaf((float)H, lam, e);
}

// A full record made room for more minima without changing any term or
// class: the entries of finished partitions (below cur) shrink to one per
// wire, the nearest minimum of its best partition (ties to the lower one), and
// vanish where that term is lambda; the current partition's entries of one
// wire merge into the nearest.  Entries of a wire stay in partition order.
// Returns the new number of entries.
static __device__ __noinline__ int record_compact(uint32_t* key, float* r, int n, int cur, float lam) {
    uint32_t keep[CDC_MAX_FOUND / 32];
    for (int q = 0; q < CDC_MAX_FOUND / 32; ++q) keep[q] = 0u;
    for (int i = 0; i < n; ++i) {
        const uint32_t k = key[i];
        const int w = key_wire(k);
        if (key_part(k) < cur) {
            bool first = true;
            for (int j = 0; j < i; ++j) first &= !(key_wire(key[j]) == w && key_part(key[j]) < cur);
            if (!first) continue;
            float best = lam, bm = 0.f, cm = r[i];
            int bp = -1, cp = key_part(k);
            for (int j = i + 1; j <= n; ++j) {
                const bool same = j < n && key_wire(key[j]) == w && key_part(key[j]) < cur;
                if (same && key_part(key[j]) == cp) {
                    cm = fminf(cm, r[j]);
                    continue;
                }
                if (j == n || same) {
                    const float t = part_term(cm, lam);
                    if (t < best) {
                        best = t;
                        bm = cm;
                        bp = cp;
                    }
                    if (j < n) {
                        cp = key_part(key[j]);
                        cm = r[j];
                    }
                }
            }
            if (bp >= 0) {
                key[i] = (uint32_t)w | ((uint32_t)bp << 16);
                r[i] = bm;
                keep[i >> 5] |= 1u << (i & 31);
            }
        } else {
            bool first = true;
            for (int j = 0; j < i; ++j) first &= key[j] != k;
            if (!first) continue;
            float cm = r[i];
            for (int j = i + 1; j < n; ++j)
                if (key[j] == k) cm = fminf(cm, r[j]);
            r[i] = cm;
            keep[i >> 5] |= 1u << (i & 31);
        }
    }
    int m = 0;
    for (int i = 0; i < n; ++i)
        if (keep[i >> 5] & (1u << (i & 31))) {
            key[m] = key[i];
            r[m] = r[i];
            ++m;
        }
    return m;
}

// Hit classification of `wire` from a record (sec. 2.2: d^2 < lambda): the
// partition of its term, or -1; returns the term (lambda without entries).
__device__ __forceinline__ float record_class(const uint32_t* key, const float* r, int n, int wire, float lam,
                                              int& part) {
    part = -1;
    for (int i = 0; i < n; ++i)
        if (key_wire(key[i]) == wire) return wire_term(key, r, n, i, wire, lam, part);
    return lam;
}

// Fired cells of layer L in the search window (half widths band [mm] in
// radius, given as the squared bounds blo2..bhi2, and d_win <= TAB_BAND [mm]
// along the layer) around (phi, z): bit b of m = cell s0 + b (mod N), from one
// 64-bit read of the layer's fired bits.  False if the window misses the layer.
__device__ __forceinline__ bool layer_cells(const DevLayer& L, const uint32_t* fired, float blo2, float bhi2, float z,
                                            float z2, float phi, float d_win, int& s0, uint32_t& m) {
    const float rl2 = fmaf(z2, L.tan2a, L.R2);
    if (rl2 > bhi2 || rl2 < blo2) return false;
    const float zt = z * L.tana_over_R, zt2 = zt * zt;
    // stereo twist atan(z tan(a) / R) by its Taylor series (|zt| < 0.2)
    const float tw = zt * fmaf(zt2, fmaf(zt2, fmaf(zt2, -1.0f / 7.0f, 0.2f), -1.0f / 3.0f), 1.0f);
    const float c = (phi - tw - L.phi_off) * L.n_over_2pi;
    if (!(fabsf(c) < 1.0e6f)) return false;  // non-finite state: nothing to look up
    const float w = d_win * L.cells_per_mm;
    const int i0 = (int)ceilf(c - w), i1 = (int)floorf(c + w);
    if (i1 < i0) return false;
    s0 = i0;  // |c| stays near N/2 at most: a few wraps at worst
    while (s0 < 0) s0 += L.N;
    while (s0 >= L.N) s0 -= L.N;
    const uint32_t* fw = fired + L.bword + (s0 >> 5);
    const unsigned long long pair = ((unsigned long long)__ldg(fw + 1) << 32) | __ldg(fw);
    // the geometry keeps i1 - i0 <= 31 (window of at most 32 cells)
    m = (uint32_t)(pair >> (s0 & 31)) & (0xffffffffu >> (31 - min(i1 - i0, 31)));
    return true;
}

// Visits the fired wires in the search window around (rho, phi, z), layer by
// layer and cell by cell: fn(wire, drift, cosa, layer).  Only fired wires touch the
// drift table.  The per-layer arithmetic is that of layer_cells, written out
// here: the stepping loop's register allocation is better that way.
template <class Fn>
__device__ __forceinline__ void visit_window(const DevLayer* s_lay, const uchar2* s_tab, const float* dtab,
                                             const uint32_t* fired, float max_drift, float band, float d_win,
                                             float rho, float phi, float z, Fn&& fn, float rlo = -1.f,
                                             float rhi = -1.f) {
    const uchar2 lr = s_tab[min((int)rho, TAB_N - 1)];
    if (lr.x > lr.y) return;
    // radial band: rho +- band, or [rlo - band, rhi + band] where the caller bounds the radii ahead
    const float blo = fmaxf((rlo >= 0.f ? rlo : rho) - band, 0.f), bhi = (rhi >= 0.f ? rhi : rho) + band;
    const float blo2 = blo * blo, bhi2 = bhi * bhi, z2 = z * z;
    for (int l = lr.x; l <= lr.y; ++l) {
        const DevLayer& L = s_lay[l];
        const float rl2 = fmaf(z2, L.tan2a, L.R2);
        if (rl2 > bhi2 || rl2 < blo2) continue;
        const float zt = z * L.tana_over_R, zt2 = zt * zt;
        const float tw = zt * fmaf(zt2, fmaf(zt2, fmaf(zt2, -1.0f / 7.0f, 0.2f), -1.0f / 3.0f), 1.0f);
        const float c = (phi - tw - L.phi_off) * L.n_over_2pi;
        if (!(fabsf(c) < 1.0e6f)) continue;
        const float w = d_win * L.cells_per_mm;
        const int i0 = (int)ceilf(c - w), i1 = (int)floorf(c + w);
        if (i1 < i0) continue;
        int s0 = i0;
        while (s0 < 0) s0 += L.N;
        while (s0 >= L.N) s0 -= L.N;
        const uint32_t* fw = fired + L.bword + (s0 >> 5);
        const unsigned long long pair = ((unsigned long long)__ldg(fw + 1) << 32) | __ldg(fw);
        uint32_t m = (uint32_t)(pair >> (s0 & 31)) & (0xffffffffu >> (31 - min(i1 - i0, 31)));
        while (m) {
            const int b = __ffs(m) - 1;
            m &= m - 1;
            int ii = s0 + b;
            if (ii >= L.N) ii -= L.N;
            const int wire = L.base + ii;
            const float d = __ldg(dtab + wire);
            if (d <= max_drift) fn(wire, d, L.cosa, l);
        }
    }
}

// Distance of closest approach inside a segment whose squared-distance
// derivative changes sign from g0 < 0 to g1 >= 0: a Newton step on the
// cubic Hermite interpolant P(u) = r_j + H10 h t_j + H01 (r_j+1 - r_j) +
// H11 h t_j+1 (u = tau h), started at the root of the linear interpolation of
// the derivative.  (ax, ay, az) = r_j - m; (Dx, Dy, Dz) = r_j+1 - r_j.  On
// 2 mm segments of 250-400 mm radius passing stereo wires at 0-10 mm, the
// start point alone leaves the distance up to 1.4e-4 mm off the interpolant's
// minimum and one Newton step brings it to rounding level (FP64 model), so one
// step is taken: a minimum runs on one lane of its warp, and each further
// step cost 3-4 % of the coarse round.  Kept out of line: it runs for a few
// percent of the steps and would otherwise set the register budget of the
// whole stepping loop.
constexpr int NEWTON_STEPS = 1;
static __device__ __noinline__ float seg_doca(float ax, float ay, float az, float otx, float oty, float otz,
                                              float Dx, float Dy, float Dz, float ntx, float nty, float ntz,
                                              float4 W, float cosa, float g0, float g1, float h) {
    const float ih = 1.0f / h;
    float u = h * (g0 / (g0 - g1));
    float wx, wy, wz, wd;
#pragma unroll
    for (int it = 0; it < NEWTON_STEPS; ++it) {
        const float t = u * ih, t2 = t * t;
        const float h10 = h * t * fmaf(t, t - 2.0f, 1.0f), h01 = t2 * fmaf(-2.0f, t, 3.0f), h11 = h * t2 * (t - 1.0f);
        wx = fmaf(h11, ntx, fmaf(h01, Dx, fmaf(h10, otx, ax)));
        wy = fmaf(h11, nty, fmaf(h01, Dy, fmaf(h10, oty, ay)));
        wz = fmaf(h11, ntz, fmaf(h01, Dz, fmaf(h10, otz, az)));
        const float d10 = fmaf(3.0f * t, t, fmaf(-4.0f, t, 1.0f)), d01 = 6.0f * t * (1.0f - t) * ih,
                    d11 = t * fmaf(3.0f, t, -2.0f);
        const float vx = fmaf(d11, ntx, fmaf(d01, Dx, d10 * otx));
        const float vy = fmaf(d11, nty, fmaf(d01, Dy, d10 * oty));
        const float vz = fmaf(d11, ntz, fmaf(d01, Dz, d10 * otz));
        const float e10 = fmaf(6.0f, t, -4.0f) * ih, e01 = fmaf(-12.0f, t, 6.0f) * ih * ih,
                    e11 = fmaf(6.0f, t, -2.0f) * ih;
        const float ax2 = fmaf(e11, ntx, fmaf(e01, Dx, e10 * otx));
        const float ay2 = fmaf(e11, nty, fmaf(e01, Dy, e10 * oty));
        const float az2 = fmaf(e11, ntz, fmaf(e01, Dz, e10 * otz));
        wd = fmaf(wx, W.z, fmaf(wy, W.w, wz * cosa));
        const float vd = fmaf(vx, W.z, fmaf(vy, W.w, vz * cosa));
        const float ad2 = fmaf(ax2, W.z, fmaf(ay2, W.w, az2 * cosa));
        const float num = fmaf(wx, vx, fmaf(wy, vy, wz * vz)) - wd * vd;
        const float den =
            fmaf(vx, vx, fmaf(vy, vy, vz * vz)) - vd * vd + (fmaf(wx, ax2, fmaf(wy, ay2, wz * az2)) - wd * ad2);
        if (den > 0.f) u = fminf(fmaxf(u - num / den, 0.f), h);
    }
    const float t = u * ih, t2 = t * t;
    const float h10 = h * t * fmaf(t, t - 2.0f, 1.0f), h01 = t2 * fmaf(-2.0f, t, 3.0f), h11 = h * t2 * (t - 1.0f);
    wx = fmaf(h11, ntx, fmaf(h01, Dx, fmaf(h10, otx, ax)));
    wy = fmaf(h11, nty, fmaf(h01, Dy, fmaf(h10, oty, ay)));
    wz = fmaf(h11, ntz, fmaf(h01, Dz, fmaf(h10, otz, az)));
    wd = fmaf(wx, W.z, fmaf(wy, W.w, wz * cosa));
    const float px = wx - wd * W.z, py = wy - wd * W.w, pz = wz - wd * cosa;
    return sqrtf(fmaf(px, px, fmaf(py, py, pz * pz)));
}

// Derivative of the squared distance to the wire line along the track, and
// |t_perp|^2, at point r with direction t.
__device__ __forceinline__ float dist_slope(float rx, float ry, float rz, float tx, float ty, float tz, float4 W,
                                            float cosa, float& tperp2) {
    const float ax = rx - W.x, ay = ry - W.y;
    const float ad = fmaf(ax, W.z, fmaf(ay, W.w, rz * cosa));
    const float td = fmaf(tx, W.z, fmaf(ty, W.w, tz * cosa));
    tperp2 = fmaf(-td, td, fmaf(tx, tx, fmaf(ty, ty, tz * tz)));
    return fmaf(ax, tx, fmaf(ay, ty, rz * tz)) - ad * td;
}

__device__ __forceinline__ float point_doca(float rx, float ry, float rz, float4 W, float cosa) {
    const float ax = rx - W.x, ay = ry - W.y;
    const float ad = fmaf(ax, W.z, fmaf(ay, W.w, rz * cosa));
    const float px = ax - ad * W.z, py = ay - ad * W.w, pz = rz - ad * cosa;
    return sqrtf(fmaf(px, px, fmaf(py, py, pz * pz)));
}

// Squared distance from point r to the wire line.
__device__ __forceinline__ float point_doca2(float rx, float ry, float rz, float4 W, float cosa) {
    const float ax = rx - W.x, ay = ry - W.y;
    const float ad = fmaf(ax, W.z, fmaf(ay, W.w, rz * cosa));
    const float px = ax - ad * W.z, py = ay - ad * W.w, pz = rz - ad * cosa;
    return fmaf(px, px, fmaf(py, py, pz * pz));
}

// An upper bound of sqrt(x), x >= 0, for the conservative filters (the
// reciprocal square root is good to a few ulp; 1e-5 relative covers it).
__device__ __forceinline__ float sqrt_ub(float x) {
    if (!(x > 0.f)) return 0.f;
    const float s = x * rsqrtf(x);
    return fmaf(s, 1.0e-5f, s);
}

__device__ __forceinline__ float rho_of(float x, float y) {
    const float r2 = fmaf(x, x, y * y);
    return r2 > 0.f ? r2 * rsqrtf(r2) : 0.f;
}

__device__ __forceinline__ bool in_chamber(const uchar2* s_tab, float rho) {
    const uchar2 lr = s_tab[min((int)rho, TAB_N - 1)];
    return lr.x <= lr.y;
}

// Signed residual D - d of the distance minimum to wire W inside the segment
// o -> n (slopes g0 < 0 <= g1, drift d), where cheap bounds do not settle it
// (with 0.01 mm to spare): +inf when D > d + sqrt(lambda) (the minimum cannot
// matter), -inf when D < d - sqrt(lambda) (it removes its partition from the
// wire's term).  D <= min(D0, D1), and with D^2' = 2 g and g' >= -kap |w_perp|
// (kap = |lam| b_max), D^2 >= D0^2 + 2 g0 h - kap (D0 + h) h^2 and
// D^2 >= D1^2 - 2 g1 h - kap (D1 + h) h^2.
__device__ __forceinline__ float seg_res(const ScanConst& P, float kap, float ox, float oy, float oz, float otx,
                                         float oty, float otz, float nx, float ny, float nz, float ntx, float nty,
                                         float ntz, float4 W, float cosa, float d, float g0, float g1) {
    const float h = P.h;
    const float D0s = point_doca2(ox, oy, oz, W, cosa), D1s = point_doca2(nx, ny, nz, W, cosa);
    const float kh2 = kap * h * h;
    const float lb2 = fmaxf(fmaf(2.0f * h, g0, fmaf(-kh2, sqrt_ub(D0s) + h, D0s)),
                            fmaf(-2.0f * h, g1, fmaf(-kh2, sqrt_ub(D1s) + h, D1s)));
    const float hi = d + P.sqrt_lam + 0.01f, lo = d - P.sqrt_lam - 0.01f;
    if (lb2 > hi * hi) return INFINITY;
    if (lo > 0.f && fminf(D0s, D1s) < lo * lo) return -INFINITY;
    return seg_doca(ox - W.x, oy - W.y, oz, otx, oty, otz, nx - ox, ny - oy, nz - oz, ntx, nty, ntz, W, cosa, g0, g1,
                    h) - d;
}

template <int KIND>
struct Tracer {
    State s;
    float bx, by, bz;                 // field at the last step's end estimate (at the seed before the first)
    float ox, oy, oz, otx, oty, otz;  // state before the last step (high words)
    const float* dtab;
    const uint32_t* fired;
    ListEntry* cand;  // this thread's list column: cand[k * stride]
    int stride;
    int n, part, nf, nc;
    bool outside, over;
    uint32_t flags;

    // A distance minimum of `wire` in partition pt with signed residual r =
    // D - drift, appended to the record if it can matter (D < drift +
    // sqrt(lambda)).
    __device__ __forceinline__ void found(const ScanConst& P, FoundList& FL, int wire, int pt, float r) {
        if (!(r < P.sqrt_lam)) return;
        if (nf < CDC_MAX_FOUND) {
            FL.key[nf] = (uint32_t)wire | ((uint32_t)pt << 16);
            FL.r[nf] = r;
            ++nf;
        } else {
            flags |= CDC_FLAG_FOUND_OVERFLOW;
        }
    }

    // Room in the record for the next LIST_M steps: compacted once it is
    // nearly full (at most LIST_CAP minima per step are appended).
    __device__ __forceinline__ void make_room(const ScanConst& P, FoundList& FL) {
        if (nf > CDC_MAX_FOUND - LIST_M * LIST_CAP) nf = record_compact(FL.key, FL.r, nf, part, P.lam);
    }

    // Candidates for the next LIST_M segments at the current state:
    // sink(wire, g, drift, cosa) stores one and returns false when full.
    template <class Sink>
    __device__ __forceinline__ void collect(const DevGeom& G, const ScanConst& P, const DevLayer* s_lay,
                                           const uchar2* s_tab, Sink&& sink) {
        over = false;
        const float x = s.rx, y = s.ry, z = s.rz, tx = s.tx, ty = s.ty, tz = s.tz;
        const float rho = rho_of(x, y);
        if (!in_chamber(s_tab, rho)) return;
        const float wide = LIST_M * P.h;
        // Growth bound of g = w_perp . t (w = r - m) along the track: dg/ds =
        // |t_perp|^2 + w_perp . t' with |t'| <= |lam| b_max = kap, |w_perp| grows
        // by at most 1 per mm and |t_perp|^2 by at most 2 kap per mm, so over an
        // arc s, g rises by at most s (|t_perp|^2 + kap (|w_perp| + 1.5 s)).
        // Distance bound: along the tangent line the distance to the wire line
        // never drops below sqrt(|w_perp|^2 - g^2 / |t_perp|^2), and over an arc
        // s <= reach the track leaves that line by at most kap reach^2 / 2.
        const float reach = wide + 0.5f;
        const float kap = fabsf(s.lam) * P.b_max;
        const float bend = fmaf(0.5f * kap, reach * reach, 0.01f);
        // Radii the track can reach within the next LIST_M segments (arc s <= wide):
        // with q = rho^2, q' = 2 (x tx + y ty) and q'' = 2 (tx^2 + ty^2) + 2 (x, y) .
        // (tx', ty') in [-2 (rho + s) kap, 2 + 2 (rho + s) kap], q stays between the
        // end values of q0 + q'0 s - (rho + wide) kap s^2 and q0 + q'0 s + (1 + (rho +
        // wide) kap) s^2 (a concave and a convex quadratic), and |rho(s) - rho| <= s.
        // The window takes those radii +- the band (0.01 mm to spare) instead of
        // rho +- (band + wide): the layers behind the track drop out.
        const float q0 = rho * rho, dq = 2.0f * wide * fmaf(x, tx, y * ty), ck = (rho + wide) * kap * wide * wide;
        const float qlo = fminf(q0, dq + q0 - ck), qhi = fmaxf(q0, dq + q0 + fmaf(wide, wide, ck));
        const float rlo = fmaxf(fmaxf(sqrtf(fmaxf(qlo, 0.f)) - 0.01f, rho - wide), 0.f);
        const float rhi = fminf(sqrtf(qhi) + 0.01f, rho + wide);
        visit_window(s_lay, s_tab, dtab, fired, P.max_drift, P.band, P.d_win + wide, rho, atan2f(y, x), z,
                     [&](int wire, float d, float cosa, int layer) {
                         const float4 W = __ldg(G.wires + wire);
                         float tp2;
                         const float g = dist_slope(x, y, z, tx, ty, tz, W, cosa, tp2);
                         bool keep = tp2 < PARALLEL_T2;
                         if (!keep && g < 0.f) {
                             // the minimum lies within the next LIST_M steps (else a later list
                             // takes the wire) and can come within d + sqrt(lambda) of the wire:
                             // |w_perp|^2 - g^2 / |t_perp|^2 <= (d + sqrt(lambda) + bend)^2
                             const float wp2 = point_doca2(x, y, z, W, cosa);
                             const float lim = d + P.sqrt_lam + bend;
                             keep = fmaf(reach, fmaf(kap, fmaf(1.5f, reach, sqrt_ub(wp2)), tp2), g) + 1e-3f >= 0.f &&
                                    fmaf(wp2, tp2, -g * g) <= lim * lim * tp2;
                         }
                         if (keep && !sink(wire, g, layer)) over = true;
                     },
                     rlo, rhi);
    }

    // Per-lane candidate list in this thread's column.
    __device__ __forceinline__ void rebuild(const DevGeom& G, const ScanConst& P, const DevLayer* s_lay,
                                            const uchar2* s_tab) {
        nc = 0;
        collect(G, P, s_lay, s_tab, [&](int wire, float g, int layer) {
            if (nc >= LIST_CAP) return false;
            cand[nc * stride] = ListEntry{(uint32_t)wire | ((uint32_t)layer << 16), g};
            ++nc;
            return true;
        });
    }

    // Seed state, the start-of-track minima and the first candidate list.
    __device__ __forceinline__ void init(const DevGeom& G, const DevField& F, const ScanConst& P,
                                         const DevLayer* s_lay, const uchar2* s_tab, const float* dtab_,
                                         ListEntry* cand_, int stride_, const float* sd, FoundList& FL) {
        seed_state(sd, G.R0d, P.charge_dir, P.direction, s);
        field_eval<KIND>(F, s.rx, s.ry, s.rz, bx, by, bz);
        dtab = dtab_;
        fired = (const uint32_t*)(dtab_ + G.n_wires);
        cand = cand_;
        stride = stride_;
        n = 0;
        part = 0;
        nf = 0;
        nc = 0;
        outside = true;
        over = false;
        flags = 0u;
        // start of the track: a minimum if the distance grows from there
        const float x = s.rx, y = s.ry, z = s.rz, tx = s.tx, ty = s.ty, tz = s.tz;
        const float rho = rho_of(x, y);
        if (in_chamber(s_tab, rho))
            visit_window(s_lay, s_tab, dtab, fired, P.max_drift, P.band, P.d_win, rho, atan2f(y, x), z,
                         [&](int wire, float d, float cosa, int) {
                             const float4 W = __ldg(G.wires + wire);
                             float tp2;
                             if (dist_slope(x, y, z, tx, ty, tz, W, cosa, tp2) > 0.f)
                                 found(P, FL, wire, 0, point_doca(x, y, z, W, cosa) - d);
                         });
        rebuild(G, P, s_lay, s_tab);
    }

    // One RKN step; the previous state stays in (ox .. otz).
    __device__ __forceinline__ void advance(const DevField& F, const ScanConst& P) {
        ox = s.rx;
        oy = s.ry;
        oz = s.rz;
        otx = s.tx;
        oty = s.ty;
        otz = s.tz;
        rkn_step_fsal<KIND>(F, s, bx, by, bz, P.h, P.h6_lo);
        ++n;
    }

    // Minima of this lane's listed wires inside the last segment.
    __device__ __forceinline__ void list_pass(const DevGeom& G, const ScanConst& P, const DevLayer* s_lay,
                                              FoundList& FL) {
        if (over) return;
        const float kap = fabsf(s.lam) * P.b_max;
        for (int k = 0; k < nc; ++k) {
            const ListEntry e = cand[k * stride];
            const int wire = (int)(e.key & 0xffffu);
            const float4 W = __ldg(G.wires + wire);
            const float cosa = s_lay[e.key >> 16].cosa;
            float tp2;
            const float g1 = dist_slope(s.rx, s.ry, s.rz, s.tx, s.ty, s.tz, W, cosa, tp2);
            if (e.g < 0.f && g1 >= 0.f)
                found(P, FL, wire, part,
                      seg_res(P, kap, ox, oy, oz, otx, oty, otz, s.rx, s.ry, s.rz, s.tx, s.ty, s.tz, W, cosa,
                              __ldg(dtab + wire), e.g, g1));
            cand[k * stride].g = g1;
        }
    }

    // Window search for a lane whose list overflowed, turn bookkeeping, stop
    // tests and the track-end minima; false once the track ended.
    __device__ __forceinline__ bool finish(const DevGeom& G, const ScanConst& P, const DevLayer* s_lay,
                                           const uchar2* s_tab, FoundList& FL) {
        const float nx = s.rx, ny = s.ry, nz = s.rz, ntx = s.tx, nty = s.ty, ntz = s.tz;
        const float rho = rho_of(nx, ny);
        if (over && in_chamber(s_tab, rho)) {
            const int pt = part;
            const float kap = fabsf(s.lam) * P.b_max;
            visit_window(s_lay, s_tab, dtab, fired, P.max_drift, P.band, P.d_win, rho, atan2f(ny, nx), nz,
                         [&](int wire, float d, float cosa, int) {
                             const float4 W = __ldg(G.wires + wire);
                             float tp2;
                             const float g0 = dist_slope(ox, oy, oz, otx, oty, otz, W, cosa, tp2);
                             if (!(g0 < 0.f)) return;
                             const float g1 = dist_slope(nx, ny, nz, ntx, nty, ntz, W, cosa, tp2);
                             if (g1 >= 0.f)
                                 found(P, FL, wire, pt,
                                       seg_res(P, kap, ox, oy, oz, otx, oty, otz, nx, ny, nz, ntx, nty, ntz, W, cosa,
                                               d, g0, g1));
                         });
        }
        const bool now_out = rho >= G.R0;
        bool stop = false;
        if (outside && !now_out) {
            ++part;
            if (part >= P.max_part) stop = true;
        }
        outside = now_out;
        if (fabsf(nz) > G.z_half || rho > G.R_out) stop = true;
        if (!stop && n >= P.max_steps) {
            stop = true;
            flags |= CDC_FLAG_STEP_CAP;
        }
        if (stop && part < P.max_part && in_chamber(s_tab, rho)) {
            // end of the track: a minimum if the distance is still shrinking
            // there (the lists hold only imminent minima, so the end looks at
            // the whole window)
            const int pe = part;
            visit_window(s_lay, s_tab, dtab, fired, P.max_drift, P.band, P.d_win, rho, atan2f(ny, nx), nz,
                         [&](int wire, float d, float cosa, int) {
                             const float4 W = __ldg(G.wires + wire);
                             float tp2;
                             if (dist_slope(nx, ny, nz, ntx, nty, ntz, W, cosa, tp2) < 0.f)
                                 found(P, FL, wire, pe, point_doca(nx, ny, nz, W, cosa) - d);
                         });
        }
        return !stop;
    }

    // One RKN step and the minima inside the new segment (per-lane list);
    // false once the track ended.
    __device__ __forceinline__ bool step(const DevGeom& G, const DevField& F, const ScanConst& P,
                                         const DevLayer* s_lay, const uchar2* s_tab, FoundList& FL) {
        advance(F, P);
        list_pass(G, P, s_lay, FL);
        return finish(G, P, s_lay, s_tab, FL);
    }

    __device__ __forceinline__ float score(const ScanConst& P, int H, const FoundList& FL) const {
        return record_score(FL.key, FL.r, nf, P.lam, H);
    }
};

}  // namespace cdc
