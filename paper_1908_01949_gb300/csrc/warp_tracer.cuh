// Warp-per-seed tracer of the scan (arXiv:1908.01949 sec. 2.2, Eq. 1) for
// rounds with few seeds.  With one lane per seed such a round leaves the GPU
// nearly empty and lasts as long as its longest track, so here the 32 lanes of
// a warp follow one seed together:
//   - every lane steps the same state with the same arithmetic as Tracer, so
//     the RKN chain runs without divergence;
//   - the candidate list holds one wire per lane and its sign tests run in
//     parallel;
//   - a window search takes one layer per lane, places the layers' fired
//     wires by a warp prefix sum in the visiting order of visit_window (layer
//     by layer, cell by cell) and hands one wire to each lane;
//   - the record of the seed's wires (tracer.cuh: FoundList) lives in shared
//     memory, where all lanes search it at once.
// Minima are recorded in the same order as by Tracer, so both compute the
// same Eq. 1 sums.
#pragma once

#include "tracer.cuh"

namespace cdc {

constexpr unsigned WARP_ALL = 0xffffffffu;
constexpr int WARP_LIST_CAP = 32;  // candidate wires per seed: one per lane
constexpr int WIN_CAP = 128;       // fired wires of one window kept in shared memory

// Per-warp shared memory: the record of the warp's seed (the entries of
// FoundList) and the fired wires of the current window (wire | layer << 16).
struct WarpFound {
    uint32_t key[CDC_MAX_FOUND];
    float r[CDC_MAX_FOUND];
    uint32_t win[WIN_CAP];
};

// Fired wire number j of the search window around (rho, phi, z), counted in
// the visiting order of visit_window, as (wire, cosa), or wire = -1; serial
// over the layers (all arguments but j equal on every lane).  Serves windows
// with more than WIN_CAP fired wires.
__device__ __forceinline__ void window_nth(const DevLayer* s_lay, const uchar2* s_tab, const uint32_t* fired,
                                           float band, float d_win, float rho, float phi, float z, int j, int& wire,
                                           float& cosa) {
    wire = -1;
    cosa = 1.f;
    const uchar2 lr = s_tab[min((int)rho, TAB_N - 1)];
    if (lr.x > lr.y) return;
    const float blo = fmaxf(rho - band, 0.f), bhi = rho + band;
    const float blo2 = blo * blo, bhi2 = bhi * bhi, z2 = z * z;
    int total = 0;
    for (int l = lr.x; l <= lr.y; ++l) {
        const DevLayer& L = s_lay[l];
        int s0;
        uint32_t m;
        if (!layer_cells(L, fired, blo2, bhi2, z, z2, phi, d_win, s0, m)) continue;
        const int cnt = __popc(m);
        if (j >= total && j < total + cnt) {
            int ii = s0 + (int)__fns(m, 0, j - total + 1);
            if (ii >= L.N) ii -= L.N;
            wire = L.base + ii;
            cosa = L.cosa;
            return;
        }
        total += cnt;
    }
}

// The fired wires of the search window around (rho, phi, z) in the visiting
// order of visit_window, written to win[0, min(total, WIN_CAP)) as wire |
// layer << 16; returns their number.  Lane k takes layer lr.x + k (+ 32 per
// chunk of layers) and a warp prefix sum of the per-layer counts places its
// wires.  Called by all lanes with equal arguments.
__device__ __forceinline__ int window_gather(const DevLayer* s_lay, const uchar2* s_tab, const uint32_t* fired,
                                             float band, float d_win, float rho, float phi, float z, int lane,
                                             uint32_t* win) {
    const uchar2 lr = s_tab[min((int)rho, TAB_N - 1)];
    if (lr.x > lr.y) return 0;
    const float blo = fmaxf(rho - band, 0.f), bhi = rho + band;
    const float blo2 = blo * blo, bhi2 = bhi * bhi, z2 = z * z;
    int total = 0;
    __syncwarp();  // the previous window's readers are done
    for (int l0 = lr.x; l0 <= lr.y; l0 += 32) {
        const int l = l0 + lane;
        int s0 = 0;
        uint32_t m = 0u;
        if (l <= lr.y && !layer_cells(s_lay[l], fired, blo2, bhi2, z, z2, phi, d_win, s0, m)) m = 0u;
        const int cnt = __popc(m);
        int inc = cnt;
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(WARP_ALL, inc, o);
            if (lane >= o) inc += v;
        }
        if (m) {
            const DevLayer& L = s_lay[l];
            int pos = total + inc - cnt;
            do {
                const int b = __ffs(m) - 1;
                m &= m - 1;
                int ii = s0 + b;
                if (ii >= L.N) ii -= L.N;
                if (pos < WIN_CAP) win[pos] = (uint32_t)(L.base + ii) | ((uint32_t)l << 16);
                ++pos;
            } while (m);
        }
        total += __shfl_sync(WARP_ALL, inc, 31);
    }
    __syncwarp();
    return total;
}

template <int KIND>
struct WarpTracer {
    State s;
    float bx, by, bz;                 // field at the last step's end estimate (at the seed before the first)
    float ox, oy, oz, otx, oty, otz;  // state before the last step (high words)
    const float* dtab;
    const uint32_t* fired;
    WarpFound* rec;
    int c_wire;  // this lane's candidate (lanes below nc): wire, its geometry, slope g, drift, cosa
    float4 c_W;
    float c_g, c_d, c_cosa;
    int n, part, nf, nc, lane;
    bool outside, over;
    uint32_t flags;

    // Entry j of the window gathered into rec->win (tot wires): (wire, cosa),
    // or wire = -1 past the end.
    __device__ __forceinline__ void window_entry(const DevLayer* s_lay, const uchar2* s_tab, float band, float d_win,
                                                 float rho, float phi, float z, int tot, int j, int& wire,
                                                 float& cosa) const {
        wire = -1;
        cosa = 1.f;
        if (j < min(tot, WIN_CAP)) {
            const uint32_t k = rec->win[j];
            wire = (int)(k & 0xffffu);
            cosa = s_lay[k >> 16].cosa;
        } else if (j < tot) {
            window_nth(s_lay, s_tab, fired, band, d_win, rho, phi, z, j, wire, cosa);
        }
    }

    // A distance minimum of `wire` in partition pt with signed residual r
    // (arguments equal on all lanes), appended to the record as by
    // Tracer::found.
    __device__ __forceinline__ void found(const ScanConst& P, int wire, int pt, float r) {
        if (!(r < P.sqrt_lam)) return;
        if (nf < CDC_MAX_FOUND) {
            if (lane == 0) {
                rec->key[nf] = (uint32_t)wire | ((uint32_t)pt << 16);
                rec->r[nf] = r;
            }
            ++nf;
        } else {
            flags |= CDC_FLAG_FOUND_OVERFLOW;
        }
    }

    // Minima found by the lanes (signed residuals; +inf where none), recorded
    // in lane order.
    __device__ __forceinline__ void record_lanes(const ScanConst& P, float r, int wire, int pt) {
        unsigned m = __ballot_sync(WARP_ALL, r < P.sqrt_lam);
        while (m) {
            const int src = __ffs(m) - 1;
            m &= m - 1;
            found(P, __shfl_sync(WARP_ALL, wire, src), pt, __shfl_sync(WARP_ALL, r, src));
        }
    }

    // Candidate list for the next LIST_M segments (the rules of Tracer::collect),
    // candidate r on lane r.
    __device__ __forceinline__ void rebuild(const DevGeom& G, const ScanConst& P, const DevLayer* s_lay,
                                            const uchar2* s_tab) {
        nc = 0;
        over = false;
        const float x = s.rx, y = s.ry, z = s.rz, tx = s.tx, ty = s.ty, tz = s.tz;
        const float rho = rho_of(x, y);
        if (!in_chamber(s_tab, rho)) return;
        const float wide = LIST_M * P.h;
        const float reach = wide + 0.5f;
        const float kap = fabsf(s.lam) * P.b_max;
        const float bend = fmaf(0.5f * kap, reach * reach, 0.01f);
        const float phi = atan2f(y, x);
        const float band = P.band + wide, d_win = P.d_win + wide;
        const int tot = window_gather(s_lay, s_tab, fired, band, d_win, rho, phi, z, lane, rec->win);
        for (int pass = 0; pass * 32 < tot; ++pass) {
            int wire;
            float cosa;
            window_entry(s_lay, s_tab, band, d_win, rho, phi, z, tot, pass * 32 + lane, wire, cosa);
            bool keep = false;
            float g = 0.f, d = 0.f;
            if (wire >= 0) {
                d = __ldg(dtab + wire);
                if (d <= P.max_drift) {
                    const float4 W = __ldg(G.wires + wire);
                    float tp2;
                    g = dist_slope(x, y, z, tx, ty, tz, W, cosa, tp2);
                    keep = tp2 < PARALLEL_T2;
                    if (!keep && g < 0.f) {
                        const float wp2 = point_doca2(x, y, z, W, cosa);
                        const float lim = d + P.sqrt_lam + bend;
                        keep = fmaf(reach, fmaf(kap, fmaf(1.5f, reach, sqrt_ub(wp2)), tp2), g) + 1e-3f >= 0.f &&
                               fmaf(wp2, tp2, -g * g) <= lim * lim * tp2;
                    }
                }
            }
            const unsigned kb = __ballot_sync(WARP_ALL, keep);
            const int nk = __popc(kb);
            const int r = lane - nc;
            const bool take = r >= 0 && r < nk;
            const int src = take ? (int)__fns(kb, 0, r + 1) : lane;
            const int w2 = __shfl_sync(WARP_ALL, wire, src);
            const float g2 = __shfl_sync(WARP_ALL, g, src), d2 = __shfl_sync(WARP_ALL, d, src),
                        a2 = __shfl_sync(WARP_ALL, cosa, src);
            if (take) {
                c_wire = w2;
                c_g = g2;
                c_d = d2;
                c_cosa = a2;
            }
            if (nc + nk > WARP_LIST_CAP) over = true;
            nc = min(nc + nk, WARP_LIST_CAP);
        }
        if (lane < nc) c_W = __ldg(G.wires + c_wire);
    }

    // Seed state, the start-of-track minima and the first candidate list.
    __device__ __forceinline__ void init(const DevGeom& G, const DevField& F, const ScanConst& P,
                                         const DevLayer* s_lay, const uchar2* s_tab, const float* dtab_,
                                         WarpFound* rec_, const float* sd) {
        seed_state(sd, G.R0d, P.charge_dir, P.direction, s);
        field_eval<KIND>(F, s.rx, s.ry, s.rz, bx, by, bz);
        dtab = dtab_;
        fired = (const uint32_t*)(dtab_ + G.n_wires);
        rec = rec_;
        lane = threadIdx.x & 31;
        n = 0;
        part = 0;
        nf = 0;
        nc = 0;
        outside = true;
        over = false;
        flags = 0u;
        c_wire = 0;
        c_W = make_float4(0.f, 0.f, 0.f, 0.f);
        c_g = c_d = 0.f;
        c_cosa = 1.f;
        const float x = s.rx, y = s.ry, z = s.rz, tx = s.tx, ty = s.ty, tz = s.tz;
        const float rho = rho_of(x, y);
        if (in_chamber(s_tab, rho)) {
            const float phi = atan2f(y, x);
            const int tot = window_gather(s_lay, s_tab, fired, P.band, P.d_win, rho, phi, z, lane, rec->win);
            for (int pass = 0; pass * 32 < tot; ++pass) {
                int wire;
                float cosa;
                window_entry(s_lay, s_tab, P.band, P.d_win, rho, phi, z, tot, pass * 32 + lane, wire, cosa);
                float r = INFINITY;
                if (wire >= 0) {
                    const float d = __ldg(dtab + wire);
                    if (d <= P.max_drift) {
                        const float4 W = __ldg(G.wires + wire);
                        float tp2;
                        if (dist_slope(x, y, z, tx, ty, tz, W, cosa, tp2) > 0.f) r = point_doca(x, y, z, W, cosa) - d;
                    }
                }
                record_lanes(P, r, wire, 0);
            }
        }
        rebuild(G, P, s_lay, s_tab);
    }

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

    // Sign tests of the listed wires, one per lane.
    __device__ __forceinline__ void list_pass(const DevGeom& G, const ScanConst& P) {
        if (over) return;
        float r = INFINITY;
        if (lane < nc) {
            const float4 W = c_W;
            float tp2;
            const float g1 = dist_slope(s.rx, s.ry, s.rz, s.tx, s.ty, s.tz, W, c_cosa, tp2);
            if (c_g < 0.f && g1 >= 0.f)
                r = seg_res(P, fabsf(s.lam) * P.b_max, ox, oy, oz, otx, oty, otz, s.rx, s.ry, s.rz, s.tx, s.ty, s.tz,
                            W, c_cosa, c_d, c_g, g1);
            c_g = g1;
        }
        record_lanes(P, r, c_wire, part);
    }

    // Window search when the list overflowed, turn bookkeeping, stop tests and
    // the track-end minima (the rules of Tracer::finish); false once ended.
    __device__ __forceinline__ bool finish(const DevGeom& G, const ScanConst& P, const DevLayer* s_lay,
                                           const uchar2* s_tab) {
        const float nx = s.rx, ny = s.ry, nz = s.rz, ntx = s.tx, nty = s.ty, ntz = s.tz;
        const float rho = rho_of(nx, ny);
        if (over && in_chamber(s_tab, rho)) {
            const float kap = fabsf(s.lam) * P.b_max;
            const float phi = atan2f(ny, nx);
            const int tot = window_gather(s_lay, s_tab, fired, P.band, P.d_win, rho, phi, nz, lane, rec->win);
            for (int pass = 0; pass * 32 < tot; ++pass) {
                int wire;
                float cosa;
                window_entry(s_lay, s_tab, P.band, P.d_win, rho, phi, nz, tot, pass * 32 + lane, wire, cosa);
                float r = INFINITY;
                if (wire >= 0) {
                    const float d = __ldg(dtab + wire);
                    if (d <= P.max_drift) {
                        const float4 W = __ldg(G.wires + wire);
                        float tp2;
                        const float g0 = dist_slope(ox, oy, oz, otx, oty, otz, W, cosa, tp2);
                        if (g0 < 0.f) {
                            const float g1 = dist_slope(nx, ny, nz, ntx, nty, ntz, W, cosa, tp2);
                            if (g1 >= 0.f)
                                r = seg_res(P, kap, ox, oy, oz, otx, oty, otz, nx, ny, nz, ntx, nty, ntz, W, cosa, d,
                                            g0, g1);
                        }
                    }
                }
                record_lanes(P, r, wire, part);
            }
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
            const float phi = atan2f(ny, nx);
            const int tot = window_gather(s_lay, s_tab, fired, P.band, P.d_win, rho, phi, nz, lane, rec->win);
            for (int pass = 0; pass * 32 < tot; ++pass) {
                int wire;
                float cosa;
                window_entry(s_lay, s_tab, P.band, P.d_win, rho, phi, nz, tot, pass * 32 + lane, wire, cosa);
                float r = INFINITY;
                if (wire >= 0) {
                    const float d = __ldg(dtab + wire);
                    if (d <= P.max_drift) {
                        const float4 W = __ldg(G.wires + wire);
                        float tp2;
                        if (dist_slope(nx, ny, nz, ntx, nty, ntz, W, cosa, tp2) < 0.f)
                            r = point_doca(nx, ny, nz, W, cosa) - d;
                    }
                }
                record_lanes(P, r, wire, part);
            }
        }
        return !stop;
    }

    // The whole track of the seed; returns the number of steps.
    __device__ __forceinline__ void run(const DevGeom& G, const DevField& F, const ScanConst& P, const DevLayer* s_lay,
                                        const uchar2* s_tab) {
        for (;;) {
            advance(F, P);
            list_pass(G, P);
            if (!finish(G, P, s_lay, s_tab)) break;
            if (n % LIST_M == 0) {
                rebuild(G, P, s_lay, s_tab);
                if (nf > CDC_MAX_FOUND - LIST_M * LIST_CAP) {  // room for the next LIST_M steps, as Tracer::make_room
                    __syncwarp();
                    int m = 0;
                    if (lane == 0) m = record_compact(rec->key, rec->r, nf, part, P.lam);
                    nf = __shfl_sync(WARP_ALL, m, 0);
                    __syncwarp();
                }
            }
        }
    }

    // Eq. 1 of the seed from its record (every lane the same value).
    __device__ __forceinline__ float score(const ScanConst& P, int H) const {
        __syncwarp();
        return record_score(rec->key, rec->r, nf, P.lam, H);
    }
};

}  // namespace cdc
