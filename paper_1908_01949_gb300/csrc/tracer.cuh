// Per-seed track tracer of the scan (arXiv:1908.01949 sec. 2.2, Eq. 1):
// RKN propagation with turn-partition bookkeeping and track-centric scoring.
//
// After every step (segment from state j to j+1) the tracer looks up the
// fired wires near the new position: the sense layers whose band contains the
// point (a per-millimetre table of candidate layers plus an exact test against
// the stereo hyperboloid r_l(z)^2 = R_l^2 + z^2 tan^2 a_l), and in each such
// layer the cells whose stereo-corrected azimuth lies within the search
// window.  For a fired wire the derivative of the squared distance to the
// wire line, g = (r - m)_perp . t, is evaluated at both ends of the segment; a
// sign change from - to + brackets a local minimum of the distance, which
// Newton iterations on the cubic Hermite interpolant of the segment locate.
// The window and band (host-computed) cover every wire whose distance of
// closest approach can enter Eq. 1 below the cutoff, so the result equals the
// brute-force definition.  Track ends count as minima when the distance is
// still decreasing there.
#pragma once

#include "cdc_dev.cuh"

namespace cdc {

template <int KIND, bool KEEP_PART>
struct Tracer {
    State s;
    const float* dtab;
    int n, part;
    bool outside;
    float eacc;
    int nf;
    unsigned long long bloom;
    uint32_t flags;
    uint32_t fkey[CDC_MAX_FOUND];  // wire | partition << 16
    float fr2[CDC_MAX_FOUND];

    // Best squared residual of `wire` below lambda; Eq. 1 accumulates
    // min(res^2, lambda) - lambda on top of H lambda.
    __device__ __forceinline__ void found(const ScanConst& P, int wire, int pt, float r2) {
        if (!(r2 < P.lam)) return;
        const unsigned long long bit = 1ull << (wire & 63);
        if (bloom & bit) {
            for (int i = 0; i < nf; ++i) {
                if ((int)(fkey[i] & 0xffffu) == wire) {
                    if (r2 < fr2[i]) {
                        eacc += r2 - fr2[i];
                        fr2[i] = r2;
                        fkey[i] = (uint32_t)wire | ((uint32_t)pt << 16);
                    }
                    return;
                }
            }
        }
        bloom |= bit;
        eacc += r2 - P.lam;
        if (nf < CDC_MAX_FOUND) {
            fkey[nf] = (uint32_t)wire | ((uint32_t)pt << 16);
            fr2[nf] = r2;
            ++nf;
        } else {
            flags |= CDC_FLAG_FOUND_OVERFLOW;
        }
    }

    __device__ __forceinline__ void lookup(int wire, int& pt, float& r2) const {
        for (int i = 0; i < nf; ++i)
            if ((int)(fkey[i] & 0xffffu) == wire) {
                pt = (int)(fkey[i] >> 16);
                r2 = fr2[i];
            }
    }

    // Calls fn(wire, drift, cosa) for every fired wire in the search window
    // around (x, y, z); returns rho.
    template <class Fn>
    __device__ __forceinline__ float for_window(const ScanConst& P, const DevLayer* s_lay, const uchar2* s_tab,
                                                float x, float y, float z, Fn&& fn) const {
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
                const float zt = z * L.tana_over_R;
                const float z2 = zt * zt;
                // stereo twist atan(z tan(a) / R) by its Taylor series (|zt| < 0.2 for any allowed stereo angle)
                const float tw = zt * fmaf(z2, fmaf(z2, fmaf(z2, -1.0f / 7.0f, 0.2f), -1.0f / 3.0f), 1.0f);
                const float c = (phi - tw - L.phi_off) * L.n_over_2pi;
                if (!(fabsf(c) < 1.0e6f)) continue;  // non-finite state: nothing to look up
                const float w = P.d_win * L.cells_per_mm;
                const int i0 = (int)ceilf(c - w), i1 = (int)floorf(c + w);
                for (int i = i0; i <= i1; ++i) {
                    int ii = i % L.N;
                    if (ii < 0) ii += L.N;
                    const int wire = L.base + ii;
                    const float d = __ldg(dtab + wire);
                    if (!(d <= P.max_drift)) continue;
                    fn(wire, d, L.cosa);
                }
            }
        }
        return rho;
    }

    __device__ __forceinline__ void init(const DevGeom& G, const ScanConst& P, const DevLayer* s_lay,
                                         const uchar2* s_tab, const float* dtab_, const float* sd) {
        seed_state(sd, G.R0d, P.charge_dir, P.direction, s);
        dtab = dtab_;
        n = 0;
        part = 0;
        outside = true;
        eacc = 0.f;
        nf = 0;
        bloom = 0ull;
        flags = 0u;
        // start of the track: a minimum if the distance grows from there
        const float x = s.rx, y = s.ry, z = s.rz, tx = s.tx, ty = s.ty, tz = s.tz;
        for_window(P, s_lay, s_tab, x, y, z, [&](int wire, float d, float cosa) {
            const float4 W = __ldg(G.wires + wire);
            const float ax = x - W.x, ay = y - W.y, az = z;
            const float ad = fmaf(ax, W.z, fmaf(ay, W.w, az * cosa));
            const float td = fmaf(tx, W.z, fmaf(ty, W.w, tz * cosa));
            const float g = fmaf(ax, tx, fmaf(ay, ty, az * tz)) - ad * td;
            if (g > 0.f) {
                const float px = ax - ad * W.z, py = ay - ad * W.w, pz = az - ad * cosa;
                const float D = sqrtf(fmaf(px, px, fmaf(py, py, pz * pz)));
                const float r = D - d;
                found(P, wire, 0, r * r);
            }
        });
    }

    __device__ __forceinline__ bool step(const DevGeom& G, const DevField& F, const ScanConst& P,
                                         const DevLayer* s_lay, const uchar2* s_tab) {
        const float ox = s.rx, oy = s.ry, oz = s.rz, otx = s.tx, oty = s.ty, otz = s.tz;
        rkn_step<KIND>(F, s, P.h);
        ++n;
        const float nx = s.rx, ny = s.ry, nz = s.rz, ntx = s.tx, nty = s.ty, ntz = s.tz;
        const int pt = part;
        const float h = P.h, ih = 1.0f / P.h;
        const float rho = for_window(P, s_lay, s_tab, nx, ny, nz, [&](int wire, float d, float cosa) {
            const float4 W = __ldg(G.wires + wire);
            const float ax = ox - W.x, ay = oy - W.y, az = oz;
            const float ad = fmaf(ax, W.z, fmaf(ay, W.w, az * cosa));
            const float t0d = fmaf(otx, W.z, fmaf(oty, W.w, otz * cosa));
            const float g0 = fmaf(ax, otx, fmaf(ay, oty, az * otz)) - ad * t0d;
            if (!(g0 < 0.f)) return;
            const float bx = nx - W.x, by = ny - W.y, bz = nz;
            const float bd = fmaf(bx, W.z, fmaf(by, W.w, bz * cosa));
            const float t1d = fmaf(ntx, W.z, fmaf(nty, W.w, ntz * cosa));
            const float g1 = fmaf(bx, ntx, fmaf(by, nty, bz * ntz)) - bd * t1d;
            if (g1 < 0.f) return;
            // local minimum inside the segment: Newton on the Hermite cubic
            // P(u) = r_j + H10 h t_j + H01 (r_j+1 - r_j) + H11 h t_j+1, u = tau h
            const float Dx = nx - ox, Dy = ny - oy, Dz = nz - oz;
            float u = h * (g0 / (g0 - g1));
            float wx = 0.f, wy = 0.f, wz = 0.f, wd = 0.f;
#pragma unroll
            for (int it = 0; it < 3; ++it) {
                const float t = u * ih, t2 = t * t;
                const float h10 = h * t * fmaf(t, t - 2.0f, 1.0f), h01 = t2 * fmaf(-2.0f, t, 3.0f),
                            h11 = h * t2 * (t - 1.0f);
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
                const float den = fmaf(vx, vx, fmaf(vy, vy, vz * vz)) - vd * vd +
                                  (fmaf(wx, ax2, fmaf(wy, ay2, wz * az2)) - wd * ad2);
                if (den > 0.f) u = fminf(fmaxf(u - num / den, 0.f), h);
            }
            {
                const float t = u * ih, t2 = t * t;
                const float h10 = h * t * fmaf(t, t - 2.0f, 1.0f), h01 = t2 * fmaf(-2.0f, t, 3.0f),
                            h11 = h * t2 * (t - 1.0f);
                wx = fmaf(h11, ntx, fmaf(h01, Dx, fmaf(h10, otx, ax)));
                wy = fmaf(h11, nty, fmaf(h01, Dy, fmaf(h10, oty, ay)));
                wz = fmaf(h11, ntz, fmaf(h01, Dz, fmaf(h10, otz, az)));
                wd = fmaf(wx, W.z, fmaf(wy, W.w, wz * cosa));
            }
            const float px = wx - wd * W.z, py = wy - wd * W.w, pz = wz - wd * cosa;
            const float D = sqrtf(fmaf(px, px, fmaf(py, py, pz * pz)));
            const float r = D - d;
            found(P, wire, pt, r * r);
        });
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
        if (stop && part < P.max_part) {
            // end of the track: a minimum if the distance is still shrinking there
            const int pe = part;
            for_window(P, s_lay, s_tab, nx, ny, nz, [&](int wire, float d, float cosa) {
                const float4 W = __ldg(G.wires + wire);
                const float ax = nx - W.x, ay = ny - W.y, az = nz;
                const float ad = fmaf(ax, W.z, fmaf(ay, W.w, az * cosa));
                const float td = fmaf(ntx, W.z, fmaf(nty, W.w, ntz * cosa));
                const float g = fmaf(ax, ntx, fmaf(ay, nty, az * ntz)) - ad * td;
                if (g < 0.f) {
                    const float px = ax - ad * W.z, py = ay - ad * W.w, pz = az - ad * cosa;
                    const float D = sqrtf(fmaf(px, px, fmaf(py, py, pz * pz)));
                    const float r = D - d;
                    found(P, wire, pe, r * r);
                }
            });
        }
        return !stop;
    }

    __device__ __forceinline__ float score(const ScanConst& P, int H) const { return fmaf((float)H, P.lam, eacc); }
};

}  // namespace cdc
