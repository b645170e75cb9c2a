// Circle Hough transform (arXiv:1908.01949 sec. 2.1, Fig. 4): integer vote
// accumulation, peak finding and the transverse seed centre.
#include <cuda_runtime.h>
#include <limits.h>
#include <stdint.h>

#include "cdc_dev.cuh"
#include "cdc_host.h"

namespace cdc {

constexpr int HOUGH_HITS = 64;      // hits staged per block iteration
constexpr int PEAK_LIST = 2048;     // sorted list of selected peaks (only overflows for counts >= PEAK_HIST)
constexpr int PEAK_HIST = 2048;     // histogram of peak counts

// Strict local maximum of the 3x3 neighbourhood; an equal neighbour with a
// lower linear index wins.
__device__ __forceinline__ bool is_peak(const int32_t* A, int nb, long long c, int v) {
    const int ix = (int)(c % nb), iy = (int)(c / nb);
    for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
            if (!dx && !dy) continue;
            const int x = ix + dx, y = iy + dy;
            if (x < 0 || y < 0 || x >= nb || y >= nb) continue;
            const long long n = (long long)y * nb + x;
            const int vn = A[n];
            if (vn > v || (vn == v && n < c)) return false;
        }
    return true;
}

// Exact floor(a / b) for 0 <= a < 2^30, b > 0, from a float estimate.
__device__ __forceinline__ int div_floor(int a, int b, float inv_b) {
    int q = (int)((float)a * inv_b);
    if (q * b > a) --q;
    else if ((q + 1) * b <= a) ++q;
    return q;
}

// Thread = one (radius, angle) vote offset; the block loops over the event's
// hits staged in shared memory.  A vote lands in bin floor((C - origin)/bin)
// of the centre C = X + O if (R - T)^2 <= |C|^2 <= (R + T)^2 (integer um).
__global__ void __launch_bounds__(256) hough_vote_kernel(const int32_t* __restrict__ hit_off,
                                                         const int32_t* __restrict__ wire_id,
                                                         const int2* __restrict__ wire_um, int n_wires,
                                                         const int2* __restrict__ offsets, cdc_hough_params H,
                                                         int32_t* acc) {
    __shared__ int2 s_xy[HOUGH_HITS];
    const int e = blockIdx.z;
    const int n_pairs = H.n_r * H.n_phi;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    const bool active = p < n_pairs;
    const int2 O = active ? offsets[p] : make_int2(0, 0);
    const long long R = (long long)H.r_min_um + (long long)(active ? p / H.n_phi : 0) * H.r_step_um;
    const long long lo = R - H.target_um, hi = R + H.target_um;
    const long long lo2 = lo > 0 ? lo * lo : 0, hi2 = hi * hi;
    const float inv_bin = 1.0f / (float)H.bin_um;
    const int nb = H.n_bins;
    const long long span = (long long)nb * H.bin_um;
    int32_t* A = acc + (size_t)e * nb * nb;
    const int h0 = hit_off[e], h1 = hit_off[e + 1];
    for (int c = h0 + blockIdx.y * HOUGH_HITS; c < h1; c += gridDim.y * HOUGH_HITS) {
        __syncthreads();
        if (threadIdx.x < HOUGH_HITS) {
            int h = c + threadIdx.x;
            int2 v = make_int2(INT_MIN, 0);
            if (h < h1) {
                int w = wire_id[h];
                if (w >= 0 && w < n_wires) v = wire_um[w];
            }
            s_xy[threadIdx.x] = v;
        }
        __syncthreads();
        if (!active) continue;
        const int nh = min(HOUGH_HITS, h1 - c);
        for (int k = 0; k < nh; ++k) {
            const int2 X = s_xy[k];
            if (X.x == INT_MIN) continue;
            const long long cx = (long long)X.x + O.x, cy = (long long)X.y + O.y;
            const long long c2 = cx * cx + cy * cy;
            if (c2 < lo2 || c2 > hi2) continue;
            const long long dx = cx - H.origin_um, dy = cy - H.origin_um;
            if (dx < 0 || dy < 0 || dx >= span || dy >= span) continue;
            const int bx = div_floor((int)dx, H.bin_um, inv_bin), by = div_floor((int)dy, H.bin_um, inv_bin);
            atomicAdd(&A[by * nb + bx], 1);
        }
    }
}

// One block per event: threshold, 3x3 peak test, ordering, radius histogram
// and the seed centre on r = R0 (FP64).
__global__ void __launch_bounds__(1024) hough_peaks_kernel(const int32_t* __restrict__ hit_off,
                                                           const int32_t* __restrict__ wire_id,
                                                           const int2* __restrict__ wire_um, int n_wires,
                                                           cdc_hough_params H, double R0,
                                                           const int32_t* __restrict__ acc, cdc_candidate* cand,
                                                           int32_t* n_cand, cdc_grid* grid_out, uint32_t* flags) {
    __shared__ unsigned long long s_list[PEAK_LIST];
    __shared__ int s_hist2[PEAK_HIST];
    __shared__ int s_wcnt[32];
    __shared__ int s_n, s_max, s_t, s_found, s_chunk;
    __shared__ int s_hist[256];
    __shared__ int s_rbin[64];
    const int e = blockIdx.x;
    const int nb = H.n_bins;
    const long long ncell = (long long)nb * nb;
    const int32_t* A = acc + (size_t)e * ncell;
    if (threadIdx.x == 0) {
        s_n = 0;
        s_max = 0;
    }
    __syncthreads();
    int mx = 0;
    for (long long c = threadIdx.x; c < ncell; c += blockDim.x) mx = max(mx, A[c]);
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_down_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) atomicMax(&s_max, mx);
    __syncthreads();
    const int thr = max(H.min_peak, (s_max + 1) / 2);
    // Exact selection of the max_cand best peaks without a bound on how many
    // peaks the accumulator holds: a histogram of peak counts gives the count
    // t of the last selected peak; peaks above t are collected directly (fewer
    // than max_cand), peaks equal to t in increasing cell order until the list
    // is full.
    for (int b = threadIdx.x; b < PEAK_HIST; b += blockDim.x) s_hist2[b] = 0;
    __syncthreads();
    for (long long c = threadIdx.x; c < ncell; c += blockDim.x) {
        const int v = A[c];
        if (v >= thr && is_peak(A, nb, c, v)) atomicAdd(&s_hist2[min(v, PEAK_HIST - 1)], 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int cum = 0, t = -1, lowest = -1;
        for (int b = PEAK_HIST - 1; b >= 0; --b) {
            if (s_hist2[b] == 0) continue;
            lowest = b;
            cum += s_hist2[b];
            if (cum >= H.max_cand) {
                t = b;
                break;
            }
        }
        s_t = t >= 0 ? t : lowest;  // fewer peaks than max_cand: take them all
    }
    __syncthreads();
    const int t_last = s_t;
    if (t_last >= 0) {
        const bool top = t_last == PEAK_HIST - 1;
        for (long long c = threadIdx.x; c < ncell; c += blockDim.x) {
            const int v = A[c];
            if ((top ? v >= t_last : v > t_last) && is_peak(A, nb, c, v)) {
                const int pos = atomicAdd(&s_n, 1);
                if (pos < PEAK_LIST)
                    s_list[pos] = ((unsigned long long)(0xffffffffu - (unsigned)v) << 32) | (unsigned)c;
            }
        }
        __syncthreads();
        if (!top) {
            const int need = H.max_cand - s_n;  // ties at t_last, lowest cell index first
            if (threadIdx.x == 0) s_found = 0;
            __syncthreads();
            for (long long base = 0; base < ncell && s_found < need; base += blockDim.x) {
                const long long c = base + threadIdx.x;
                const bool tie = c < ncell && A[c] == t_last && is_peak(A, nb, c, t_last);
                const unsigned m = __ballot_sync(0xffffffffu, tie);
                if ((threadIdx.x & 31) == 0) s_wcnt[threadIdx.x >> 5] = __popc(m);
                __syncthreads();
                if (threadIdx.x == 0) {
                    int acc2 = 0;
                    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
                        const int k = s_wcnt[w];
                        s_wcnt[w] = acc2;
                        acc2 += k;
                    }
                    s_chunk = acc2;
                }
                __syncthreads();
                if (tie) {
                    const int pos = s_found + s_wcnt[threadIdx.x >> 5] + __popc(m & ((1u << (threadIdx.x & 31)) - 1u));
                    if (pos < need)
                        s_list[s_n + pos] = ((unsigned long long)(0xffffffffu - (unsigned)t_last) << 32) | (unsigned)c;
                }
                __syncthreads();
                if (threadIdx.x == 0) s_found += s_chunk;
                __syncthreads();
            }
            if (threadIdx.x == 0) s_n += min(s_found, need);
            __syncthreads();
        }
    }
    const int np = min(s_n, PEAK_LIST);
    if (threadIdx.x == 0 && s_n > PEAK_LIST) atomicOr(&flags[e], CDC_FLAG_FOUND_OVERFLOW);
    for (int i = np + threadIdx.x; i < PEAK_LIST; i += blockDim.x) s_list[i] = ~0ull;
    __syncthreads();
    // bitonic sort of the selected peak keys: (count desc, index asc)
    for (int k = 2; k <= PEAK_LIST; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < PEAK_LIST; i += blockDim.x) {
                const int l = i ^ j;
                if (l > i) {
                    const unsigned long long a = s_list[i], b = s_list[l];
                    const bool up = (i & k) == 0;
                    if ((a > b) == up) {
                        s_list[i] = b;
                        s_list[l] = a;
                    }
                }
            }
            __syncthreads();
        }
    const int nc = min(np, H.max_cand);
    const int h0 = hit_off[e], h1 = hit_off[e + 1];
    for (int q = 0; q < nc; ++q) {
        const int c = (int)(s_list[q] & 0xffffffffu);
        const long long cx = (long long)H.origin_um + (long long)(c % nb) * H.bin_um + H.bin_um / 2;
        const long long cy = (long long)H.origin_um + (long long)(c / nb) * H.bin_um + H.bin_um / 2;
        for (int j = threadIdx.x; j < H.n_r; j += blockDim.x) s_hist[j] = 0;
        __syncthreads();
        for (int h = h0 + threadIdx.x; h < h1; h += blockDim.x) {
            const int w = wire_id[h];
            if (w < 0 || w >= n_wires) continue;
            const int2 X = wire_um[w];
            const long long dx = X.x - cx, dy = X.y - cy;
            const long long d2 = dx * dx + dy * dy;
            for (int j = 0; j < H.n_r; ++j) {
                const long long R = (long long)H.r_min_um + (long long)j * H.r_step_um;
                const long long a = R - H.r_hist_half_um, b = R + H.r_hist_half_um;
                if (d2 >= a * a && d2 < b * b) atomicAdd(&s_hist[j], 1);
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            int bj = -1, bc = 0;
            for (int j = 0; j < H.n_r; ++j)
                if (s_hist[j] > bc) {
                    bc = s_hist[j];
                    bj = j;
                }
            s_rbin[q] = bj;
        }
        __syncthreads();
    }
    if (threadIdx.x < nc) {
        const int q = threadIdx.x;
        const int c = (int)(s_list[q] & 0xffffffffu);
        const int ix = c % nb, iy = c / nb;
        const int bj = s_rbin[q];
        const double qnan = __longlong_as_double(0x7ff8000000000000ll);
        double th = qnan, px = qnan, py = qnan;
        if (bj >= 0) {
            const double Cx = ((double)H.origin_um + (double)ix * H.bin_um + H.bin_um / 2) / 1000.0;
            const double Cy = ((double)H.origin_um + (double)iy * H.bin_um + H.bin_um / 2) / 1000.0;
            const double R = ((double)H.r_min_um + (double)bj * H.r_step_um) / 1000.0;
            const double dd = sqrt(Cx * Cx + Cy * Cy);
            if (dd > 0.0 && R0 <= dd + R && R0 >= fabs(dd - R)) {
                const double a = (R0 * R0 - R * R + dd * dd) / (2.0 * dd);
                const double hp = sqrt(fmax(R0 * R0 - a * a, 0.0));
                const double ccw = ((double)H.charge * (double)H.b_nominal < 0.0) ? 1.0 : -1.0;
                for (int sgn = 1; sgn >= -1; sgn -= 2) {
                    const double Px = a * Cx / dd - sgn * hp * Cy / dd;
                    const double Py = a * Cy / dd + sgn * hp * Cx / dd;
                    const double tx = -ccw * (Py - Cy) / R, ty = ccw * (Px - Cx) / R;
                    if (tx * Px + ty * Py > 0.0) {  // the outward crossing
                        const double pt = KAPPA_D * fabs((double)H.b_nominal) * R;
                        th = atan2(Py, Px);
                        px = pt * tx;
                        py = pt * ty;
                        break;
                    }
                }
            }
        }
        cdc_candidate cd;
        cd.ix = ix;
        cd.iy = iy;
        cd.count = (int)(0xffffffffu - (unsigned)(s_list[q] >> 32));
        cd.r_bin = bj;
        cd.theta0 = (float)th;
        cd.px0 = (float)px;
        cd.py0 = (float)py;
        cand[(size_t)e * H.max_cand + q] = cd;
        if (q == 0 && grid_out) {
            cdc_grid g = H.grid_template;
            g.centre[0] = (float)th;
            g.centre[2] = (float)px;
            g.centre[3] = (float)py;
            if (!(th == th)) {
                for (int a2 = 0; a2 < 5; ++a2) g.n[a2] = 0;
                atomicOr(&flags[e], CDC_FLAG_EMPTY);
            }
            grid_out[e] = g;
        }
    }
    if (threadIdx.x == 0) {
        n_cand[e] = nc;
        if (nc == 0) {
            atomicOr(&flags[e], CDC_FLAG_EMPTY);
            if (grid_out) {
                cdc_grid g = H.grid_template;
                for (int a2 = 0; a2 < 5; ++a2) g.n[a2] = 0;
                grid_out[e] = g;
            }
        }
    }
}

cudaError_t launch_hough(const DevGeom& G, const cdc_hough_params& H, const HoughLaunch& L, cudaStream_t st) {
    const size_t cells = (size_t)H.n_bins * H.n_bins;
    cudaError_t err = cudaMemsetAsync(L.acc, 0, sizeof(int32_t) * cells * L.n_events, st);
    if (err != cudaSuccess) return err;
    const int n_pairs = H.n_r * H.n_phi;
    dim3 grid((n_pairs + 255) / 256, 8, L.n_events);
    hough_vote_kernel<<<grid, 256, 0, st>>>(L.hit_off, L.wire_id, G.wire_um, G.n_wires, L.offsets, H, L.acc);
    hough_peaks_kernel<<<L.n_events, 1024, 0, st>>>(L.hit_off, L.wire_id, G.wire_um, G.n_wires, H, G.R0d, L.acc,
                                                    L.cand, L.n_cand, L.grid_out, L.flags);
    return cudaGetLastError();
}

// One grid per (event, candidate slot): the template centred on the
// candidate's seed, or a grid of zero seeds past the event's candidates and
// where the circle never crosses r = R0 (the rule of the top candidate's
// grid in hough_peaks_kernel).
__global__ void candidate_grids_kernel(int n_events, int max_cand, cdc_grid tmpl, const cdc_candidate* __restrict__ cand,
                                       const int32_t* __restrict__ n_cand, cdc_grid* grids) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_events * max_cand) return;
    const int e = i / max_cand, q = i - e * max_cand;
    cdc_grid g = tmpl;
    bool empty = q >= n_cand[e];
    if (!empty) {
        const cdc_candidate cd = cand[i];
        g.centre[0] = cd.theta0;
        g.centre[2] = cd.px0;
        g.centre[3] = cd.py0;
        empty = !(cd.theta0 == cd.theta0);
    }
    if (empty)
        for (int a = 0; a < 5; ++a) g.n[a] = 0;
    grids[i] = g;
}

cudaError_t launch_candidate_grids(int n_events, const cdc_hough_params& H, const cdc_candidate* cand,
                                   const int32_t* n_cand, cdc_grid* grids, cudaStream_t st) {
    const int n = n_events * H.max_cand;
    candidate_grids_kernel<<<(n + 127) / 128, 128, 0, st>>>(n_events, H.max_cand, H.grid_template, cand, n_cand,
                                                            grids);
    return cudaGetLastError();
}

}  // namespace cdc
