// Circle Hough transform (arXiv:1908.01949 sec. 2.1, Fig. 4): integer vote
// accumulation, peak finding and the transverse seed centre.
#include <cuda_runtime.h>
#include <limits.h>
#include <stdint.h>

#include "cdc_dev.cuh"
#include "cdc_host.h"

namespace cdc {

constexpr int HOUGH_HITS = 64;      // hits staged per block iteration
constexpr int PEAK_BLOCKS = HOUGH_SLICES;    // blocks per event of the peak search, one slice of cells each
constexpr int PEAK_KEYS = HOUGH_SLICE_KEYS;  // entries of a slice's list (max_cand <= 64)
constexpr int PEAK_THREADS = 256;
constexpr int SELECT_RUN = 16;      // counts each lane loads before testing them
constexpr int HIST_CAP = 4096;      // radius-histogram bins of one pass over the hits (n_r <= 256)
static_assert(PEAK_BLOCKS % (PEAK_THREADS / 32) == 0, "each warp merges the same number of slices");
static_assert(PEAK_KEYS <= PEAK_THREADS, "a thread per candidate of a histogram pass");

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

// The peak search runs in three launches so that an event's 262144 cells are
// read by many blocks: the event's maximum (the threshold), each block's
// PEAK_KEYS best peaks of its slice, and one block per event that merges the
// slices' lists and forms the radius histogram and the seed centre.  A peak's
// key is (~count << 32 | cell), so ascending keys are the order (count desc,
// index asc) and the selection is exact however many peaks there are.
__device__ __forceinline__ void peak_slice(long long ncell, int b, long long& c0, long long& c1) {
    const long long per = (ncell + PEAK_BLOCKS - 1) / PEAK_BLOCKS;
    c0 = min(ncell, (long long)b * per);
    c1 = min(ncell, c0 + per);
}

__device__ __forceinline__ uint64_t peak_key(int v, long long c) {
    return ((uint64_t)(0xffffffffu - (unsigned)v) << 32) | (uint32_t)c;
}

// The warps' lists of a block, merged into warp 0's (la, lb).
__device__ __forceinline__ void merge_warp_lists(uint64_t& la, uint64_t& lb, int K,
                                                 uint64_t (*s_keys)[PEAK_KEYS]) {
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    s_keys[w][lane] = la;
    s_keys[w][32 + lane] = lb;
    __syncthreads();
    if (w == 0)
        for (int o = 1; o < PEAK_THREADS / 32; ++o) {
            const uint64_t ka = s_keys[o][lane], kb = s_keys[o][32 + lane];
            list_insert(la, lb, ka, ka != KEY_NONE, K);
            list_insert(la, lb, kb, kb != KEY_NONE, K);
        }
}

__global__ void __launch_bounds__(PEAK_THREADS) hough_max_kernel(int nb, const int32_t* __restrict__ acc,
                                                                 int32_t* emax) {
    __shared__ int s_max;
    const int e = blockIdx.y;
    const long long ncell = (long long)nb * nb;
    const int32_t* A = acc + (size_t)e * ncell;
    long long c0, c1;
    peak_slice(ncell, blockIdx.x, c0, c1);
    if (threadIdx.x == 0) s_max = 0;
    __syncthreads();
    int mx = 0;
    for (long long c = c0 + threadIdx.x; c < c1; c += blockDim.x) mx = max(mx, A[c]);
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_down_sync(FULL, mx, o));
    if ((threadIdx.x & 31) == 0) atomicMax(&s_max, mx);
    __syncthreads();
    if (threadIdx.x == 0 && s_max > 0) atomicMax(&emax[e], s_max);
}

// Peaks of one slice: count >= max(min_peak, ceil(max / 2)) and the strict
// 3x3 maximum test; the block's max_cand smallest keys go to
// keys[e][blockIdx.x][0 .. PEAK_KEYS).
__global__ void __launch_bounds__(PEAK_THREADS) hough_select_kernel(cdc_hough_params H,
                                                                    const int32_t* __restrict__ acc,
                                                                    const int32_t* __restrict__ emax,
                                                                    uint64_t* keys) {
    __shared__ uint64_t s_keys[PEAK_THREADS / 32][PEAK_KEYS];
    const int e = blockIdx.y, nb = H.n_bins, K = H.max_cand;
    const long long ncell = (long long)nb * nb;
    const int32_t* A = acc + (size_t)e * ncell;
    const int thr = max(H.min_peak, (emax[e] + 1) / 2);
    long long c0, c1;
    peak_slice(ncell, blockIdx.x, c0, c1);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint64_t la = KEY_NONE, lb = KEY_NONE;
    // a warp takes runs of 32 x SELECT_RUN cells; the run's counts are loaded
    // before any is tested, so the loads overlap instead of waiting in turn
    for (long long base = c0 + (long long)w * 32 * SELECT_RUN; base < c1;
         base += (long long)(PEAK_THREADS / 32) * 32 * SELECT_RUN) {  // warp-uniform
        int v[SELECT_RUN];
#pragma unroll
        for (int k = 0; k < SELECT_RUN; ++k) {
            const long long c = base + k * 32 + lane;
            v[k] = c < c1 ? A[c] : 0;
        }
#pragma unroll
        for (int k = 0; k < SELECT_RUN; ++k) {
            const long long c = base + k * 32 + lane;
            const bool peak = c < c1 && v[k] >= thr && is_peak(A, nb, c, v[k]);
            if (__any_sync(FULL, peak)) list_insert(la, lb, peak ? peak_key(v[k], c) : KEY_NONE, peak, K);
        }
    }
    merge_warp_lists(la, lb, K, s_keys);
    if (threadIdx.x < 32) {
        uint64_t* out = keys + ((size_t)e * PEAK_BLOCKS + blockIdx.x) * PEAK_KEYS;
        out[threadIdx.x] = la;
        out[32 + threadIdx.x] = lb;
    }
}

// One block per event: the slices' lists merged into the event's max_cand
// best peaks, then per peak the radius histogram and the seed centre on
// r = R0 (FP64).
__global__ void __launch_bounds__(PEAK_THREADS) hough_finish_kernel(const int32_t* __restrict__ hit_off,
                                                                    const int32_t* __restrict__ wire_id,
                                                                    const int2* __restrict__ wire_um, int n_wires,
                                                                    cdc_hough_params H, double R0,
                                                                    const uint64_t* __restrict__ keys,
                                                                    cdc_candidate* cand, int32_t* n_cand,
                                                                    cdc_grid* grid_out, uint32_t* flags) {
    __shared__ uint64_t s_keys[PEAK_THREADS / 32][PEAK_KEYS];
    __shared__ uint64_t s_list[PEAK_KEYS];
    __shared__ int s_hist[HIST_CAP];
    __shared__ int s_rbin[PEAK_KEYS];
    __shared__ int s_n;
    const int e = blockIdx.x;
    const int nb = H.n_bins, K = H.max_cand;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint64_t la = KEY_NONE, lb = KEY_NONE;
    {
        constexpr int PER_WARP = PEAK_BLOCKS / (PEAK_THREADS / 32);  // slices merged by each warp
        uint64_t ka[PER_WARP], kb[PER_WARP];
#pragma unroll
        for (int i = 0; i < PER_WARP; ++i) {  // all loads first
            const uint64_t* src = keys + ((size_t)e * PEAK_BLOCKS + w + i * (PEAK_THREADS / 32)) * PEAK_KEYS;
            ka[i] = src[lane];
            kb[i] = src[32 + lane];
        }
#pragma unroll
        for (int i = 0; i < PER_WARP; ++i) {
            list_insert(la, lb, ka[i], ka[i] != KEY_NONE, K);
            list_insert(la, lb, kb[i], kb[i] != KEY_NONE, K);
        }
    }
    merge_warp_lists(la, lb, K, s_keys);
    if (w == 0) {
        s_list[lane] = la;
        s_list[32 + lane] = lb;
        const int n = __popc(__ballot_sync(FULL, la != KEY_NONE)) + __popc(__ballot_sync(FULL, lb != KEY_NONE));
        if (lane == 0) s_n = min(n, K);
    }
    __syncthreads();
    const int nc = s_n;
    const int h0 = hit_off[e], h1 = hit_off[e + 1];
    // radius histograms of up to HIST_CAP / n_r candidates per pass over the hits
    const int group = HIST_CAP / H.n_r;
    for (int q0 = 0; q0 < nc; q0 += group) {
        const int qn = min(group, nc - q0);
        for (int i = threadIdx.x; i < qn * H.n_r; i += blockDim.x) s_hist[i] = 0;
        __syncthreads();
        for (int h = h0 + threadIdx.x; h < h1; h += blockDim.x) {
            const int wi = wire_id[h];
            if (wi < 0 || wi >= n_wires) continue;
            const int2 X = wire_um[wi];
            for (int q = 0; q < qn; ++q) {
                const int c = (int)(s_list[q0 + q] & 0xffffffffu);
                const long long cx = (long long)H.origin_um + (long long)(c % nb) * H.bin_um + H.bin_um / 2;
                const long long cy = (long long)H.origin_um + (long long)(c / nb) * H.bin_um + H.bin_um / 2;
                const long long dx = X.x - cx, dy = X.y - cy;
                const long long d2 = dx * dx + dy * dy;
                for (int j = 0; j < H.n_r; ++j) {
                    const long long R = (long long)H.r_min_um + (long long)j * H.r_step_um;
                    const long long a = R - H.r_hist_half_um, b = R + H.r_hist_half_um;
                    if (d2 >= a * a && d2 < b * b) atomicAdd(&s_hist[q * H.n_r + j], 1);
                }
            }
        }
        __syncthreads();
        if (threadIdx.x < qn) {  // the most populated radius, ties to the lower j
            int bj = -1, bc = 0;
            for (int j = 0; j < H.n_r; ++j)
                if (s_hist[threadIdx.x * H.n_r + j] > bc) {
                    bc = s_hist[threadIdx.x * H.n_r + j];
                    bj = j;
                }
            s_rbin[q0 + threadIdx.x] = bj;
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
    err = cudaMemsetAsync(L.emax, 0, sizeof(int32_t) * L.n_events, st);
    if (err != cudaSuccess) return err;
    const dim3 pg(PEAK_BLOCKS, L.n_events);
    hough_max_kernel<<<pg, PEAK_THREADS, 0, st>>>(H.n_bins, L.acc, L.emax);
    hough_select_kernel<<<pg, PEAK_THREADS, 0, st>>>(H, L.acc, L.emax, L.keys);
    hough_finish_kernel<<<L.n_events, PEAK_THREADS, 0, st>>>(L.hit_off, L.wire_id, G.wire_um, G.n_wires, H, G.R0d,
                                                             L.keys, L.cand, L.n_cand, L.grid_out, L.flags);
    return cudaGetLastError();
}

// One grid per (event, candidate slot): the template centred on the
// candidate's seed, or a grid of zero seeds past the event's candidates and
// where the circle never crosses r = R0 (the rule of the top candidate's
// grid in hough_finish_kernel).
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
