// Seed scan kernels (arXiv:1908.01949 sec. 2.2, Eq. 1): hit staging, the
// persistent thread-per-seed RKN scorer, warp-level top-K, the zoom re-scan
// grids and the hit-to-turn classification of the best seed.
#include <cuda_runtime.h>

#include <algorithm>
#include <stdint.h>

#include "cdc_dev.cuh"
#include "cdc_host.h"
#include "tracer.cuh"
#include "warp_tracer.cuh"

namespace cdc {

constexpr float NOT_FIRED = 3.0e38f;   // drift-table sentinel (above any valid drift)

// ---------------------------------------------------------------- staging
// Event table of event e: tab[e][wire] = drift of the event's hit on that wire
// and the fired bit of the wire; validates the wire id and drift range;
// duplicate wires keep the smaller drift and flag.
__global__ void clear_tables_kernel(float* tab, int n_events, int n_wires) {
    const int stride = (int)event_stride(n_wires);
    for (int e = blockIdx.y; e < n_events; e += gridDim.y) {
        float* t = tab + (size_t)e * stride;
        for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < stride; j += gridDim.x * blockDim.x)
            t[j] = j < n_wires ? NOT_FIRED : 0.f;  // 0.f: all fired bits clear
    }
}

__global__ void stage_kernel(DevGeom G, int n_events, const int32_t* __restrict__ hit_off,
                             const int32_t* __restrict__ wire_id, const float* __restrict__ drift, float max_drift,
                             float* tab, uint32_t* flags) {
    const int n_wires = G.n_wires;
    const size_t stride = event_stride(n_wires);
    const int total = hit_off[n_events];
    for (int h = blockIdx.x * blockDim.x + threadIdx.x; h < total; h += gridDim.x * blockDim.x) {
        int lo = 0, hi = n_events - 1;
        while (lo < hi) {  // event e with hit_off[e] <= h < hit_off[e+1]
            int mid = (lo + hi + 1) >> 1;
            if (hit_off[mid] <= h) lo = mid; else hi = mid - 1;
        }
        int w = wire_id[h];
        float d = drift[h];
        if (w < 0 || w >= n_wires || !(d >= 0.f && d <= max_drift)) {
            if (flags) atomicOr(&flags[lo], CDC_FLAG_BAD_HIT);
            continue;
        }
        float* t = tab + (size_t)lo * stride;
        int old = atomicMin((int*)&t[w], __float_as_int(d));
        if (old != __float_as_int(NOT_FIRED) && flags) atomicOr(&flags[lo], CDC_FLAG_BAD_HIT);
        int a = 0, b = G.n_layers - 1;  // layer of the wire
        while (a < b) {
            const int mid = (a + b + 1) >> 1;
            if (G.layers[mid].base <= w) a = mid; else b = mid - 1;
        }
        const DevLayer& L = G.layers[a];
        uint32_t* bits = (uint32_t*)(t + n_wires) + L.bword;
        const int i = w - L.base;
        atomicOr(bits + (i >> 5), 1u << (i & 31));
        if (i < 32) atomicOr(bits + ((L.N + i) >> 5), 1u << ((L.N + i) & 31));
    }
}

cudaError_t launch_stage(const DevGeom& G, int n_events, const int32_t* hit_off, const int32_t* wire_id,
                         const float* drift, float max_drift, float* tab, uint32_t* flags, int num_sms,
                         cudaStream_t st) {
    if (n_events <= 0) return cudaSuccess;
    const int stride = (int)event_stride(G.n_wires);
    const dim3 cg((stride + 255) / 256, n_events < 65535 ? n_events : 65535);
    clear_tables_kernel<<<cg, 256, 0, st>>>(tab, n_events, G.n_wires);
    stage_kernel<<<num_sms * 4, 256, 0, st>>>(G, n_events, hit_off, wire_id, drift, max_drift, tab, flags);
    return cudaGetLastError();
}

// --------------------------------------------------------------- prologue
// Seed and top-K segment offsets of every event for one round; resets the
// work counter.  One block.
__global__ void prologue_kernel(int n_events, const cdc_grid* __restrict__ grids, int gpe, long long cap,
                                long long seg_cap, long long* seed_off, int* seg_off, unsigned long long* counters,
                                uint32_t* flags) {
    __shared__ long long s_sum[1024];
    __shared__ int s_seg[1024];
    __shared__ long long s_base;
    __shared__ int s_sbase;
    if (threadIdx.x == 0) {
        s_base = 0;
        s_sbase = 0;
    }
    __syncthreads();
    for (int c0 = 0; c0 < n_events; c0 += blockDim.x) {
        int e = c0 + threadIdx.x;
        long long n = 0;
        if (e < n_events) {
            for (int g = 0; g < gpe; ++g) n += grid_count(grids[(size_t)e * gpe + g]);
            if (n >= (1ll << ROUND_SHIFT)) {
                atomicOr(&flags[e], CDC_FLAG_EMPTY);
                n = 0;
            }
        }
        int sg = (int)((n + SEG - 1) / SEG);
        s_sum[threadIdx.x] = n;
        s_seg[threadIdx.x] = sg;
        __syncthreads();
        for (int off = 1; off < blockDim.x; off <<= 1) {  // inclusive scan
            long long a = threadIdx.x >= off ? s_sum[threadIdx.x - off] : 0;
            int b = threadIdx.x >= off ? s_seg[threadIdx.x - off] : 0;
            __syncthreads();
            s_sum[threadIdx.x] += a;
            s_seg[threadIdx.x] += b;
            __syncthreads();
        }
        if (e < n_events) {
            seed_off[e] = s_base + s_sum[threadIdx.x] - n;
            seg_off[e] = s_sbase + s_seg[threadIdx.x] - sg;
        }
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) {
            s_base += s_sum[threadIdx.x];
            s_sbase += s_seg[threadIdx.x];
        }
        __syncthreads();
    }
    // beyond the buffers: scan nothing (every event gets empty seed and segment
    // ranges, so no later kernel reads past them) and flag every event
    const bool over = s_base > cap || (long long)s_sbase > seg_cap;
    if (over)
        for (int e = threadIdx.x; e <= n_events; e += blockDim.x) {
            seed_off[e] = 0;
            seg_off[e] = 0;
            if (e < n_events) atomicOr(&flags[e], CDC_FLAG_EMPTY);
        }
    if (threadIdx.x == 0) {
        const long long tot = over ? 0 : s_base;
        seed_off[n_events] = tot;
        seg_off[n_events] = tot ? s_sbase : 0;
        counters[0] = 0;
        counters[1] = (unsigned long long)tot;
        counters[2] = (unsigned long long)(tot ? s_sbase : 0);
    }
}

// ------------------------------------------------------------- the scan
struct ScanIO {
    const float* drift_tab;
    const int32_t* hit_off;
    const cdc_grid* grids;
    int gpe;
    const long long* seed_off;
    int n_events;
    unsigned long long* counters;
    float* E;
    uint32_t* flags;
    unsigned long long* steps;
    const uint16_t* perm;  // [n_events][PERM_CAP] block order of single-grid rounds, or nullptr
    SeedRecord* recs;      // [n_events][REC_SLOTS] records of improving seeds (zoom rounds), or nullptr
    unsigned* rec_count;   // [n_events]
    unsigned* run_best;    // [n_events] best score so far (float bits)
    int round;
};

// A slot for the record of a zoom-round seed whose score is at most its
// event's best so far (the running minimum starts each round at the best of
// the previous rounds), or -1: only such a seed can become the event's best.
__device__ __forceinline__ int record_slot(const ScanIO& io, int ev, float score) {
    if (!(score >= 0.f)) return -1;
    const unsigned bits = __float_as_uint(score);  // non-negative floats order as their bits
    if (bits > atomicMin(io.run_best + ev, bits)) return -1;
    const unsigned slot = atomicAdd(io.rec_count + ev, 1u);
    return slot < (unsigned)REC_SLOTS ? (int)slot : -1;
}

// Per event, the (z0, pz0) blocks of its coarse grid in the order the scan
// takes them: longest estimated track first, so that the persistent scan ends
// on short tracks and its warps run out of work together.  Estimate: the path
// to the end plate the track heads for, (z_half - z0 sgn(pz dir)) p / |pz|,
// capped at max_part turns of 2 pi p / (kappa b_max), with (px, py) at the
// grid centre.  Only the order in which seeds are processed changes, not their
// scores or indices.  Rank of block i = number of blocks with a larger key, or
// an equal key and a lower index (a permutation).
__global__ void __launch_bounds__(1024) order_blocks_kernel(int n_events, const cdc_grid* __restrict__ grids,
                                                            float z_half, float b_max, int max_part, int direction,
                                                            uint16_t* perm) {
    __shared__ float s_key[PERM_CAP];
    const int e = blockIdx.x;
    if (e >= n_events) return;
    const cdc_grid g = grids[e];
    const int nz = g.n[1], np = g.n[4];
    if (nz < 1 || np < 1 || (long long)nz * np > PERM_CAP) return;  // scan_order_index keeps the natural order
    const int nb = nz * np;
    const float px = g.centre[2], py = g.centre[3];
    for (int i = threadIdx.x; i < nb; i += blockDim.x) {
        const float z0 = fmaf((float)(i / np) - 0.5f * (float)(nz - 1), g.step[1], g.centre[1]);
        const float pz = fmaf((float)(i % np) - 0.5f * (float)(np - 1), g.step[4], g.centre[4]);
        const float p = sqrtf(fmaf(px, px, fmaf(py, py, pz * pz)));
        const float turn = b_max > 0.f ? 6.28318531f * p / (KAPPA * b_max) : INFINITY;
        const float side = pz * (float)direction >= 0.f ? 1.f : -1.f;
        const float sz = fabsf(pz) > 0.f ? fmaxf(z_half - side * z0, 0.f) * p / fabsf(pz) : INFINITY;
        const float key = fminf(sz, (float)max_part * turn);
        s_key[i] = key == key ? key : 0.f;
    }
    __syncthreads();
    uint16_t* out = perm + (size_t)e * PERM_CAP;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) {
        const float k = s_key[i];
        int rank = 0;
        for (int j = 0; j < nb; ++j) {
            const float kj = s_key[j];
            rank += (kj > k || (kj == k && j < i)) ? 1 : 0;
        }
        out[rank] = (uint16_t)i;
    }
}

// Persistent thread-per-seed scorer.  A warp takes 32 consecutive seeds in
// scan order (neighbours in theta0, px0, py0 at equal z0, pz0: nearly the same
// path, so the lanes search nearly the same wires and stay converged) from a
// global counter, steps them in chunks of CHUNK RKN steps, and takes the next
// 32 once all its lanes have ended; in a coarse round the (z0, pz0) blocks
// come longest estimated track first (order_blocks_kernel), so the round ends
// on short tracks.  Scores are written at the seeds' row-major indices; in
// zoom rounds a seed that reaches its event's best score so far also keeps
// its record of scored wires (record_slot).
// BS threads per block: seven 128-thread blocks per SM (28 warps, 72 registers
// per thread) or three 256-thread blocks (24 warps, 80 registers); the
// shorter register budget costs a few spilled words and its extra warps hide
// more of the field-load latency.
template <int KIND, int BS, int CHUNK>
__global__ void __launch_bounds__(BS, 896 / BS) scan_kernel(DevGeom G, DevField F, ScanConst P, ScanIO io) {
    static_assert(CHUNK % LIST_M == 0, "candidate lists restart at chunk boundaries");
    extern __shared__ DevLayer s_lay[];  // [G.n_layers]: dynamic, so three blocks' lists and tables leave 192 KB of L1
    __shared__ uchar2 s_tab[TAB_N];
    __shared__ ListEntry s_cand[LIST_CAP][BS];
    for (int i = threadIdx.x; i < G.n_layers; i += blockDim.x) s_lay[i] = G.layers[i];
    for (int i = threadIdx.x; i < TAB_N; i += blockDim.x) s_tab[i] = G.tab[i];
    __syncthreads();
    const long long total = (long long)io.counters[1];
    const int lane = threadIdx.x & 31;
    Tracer<KIND> T;
    FoundList FL;
    long long my = -1;   // this lane's seed; -1: ended (or none yet), -2: no seeds left
    long long done = -1; // an ended seed whose score is still to be formed
    int ev = 0;
    unsigned long long nsteps = 0;
    for (;;) {
        if (__all_sync(FULL, my < 0)) {
            // the cohort ended: its seeds' scores are formed from their records
            // together (converged), then whole cohorts are refilled
            if (done >= 0) {
                const int H = io.hit_off[ev + 1] - io.hit_off[ev];
                const float score = T.score(P, H, FL);
                io.E[done] = score;
                if (io.recs) {
                    const int slot = record_slot(io, ev, score);
                    if (slot >= 0) {
                        SeedRecord& R = io.recs[(size_t)ev * REC_SLOTS + slot];
                        R.round = io.round;
                        R.index = (int)(done - io.seed_off[ev]);
                        R.nf = T.nf;
                        for (int i = 0; i < T.nf; ++i) {
                            R.key[i] = FL.key[i];
                            R.r[i] = FL.r[i];
                        }
                    }
                }
                if (T.flags) atomicOr(&io.flags[ev], T.flags);
                nsteps += (unsigned long long)T.n;
                done = -1;
            }
            const unsigned need = __ballot_sync(FULL, my == -1);
            if (!need) break;
            const int leader = __ffs(need) - 1;
            unsigned long long base = 0;
            if (lane == leader) base = atomicAdd(&io.counters[0], (unsigned long long)__popc(need));
            base = __shfl_sync(FULL, base, leader);
            if (my == -1) {
                const long long s = (long long)base + __popc(need & ((1u << lane) - 1u));
                if (s < total) {
                    ev = find_event(io.seed_off, io.n_events, s);
                    float sd[5];
                    my = io.seed_off[ev] + event_seed_ordered(io.grids, io.gpe, ev, s - io.seed_off[ev], sd,
                                                              io.perm ? io.perm + (size_t)ev * PERM_CAP : nullptr);
                    T.init(G, F, P, s_lay, s_tab, io.drift_tab + (size_t)ev * event_stride(G.n_wires),
                           &s_cand[0][threadIdx.x], BS, sd, FL);
                } else {
                    my = -2;
                }
            }
        }
        if (my >= 0) {
            for (int it = 0; it < CHUNK; ++it) {
                if (!T.step(G, F, P, s_lay, s_tab, FL)) {
                    done = my;
                    my = -1;
                    break;
                }
                if ((it % LIST_M) == LIST_M - 1) {  // seeds start at chunk starts
                    T.rebuild(G, P, s_lay, s_tab);
                    T.make_room(P, FL);
                }
            }
        }
    }
    if (io.steps) {
        for (int o = 16; o > 0; o >>= 1) nsteps += __shfl_down_sync(FULL, nsteps, o);
        if (lane == 0 && nsteps) atomicAdd(io.steps, nsteps);
    }
}

// ------------------------------------------------------------------ top-K
// One warp per segment of SEG seeds: the K lowest (E, index) keys.
__global__ void topk_partial_kernel(const float* __restrict__ E, const long long* __restrict__ seed_off,
                                    const int* __restrict__ seg_off, int n_events,
                                    const unsigned long long* counters, int K, uint64_t* seg_keys) {
    const int lane = threadIdx.x & 31;
    const int warps = gridDim.x * (blockDim.x >> 5);
    const long long n_seg = (long long)counters[2];
    for (long long s = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); s < n_seg; s += warps) {
        int lo = 0, hi = n_events - 1;
        while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if (seg_off[mid] <= s) lo = mid; else hi = mid - 1;
        }
        const int e = lo;
        const long long n_e = seed_off[e + 1] - seed_off[e];
        const long long a0 = (s - seg_off[e]) * (long long)SEG;
        const long long a1 = min(a0 + SEG, n_e);
        uint64_t la = KEY_NONE, lb = KEY_NONE;
        for (long long i0 = a0; i0 < a1; i0 += 32) {
            long long i = i0 + lane;
            bool ok = i < a1;
            uint64_t key = ok ? make_key(E[seed_off[e] + i], (uint32_t)i) : KEY_NONE;
            list_insert(la, lb, key, ok, K);
        }
        uint64_t* out = seg_keys + s * CDC_MAX_K;
        if (lane < K) out[lane] = la;
        if (32 + lane < K) out[32 + lane] = lb;
    }
}

// One warp per event: merge the segment lists into the round's top-K.
__global__ void topk_merge_kernel(const int* __restrict__ seg_off, int n_events, int K,
                                  const uint64_t* __restrict__ seg_keys, uint64_t* round_keys) {
    const int lane = threadIdx.x & 31;
    const int e = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (e >= n_events) return;
    uint64_t la = KEY_NONE, lb = KEY_NONE;
    const long long total = (long long)(seg_off[e + 1] - seg_off[e]) * K;
    const uint64_t* src = seg_keys + (long long)seg_off[e] * CDC_MAX_K;
    for (long long i0 = 0; i0 < total; i0 += 32) {
        long long i = i0 + lane;
        bool ok = i < total;
        uint64_t key = ok ? src[(i / K) * CDC_MAX_K + (i % K)] : KEY_NONE;
        list_insert(la, lb, key, ok && key != KEY_NONE, K);
    }
    uint64_t* out = round_keys + (size_t)e * CDC_MAX_K;
    if (lane < K) out[lane] = la;
    if (32 + lane < K) out[32 + lane] = lb;
}

// One thread per event: merge round r's top-K into the best list over all
// rounds, ordered by (E, round, index); seeds decoded from round r's grids.
__global__ void merge_best_kernel(int n_events, int K, int round, const uint64_t* __restrict__ round_keys,
                                  const cdc_grid* __restrict__ grids, int gpe, uint64_t* best_keys, float* best_E,
                                  float* best_seed, uint64_t* topk0, unsigned* run_best) {
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n_events) return;
    uint64_t ok[CDC_MAX_K];
    float os[CDC_MAX_K][5];
    const uint64_t* rk = round_keys + (size_t)e * CDC_MAX_K;
    uint64_t* bk = best_keys + (size_t)e * CDC_MAX_K;
    for (int i = 0; i < K; ++i) {
        ok[i] = round == 0 ? KEY_NONE : bk[i];
        for (int a = 0; a < 5; ++a) os[i][a] = round == 0 ? 0.f : best_seed[((size_t)e * K + i) * 5 + a];
    }
    if (round == 0 && topk0)
        for (int i = 0; i < K; ++i) topk0[(size_t)e * K + i] = rk[i];
    int p = 0, q = 0;
    for (int i = 0; i < K; ++i) {
        uint64_t nk = rk[q] == KEY_NONE ? KEY_NONE
                                        : ((rk[q] & 0xffffffff00000000ull) | ((uint64_t)round << ROUND_SHIFT) |
                                           (rk[q] & ((1ull << ROUND_SHIFT) - 1)));
        bool take_new = (q < K) && nk < ok[p];
        uint64_t key;
        float sd[5];
        if (take_new) {
            key = nk;
            event_seed(grids, gpe, e, (long long)(rk[q] & 0xffffffffull), sd);
            ++q;
        } else {
            key = ok[p];
            for (int a = 0; a < 5; ++a) sd[a] = os[p][a];
            ++p;
        }
        bk[i] = key;
        best_E[(size_t)e * K + i] = key == KEY_NONE ? __int_as_float(0x7f800000) : __uint_as_float((uint32_t)(key >> 32));
        for (int a = 0; a < 5; ++a)
            best_seed[((size_t)e * K + i) * 5 + a] = key == KEY_NONE ? __int_as_float(0x7fffffff) : sd[a];
    }
    // the next round records the seeds that reach this score (record_slot)
    if (run_best) run_best[e] = bk[0] == KEY_NONE ? 0x7f800000u : (uint32_t)(bk[0] >> 32);
}

// Zoom grids of round r (sec. 2.2: finer seed sets around the candidates):
// around each of the previous round's n_zoom best seeds a 3^5 grid with the
// coarse step times 2^-r.
__global__ void zoom_grid_kernel(int n_events, int n_zoom, int round, const uint64_t* __restrict__ prev_keys,
                                 const cdc_grid* __restrict__ prev_grids, int prev_gpe,
                                 const cdc_grid* __restrict__ grids0, cdc_grid* out, cdc_grid* record) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_events * n_zoom) return;
    int e = t / n_zoom, c = t % n_zoom;
    uint64_t key = prev_keys[(size_t)e * CDC_MAX_K + c];
    cdc_grid g;
    float f = ldexpf(1.0f, -round);
    for (int a = 0; a < 5; ++a) {
        g.step[a] = grids0[e].step[a] * f;
        g.n[a] = key == KEY_NONE ? 0 : 3;
        g.centre[a] = 0.f;
    }
    if (key != KEY_NONE) event_seed(prev_grids, prev_gpe, e, (long long)(key & 0xffffffffull), g.centre);
    out[(size_t)e * CDC_MAX_ZOOM + c] = g;
    if (record) record[(size_t)e * n_zoom + c] = g;
}

__global__ void record_round0_kernel(int n_events, int n_zoom, const cdc_grid* grids0, cdc_grid* record) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_events * n_zoom) return;
    int e = t / n_zoom, c = t % n_zoom;
    cdc_grid g = grids0[e];
    if (c > 0)
        for (int a = 0; a < 5; ++a) g.n[a] = 0;
    record[(size_t)e * n_zoom + c] = g;
}

// Warp-per-seed scorer for rounds with few seeds (the zoom rounds of a few
// events): each warp takes one seed at a time from the global counter and its
// 32 lanes follow it together (warp_tracer.cuh), which shortens the round,
// bounded by its longest track, without changing any score.
template <int KIND>
__global__ void __launch_bounds__(128) scan_warp_kernel(DevGeom G, DevField F, ScanConst P, ScanIO io) {
    __shared__ DevLayer s_lay[CDC_MAX_LAYERS];
    __shared__ uchar2 s_tab[TAB_N];
    __shared__ WarpFound s_rec[4];
    for (int i = threadIdx.x; i < G.n_layers; i += blockDim.x) s_lay[i] = G.layers[i];
    for (int i = threadIdx.x; i < TAB_N; i += blockDim.x) s_tab[i] = G.tab[i];
    __syncthreads();
    const long long total = (long long)io.counters[1];
    const int lane = threadIdx.x & 31;
    WarpTracer<KIND> T;
    unsigned long long nsteps = 0;
    for (;;) {
        unsigned long long s = 0;
        if (lane == 0) s = atomicAdd(&io.counters[0], 1ull);
        s = __shfl_sync(FULL, s, 0);
        if ((long long)s >= total) break;
        const int ev = find_event(io.seed_off, io.n_events, (long long)s);
        float sd[5];
        event_seed(io.grids, io.gpe, ev, (long long)s - io.seed_off[ev], sd);
        T.init(G, F, P, s_lay, s_tab, io.drift_tab + (size_t)ev * event_stride(G.n_wires), &s_rec[threadIdx.x >> 5],
               sd);
        T.run(G, F, P, s_lay, s_tab);
        const float score = T.score(P, io.hit_off[ev + 1] - io.hit_off[ev]);
        if (lane == 0) {
            io.E[s] = score;
            if (T.flags) atomicOr(&io.flags[ev], T.flags);
            nsteps += (unsigned long long)T.n;
        }
        if (io.recs) {
            int slot = lane == 0 ? record_slot(io, ev, score) : -1;
            slot = __shfl_sync(FULL, slot, 0);
            if (slot >= 0) {
                SeedRecord& R = io.recs[(size_t)ev * REC_SLOTS + slot];
                const WarpFound* wr = &s_rec[threadIdx.x >> 5];
                if (lane == 0) {
                    R.round = io.round;
                    R.index = (int)((long long)s - io.seed_off[ev]);
                    R.nf = T.nf;
                }
                for (int i = lane; i < T.nf; i += 32) {
                    R.key[i] = wr->key[i];
                    R.r[i] = wr->r[i];
                }
            }
            __syncwarp();  // the record is read before the next seed overwrites it
        }
    }
    if (io.steps && lane == 0 && nsteps) atomicAdd(io.steps, nsteps);
}

// Hit classification of each event's best seed (sec. 2.2: hits with
// d^2 < lambda belong to the partition under investigation), one warp per
// event: from the record of scored wires the seed's zoom round kept
// (record_slot), else by following the seed again (warp_tracer.cuh); then the
// lanes classify the hits.
template <int KIND>
__global__ void __launch_bounds__(128) assign_kernel(DevGeom G, DevField F, ScanConst P, int n_events,
                                                     const float* __restrict__ drift_tab,
                                                     const int32_t* __restrict__ hit_off,
                                                     const int32_t* __restrict__ wire_id,
                                                     const float* __restrict__ best_seed, int K, int8_t* hit_part,
                                                     float* hit_res2, const uint64_t* __restrict__ best_keys,
                                                     const SeedRecord* __restrict__ recs,
                                                     const unsigned* __restrict__ rec_count) {
    __shared__ DevLayer s_lay[CDC_MAX_LAYERS];
    __shared__ uchar2 s_tab[TAB_N];
    __shared__ WarpFound s_rec[4];
    for (int i = threadIdx.x; i < G.n_layers; i += blockDim.x) s_lay[i] = G.layers[i];
    for (int i = threadIdx.x; i < TAB_N; i += blockDim.x) s_tab[i] = G.tab[i];
    __syncthreads();
    const int e = blockIdx.x * 4 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (e >= n_events) return;
    float sd[5];
    bool valid = true;
    for (int a = 0; a < 5; ++a) {
        sd[a] = best_seed[(size_t)e * K * 5 + a];
        valid &= (sd[a] == sd[a]);
    }
    const int h0 = hit_off[e], h1 = hit_off[e + 1];
    if (!valid) {
        for (int h = h0 + lane; h < h1; h += 32) {
            if (hit_part) hit_part[h] = -1;
            if (hit_res2) hit_res2[h] = P.lam;
        }
        return;
    }
    // the best seed came from a zoom round and its record was kept (record_slot):
    // the same scored wires as tracing it again
    if (recs) {
        const uint64_t bk = best_keys[(size_t)e * CDC_MAX_K];
        const int round = (int)((bk >> ROUND_SHIFT) & 0x1fu), index = (int)(bk & ((1ull << ROUND_SHIFT) - 1));
        const int n = min(rec_count[e], (unsigned)REC_SLOTS);
        int slot = -1;
        for (int b = 0; b < n; b += 32) {
            const int i = b + lane;
            const SeedRecord* R = recs + (size_t)e * REC_SLOTS + i;
            const unsigned m = __ballot_sync(0xffffffffu, i < n && R->round == round && R->index == index);
            if (m) {
                slot = b + __ffs(m) - 1;
                break;
            }
        }
        if (bk != KEY_NONE && round > 0 && slot >= 0) {
            const SeedRecord& R = recs[(size_t)e * REC_SLOTS + slot];
            for (int h = h0 + lane; h < h1; h += 32) {
                const int w = wire_id[h];
                int part;
                const float r2 = record_class(R.key, R.r, R.nf, w, P.lam, part);
                if (hit_part) hit_part[h] = (int8_t)part;
                if (hit_res2) hit_res2[h] = r2;
            }
            return;
        }
    }
    WarpFound* rec = &s_rec[threadIdx.x >> 5];
    WarpTracer<KIND> T;
    T.init(G, F, P, s_lay, s_tab, drift_tab + (size_t)e * event_stride(G.n_wires), rec, sd);
    T.run(G, F, P, s_lay, s_tab);
    for (int h = h0 + lane; h < h1; h += 32) {
        const int w = wire_id[h];
        int part;
        const float r2 = record_class(rec->key, rec->r, T.nf, w, P.lam, part);
        if (hit_part) hit_part[h] = (int8_t)part;
        if (hit_res2) hit_res2[h] = r2;
    }
}

// ------------------------------------------------- classification counts
// counts[e][truth + 1][class + 1] += 1 per hit (sec. 3.1, Eqs. 2-3).
__global__ void class_counts_kernel(int n_events, const int32_t* __restrict__ hit_off,
                                    const int8_t* __restrict__ hit_part, const int8_t* __restrict__ truth_part,
                                    int n_part, int32_t* counts) {
    const int total = hit_off[n_events];
    const int np1 = n_part + 1;
    for (int h = blockIdx.x * blockDim.x + threadIdx.x; h < total; h += gridDim.x * blockDim.x) {
        const int e = find_event_i32(hit_off, n_events, h);
        int t = truth_part[h], c = hit_part[h];
        t = (t < 0 || t >= n_part) ? 0 : t + 1;
        c = (c < 0 || c >= n_part) ? 0 : c + 1;
        atomicAdd(&counts[((size_t)e * np1 + t) * np1 + c], 1);
    }
}

// Eqs. 2-3 from the counts of n_sets events (one thread per partition j):
// eff[j] = C_{j->j} / C_j, pur[j] = C_{j->j} / sum_{i >= 0} C_{i->j}, counts
// summed over the events first (64-bit), NaN for a zero denominator.
__global__ void efficiency_purity_kernel(int n_sets, const int32_t* __restrict__ counts, int n_part, float* eff,
                                         float* pur) {
    const int np1 = n_part + 1;
    for (int k = threadIdx.x; k < n_part; k += blockDim.x) {
        long long diag = 0, row = 0, col = 0;
        for (int e = 0; e < n_sets; ++e) {
            const int32_t* C = counts + (size_t)e * np1 * np1;
            diag += C[(k + 1) * np1 + (k + 1)];
            for (int j = 0; j <= n_part; ++j) row += C[(k + 1) * np1 + j];
            for (int i = 1; i <= n_part; ++i) col += C[i * np1 + (k + 1)];
        }
        const float nan = __int_as_float(0x7fc00000);
        eff[k] = row ? (float)((double)diag / (double)row) : nan;
        pur[k] = col ? (float)((double)diag / (double)col) : nan;
    }
}

cudaError_t launch_efficiency_purity(int n_sets, const int32_t* counts, int n_part, float* eff, float* pur,
                                     cudaStream_t st) {
    efficiency_purity_kernel<<<1, 32, 0, st>>>(n_sets, counts, n_part, eff, pur);
    return cudaGetLastError();
}

// n_common[e] = hits of event e classified pa by one scan and pb by the other.
__global__ void common_hits_kernel(int n_events, const int32_t* __restrict__ hit_off,
                                   const int8_t* __restrict__ part_a, const int8_t* __restrict__ part_b, int pa,
                                   int pb, int32_t* n_common) {
    for (int e = blockIdx.x; e < n_events; e += gridDim.x) {
        int c = 0;
        for (int h = hit_off[e] + threadIdx.x; h < hit_off[e + 1]; h += blockDim.x)
            c += (part_a[h] == pa && part_b[h] == pb) ? 1 : 0;
        for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(FULL, c, o);
        __shared__ int s_c[8];
        if ((threadIdx.x & 31) == 0) s_c[threadIdx.x >> 5] = c;
        __syncthreads();
        if (threadIdx.x == 0) {
            int t = 0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s_c[w];
            n_common[e] = t;
        }
        __syncthreads();
    }
}

cudaError_t launch_common_hits(int n_events, const int32_t* hit_off, const int8_t* part_a, const int8_t* part_b,
                               int pa, int pb, int32_t* n_common, int num_sms, cudaStream_t st) {
    common_hits_kernel<<<std::min(n_events, num_sms * 8), 256, 0, st>>>(n_events, hit_off, part_a, part_b, pa, pb,
                                                                       n_common);
    return cudaGetLastError();
}

cudaError_t launch_class_counts(int n_events, const int32_t* hit_off, const int8_t* hit_part,
                                const int8_t* truth_part, int n_part, int32_t* counts, int num_sms, cudaStream_t st) {
    const size_t n = (size_t)n_events * (n_part + 1) * (n_part + 1);
    cudaError_t e = cudaMemsetAsync(counts, 0, n * sizeof(int32_t), st);
    if (e != cudaSuccess) return e;
    class_counts_kernel<<<num_sms * 2, 256, 0, st>>>(n_events, hit_off, hit_part, truth_part, n_part, counts);
    return cudaGetLastError();
}

// ------------------------------------------------- neighbouring turn (sec. 2.3)
// Seed of the previous (direction -1) or next (+1) turn from the seed of a
// turn: propagate (refine stepper) to the second change of side of the R0
// cylinder (starting inside for -1, outside for +1), interpolate the crossing
// linearly in rho between the two states, project it onto the cylinder and
// return the momentum along the forward motion.  FP64 for the interpolation.
template <int KIND>
__global__ void extrapolate_turn_kernel(DevGeom G, DevField F, ScanConst P, int n_seeds, const float* __restrict__ seeds,
                                        float* out, int32_t* status) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_seeds) return;
    const int direction = P.direction;
    float sd[5];
    for (int a = 0; a < 5; ++a) sd[a] = seeds[(size_t)i * 5 + a];
    State s;
    seed_state(sd, G.R0d, P.charge_dir, direction, s);
    const double p = sqrt((double)sd[2] * sd[2] + (double)sd[3] * sd[3] + (double)sd[4] * sd[4]);
    bool outside = direction > 0;
    int changes = 0, st = 2;
    for (int n = 0; n < P.max_steps; ++n) {
        const double x0 = (double)s.rx + s.lx, y0 = (double)s.ry + s.ly, z0 = (double)s.rz + s.lz;
        const double tx0 = (double)s.tx + s.mx, ty0 = (double)s.ty + s.my, tz0 = (double)s.tz + s.mz;
        rkn_step<KIND, true>(F, s, P.h, P.h6_lo);
        const double x1 = (double)s.rx + s.lx, y1 = (double)s.ry + s.ly, z1 = (double)s.rz + s.lz;
        const double rho0 = sqrt(x0 * x0 + y0 * y0), rho1 = sqrt(x1 * x1 + y1 * y1);
        const bool now_out = rho1 >= G.R0d;
        if (now_out != outside) {
            outside = now_out;
            if (++changes == 2) {
                const double w = (G.R0d - rho0) / (rho1 - rho0);
                const double qx = x0 + w * (x1 - x0), qy = y0 + w * (y1 - y0), qz = z0 + w * (z1 - z0);
                const double dx = tx0 + w * ((double)s.tx + s.mx - tx0), dy = ty0 + w * ((double)s.ty + s.my - ty0),
                             dz = tz0 + w * ((double)s.tz + s.mz - tz0);
                const double dn = sqrt(dx * dx + dy * dy + dz * dz), sign = direction < 0 ? -1.0 : 1.0;
                out[(size_t)i * 5 + 0] = (float)atan2(qy, qx);
                out[(size_t)i * 5 + 1] = (float)qz;
                out[(size_t)i * 5 + 2] = (float)(sign * p * dx / dn);
                out[(size_t)i * 5 + 3] = (float)(sign * p * dy / dn);
                out[(size_t)i * 5 + 4] = (float)(sign * p * dz / dn);
                st = 0;
                break;
            }
        }
        if (fabs(z1) > G.z_half || rho1 > G.R_out) {
            st = 1;
            break;
        }
    }
    if (st != 0)
        for (int a = 0; a < 5; ++a) out[(size_t)i * 5 + a] = __int_as_float(0x7fc00000);
    status[i] = st;
}

cudaError_t launch_extrapolate_turn(const DevGeom& G, const DevField& F, const ScanConst& P, int n_seeds,
                                    const float* seeds, float* out, int32_t* status, cudaStream_t st) {
    const int bs = 128, nb = (n_seeds + bs - 1) / bs;
    if (F.kind == 0)
        extrapolate_turn_kernel<0><<<nb, bs, 0, st>>>(G, F, P, n_seeds, seeds, out, status);
    else
        extrapolate_turn_kernel<1><<<nb, bs, 0, st>>>(G, F, P, n_seeds, seeds, out, status);
    return cudaGetLastError();
}

// ------------------------------------------------------------ propagation
template <int KIND, bool LAM2>
__global__ void propagate_kernel(DevGeom G, DevField F, ScanConst P, int n_seeds, const float* __restrict__ seeds,
                                 int every, int n_rec, double* pos, int32_t* n_steps, double* path) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_seeds) return;
    State s;
    seed_state(seeds + 5 * (size_t)i, G.R0d, P.charge_dir, P.direction, s);
    const double nan = __longlong_as_double(0x7ff8000000000000ll);
    for (int r = 0; r < n_rec; ++r)
        for (int a = 0; a < 3; ++a) pos[((size_t)i * n_rec + r) * 3 + a] = nan;
    int n = 0, part = 0;
    bool outside = true;
    float bx, by, bz;  // the scan stepper's field of the last end estimate
    field_eval<KIND>(F, s.rx, s.ry, s.rz, bx, by, bz);
    for (;;) {
        if (n >= P.max_steps) break;
        if (LAM2)
            rkn_step<KIND, true>(F, s, P.h, P.h6_lo);
        else
            rkn_step_fsal<KIND>(F, s, bx, by, bz, P.h, P.h6_lo);
        ++n;
        if (n % every == 0 && n / every <= n_rec) {
            double* o = pos + ((size_t)i * n_rec + (n / every - 1)) * 3;
            o[0] = (double)s.rx + (double)s.lx;
            o[1] = (double)s.ry + (double)s.ly;
            o[2] = (double)s.rz + (double)s.lz;
        }
        float rho = sqrtf(fmaf(s.rx, s.rx, s.ry * s.ry));
        bool now_out = rho >= G.R0;
        bool stop = false;
        if (outside && !now_out) {
            ++part;
            stop = part >= P.max_part;
        }
        outside = now_out;
        if (fabsf(s.rz) > G.z_half || rho > G.R_out) stop = true;
        if (stop) break;
    }
    n_steps[i] = n;
    path[i] = (double)n * (double)P.h;  // fixed step: the FP64 path length is the step count times h
}

// FP64 reference stepper on the GPU (precision sweep).
template <int KIND>
__device__ void field_eval_d(const DevField& F, double x, double y, double z, double& bx, double& by, double& bz) {
    if (KIND == 0) {
        bx = 0;
        by = 0;
        bz = F.B0;
        return;
    }
    double rho = sqrt(x * x + y * y);
    double rmax = F.r_min + F.dr * (F.nr - 1), zmax = F.z_min + F.dz * (F.nz - 1);
    double rc = fmin(fmax(rho, (double)F.r_min), rmax), zc = fmin(fmax(z, (double)F.z_min), zmax);
    double u = (rc - F.r_min) / F.dr, v = (zc - F.z_min) / F.dz;
    int i = min((int)u, F.nr - 2), j = min((int)v, F.nz - 2);
    u -= i;
    v -= j;
    const float4* c = F.cells + 2 * ((i + 1) * (F.nz + 1) + (j + 1));  // interior cell of the padded table
    float4 cz = c[0], cr = c[1];
    bz = (double)cz.x + (double)cz.y * u + (double)cz.z * v + (double)cz.w * u * v;
    double br = (double)cr.x + (double)cr.y * u + (double)cr.z * v + (double)cr.w * u * v;
    bx = rho > 0 ? br * x / rho : 0.0;
    by = rho > 0 ? br * y / rho : 0.0;
}

template <int KIND>
__global__ void propagate_fp64_kernel(DevGeom G, DevField F, ScanConst P, int n_seeds, const float* __restrict__ seeds,
                                      int every, int n_rec, double* pos, int32_t* n_steps, double* path) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_seeds) return;
    const float* sd = seeds + 5 * (size_t)i;
    double st, ct;
    sincos((double)sd[0], &st, &ct);
    double r[3] = {G.R0d * ct, G.R0d * st, (double)sd[1]};
    double p = sqrt((double)sd[2] * sd[2] + (double)sd[3] * sd[3] + (double)sd[4] * sd[4]);
    double ip = (P.direction < 0 ? -1.0 : 1.0) / p;
    double t[3] = {sd[2] * ip, sd[3] * ip, sd[4] * ip};
    double lam = (double)P.charge_dir * KAPPA_D / p, h = P.h;
    const double nan = __longlong_as_double(0x7ff8000000000000ll);
    for (int q = 0; q < n_rec; ++q)
        for (int a = 0; a < 3; ++a) pos[((size_t)i * n_rec + q) * 3 + a] = nan;
    int n = 0, part = 0;
    bool outside = true;
    for (;;) {
        if (n >= P.max_steps) break;
        double B[3], k1[3], k2[3], k3[3], k4[3], tt[3], pm[3];
        field_eval_d<KIND>(F, r[0], r[1], r[2], B[0], B[1], B[2]);
        k1[0] = lam * (t[1] * B[2] - t[2] * B[1]);
        k1[1] = lam * (t[2] * B[0] - t[0] * B[2]);
        k1[2] = lam * (t[0] * B[1] - t[1] * B[0]);
        for (int a = 0; a < 3; ++a) {
            pm[a] = r[a] + 0.5 * h * t[a] + h * h / 8.0 * k1[a];
            tt[a] = t[a] + 0.5 * h * k1[a];
        }
        field_eval_d<KIND>(F, pm[0], pm[1], pm[2], B[0], B[1], B[2]);
        k2[0] = lam * (tt[1] * B[2] - tt[2] * B[1]);
        k2[1] = lam * (tt[2] * B[0] - tt[0] * B[2]);
        k2[2] = lam * (tt[0] * B[1] - tt[1] * B[0]);
        for (int a = 0; a < 3; ++a) tt[a] = t[a] + 0.5 * h * k2[a];
        k3[0] = lam * (tt[1] * B[2] - tt[2] * B[1]);
        k3[1] = lam * (tt[2] * B[0] - tt[0] * B[2]);
        k3[2] = lam * (tt[0] * B[1] - tt[1] * B[0]);
        for (int a = 0; a < 3; ++a) {
            pm[a] = r[a] + h * t[a] + 0.5 * h * h * k3[a];
            tt[a] = t[a] + h * k3[a];
        }
        field_eval_d<KIND>(F, pm[0], pm[1], pm[2], B[0], B[1], B[2]);
        k4[0] = lam * (tt[1] * B[2] - tt[2] * B[1]);
        k4[1] = lam * (tt[2] * B[0] - tt[0] * B[2]);
        k4[2] = lam * (tt[0] * B[1] - tt[1] * B[0]);
        for (int a = 0; a < 3; ++a) {
            r[a] += h * t[a] + h * h / 6.0 * (k1[a] + k2[a] + k3[a]);
            t[a] += h / 6.0 * (k1[a] + 2.0 * k2[a] + 2.0 * k3[a] + k4[a]);
        }
        ++n;
        if (n % every == 0 && n / every <= n_rec) {
            double* o = pos + ((size_t)i * n_rec + (n / every - 1)) * 3;
            o[0] = r[0];
            o[1] = r[1];
            o[2] = r[2];
        }
        double rho = sqrt(r[0] * r[0] + r[1] * r[1]);
        bool now_out = rho >= G.R0d;
        bool stop = false;
        if (outside && !now_out) {
            ++part;
            stop = part >= P.max_part;
        }
        outside = now_out;
        if (fabs(r[2]) > (double)G.z_half || rho > (double)G.R_out) stop = true;
        if (stop) break;
    }
    n_steps[i] = n;
    path[i] = (double)n * h;
}

// ----------------------------------------------------------- launchers
static int blocks_for(long long n, int bs) { return (int)((n + bs - 1) / bs); }

// A timer mark on stream st: recorded at once, or, while st is being captured
// into a CUDA graph, as an event-record node that every replay of the graph
// records again.
static void timer_mark(cudaEvent_t ev, cudaStream_t st) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusActive)
        cudaEventRecordWithFlags(ev, st, cudaEventRecordExternal);
    else
        cudaEventRecord(ev, st);
}

using ScanKernel = void (*)(DevGeom, DevField, ScanConst, ScanIO);

template <int KIND>
static ScanKernel scan_kernel_of(int block, int chunk) {
    if (block == 128) return chunk == 32 ? scan_kernel<KIND, 128, 32> : scan_kernel<KIND, 128, 16>;
    return chunk == 32 ? scan_kernel<KIND, 256, 32> : scan_kernel<KIND, 256, 16>;
}

cudaError_t launch_seed_offsets(int n_events, const cdc_grid* grids, int gpe, const Workspace& W, uint32_t* flags,
                                cudaStream_t st) {
    prologue_kernel<<<1, 1024, 0, st>>>(n_events, grids, gpe, W.e_cap, W.seg_cap, W.seed_off, W.seg_off, W.counters,
                                        flags);
    return cudaGetLastError();
}

cudaError_t launch_scan(const DevGeom& G, const DevField& F, const ScanConst& P, const Workspace& W,
                        const ScanLaunch& L, int num_sms, cudaStream_t st) {
    cudaError_t err;
    const int ne = L.n_events;
    // stage the event hits into per-event hit tables
    if ((err = launch_stage(G, ne, L.hit_off, L.wire_id, L.drift, P.max_drift, W.drift_tab, L.flags, num_sms, st)) !=
        cudaSuccess)
        return err;
    const int bs = L.block == 128 ? 128 : 256;
    const ScanKernel kern = F.kind == 0 ? scan_kernel_of<0>(bs, L.chunk) : scan_kernel_of<1>(bs, L.chunk);
    const size_t lay_smem = sizeof(DevLayer) * (size_t)G.n_layers;
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, bs, lay_smem);
    const int scan_blocks = num_sms * (occ > 0 ? occ : 1);
    if (W.rec_count && L.n_rounds > 1 && (L.hit_part || L.hit_res2) &&
        (err = cudaMemsetAsync(W.rec_count, 0, sizeof(unsigned) * ne, st)) != cudaSuccess)
        return err;
    for (int r = 0; r < L.n_rounds; ++r) {
        const cdc_grid* grids = r == 0 ? L.grids0 : W.zgrids + (size_t)(r & 1) * W.max_events * CDC_MAX_ZOOM;
        const int gpe = r == 0 ? 1 : CDC_MAX_ZOOM;
        if (r > 0) {
            const cdc_grid* pg = r == 1 ? L.grids0 : W.zgrids + (size_t)((r - 1) & 1) * W.max_events * CDC_MAX_ZOOM;
            const int pgpe = r == 1 ? 1 : CDC_MAX_ZOOM;
            const uint64_t* pk = W.round_keys + (size_t)((r - 1) & 1) * W.max_events * CDC_MAX_K;
            cdc_grid* out = const_cast<cdc_grid*>(grids);
            // slots beyond n_zoom stay empty grids
            cudaMemsetAsync(out, 0, sizeof(cdc_grid) * (size_t)ne * CDC_MAX_ZOOM, st);
            zoom_grid_kernel<<<blocks_for((long long)ne * L.n_zoom, 128), 128, 0, st>>>(
                ne, L.n_zoom, r, pk, pg, pgpe, L.grids0, out,
                L.zoom_grids ? L.zoom_grids + (size_t)r * ne * L.n_zoom : nullptr);
        } else if (L.zoom_grids) {
            record_round0_kernel<<<blocks_for((long long)ne * L.n_zoom, 128), 128, 0, st>>>(ne, L.n_zoom, L.grids0,
                                                                                           L.zoom_grids);
        }
        float* E = (r == 0 && L.E0) ? L.E0 : W.E;
        long long cap = (r == 0 && L.E0) ? (1ll << 62) : W.e_cap;
        if (r == 0 && L.e0_cap >= 0) cap = std::min(cap, L.e0_cap);
        prologue_kernel<<<1, 1024, 0, st>>>(ne, grids, gpe, cap, W.seg_cap, W.seed_off, W.seg_off, W.counters,
                                            L.flags);
        if (r == 0 && W.perm)
            order_blocks_kernel<<<ne, 1024, 0, st>>>(ne, grids, G.z_half, P.b_max, P.max_part, P.direction, W.perm);
        const bool rec = r > 0 && W.recs && (L.hit_part || L.hit_res2);
        ScanIO io{W.drift_tab, L.hit_off, grids, gpe, W.seed_off, ne, W.counters, E, L.flags,
                  L.steps ? L.steps + r : nullptr, r == 0 ? W.perm : nullptr, rec ? W.recs : nullptr,
                  W.rec_count, W.run_best, r};
        const bool timed = L.timer.ev && *L.timer.used + 2 <= L.timer.cap;
        if (timed) timer_mark(L.timer.ev[*L.timer.used], st);
        // a round of few seeds (host bound: zoom grids of 3^5 seeds) runs one warp per seed
        const long long round_seeds = (long long)ne * L.n_zoom * ZOOM_GRID;
        if (r > 0 && round_seeds <= L.warp_seeds) {
            const int nb = (int)std::min<long long>((round_seeds + 3) / 4, (long long)num_sms * 16);
            if (F.kind == 0)
                scan_warp_kernel<0><<<nb, 128, 0, st>>>(G, F, P, io);
            else
                scan_warp_kernel<1><<<nb, 128, 0, st>>>(G, F, P, io);
        } else {
            // a zoom round has at most round_seeds seeds: one block per 32 of them (one
            // cohort each, spread over SMs) instead of the full persistent grid, whose idle
            // blocks would only contend for SM slots with other streams' work
            const int nb = r == 0 ? scan_blocks
                                  : (int)std::min<long long>(scan_blocks, std::max<long long>(1, (round_seeds + 31) / 32));
            kern<<<nb, bs, lay_smem, st>>>(G, F, P, io);
        }
        if (timed) {
            timer_mark(L.timer.ev[*L.timer.used + 1], st);
            *L.timer.used += 2;
        }
        // one warp per 4096-seed segment; a zoom round has at most round_seeds / SEG + ne segments
        const int tb = r == 0 ? num_sms * 2
                              : (int)std::min<long long>(num_sms * 2, (round_seeds / SEG + ne + 7) / 8);
        topk_partial_kernel<<<tb, 256, 0, st>>>(E, W.seed_off, W.seg_off, ne, W.counters, P.k, W.seg_keys);
        uint64_t* rk = W.round_keys + (size_t)(r & 1) * W.max_events * CDC_MAX_K;
        topk_merge_kernel<<<blocks_for((long long)ne * 32, 256), 256, 0, st>>>(W.seg_off, ne, P.k, W.seg_keys, rk);
        merge_best_kernel<<<blocks_for(ne, 64), 64, 0, st>>>(ne, P.k, r, rk, grids, gpe, W.best_keys, L.best_E,
                                                             L.best_seed, L.topk0, W.run_best);
        if ((err = cudaGetLastError()) != cudaSuccess) return err;
    }
    if (L.hit_part || L.hit_res2) {
        const SeedRecord* recs = L.n_rounds > 1 ? W.recs : nullptr;
        if (F.kind == 0)
            assign_kernel<0><<<blocks_for(ne, 4), 128, 0, st>>>(G, F, P, ne, W.drift_tab, L.hit_off, L.wire_id,
                                                                L.best_seed, P.k, L.hit_part, L.hit_res2,
                                                                W.best_keys, recs, W.rec_count);
        else
            assign_kernel<1><<<blocks_for(ne, 4), 128, 0, st>>>(G, F, P, ne, W.drift_tab, L.hit_off, L.wire_id,
                                                                L.best_seed, P.k, L.hit_part, L.hit_res2,
                                                                W.best_keys, recs, W.rec_count);
    }
    return cudaGetLastError();
}

cudaError_t launch_propagate(const DevGeom& G, const DevField& F, const ScanConst& P, int n_seeds,
                             const float* seeds, int every, int n_rec, int precision, double* pos, int32_t* n_steps,
                             double* path, cudaStream_t st) {
    const int bs = 128, nb = blocks_for(n_seeds, bs);
    if (precision == 0) {
        if (F.kind == 0)
            propagate_kernel<0, false><<<nb, bs, 0, st>>>(G, F, P, n_seeds, seeds, every, n_rec, pos, n_steps, path);
        else
            propagate_kernel<1, false><<<nb, bs, 0, st>>>(G, F, P, n_seeds, seeds, every, n_rec, pos, n_steps, path);
    } else if (precision == 2) {
        if (F.kind == 0)
            propagate_kernel<0, true><<<nb, bs, 0, st>>>(G, F, P, n_seeds, seeds, every, n_rec, pos, n_steps, path);
        else
            propagate_kernel<1, true><<<nb, bs, 0, st>>>(G, F, P, n_seeds, seeds, every, n_rec, pos, n_steps, path);
    } else {
        if (F.kind == 0)
            propagate_fp64_kernel<0><<<nb, bs, 0, st>>>(G, F, P, n_seeds, seeds, every, n_rec, pos, n_steps, path);
        else
            propagate_fp64_kernel<1><<<nb, bs, 0, st>>>(G, F, P, n_seeds, seeds, every, n_rec, pos, n_steps, path);
    }
    return cudaGetLastError();
}

}  // namespace cdc
