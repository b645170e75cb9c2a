// The paper's two-kernel organisation of the scan (arXiv:1908.01949 sec. 4.2:
// propagation and distance search in separate kernels), kept as an A/B
// reference for the fused scan:
//   A. one thread per seed propagates the seed to the end of its track and
//      records the state after every RKN step;
//   B. one block per seed and one thread per hit of the event (the paper's
//      block-per-seed, thread-per-wire layout, sec. 2.2) find each wire's
//      distance of closest approach from the recorded states.
// B takes the same minima as the fused scan (sign changes of the distance
// slope g between recorded states, refined on the cubic Hermite segment; the
// track start and end) and sums Eq. 1 per seed, so both produce the same
// scores.  The per-seed states live in global memory between the kernels and
// in shared memory while B reads them.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "cdc_dev.cuh"
#include "cdc_host.h"
#include "tracer.cuh"

namespace cdc {

namespace {
constexpr unsigned FULL_MASK = 0xffffffffu;
}

// A: states of seeds [s0, s0 + n) (global seed indices in row-major order):
// rec_r[i * stride + j] = (x, y, z, partition), rec_t[...] = (tx, ty, tz, 0) after
// step j (j = 0: the seed), n_rec[i] = steps taken, end_ok[i] = 1 + the
// partition of the end point if the track did not end at the partition limit
// (its end may then be a minimum), else 0.
template <int KIND>
__global__ void __launch_bounds__(128) record_kernel(DevGeom G, DevField F, ScanConst P, const cdc_grid* grids,
                                                     const long long* seed_off, const unsigned long long* counters,
                                                     int n_events, long long s0, int n, int stride, float4* rec_r,
                                                     float4* rec_t, int* n_rec, int8_t* end_ok) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const long long s = s0 + i;
    if (s >= (long long)counters[1]) {  // beyond the grids' seeds: nothing to score
        n_rec[i] = -1;
        return;
    }
    const int ev = find_event(seed_off, n_events, s);
    float sd[5];
    event_seed(grids, 1, ev, s - seed_off[ev], sd);
    State st;
    seed_state(sd, G.R0d, P.charge_dir, P.direction, st);
    float4* rr = rec_r + (size_t)i * stride;
    float4* rt = rec_t + (size_t)i * stride;
    int part = 0, k = 0;
    bool outside = true, stop = false;
    rr[0] = make_float4(st.rx, st.ry, st.rz, __int_as_float(0));
    rt[0] = make_float4(st.tx, st.ty, st.tz, 0.f);
    float bx, by, bz;  // field of the last end estimate (the scan's stepper)
    field_eval<KIND>(F, st.rx, st.ry, st.rz, bx, by, bz);
    while (!stop) {
        rkn_step_fsal<KIND>(F, st, bx, by, bz, P.h, P.h6_lo);
        ++k;
        const float rho = rho_of(st.rx, st.ry);
        const bool now_out = rho >= G.R0;
        const int pt = part;  // a segment belongs to the partition at its start
        if (outside && !now_out) {
            ++part;
            if (part >= P.max_part) stop = true;
        }
        outside = now_out;
        if (fabsf(st.rz) > G.z_half || rho > G.R_out) stop = true;
        if (!stop && k >= P.max_steps) stop = true;
        rr[k] = make_float4(st.rx, st.ry, st.rz, __int_as_float(pt));
        rt[k] = make_float4(st.tx, st.ty, st.tz, 0.f);
    }
    n_rec[i] = k;
    end_ok[i] = part < P.max_part ? (int8_t)(part + 1) : (int8_t)0;
}

// B: Eq. 1 of seed i = one block; the recorded states are staged in shared
// memory, then every thread takes hits of the seed's event: per turn partition
// the DCA of the hit's wire is the smallest distance over the partition's
// minima, and the hit's term is the smallest min((DCA - drift)^2, lambda) over
// the partitions (minima come in track order, so a partition's DCA is final
// once a later partition's minimum appears).
template <int KIND>
__global__ void split_doca_kernel(DevGeom G, ScanConst P, const long long* seed_off, int n_events, long long s0,
                                  int stride, const float4* __restrict__ rec_r, const float4* __restrict__ rec_t,
                                  const int* __restrict__ n_rec, const int8_t* __restrict__ end_ok,
                                  const int32_t* __restrict__ hit_off, const int32_t* __restrict__ wire_id,
                                  const float* __restrict__ drift, float* E) {
    extern __shared__ float4 s_mem[];
    __shared__ DevLayer s_lay[CDC_MAX_LAYERS];
    __shared__ float s_part[32];
    const int i = blockIdx.x;
    const long long s = s0 + i;
    const int n = n_rec[i];
    if (n < 0) return;
    const int ev = find_event(seed_off, n_events, s);
    float4* sr = s_mem;
    float4* stt = s_mem + stride;
    for (int j = threadIdx.x; j <= n; j += blockDim.x) {
        sr[j] = rec_r[(size_t)i * stride + j];
        stt[j] = rec_t[(size_t)i * stride + j];
    }
    for (int l = threadIdx.x; l < G.n_layers; l += blockDim.x) s_lay[l] = G.layers[l];
    __syncthreads();
    const int end_part = (int)end_ok[i] - 1;  // -1: the end is no minimum
    float acc = 0.f;
    for (int h = hit_off[ev] + threadIdx.x; h < hit_off[ev + 1]; h += blockDim.x) {
        const int w = wire_id[h];
        const float d = drift[h];
        if (w < 0 || w >= G.n_wires || !(d >= 0.f && d <= P.max_drift)) {
            acc += P.lam;
            continue;
        }
        int a = 0, b = G.n_layers - 1;  // layer of the wire
        while (a < b) {
            const int mid = (a + b + 1) >> 1;
            if (s_lay[mid].base <= w) a = mid; else b = mid - 1;
        }
        const float cosa = s_lay[a].cosa;
        const float4 W = __ldg(G.wires + w);
        float best = P.lam, dmin = INFINITY, tp2;  // best term of the finished partitions; DCA of partition cp
        int cp = 0;
        auto minimum = [&](int k, float D) {
            if (k != cp) {
                const float r = dmin - d;
                best = fminf(best, fminf(r * r, P.lam));
                cp = k;
                dmin = D;
            } else {
                dmin = fminf(dmin, D);
            }
        };
        float4 r0 = sr[0], t0 = stt[0];
        float g0 = dist_slope(r0.x, r0.y, r0.z, t0.x, t0.y, t0.z, W, cosa, tp2);
        // the start of the track: a minimum if the distance grows from there
        if (g0 > 0.f) minimum(0, point_doca(r0.x, r0.y, r0.z, W, cosa));
        for (int j = 1; j <= n; ++j) {
            const float4 r1 = sr[j], t1 = stt[j];
            const float g1 = dist_slope(r1.x, r1.y, r1.z, t1.x, t1.y, t1.z, W, cosa, tp2);
            if (g0 < 0.f && g1 >= 0.f)  // a segment belongs to the partition at its start
                minimum(__float_as_int(r1.w), seg_doca(r0.x - W.x, r0.y - W.y, r0.z, t0.x, t0.y, t0.z, r1.x - r0.x,
                                                       r1.y - r0.y, r1.z - r0.z, t1.x, t1.y, t1.z, W, cosa, g0, g1,
                                                       P.h));
            r0 = r1;
            t0 = t1;
            g0 = g1;
        }
        // the end of the track, still approaching
        if (end_part >= 0 && g0 < 0.f) minimum(end_part, point_doca(r0.x, r0.y, r0.z, W, cosa));
        const float r = dmin - d;
        acc += fminf(best, fminf(r * r, P.lam));
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(FULL_MASK, acc, o);
    if ((threadIdx.x & 31) == 0) s_part[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += s_part[q];
        E[s] = t;
    }
}

cudaError_t launch_split(const DevGeom& G, const DevField& F, const ScanConst& P, const SplitLaunch& L,
                         cudaStream_t st) {
    cudaError_t err;
    if ((err = launch_seed_offsets(L.n_events, L.grids, 1, L.W, L.flags, st)) != cudaSuccess) return err;
    const int stride = P.max_steps + 1;
    const size_t smem = (size_t)2 * stride * sizeof(float4);
    if (F.kind == 0)
        err = cudaFuncSetAttribute(split_doca_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    else
        err = cudaFuncSetAttribute(split_doca_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    for (long long s0 = 0; s0 < L.n_seeds; s0 += L.chunk) {
        const int n = (int)std::min<long long>(L.chunk, L.n_seeds - s0);
        if (F.kind == 0)
            record_kernel<0><<<(n + 127) / 128, 128, 0, st>>>(G, F, P, L.grids, L.W.seed_off, L.W.counters,
                                                              L.n_events, s0, n, stride, L.rec_r, L.rec_t, L.n_rec,
                                                              L.end_ok);
        else
            record_kernel<1><<<(n + 127) / 128, 128, 0, st>>>(G, F, P, L.grids, L.W.seed_off, L.W.counters,
                                                              L.n_events, s0, n, stride, L.rec_r, L.rec_t, L.n_rec,
                                                              L.end_ok);
        if (F.kind == 0)
            split_doca_kernel<0><<<n, L.block, smem, st>>>(G, P, L.W.seed_off, L.n_events, s0, stride, L.rec_r,
                                                           L.rec_t, L.n_rec, L.end_ok, L.hit_off, L.wire_id, L.drift,
                                                           L.E);
        else
            split_doca_kernel<1><<<n, L.block, smem, st>>>(G, P, L.W.seed_off, L.n_events, s0, stride, L.rec_r,
                                                           L.rec_t, L.n_rec, L.end_ok, L.hit_off, L.wire_id, L.drift,
                                                           L.E);
        if ((err = cudaGetLastError()) != cudaSuccess) return err;
    }
    return cudaSuccess;
}

}  // namespace cdc
