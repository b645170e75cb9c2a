// Host-side declarations shared by the C-ABI layer and the kernel launchers.
#pragma once

#include <cuda_runtime.h>

#include "cdc_dev.cuh"

namespace cdc {

// Device workspace owned by a context, sized by cdc_reserve.
// Hough peak search: each event's accumulator is searched in HOUGH_SLICES
// slices, each keeping its HOUGH_SLICE_KEYS (>= max_cand) best peaks.
constexpr int HOUGH_SLICES = 64;
constexpr int HOUGH_SLICE_KEYS = 64;

struct Workspace {
    float* drift_tab = nullptr;            // [max_events][event_stride(n_wires)]: drifts, then fired-wire bits
    float* E = nullptr;                    // [e_cap] scores of the current round
    long long* seed_off = nullptr;         // [max_events + 1]
    int* seg_off = nullptr;                // [max_events + 1]
    unsigned long long* counters = nullptr;// [4]: work counter, total seeds, total segments, spare
    uint64_t* seg_keys = nullptr;          // [seg_cap][CDC_MAX_K]
    uint64_t* round_keys = nullptr;        // [2][max_events][CDC_MAX_K]
    uint64_t* best_keys = nullptr;         // [max_events][CDC_MAX_K]
    cdc_grid* zgrids = nullptr;            // [2][max_events][CDC_MAX_ZOOM]
    uint16_t* perm = nullptr;              // [max_events][PERM_CAP]: coarse-grid block order (nullptr: natural)
    SeedRecord* recs = nullptr;            // [max_events][REC_SLOTS]: records of improving zoom-round seeds
    unsigned* rec_count = nullptr;         // [max_events]: records claimed in this call
    unsigned* run_best = nullptr;          // [max_events]: the event's best score so far (float bits)
    int32_t* hough_max = nullptr;          // [max_events]: the Hough accumulator's maximum
    uint64_t* hough_keys = nullptr;        // [max_events][HOUGH_SLICES][HOUGH_SLICE_KEYS]: peaks of each slice
    int max_events = 0;
    long long e_cap = 0, seg_cap = 0;
    int n_wires = 0;
};

// Optional CUDA-event pairs recorded around each scan-kernel launch.
struct KernelTimer {
    cudaEvent_t* ev = nullptr;  // [cap]: start, end, start, end, ...
    int cap = 0;
    int* used = nullptr;
};

struct ScanLaunch {
    int n_events;
    const int32_t* hit_off;
    const int32_t* wire_id;
    const float* drift;
    const cdc_grid* grids0;   // caller's coarse grids, one per event
    float* E0;                // caller's coarse-round E output or nullptr
    uint64_t* topk0;
    float* best_E;
    float* best_seed;
    int8_t* hit_part;
    float* hit_res2;
    cdc_grid* zoom_grids;
    uint32_t* flags;
    unsigned long long* steps;
    int n_rounds, n_zoom;
    KernelTimer timer;
    int block = 256, chunk = 16;  // scan-kernel launch shape (cdc_scan_config)
    long long warp_seeds = 0;     // zoom rounds of at most this many seeds run one warp per seed
    long long e0_cap = -1;        // >= 0: most seeds the coarse round may hold (E0 and workspace sized for it)
};

// Kernel launchers (scan.cu).  Return cudaSuccess or the launch error.

// Seed offsets of every event (W.seed_off), the seed total and a reset work
// counter (W.counters) for grids with gpe grids per event.
cudaError_t launch_seed_offsets(int n_events, const cdc_grid* grids, int gpe, const Workspace& W, uint32_t* flags,
                                cudaStream_t st);

// Fills the per-event hit tables of n_events events from the CSR hit lists;
// flags (nullable) receives CDC_FLAG_BAD_HIT for invalid or duplicate hits.
cudaError_t launch_stage(const DevGeom& G, int n_events, const int32_t* hit_off, const int32_t* wire_id,
                         const float* drift, float max_drift, float* tab, uint32_t* flags, int num_sms,
                         cudaStream_t st);
cudaError_t launch_scan(const DevGeom& G, const DevField& F, const ScanConst& P, const Workspace& W,
                        const ScanLaunch& L, int num_sms, cudaStream_t st);

cudaError_t launch_common_hits(int n_events, const int32_t* hit_off, const int8_t* part_a, const int8_t* part_b,
                               int pa, int pb, int32_t* n_common, int num_sms, cudaStream_t st);

cudaError_t launch_extrapolate_turn(const DevGeom& G, const DevField& F, const ScanConst& P, int n_seeds,
                                    const float* seeds, float* out, int32_t* status, cudaStream_t st);

cudaError_t launch_class_counts(int n_events, const int32_t* hit_off, const int8_t* hit_part,
                                const int8_t* truth_part, int n_part, int32_t* counts, int num_sms, cudaStream_t st);
cudaError_t launch_efficiency_purity(int n_sets, const int32_t* counts, int n_part, float* eff, float* pur,
                                     cudaStream_t st);

cudaError_t launch_propagate(const DevGeom& G, const DevField& F, const ScanConst& P, int n_seeds,
                             const float* seeds, int every, int n_rec, int precision, double* pos, int32_t* n_steps,
                             double* path, cudaStream_t st);

// The paper's two-kernel scan (split.cu): record states, then DOCA per hit.
struct SplitLaunch {
    int n_events;
    const int32_t* hit_off;
    const int32_t* wire_id;
    const float* drift;
    const cdc_grid* grids;  // one per event
    long long n_seeds;      // the grids' total
    int chunk;              // seeds recorded at a time
    int block;              // threads per seed block of the DOCA kernel
    Workspace W;
    uint32_t* flags;
    float* E;
    float4* rec_r;          // [chunk][max_steps + 1]
    float4* rec_t;
    int* n_rec;             // [chunk]
    int8_t* end_ok;         // [chunk]
};
cudaError_t launch_split(const DevGeom& G, const DevField& F, const ScanConst& P, const SplitLaunch& L,
                         cudaStream_t st);

// Hough (hough.cu).
struct HoughLaunch {
    int n_events;
    const int32_t* hit_off;
    const int32_t* wire_id;
    const int2* offsets;       // [n_r * n_phi] integer (dx, dy) of each vote [um]
    int32_t* acc;
    cdc_candidate* cand;
    int32_t* n_cand;
    cdc_grid* grid_out;
    uint32_t* flags;
    int32_t* emax;             // [n_events] scratch: accumulator maxima
    uint64_t* keys;            // [n_events][HOUGH_SLICES][HOUGH_SLICE_KEYS] scratch
};
cudaError_t launch_hough(const DevGeom& G, const cdc_hough_params& H, const HoughLaunch& L, cudaStream_t st);
cudaError_t launch_candidate_grids(int n_events, const cdc_hough_params& H, const cdc_candidate* cand,
                                   const int32_t* n_cand, cdc_grid* grids, cudaStream_t st);

// Refine (refine.cu).
struct RefineLaunch {
    int n_seeds;
    const int32_t* seed_event;
    const float* seeds;
    int n_events;
    const int32_t* hit_off;
    const int32_t* wire_id;
    const float* drift;
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
cudaError_t launch_refine(const DevGeom& G, const DevField& F, const ScanConst& P, const RefineLaunch& L,
                          float* drift_tab, int num_sms, int do_gn, cudaStream_t st);

// FP32 FMA throughput measurement (peak.cu): one launch filling every SM;
// fma_count = FMAs it executes.  sink: device float[grid] (written never).
cudaError_t launch_ffma(int num_sms, int iters, float* sink, cudaStream_t st, double* fma_count);

}  // namespace cdc
