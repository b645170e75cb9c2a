// Seed scan that allocates no device memory.
//
// Some callers cannot call cudaMalloc: code running inside a memory pool or an
// allocator callback that must not re-enter the allocator, processes whose
// device memory is fully handed to another framework's caching allocator, and
// real-time paths that forbid allocation after start-up.  For them this entry
// point runs the same single-round scan as cdc_scan_seeds, but its workspace
// (per-event drift tables, scores, offsets, top-K keys) lives in one
// file-scope __device__ array of fixed size instead of the context's
// cdc_reserve buffers.  Only the caller's inputs and outputs are touched
// otherwise; the array exists on every device that loads the library, for the
// life of the process.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "../../include/cdc.h"
#include "cdc_host.h"

namespace cdc {
int scan_view(cdc_ctx* c, const cdc_scan_params* p, DevGeom* G, DevField* F, ScanConst* P, int* num_sms,
              int* device, int* block, int* chunk);
int set_error(cdc_ctx* c, int code, const char* msg);
}  // namespace cdc

namespace {

using namespace cdc;

constexpr size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

constexpr long long NA_SEG_CAP = CDC_NOALLOC_MAX_SEEDS / SEG + CDC_NOALLOC_MAX_EVENTS + 1;
constexpr size_t OFF_DRIFT = 0;
constexpr size_t OFF_E = OFF_DRIFT + align256(sizeof(float) * CDC_NOALLOC_MAX_EVENTS * (CDC_MAX_WIRES + FIRED_WORDS));
constexpr size_t OFF_SEEDOFF = OFF_E + align256(sizeof(float) * CDC_NOALLOC_MAX_SEEDS);
constexpr size_t OFF_SEGOFF = OFF_SEEDOFF + align256(sizeof(long long) * (CDC_NOALLOC_MAX_EVENTS + 1));
constexpr size_t OFF_COUNT = OFF_SEGOFF + align256(sizeof(int) * (CDC_NOALLOC_MAX_EVENTS + 1));
constexpr size_t OFF_SEGK = OFF_COUNT + align256(sizeof(unsigned long long) * 4);
constexpr size_t OFF_ROUNDK = OFF_SEGK + align256(sizeof(uint64_t) * NA_SEG_CAP * CDC_MAX_K);
constexpr size_t OFF_BESTK = OFF_ROUNDK + align256(sizeof(uint64_t) * 2 * CDC_NOALLOC_MAX_EVENTS * CDC_MAX_K);
constexpr size_t OFF_ZGRID = OFF_BESTK + align256(sizeof(uint64_t) * CDC_NOALLOC_MAX_EVENTS * CDC_MAX_K);
constexpr size_t SCRATCH_BYTES = OFF_ZGRID + align256(sizeof(cdc_grid) * 2 * CDC_NOALLOC_MAX_EVENTS * CDC_MAX_ZOOM);

// The workspace.  In host code the name below is only a handle for the
// runtime, not a device address: the address is looked up per device with
// cudaGetSymbolAddress.  Every call shares it and it keeps the previous call's
// contents; the scan's own kernels initialise every part they read (drift
// tables, offsets, counters, keys), so nothing is cleared here.
static __device__ __align__(256) unsigned char g_scratch[SCRATCH_BYTES];

constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
void* g_addr[MAX_DEVICES] = {};

// Device address of g_scratch on `device`, looked up on the first call for
// that device (the device must be current).
cudaError_t scratch_address(int device, void** out) {
    if (device < 0 || device >= MAX_DEVICES) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[device]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess) return e;
        g_addr[device] = p;
    }
    *out = g_addr[device];
    return cudaSuccess;
}

struct CurrentDevice {
    int prev = -1;
    bool ok = true;
    explicit CurrentDevice(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~CurrentDevice() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

}  // namespace

extern "C" int cdc_scan_seeds_noalloc(cdc_ctx* c, int n_events, int64_t n_seeds, const int32_t* hit_off,
                                      const int32_t* wire_id, const float* drift, const cdc_grid* grids,
                                      const cdc_scan_params* p, float* E, uint64_t* topk0, float* best_E,
                                      float* best_seed, int8_t* hit_part, float* hit_res2, uint32_t* flags,
                                      unsigned long long* steps, void* stream) {
    if (!c) return CDC_ERR_ARG;
    if (n_events < 0 || n_seeds < 0) return set_error(c, CDC_ERR_ARG, "n_events and n_seeds must be >= 0");
    if (n_events > CDC_NOALLOC_MAX_EVENTS)
        return set_error(c, CDC_ERR_RANGE, "cdc_scan_seeds_noalloc: more than CDC_NOALLOC_MAX_EVENTS (8) events");
    if (n_seeds > CDC_NOALLOC_MAX_SEEDS)
        return set_error(c, CDC_ERR_RANGE, "cdc_scan_seeds_noalloc: more than CDC_NOALLOC_MAX_SEEDS (65536) seeds");
    if (!p) return set_error(c, CDC_ERR_ARG, "scan params is NULL");
    if (p->n_rounds != 1)
        return set_error(c, CDC_ERR_RANGE, "cdc_scan_seeds_noalloc: only the single-round scan (n_rounds = 1)");
    DevGeom G;
    DevField F;
    ScanConst P;
    int sms = 1, dev = 0, block = 256, chunk = 16;
    int rc = scan_view(c, p, &G, &F, &P, &sms, &dev, &block, &chunk);
    if (rc) return rc;
    if (n_events == 0) return CDC_OK;
    if (!hit_off || !wire_id || !drift || !grids || !best_E || !best_seed || !flags)
        return set_error(c, CDC_ERR_ARG, "NULL argument");
    CurrentDevice guard(dev);
    if (!guard.ok) return set_error(c, CDC_ERR_CUDA, "cudaSetDevice failed");
    void* base = nullptr;
    if (scratch_address(dev, &base) != cudaSuccess)
        return set_error(c, CDC_ERR_CUDA, "cudaGetSymbolAddress of the no-allocation workspace failed");
    unsigned char* b = (unsigned char*)base;
    Workspace W;
    W.drift_tab = (float*)(b + OFF_DRIFT);
    W.E = (float*)(b + OFF_E);
    W.seed_off = (long long*)(b + OFF_SEEDOFF);
    W.seg_off = (int*)(b + OFF_SEGOFF);
    W.counters = (unsigned long long*)(b + OFF_COUNT);
    W.seg_keys = (uint64_t*)(b + OFF_SEGK);
    W.round_keys = (uint64_t*)(b + OFF_ROUNDK);
    W.best_keys = (uint64_t*)(b + OFF_BESTK);
    W.zgrids = (cdc_grid*)(b + OFF_ZGRID);
    W.max_events = CDC_NOALLOC_MAX_EVENTS;
    W.e_cap = CDC_NOALLOC_MAX_SEEDS;
    W.seg_cap = NA_SEG_CAP;
    W.n_wires = G.n_wires;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(flags, 0, sizeof(uint32_t) * n_events, st);
    if (e != cudaSuccess) return set_error(c, CDC_ERR_CUDA, "flags reset failed");
    ScanLaunch L{n_events, hit_off, wire_id, drift, grids, E, topk0, best_E, best_seed, hit_part, hit_res2, nullptr,
                 flags, steps, 1, 1, KernelTimer{}};
    L.block = block;
    L.chunk = chunk;
    // the caller sized E (and the array holds the scores) for n_seeds: grids that
    // hold more scan nothing and flag every event empty, with or without E
    L.e0_cap = n_seeds;
    e = launch_scan(G, F, P, W, L, sms, st);
    if (e != cudaSuccess) return set_error(c, CDC_ERR_CUDA, cudaGetErrorString(e));
    return CDC_OK;
}
