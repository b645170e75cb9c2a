// C ABI of the seed-scanning track finder: context, loading, validation and
// the compute entry points declared in include/cdc.h.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "../../include/cdc.h"
#include "cdc_dev.cuh"
#include "cdc_host.h"

using namespace cdc;

struct cdc_ctx {
    int device = 0;
    int num_sms = 1;
    std::string err;
    // geometry
    bool geom = false;
    DevGeom G{};
    DevLayer* d_layers = nullptr;
    float4* d_wires = nullptr;
    uchar2* d_tab = nullptr;
    int2* d_wire_um = nullptr;
    float4* d_wires_lo = nullptr;
    double tan_max = 0.0;
    // field
    bool field = false;
    DevField F{};
    float b_max = 0.f;
    float4* d_cells = nullptr;
    // workspace
    Workspace W{};
    // Hough vote offsets for the last parameter set
    int2* d_offsets = nullptr;
    size_t offsets_cap = 0;
    int off_key[4] = {-1, -1, -1, -1};
    // the two-kernel scan's recorded states (cdc_reserve_split)
    float4 *split_r = nullptr, *split_t = nullptr;
    int* split_n = nullptr;
    int8_t* split_end = nullptr;
    int split_chunk = 0, split_steps = 0;
    // scan-kernel launch shape (cdc_scan_config)
    int scan_block = 128, scan_chunk = 32, scan_warp_seeds = 0;
    // kernel timer
    bool timer_on = false, timer_keep = false;
    std::vector<cudaEvent_t> timer_ev;
    int timer_used = 0;
    // FP32 throughput measurement
    float* d_sink = nullptr;
    int sink_n = 0;
};

namespace {

const double PI = 3.14159265358979323846;

int fail(cdc_ctx* c, int code, const std::string& msg) {
    if (c) c->err = msg;
    return code;
}

int cuda_fail(cdc_ctx* c, cudaError_t e, const char* what) {
    return fail(c, CDC_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

template <class T>
void dfree(T*& p) {
    if (p) cudaFree(p);
    p = nullptr;
}

template <class T>
cudaError_t dalloc(T*& p, size_t n) {
    dfree(p);
    if (n == 0) n = 1;
    return cudaMalloc((void**)&p, n * sizeof(T));
}

void free_workspace(Workspace& W) {
    dfree(W.drift_tab);
    dfree(W.E);
    dfree(W.seed_off);
    dfree(W.seg_off);
    dfree(W.counters);
    dfree(W.seg_keys);
    dfree(W.round_keys);
    dfree(W.best_keys);
    dfree(W.zgrids);
    dfree(W.perm);
    dfree(W.recs);
    dfree(W.rec_count);
    dfree(W.run_best);
    dfree(W.hough_max);
    dfree(W.hough_keys);
    W = Workspace{};
}

// Window and band half-width [mm] that cover every wire whose distance of
// closest approach can score below lambda (see tracer.cuh).
float search_width(const cdc_ctx* c, const cdc_scan_params* p) {
    double dmax = (double)p->max_drift + sqrt((double)p->lambda);
    return (float)((1.0 + c->tan_max) * dmax + 1.1 * (double)p->h + 1.0);
}

int check_scan_params(cdc_ctx* c, const cdc_scan_params* p, bool need_k) {
    if (!p) return fail(c, CDC_ERR_ARG, "scan params is NULL");
    if (!(p->h > 0.f) || !(p->lambda > 0.f) || !(p->max_drift >= 0.f) || !(p->charge == p->charge) || p->charge == 0.f)
        return fail(c, CDC_ERR_ARG, "scan params: h, lambda, charge must be non-zero, max_drift >= 0");
    if (p->max_steps < 1 || p->max_steps > (1 << 20)) return fail(c, CDC_ERR_RANGE, "max_steps outside 1..2^20");
    if (p->max_partitions < 1 || p->max_partitions > 16)
        return fail(c, CDC_ERR_RANGE, "max_partitions outside 1..16");
    if (p->direction != 1 && p->direction != -1) return fail(c, CDC_ERR_ARG, "direction must be +1 or -1");
    if (need_k) {
        if (p->k < 1 || p->k > CDC_MAX_K) return fail(c, CDC_ERR_RANGE, "k outside 1..64");
        if (p->n_rounds < 1 || p->n_rounds > CDC_MAX_ROUNDS) return fail(c, CDC_ERR_RANGE, "n_rounds outside 1..16");
        if (p->n_rounds > 1 && (p->n_zoom < 1 || p->n_zoom > CDC_MAX_ZOOM || p->n_zoom > p->k))
            return fail(c, CDC_ERR_RANGE, "n_zoom outside 1..min(k, 8)");
    }
    if (search_width(c, p) + LIST_M * p->h > TAB_BAND)  // the candidate lists widen the window by LIST_M h
        return fail(c, CDC_ERR_RANGE, "max_drift + sqrt(lambda) (or h) too large for the wire search window");
    return CDC_OK;
}

ScanConst make_const(const cdc_ctx* c, const cdc_scan_params* p) {
    ScanConst P{};
    P.h = p->h;
    P.h6_lo = (float)((double)p->h / 6.0 - (double)(p->h * (1.0f / 6.0f)));
    P.lam = p->lambda;
    P.sqrt_lam = sqrtf(p->lambda);
    P.charge_dir = p->charge * (float)p->direction;
    P.band = search_width(c, p);
    P.d_win = P.band;
    P.max_drift = p->max_drift;
    P.b_max = c->b_max;
    P.max_steps = p->max_steps;
    P.max_part = p->max_partitions;
    P.direction = p->direction;
    P.k = p->k;
    return P;
}

}  // namespace

extern "C" {

int cdc_create(cdc_ctx** out, int device) {
    if (!out) return CDC_ERR_ARG;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) return CDC_ERR_CUDA;
    cdc_ctx* c = new cdc_ctx();
    c->device = device;
    DeviceGuard g(device);
    if (!g.ok || cudaFree(0) != cudaSuccess ||
        cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
        delete c;
        return CDC_ERR_CUDA;
    }
    c->scan_warp_seeds = 16 * c->num_sms;
    *out = c;
    return CDC_OK;
}

void cdc_destroy(cdc_ctx* c) {
    if (!c) return;
    DeviceGuard g(c->device);
    dfree(c->d_layers);
    dfree(c->d_wires);
    dfree(c->d_tab);
    dfree(c->d_wire_um);
    dfree(c->d_wires_lo);
    dfree(c->d_cells);
    dfree(c->d_offsets);
    free_workspace(c->W);
    dfree(c->split_r);
    dfree(c->split_t);
    dfree(c->split_n);
    dfree(c->split_end);
    for (cudaEvent_t e : c->timer_ev) cudaEventDestroy(e);
    dfree(c->d_sink);
    delete c;
}

const char* cdc_last_error(const cdc_ctx* c) {
    if (!c) return "NULL context";
    return c->err.c_str();
}

int cdc_load_geometry(cdc_ctx* c, int n_layers, const double* R, const double* alpha, const int32_t* N,
                      const double* phi_off, double z_half, double R0, double R_out) {
    if (!c) return CDC_ERR_ARG;
    if (!R || !alpha || !N || !phi_off) return fail(c, CDC_ERR_ARG, "geometry array is NULL");
    if (n_layers < 1 || n_layers > CDC_MAX_LAYERS) return fail(c, CDC_ERR_RANGE, "n_layers outside 1..64");
    if (!(z_half > 0) || !(R0 > 0) || !(R_out > R0)) return fail(c, CDC_ERR_ARG, "need z_half > 0, 0 < R0 < R_out");
    if (R_out + TAB_BAND + 10.0 >= TAB_N) return fail(c, CDC_ERR_RANGE, "R_out + 42 mm beyond the radial table (1024 mm)");
    int nw = 0;
    double tmax = 0.0;
    for (int l = 0; l < n_layers; ++l) {
        if (N[l] < 32 || N[l] > 65535) return fail(c, CDC_ERR_RANGE, "wires per layer outside 32..65535");
        // a window of half width TAB_BAND spans at most 32 cells of the fired-wire bits
        if (2.0 * TAB_BAND * (N[l] / (2.0 * PI * (R[l] - TAB_BAND)) * 1.01) > 31.0)
            return fail(c, CDC_ERR_RANGE, "wire pitch below 2.1 mm: the search window spans more than 32 cells");
        if (!(R[l] > TAB_BAND) || (l > 0 && !(R[l] > R[l - 1])))
            return fail(c, CDC_ERR_RANGE, "layer radii must increase and exceed 32 mm");
        if (!(fabs(alpha[l]) < 0.19)) return fail(c, CDC_ERR_RANGE, "|stereo angle| must be below 0.19 rad");
        nw += N[l];
        tmax = std::max(tmax, fabs(tan(alpha[l])));
    }
    if (nw > CDC_MAX_WIRES) return fail(c, CDC_ERR_RANGE, "more than 8192 wires");
    std::vector<DevLayer> lay(n_layers);
    std::vector<float4> wires(nw);
    std::vector<int2> wum(nw);
    std::vector<float4> wlo(nw);
    int base = 0, bword = 0;
    for (int l = 0; l < n_layers; ++l) {
        DevLayer& L = lay[l];
        L.bword = bword;
        bword += (N[l] >> 5) + 3;
        double ta = tan(alpha[l]);
        L.R2 = (float)(R[l] * R[l]);
        L.tan2a = (float)(ta * ta);
        L.tana_over_R = (float)(ta / R[l]);
        L.phi_off = (float)phi_off[l];
        L.n_over_2pi = (float)(N[l] / (2.0 * PI));
        L.cells_per_mm = (float)(N[l] / (2.0 * PI * (R[l] - TAB_BAND)) * 1.01);
        L.cosa = (float)cos(alpha[l]);
        L.cosa_lo = (float)(cos(alpha[l]) - (double)L.cosa);
        L.N = N[l];
        L.base = base;
        double sa = sin(alpha[l]);
        for (int i = 0; i < N[l]; ++i) {
            double phi = phi_off[l] + 2.0 * PI * (double)i / (double)N[l];
            double mx = R[l] * cos(phi), my = R[l] * sin(phi);
            wires[base + i] = make_float4((float)mx, (float)my, (float)(-sa * sin(phi)), (float)(sa * cos(phi)));
            wum[base + i] = make_int2((int)llround(1000.0 * mx), (int)llround(1000.0 * my));
            const double dx = -sa * sin(phi), dy = sa * cos(phi);
            wlo[base + i] = make_float4((float)(mx - (double)(float)mx), (float)(my - (double)(float)my),
                                        (float)(dx - (double)(float)dx), (float)(dy - (double)(float)dy));
        }
        base += N[l];
    }
    // candidate layers per millimetre of rho: bands [R_l - B, r_l(z_half + 10) + B]
    std::vector<uchar2> tab(TAB_N);
    for (int b = 0; b < TAB_N; ++b) {
        int lo = n_layers, hi = -1;
        for (int l = 0; l < n_layers; ++l) {
            double ta = tan(alpha[l]);
            double rmax = sqrt(R[l] * R[l] + (z_half + 10.0) * (z_half + 10.0) * ta * ta);
            if (rmax + TAB_BAND >= b && R[l] - TAB_BAND <= b + 1) {
                lo = std::min(lo, l);
                hi = std::max(hi, l);
            }
        }
        tab[b] = hi < 0 ? make_uchar2(1, 0) : make_uchar2((unsigned char)lo, (unsigned char)hi);
    }
    DeviceGuard g(c->device);
    cudaError_t e;
    if ((e = dalloc(c->d_layers, lay.size())) != cudaSuccess || (e = dalloc(c->d_wires, wires.size())) != cudaSuccess ||
        (e = dalloc(c->d_tab, tab.size())) != cudaSuccess || (e = dalloc(c->d_wire_um, wum.size())) != cudaSuccess ||
        (e = dalloc(c->d_wires_lo, wlo.size())) != cudaSuccess)
        return fail(c, CDC_ERR_NOMEM, std::string("geometry allocation: ") + cudaGetErrorString(e));
    if ((e = cudaMemcpy(c->d_layers, lay.data(), lay.size() * sizeof(DevLayer), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(c->d_wires, wires.data(), wires.size() * sizeof(float4), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(c->d_tab, tab.data(), tab.size() * sizeof(uchar2), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(c->d_wire_um, wum.data(), wum.size() * sizeof(int2), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(c->d_wires_lo, wlo.data(), wlo.size() * sizeof(float4), cudaMemcpyHostToDevice)) != cudaSuccess)
        return cuda_fail(c, e, "geometry upload");
    c->G.layers = c->d_layers;
    c->G.wires = c->d_wires;
    c->G.tab = c->d_tab;
    c->G.wire_um = c->d_wire_um;
    c->G.wires_lo = c->d_wires_lo;
    c->G.n_layers = n_layers;
    c->G.n_wires = nw;
    c->G.z_half = (float)z_half;
    c->G.R0 = (float)R0;
    c->G.R_out = (float)R_out;
    c->G.R0d = R0;
    c->tan_max = tmax;
    c->geom = true;
    return CDC_OK;
}

int cdc_load_field(cdc_ctx* c, int kind, float b0, const float* bz, const float* br, int nr, int nz, float r_min,
                   float z_min, float dr, float dz) {
    if (!c) return CDC_ERR_ARG;
    DeviceGuard g(c->device);
    if (kind == 0) {
        if (!(b0 == b0)) return fail(c, CDC_ERR_ARG, "b0 is NaN");
        c->F = DevField{};
        c->F.kind = 0;
        c->F.B0 = b0;
        c->b_max = fabsf(b0);
        c->field = true;
        return CDC_OK;
    }
    if (kind != 1) return fail(c, CDC_ERR_ARG, "field kind must be 0 or 1");
    if (!bz || !br) return fail(c, CDC_ERR_ARG, "field map array is NULL");
    if (nr < 2 || nz < 2 || (long long)nr * nz > (1ll << 28)) return fail(c, CDC_ERR_RANGE, "map size");
    if (!(dr > 0.f) || !(dz > 0.f) || !(r_min >= 0.f)) return fail(c, CDC_ERR_ARG, "need dr, dz > 0 and r_min >= 0");
    // Cell (ip, jp) of the (nr + 1) x (nz + 1) table covers the map cell (ip - 1, jp - 1); the border
    // rows and columns hold the edge values with no dependence on the clamped coordinate, so a
    // position beyond the grid, whose cell index is clamped into the border, reads the field at the
    // nearest edge point (the map's clamped interpolation) without clamping its coordinates.
    const size_t ncell = (size_t)(nr + 1) * (nz + 1);
    std::vector<float4> cells(2 * ncell);
    double bmax = 0.0;  // |B| of the bilinear field never exceeds the largest sample norm
    for (size_t q = 0; q < (size_t)nr * nz; ++q) bmax = std::max(bmax, hypot((double)bz[q], (double)br[q]));
    for (int ip = 0; ip <= nr; ++ip)
        for (int jp = 0; jp <= nz; ++jp) {
            // the map cell's corner indices, each clamped into the grid; a border cell repeats its edge
            const int i0 = std::min(std::max(ip - 1, 0), nr - 1), i1 = std::min(ip, nr - 1);
            const int j0 = std::min(std::max(jp - 1, 0), nz - 1), j1 = std::min(jp, nz - 1);
            const float* m[2] = {bz, br};
            for (int q = 0; q < 2; ++q) {
                double v00 = m[q][(size_t)i0 * nz + j0], v10 = m[q][(size_t)i1 * nz + j0];
                double v01 = m[q][(size_t)i0 * nz + j1], v11 = m[q][(size_t)i1 * nz + j1];
                cells[2 * ((size_t)ip * (nz + 1) + jp) + q] =
                    make_float4((float)v00, (float)(v10 - v00), (float)(v01 - v00), (float)(v11 - v10 - v01 + v00));
            }
        }
    cudaError_t e;
    if ((e = dalloc(c->d_cells, cells.size())) != cudaSuccess)
        return fail(c, CDC_ERR_NOMEM, std::string("field allocation: ") + cudaGetErrorString(e));
    if ((e = cudaMemcpy(c->d_cells, cells.data(), cells.size() * sizeof(float4), cudaMemcpyHostToDevice)) != cudaSuccess)
        return cuda_fail(c, e, "field upload");
    DevField F{};
    F.kind = 1;
    F.B0 = b0;
    F.cells = c->d_cells;
    F.nr = nr;
    F.nz = nz;
    F.r_min = r_min;
    F.z_min = z_min;
    F.inv_dr = 1.0f / dr;
    F.inv_dz = 1.0f / dz;
    F.u_off = 1.0f - r_min * F.inv_dr;  // padded cell coordinates: (rho - r_min) / dr + 1
    F.v_off = 1.0f - z_min * F.inv_dz;
    F.r_max = r_min + dr * (float)(nr - 1);
    F.z_max = z_min + dz * (float)(nz - 1);
    F.dr = dr;
    F.dz = dz;
    c->F = F;
    c->b_max = (float)(bmax * (1.0 + 1e-6));
    c->field = true;
    return CDC_OK;
}

int cdc_reserve(cdc_ctx* c, int max_events, int64_t max_seeds, int64_t max_hits) {
    if (!c) return CDC_ERR_ARG;
    if (!c->geom) return fail(c, CDC_ERR_NOT_LOADED, "load the geometry before cdc_reserve");
    if (max_events < 1 || max_seeds < 0 || max_hits < 0) return fail(c, CDC_ERR_ARG, "reserve sizes");
    if (max_events > (1 << 20)) return fail(c, CDC_ERR_RANGE, "max_events above 2^20");
    DeviceGuard g(c->device);
    free_workspace(c->W);
    Workspace W;
    W.max_events = max_events;
    W.n_wires = c->G.n_wires;
    W.e_cap = std::max<long long>(max_seeds, (long long)max_events * CDC_MAX_ZOOM * ZOOM_GRID);
    W.seg_cap = W.e_cap / SEG + max_events + 1;
    cudaError_t e = cudaSuccess;
    if ((e = dalloc(W.drift_tab, (size_t)max_events * event_stride(W.n_wires))) != cudaSuccess ||
        (e = dalloc(W.E, (size_t)W.e_cap)) != cudaSuccess || (e = dalloc(W.seed_off, (size_t)max_events + 1)) != cudaSuccess ||
        (e = dalloc(W.seg_off, (size_t)max_events + 1)) != cudaSuccess || (e = dalloc(W.counters, 4)) != cudaSuccess ||
        (e = dalloc(W.seg_keys, (size_t)W.seg_cap * CDC_MAX_K)) != cudaSuccess ||
        (e = dalloc(W.round_keys, (size_t)2 * max_events * CDC_MAX_K)) != cudaSuccess ||
        (e = dalloc(W.best_keys, (size_t)max_events * CDC_MAX_K)) != cudaSuccess ||
        (e = dalloc(W.zgrids, (size_t)2 * max_events * CDC_MAX_ZOOM)) != cudaSuccess ||
        (e = dalloc(W.perm, (size_t)max_events * PERM_CAP)) != cudaSuccess ||
        (e = dalloc(W.recs, (size_t)max_events * REC_SLOTS)) != cudaSuccess ||
        (e = dalloc(W.rec_count, (size_t)max_events)) != cudaSuccess ||
        (e = dalloc(W.run_best, (size_t)max_events)) != cudaSuccess ||
        (e = dalloc(W.hough_max, (size_t)max_events)) != cudaSuccess ||
        (e = dalloc(W.hough_keys, (size_t)max_events * HOUGH_SLICES * HOUGH_SLICE_KEYS)) != cudaSuccess) {
        free_workspace(W);
        return fail(c, CDC_ERR_NOMEM, std::string("workspace allocation: ") + cudaGetErrorString(e));
    }
    c->W = W;
    return CDC_OK;
}

int cdc_hough_seeds(cdc_ctx* c, int n_events, const int32_t* hit_off, const int32_t* wire_id,
                    const cdc_hough_params* p, int32_t* acc, cdc_candidate* cand, int32_t* n_cand, cdc_grid* grid_out,
                    uint32_t* flags, void* stream) {
    if (!c) return CDC_ERR_ARG;
    if (!c->geom) return fail(c, CDC_ERR_NOT_LOADED, "geometry not loaded");
    if (n_events < 0) return fail(c, CDC_ERR_ARG, "n_events < 0");
    if (n_events == 0) return CDC_OK;
    if (n_events > 65535) return fail(c, CDC_ERR_RANGE, "more than 65535 events per Hough call");
    if (!p || !hit_off || !wire_id || !acc || !cand || !n_cand || !flags)
        return fail(c, CDC_ERR_ARG, "NULL argument");
    if (n_events > c->W.max_events)
        return fail(c, CDC_ERR_NOT_LOADED, "workspace too small: cdc_reserve at least n_events events");
    if (p->n_bins < 3 || p->n_bins > 4096 || p->bin_um < 2 || (p->bin_um & 1) || p->n_r < 1 || p->n_r > 256 ||
        p->n_phi < 1 || p->n_phi > 8192 || p->r_min_um < 0 || p->r_step_um < 0 || p->target_um < 0 ||
        p->min_peak < 1 || p->max_cand < 1 || p->max_cand > 64 || p->r_hist_half_um < 0)
        return fail(c, CDC_ERR_RANGE, "Hough parameters out of range");
    if ((long long)p->n_bins * p->bin_um >= (1ll << 30) || llabs((long long)p->origin_um) >= (1ll << 29) ||
        (long long)p->r_min_um + (long long)p->n_r * p->r_step_um >= (1ll << 29))
        return fail(c, CDC_ERR_RANGE, "Hough coordinates beyond 2^29 um");
    DeviceGuard g(c->device);
    cudaStream_t st = (cudaStream_t)stream;
    // integer vote offsets round(R_j (cos, sin)(2 pi k / n_phi)) [um], uploaded once per parameter set
    const int key[4] = {p->n_r, p->r_min_um, p->r_step_um, p->n_phi};
    if (memcmp(key, c->off_key, sizeof key) != 0) {
        const size_t n = (size_t)p->n_r * p->n_phi;
        std::vector<int2> off(n);
        for (int j = 0; j < p->n_r; ++j) {
            const long long R = (long long)p->r_min_um + (long long)j * p->r_step_um;
            for (int k = 0; k < p->n_phi; ++k) {
                const double ph = 2.0 * PI * (double)k / (double)p->n_phi;
                off[(size_t)j * p->n_phi + k] = make_int2((int)llround((double)R * cos(ph)), (int)llround((double)R * sin(ph)));
            }
        }
        if (n > c->offsets_cap) {
            cudaError_t e = dalloc(c->d_offsets, n);
            if (e != cudaSuccess) return fail(c, CDC_ERR_NOMEM, "Hough offset table allocation");
            c->offsets_cap = n;
        }
        cudaError_t e = cudaMemcpy(c->d_offsets, off.data(), n * sizeof(int2), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return cuda_fail(c, e, "Hough offset upload");
        memcpy(c->off_key, key, sizeof key);
    }
    cudaError_t e = cudaMemsetAsync(flags, 0, sizeof(uint32_t) * n_events, st);
    if (e != cudaSuccess) return cuda_fail(c, e, "flags reset");
    HoughLaunch L{n_events, hit_off, wire_id, c->d_offsets, acc, cand, n_cand, grid_out, flags,
                  c->W.hough_max, c->W.hough_keys};
    e = launch_hough(c->G, *p, L, st);
    if (e != cudaSuccess) return cuda_fail(c, e, "Hough launch");
    return CDC_OK;
}

int cdc_candidate_grids(cdc_ctx* c, int n_events, const cdc_hough_params* p, const cdc_candidate* cand,
                        const int32_t* n_cand, cdc_grid* grids, void* stream) {
    if (!c) return CDC_ERR_ARG;
    if (n_events < 0) return fail(c, CDC_ERR_ARG, "n_events < 0");
    if (!p || !cand || !n_cand || !grids) return fail(c, CDC_ERR_ARG, "NULL argument");
    if (p->max_cand < 1 || p->max_cand > 64) return fail(c, CDC_ERR_RANGE, "max_cand outside 1..64");
    if (n_events > 65535) return fail(c, CDC_ERR_RANGE, "more than 65535 events");
    if (n_events == 0) return CDC_OK;
    DeviceGuard g(c->device);
    cudaError_t e = launch_candidate_grids(n_events, *p, cand, n_cand, grids, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "candidate grids launch");
    return CDC_OK;
}

int cdc_scan_seeds(cdc_ctx* c, int n_events, const int32_t* hit_off, const int32_t* wire_id, const float* drift,
                   const cdc_grid* grids, const cdc_scan_params* p, float* E, uint64_t* topk0, float* best_E,
                   float* best_seed, int8_t* hit_part, float* hit_res2, cdc_grid* zoom_grids, uint32_t* flags,
                   unsigned long long* steps, void* stream) {
    if (!c) return CDC_ERR_ARG;
    if (!c->geom || !c->field) return fail(c, CDC_ERR_NOT_LOADED, "geometry or field not loaded");
    if (n_events < 0) return fail(c, CDC_ERR_ARG, "n_events < 0");
    if (n_events == 0) return CDC_OK;
    int rc = check_scan_params(c, p, true);
    if (rc) return rc;
    if (!hit_off || !wire_id || !drift || !grids || !best_E || !best_seed || !flags)
        return fail(c, CDC_ERR_ARG, "NULL argument");
    if (n_events > c->W.max_events || c->W.n_wires < c->G.n_wires)
        return fail(c, CDC_ERR_NOT_LOADED, "workspace too small: call cdc_reserve");
    DeviceGuard g(c->device);
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(flags, 0, sizeof(uint32_t) * n_events, st);
    if (e != cudaSuccess) return cuda_fail(c, e, "flags reset");
    ScanLaunch L{n_events, hit_off, wire_id, drift, grids, E, topk0, best_E, best_seed, hit_part, hit_res2, zoom_grids,
                 flags, steps, p->n_rounds, p->n_rounds > 1 ? p->n_zoom : 1, KernelTimer{}};
    if (c->timer_on) L.timer = KernelTimer{c->timer_ev.data(), (int)c->timer_ev.size(), &c->timer_used};
    L.block = c->scan_block;
    L.chunk = c->scan_chunk;
    L.warp_seeds = c->scan_warp_seeds;
    e = launch_scan(c->G, c->F, make_const(c, p), c->W, L, c->num_sms, st);
    if (e != cudaSuccess) return cuda_fail(c, e, "scan launch");
    return CDC_OK;
}

int cdc_classification_counts(cdc_ctx* c, int n_events, const int32_t* hit_off, const int8_t* hit_part,
                              const int8_t* truth_part, int n_part, int32_t* counts, void* stream) {
    if (!c) return CDC_ERR_ARG;
    if (n_events < 0) return fail(c, CDC_ERR_ARG, "n_events < 0");
    if (n_events == 0) return CDC_OK;
    if (n_part < 1 || n_part > 16) return fail(c, CDC_ERR_RANGE, "n_part outside 1..16");
    if (!hit_off || !hit_part || !truth_part || !counts) return fail(c, CDC_ERR_ARG, "NULL argument");
    DeviceGuard g(c->device);
    cudaError_t e = launch_class_counts(n_events, hit_off, hit_part, truth_part, n_part, counts, c->num_sms,
                                        (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "classification counts");
    return CDC_OK;
}

int cdc_efficiency_purity(cdc_ctx* c, int n_sets, const int32_t* counts, int n_part, float* eff, float* pur,
                          void* stream) {
    if (!c) return CDC_ERR_ARG;
    if (n_sets < 1) return fail(c, CDC_ERR_ARG, "n_sets < 1");
    if (n_part < 1 || n_part > 16) return fail(c, CDC_ERR_RANGE, "n_part outside 1..16");
    if (!counts || !eff || !pur) return fail(c, CDC_ERR_ARG, "NULL argument");
    DeviceGuard g(c->device);
    cudaError_t e = launch_efficiency_purity(n_sets, counts, n_part, eff, pur, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "efficiency and purity");
    return CDC_OK;
}

int cdc_reserve_split(cdc_ctx* c, int chunk, int max_steps) {
    if (!c) return CDC_ERR_ARG;
    if (chunk < 1 || chunk > (1 << 20) || max_steps < 1 || max_steps > 6900)
        return fail(c, CDC_ERR_RANGE, "split reserve: chunk outside 1..2^20 or max_steps outside 1..6900");
    DeviceGuard g(c->device);
    dfree(c->split_r);
    dfree(c->split_t);
    dfree(c->split_n);
    dfree(c->split_end);
    c->split_chunk = c->split_steps = 0;
    const size_t n = (size_t)chunk * (max_steps + 1);
    cudaError_t e;
    if ((e = dalloc(c->split_r, n)) != cudaSuccess || (e = dalloc(c->split_t, n)) != cudaSuccess ||
        (e = dalloc(c->split_n, (size_t)chunk)) != cudaSuccess || (e = dalloc(c->split_end, (size_t)chunk)) != cudaSuccess)
        return fail(c, CDC_ERR_NOMEM, std::string("split workspace: ") + cudaGetErrorString(e));
    c->split_chunk = chunk;
    c->split_steps = max_steps;
    return CDC_OK;
}

int cdc_scan_seeds_split(cdc_ctx* c, int n_events, int64_t n_seeds, const int32_t* hit_off, const int32_t* wire_id,
                         const float* drift, const cdc_grid* grids, const cdc_scan_params* p, float* E,
                         uint32_t* flags, void* stream) {
    if (!c) return CDC_ERR_ARG;
    if (!c->geom || !c->field) return fail(c, CDC_ERR_NOT_LOADED, "geometry or field not loaded");
    if (n_events < 0 || n_seeds < 0) return fail(c, CDC_ERR_ARG, "n_events or n_seeds < 0");
    if (n_events == 0) return CDC_OK;
    if (!p) return fail(c, CDC_ERR_ARG, "scan params is NULL");
    cdc_scan_params p1 = *p;
    p1.n_rounds = 1;
    int rc = check_scan_params(c, &p1, true);
    if (rc) return rc;
    if (!hit_off || !wire_id || !drift || !grids || !E || !flags) return fail(c, CDC_ERR_ARG, "NULL argument");
    if (n_events > c->W.max_events || c->W.n_wires < c->G.n_wires)
        return fail(c, CDC_ERR_NOT_LOADED, "workspace too small: call cdc_reserve");
    if (!c->split_r || p->max_steps > c->split_steps)
        return fail(c, CDC_ERR_NOT_LOADED, "split workspace missing or max_steps above its reserve");
    if (n_seeds > c->W.e_cap) return fail(c, CDC_ERR_RANGE, "n_seeds above the reserved seed capacity");
    DeviceGuard g(c->device);
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(flags, 0, sizeof(uint32_t) * n_events, st);
    if (e != cudaSuccess) return cuda_fail(c, e, "flags reset");
    const ScanConst P = make_const(c, &p1);
    if ((e = launch_stage(c->G, n_events, hit_off, wire_id, drift, P.max_drift, c->W.drift_tab, flags, c->num_sms,
                          st)) != cudaSuccess)
        return cuda_fail(c, e, "staging");
    SplitLaunch L{n_events, hit_off, wire_id, drift, grids, n_seeds, c->split_chunk, 256, c->W, flags, E,
                  c->split_r, c->split_t, c->split_n, c->split_end};
    if ((e = launch_split(c->G, c->F, P, L, st)) != cudaSuccess) return cuda_fail(c, e, "split scan launch");
    return CDC_OK;
}

int cdc_extrapolate_turn(cdc_ctx* c, int n_seeds, const float* seeds, const cdc_scan_params* p, int direction,
                         float* seeds_out, int32_t* status, void* stream) {
    if (!c) return CDC_ERR_ARG;
    if (!c->geom || !c->field) return fail(c, CDC_ERR_NOT_LOADED, "geometry or field not loaded");
    if (n_seeds < 0) return fail(c, CDC_ERR_ARG, "n_seeds < 0");
    if (n_seeds == 0) return CDC_OK;
    if (direction != 1 && direction != -1) return fail(c, CDC_ERR_ARG, "direction must be +1 or -1");
    if (!p) return fail(c, CDC_ERR_ARG, "scan params is NULL");
    cdc_scan_params p1 = *p;
    p1.direction = direction;
    p1.n_rounds = 1;
    int rc = check_scan_params(c, &p1, false);
    if (rc) return rc;
    if (!seeds || !seeds_out || !status) return fail(c, CDC_ERR_ARG, "NULL argument");
    DeviceGuard g(c->device);
    cudaError_t e = launch_extrapolate_turn(c->G, c->F, make_const(c, &p1), n_seeds, seeds, seeds_out, status,
                                            (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "extrapolation launch");
    return CDC_OK;
}

int cdc_common_hits(cdc_ctx* c, int n_events, const int32_t* hit_off, const int8_t* part_a, const int8_t* part_b,
                    int pa, int pb, int32_t* n_common, void* stream) {
    if (!c) return CDC_ERR_ARG;
    if (n_events < 0) return fail(c, CDC_ERR_ARG, "n_events < 0");
    if (n_events == 0) return CDC_OK;
    if (!hit_off || !part_a || !part_b || !n_common) return fail(c, CDC_ERR_ARG, "NULL argument");
    DeviceGuard g(c->device);
    cudaError_t e = launch_common_hits(n_events, hit_off, part_a, part_b, pa, pb, n_common, c->num_sms,
                                       (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "common hits");
    return CDC_OK;
}

static const cdc_scan_config SCAN_CONFIGS[CDC_SCAN_CONFIGS] = {{256, 16, 0}, {256, 32, 0}, {128, 16, 0}, {128, 32, 0}};

int cdc_set_scan_config(cdc_ctx* c, const cdc_scan_config* cfg) {
    if (!c || !cfg) return c ? fail(c, CDC_ERR_ARG, "NULL config") : CDC_ERR_ARG;
    if ((cfg->block != 128 && cfg->block != 256) || (cfg->chunk != 16 && cfg->chunk != 32) || cfg->warp_seeds < 0)
        return fail(c, CDC_ERR_RANGE, "scan config: block must be 128 or 256, chunk 16 or 32, warp_seeds >= 0");
    c->scan_block = cfg->block;
    c->scan_chunk = cfg->chunk;
    c->scan_warp_seeds = cfg->warp_seeds;
    return CDC_OK;
}

int cdc_get_scan_config(const cdc_ctx* c, cdc_scan_config* cfg) {
    if (!c || !cfg) return CDC_ERR_ARG;
    cfg->block = c->scan_block;
    cfg->chunk = c->scan_chunk;
    cfg->warp_seeds = c->scan_warp_seeds;
    return CDC_OK;
}

int cdc_tune_scan(cdc_ctx* c, int n_events, const int32_t* hit_off, const int32_t* wire_id, const float* drift,
                  const cdc_grid* grids, const cdc_scan_params* p, int reps, cdc_scan_config* best, float* ms,
                  void* stream) {
    if (!c) return CDC_ERR_ARG;
    if (!c->geom || !c->field) return fail(c, CDC_ERR_NOT_LOADED, "geometry or field not loaded");
    if (!p) return fail(c, CDC_ERR_ARG, "scan params is NULL");
    if (n_events < 1) return fail(c, CDC_ERR_ARG, "n_events must be >= 1");
    if (reps < 1 || reps > 20) return fail(c, CDC_ERR_RANGE, "reps outside 1..20");
    cdc_scan_params p1 = *p;
    p1.n_rounds = 1;
    int rc = check_scan_params(c, &p1, true);
    if (rc) return rc;
    if (!hit_off || !wire_id || !drift || !grids) return fail(c, CDC_ERR_ARG, "NULL argument");
    if (n_events > c->W.max_events || c->W.n_wires < c->G.n_wires)
        return fail(c, CDC_ERR_NOT_LOADED, "workspace too small: call cdc_reserve");
    DeviceGuard g(c->device);
    cudaStream_t st = (cudaStream_t)stream;
    float *bE = nullptr, *bS = nullptr;
    uint32_t* fl = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e;
    if ((e = dalloc(bE, (size_t)n_events * p1.k)) != cudaSuccess ||
        (e = dalloc(bS, (size_t)n_events * p1.k * 5)) != cudaSuccess || (e = dalloc(fl, (size_t)n_events)) != cudaSuccess) {
        dfree(bE);
        dfree(bS);
        dfree(fl);
        return fail(c, CDC_ERR_NOMEM, std::string("tuner buffers: ") + cudaGetErrorString(e));
    }
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const ScanConst P = make_const(c, &p1);
    float med[CDC_SCAN_CONFIGS];
    int bi = 0;
    for (int i = 0; i < CDC_SCAN_CONFIGS && e == cudaSuccess; ++i) {
        ScanLaunch L{n_events, hit_off, wire_id, drift, grids, nullptr, nullptr, bE, bS, nullptr, nullptr, nullptr,
                     fl, nullptr, 1, 1, KernelTimer{}};
        L.block = SCAN_CONFIGS[i].block;
        L.chunk = SCAN_CONFIGS[i].chunk;
        std::vector<float> t;
        for (int r = 0; r <= reps && e == cudaSuccess; ++r) {
            cudaEventRecord(e0, st);
            e = launch_scan(c->G, c->F, P, c->W, L, c->num_sms, st);
            cudaEventRecord(e1, st);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float x = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&x, e0, e1);
            if (r > 0) t.push_back(x);  // the first run warms up
        }
        if (e != cudaSuccess) break;
        std::sort(t.begin(), t.end());
        med[i] = t[t.size() / 2];
        if (med[i] < med[bi]) bi = i;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    dfree(bE);
    dfree(bS);
    dfree(fl);
    if (e != cudaSuccess) return cuda_fail(c, e, "tuning run");
    c->scan_block = SCAN_CONFIGS[bi].block;
    c->scan_chunk = SCAN_CONFIGS[bi].chunk;
    if (best) {
        *best = SCAN_CONFIGS[bi];
        best->warp_seeds = c->scan_warp_seeds;
    }
    if (ms)
        for (int i = 0; i < CDC_SCAN_CONFIGS; ++i) ms[i] = med[i];
    return CDC_OK;
}

}  // extern "C"

namespace {
int refine_common(cdc_ctx* c, int n_seeds, const int32_t* seed_event, const float* seeds, int n_events,
                  const int32_t* hit_off, const int32_t* wire_id, const float* drift, const cdc_scan_params* scan,
                  const cdc_refine_params* rp, float* seeds_out, double* chi2, float* grad, int32_t* n_used,
                  uint32_t* flags, void* stream, int do_gn) {
    if (!c) return CDC_ERR_ARG;
    if (!c->geom || !c->field) return fail(c, CDC_ERR_NOT_LOADED, "geometry or field not loaded");
    if (n_seeds < 0 || n_events < 0) return fail(c, CDC_ERR_ARG, "n_seeds, n_events < 0");
    if (n_seeds == 0) return CDC_OK;
    int rc = check_scan_params(c, scan, false);
    if (rc) return rc;
    if (!rp) return fail(c, CDC_ERR_ARG, "refine params is NULL");
    if (!seed_event || !seeds || !hit_off || !wire_id || !drift || !chi2 || !flags || (do_gn && !seeds_out))
        return fail(c, CDC_ERR_ARG, "NULL argument");
    if (n_events < 1) return fail(c, CDC_ERR_ARG, "n_events must be >= 1");
    if (rp->n_iter < 0 || rp->n_iter > 32) return fail(c, CDC_ERR_RANGE, "n_iter outside 0..32");
    if (!(rp->sigma > 0.f)) return fail(c, CDC_ERR_ARG, "sigma must be > 0");
    for (int m = 0; m < 5; ++m)
        if (!(rp->scale[m] > 0.f)) return fail(c, CDC_ERR_ARG, "scales must be > 0");
    if (rp->checkpoint < 8 || rp->checkpoint > 256) return fail(c, CDC_ERR_RANGE, "checkpoint outside 8..256");
    if (scan->max_steps >= 64 * rp->checkpoint) return fail(c, CDC_ERR_RANGE, "max_steps >= 64 * checkpoint");
    if (n_events > c->W.max_events || c->W.n_wires < c->G.n_wires)
        return fail(c, CDC_ERR_NOT_LOADED, "workspace too small: call cdc_reserve");
    DeviceGuard g(c->device);
    RefineLaunch L{n_seeds, seed_event, seeds, n_events, hit_off, wire_id, drift, rp->n_iter, rp->sigma,
                   {rp->scale[0], rp->scale[1], rp->scale[2], rp->scale[3], rp->scale[4]}, rp->checkpoint, seeds_out,
                   chi2, grad, n_used, flags};
    cudaError_t e = launch_refine(c->G, c->F, make_const(c, scan), L, c->W.drift_tab, c->num_sms, do_gn,
                                  (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "refine launch");
    return CDC_OK;
}
}  // namespace

extern "C" {

int cdc_refine_seeds(cdc_ctx* c, int n_seeds, const int32_t* seed_event, const float* seeds, int n_events,
                     const int32_t* hit_off, const int32_t* wire_id, const float* drift, const cdc_scan_params* scan,
                     const cdc_refine_params* params, float* seeds_out, double* chi2, float* grad, int32_t* n_used,
                     uint32_t* flags, void* stream) {
    return refine_common(c, n_seeds, seed_event, seeds, n_events, hit_off, wire_id, drift, scan, params, seeds_out,
                         chi2, grad, n_used, flags, stream, 1);
}

int cdc_chi2_grad(cdc_ctx* c, int n_seeds, const int32_t* seed_event, const float* seeds, int n_events,
                  const int32_t* hit_off, const int32_t* wire_id, const float* drift, const cdc_scan_params* scan,
                  const cdc_refine_params* params, double* chi2, float* grad, int32_t* n_used, uint32_t* flags,
                  void* stream) {
    return refine_common(c, n_seeds, seed_event, seeds, n_events, hit_off, wire_id, drift, scan, params, nullptr,
                         chi2, grad, n_used, flags, stream, 0);
}

int cdc_propagate(cdc_ctx* c, int n_seeds, const float* seeds, const cdc_scan_params* p, int every, int n_rec,
                  int precision, double* pos, int32_t* n_steps, double* path, void* stream) {
    if (!c) return CDC_ERR_ARG;
    if (!c->geom || !c->field) return fail(c, CDC_ERR_NOT_LOADED, "geometry or field not loaded");
    if (n_seeds < 0) return fail(c, CDC_ERR_ARG, "n_seeds < 0");
    if (n_seeds == 0) return CDC_OK;
    int rc = check_scan_params(c, p, false);
    if (rc) return rc;
    if (!seeds || !pos || !n_steps || !path) return fail(c, CDC_ERR_ARG, "NULL argument");
    if (every < 1 || n_rec < 1) return fail(c, CDC_ERR_ARG, "every and n_rec must be >= 1");
    if (precision < 0 || precision > 2) return fail(c, CDC_ERR_ARG, "precision must be 0, 1 or 2");
    DeviceGuard g(c->device);
    cudaError_t e = launch_propagate(c->G, c->F, make_const(c, p), n_seeds, seeds, every, n_rec, precision, pos,
                                     n_steps, path, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "propagate launch");
    return CDC_OK;
}

int cdc_kernel_timer(cdc_ctx* c, int enable) {
    if (!c) return CDC_ERR_ARG;
    DeviceGuard g(c->device);
    if (enable && c->timer_ev.empty()) {
        c->timer_ev.resize(2048);
        for (auto& e : c->timer_ev)
            if (cudaEventCreate(&e) != cudaSuccess) return fail(c, CDC_ERR_CUDA, "cudaEventCreate");
    }
    c->timer_on = enable != 0;
    c->timer_keep = enable == 2;
    c->timer_used = 0;
    return CDC_OK;
}

int cdc_kernel_time(cdc_ctx* c, double* total_ms, int64_t* launches, float* per_launch_ms, int cap) {
    if (!c || !total_ms || !launches) return c ? fail(c, CDC_ERR_ARG, "NULL argument") : CDC_ERR_ARG;
    DeviceGuard g(c->device);
    double tot = 0.0;
    for (int i = 0; i + 1 < c->timer_used; i += 2) {
        cudaError_t e = cudaEventSynchronize(c->timer_ev[i + 1]);
        if (e != cudaSuccess) return cuda_fail(c, e, "kernel timer");
        float ms = 0.f;
        e = cudaEventElapsedTime(&ms, c->timer_ev[i], c->timer_ev[i + 1]);
        if (e != cudaSuccess) return cuda_fail(c, e, "kernel timer");
        tot += ms;
        if (per_launch_ms && i / 2 < cap) per_launch_ms[i / 2] = ms;
    }
    *total_ms = tot;
    *launches = c->timer_used / 2;
    if (!c->timer_keep) c->timer_used = 0;
    return CDC_OK;
}

int cdc_fp32_peak(cdc_ctx* c, int iters, double* tflops, double* ms, void* stream) {
    if (!c || !tflops || !ms) return c ? fail(c, CDC_ERR_ARG, "NULL argument") : CDC_ERR_ARG;
    if (iters < 1 || iters > (1 << 20)) return fail(c, CDC_ERR_RANGE, "iters outside 1..2^20");
    DeviceGuard g(c->device);
    cudaStream_t st = (cudaStream_t)stream;
    const int need = c->num_sms * 64;  // >= blocks of one launch (at most 8 blocks of 256 threads per SM)
    cudaError_t e;
    if (c->sink_n < need) {
        dfree(c->d_sink);
        c->sink_n = 0;
        if ((e = dalloc(c->d_sink, (size_t)need)) != cudaSuccess) return cuda_fail(c, e, "sink allocation");
        c->sink_n = need;
    }
    cudaEvent_t ev[2];
    if (cudaEventCreate(&ev[0]) != cudaSuccess) return fail(c, CDC_ERR_CUDA, "cudaEventCreate");
    if (cudaEventCreate(&ev[1]) != cudaSuccess) {
        cudaEventDestroy(ev[0]);
        return fail(c, CDC_ERR_CUDA, "cudaEventCreate");
    }
    double fmas = 0.0;
    float t = 0.f;
    e = launch_ffma(c->num_sms, iters, c->d_sink, st, &fmas);  // warm-up
    if (e == cudaSuccess) e = cudaEventRecord(ev[0], st);
    if (e == cudaSuccess) e = launch_ffma(c->num_sms, iters, c->d_sink, st, &fmas);
    if (e == cudaSuccess) e = cudaEventRecord(ev[1], st);
    if (e == cudaSuccess) e = cudaEventSynchronize(ev[1]);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, ev[0], ev[1]);
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
    if (e != cudaSuccess) return cuda_fail(c, e, "FP32 peak measurement");
    *ms = t;
    *tflops = 2.0 * fmas / (t * 1e-3) / 1e12;
    return CDC_OK;
}

}  // extern "C"

namespace cdc {

// Context view for the allocation-free scan (noalloc.cu): validates the scan
// parameters exactly as cdc_scan_seeds does and hands out the loaded tables.
int scan_view(cdc_ctx* c, const cdc_scan_params* p, DevGeom* G, DevField* F, ScanConst* P, int* num_sms,
              int* device, int* block, int* chunk) {
    if (!c) return CDC_ERR_ARG;
    if (!c->geom || !c->field) return fail(c, CDC_ERR_NOT_LOADED, "geometry or field not loaded");
    int rc = check_scan_params(c, p, true);
    if (rc) return rc;
    *G = c->G;
    *F = c->F;
    *P = make_const(c, p);
    *num_sms = c->num_sms;
    *device = c->device;
    *block = c->scan_block;
    *chunk = c->scan_chunk;
    return CDC_OK;
}

int set_error(cdc_ctx* c, int code, const char* msg) { return fail(c, code, msg); }

}  // namespace cdc
