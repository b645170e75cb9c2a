"""ctypes binding of libcdc.so (include/cdc.h): argument marshalling only.

Every compute step runs in the CUDA library; this module checks tensor
dtypes/devices, turns torch tensors into device pointers and numpy arrays into
host pointers, and raises on a non-zero status with the library's message.
If the library has not been built it raises: there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libcdc.so")

CDC_MAX_K = 64
CDC_MAX_ZOOM = 8
CDC_MAX_ROUNDS = 16
CDC_MAX_FOUND = 256

FLAG_STEP_CAP = 1
FLAG_FOUND_OVERFLOW = 2
FLAG_EMPTY = 4
FLAG_NOT_SPD = 8
FLAG_DOCA_ZERO = 16
FLAG_LOST_HIT = 32
FLAG_BAD_HIT = 64

STATUS = {0: "CDC_OK", -1: "CDC_ERR_ARG", -2: "CDC_ERR_RANGE", -3: "CDC_ERR_CUDA", -4: "CDC_ERR_NOT_LOADED",
          -5: "CDC_ERR_TIMEOUT", -6: "CDC_ERR_NOMEM"}

# All entry points of include/cdc.h.
EXPORTS = ["cdc_create", "cdc_destroy", "cdc_last_error", "cdc_load_geometry", "cdc_load_field", "cdc_reserve",
           "cdc_hough_seeds", "cdc_scan_seeds", "cdc_refine_seeds", "cdc_chi2_grad", "cdc_propagate",
           "cdc_kernel_timer", "cdc_kernel_time", "cdc_set_scan_config", "cdc_get_scan_config", "cdc_tune_scan",
           "cdc_reserve_split", "cdc_scan_seeds_split", "cdc_extrapolate_turn", "cdc_classification_counts",
           "cdc_common_hits", "cdc_fp32_peak", "cdc_efficiency_purity", "cdc_candidate_grids",
           "cdc_scan_seeds_noalloc"]


class cdc_grid(C.Structure):
    _fields_ = [("centre", C.c_float * 5), ("step", C.c_float * 5), ("n", C.c_int32 * 5)]


class cdc_scan_params(C.Structure):
    _fields_ = [("h", C.c_float), ("max_steps", C.c_int32), ("lambda_", C.c_float), ("max_partitions", C.c_int32),
                ("direction", C.c_int32), ("charge", C.c_float), ("k", C.c_int32), ("n_rounds", C.c_int32),
                ("n_zoom", C.c_int32), ("max_drift", C.c_float)]


class cdc_hough_params(C.Structure):
    _fields_ = [("n_bins", C.c_int32), ("bin_um", C.c_int32), ("origin_um", C.c_int32), ("n_r", C.c_int32),
                ("r_min_um", C.c_int32), ("r_step_um", C.c_int32), ("n_phi", C.c_int32), ("target_um", C.c_int32),
                ("min_peak", C.c_int32), ("max_cand", C.c_int32), ("r_hist_half_um", C.c_int32),
                ("b_nominal", C.c_float), ("charge", C.c_float), ("grid_template", cdc_grid)]


class cdc_candidate(C.Structure):
    _fields_ = [("ix", C.c_int32), ("iy", C.c_int32), ("count", C.c_int32), ("r_bin", C.c_int32),
                ("theta0", C.c_float), ("px0", C.c_float), ("py0", C.c_float)]


class cdc_refine_params(C.Structure):
    _fields_ = [("n_iter", C.c_int32), ("sigma", C.c_float), ("scale", C.c_float * 5), ("checkpoint", C.c_int32)]


class cdc_scan_config(C.Structure):
    _fields_ = [("block", C.c_int32), ("chunk", C.c_int32), ("warp_seeds", C.c_int32)]


CDC_SCAN_CONFIGS = 4
SCAN_CONFIGS = [(256, 16), (256, 32), (128, 16), (128, 32)]   # the order cdc_tune_scan times them in

GRID_BYTES = C.sizeof(cdc_grid)            # 60
CAND_BYTES = C.sizeof(cdc_candidate)       # 28
GRID_DTYPE = np.dtype([("centre", np.float32, 5), ("step", np.float32, 5), ("n", np.int32, 5)])
CAND_DTYPE = np.dtype([("ix", np.int32), ("iy", np.int32), ("count", np.int32), ("r_bin", np.int32),
                       ("theta0", np.float32), ("px0", np.float32), ("py0", np.float32)])
assert GRID_DTYPE.itemsize == GRID_BYTES and CAND_DTYPE.itemsize == CAND_BYTES

_lib = None


def lib():
    """Load libcdc.so; raise if it is missing (the CUDA path has no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library {LIB_PATH} is missing: run `python -c \"import __graft_entry__ as g; "
                               f"g.build()\"` (nvcc, sm_103a) first")
        L = C.CDLL(LIB_PATH)
        vp, i32, i64 = C.c_void_p, C.c_int32, C.c_int64
        P = C.POINTER
        L.cdc_create.argtypes = [P(vp), C.c_int]
        L.cdc_destroy.argtypes = [vp]
        L.cdc_destroy.restype = None
        L.cdc_last_error.argtypes = [vp]
        L.cdc_last_error.restype = C.c_char_p
        L.cdc_load_geometry.argtypes = [vp, C.c_int, vp, vp, vp, vp, C.c_double, C.c_double, C.c_double]
        L.cdc_load_field.argtypes = [vp, C.c_int, C.c_float, vp, vp, C.c_int, C.c_int, C.c_float, C.c_float,
                                     C.c_float, C.c_float]
        L.cdc_reserve.argtypes = [vp, C.c_int, i64, i64]
        L.cdc_hough_seeds.argtypes = [vp, C.c_int, vp, vp, P(cdc_hough_params), vp, vp, vp, vp, vp, vp]
        L.cdc_candidate_grids.argtypes = [vp, C.c_int, P(cdc_hough_params), vp, vp, vp, vp]
        L.cdc_scan_seeds.argtypes = [vp, C.c_int, vp, vp, vp, vp, P(cdc_scan_params), vp, vp, vp, vp, vp, vp, vp, vp,
                                     vp, vp]
        L.cdc_refine_seeds.argtypes = [vp, C.c_int, vp, vp, C.c_int, vp, vp, vp, P(cdc_scan_params),
                                       P(cdc_refine_params), vp, vp, vp, vp, vp, vp]
        L.cdc_chi2_grad.argtypes = [vp, C.c_int, vp, vp, C.c_int, vp, vp, vp, P(cdc_scan_params), P(cdc_refine_params),
                                    vp, vp, vp, vp, vp]
        L.cdc_propagate.argtypes = [vp, C.c_int, vp, P(cdc_scan_params), C.c_int, C.c_int, C.c_int, vp, vp, vp, vp]
        L.cdc_kernel_timer.argtypes = [vp, C.c_int]
        L.cdc_scan_seeds_noalloc.argtypes = [vp, C.c_int, i64, vp, vp, vp, vp, P(cdc_scan_params), vp, vp, vp, vp, vp,
                                             vp, vp, vp, vp]
        L.cdc_kernel_time.argtypes = [vp, P(C.c_double), P(C.c_int64), vp, C.c_int]
        L.cdc_classification_counts.argtypes = [vp, C.c_int, vp, vp, vp, C.c_int, vp, vp]
        L.cdc_reserve_split.argtypes = [vp, C.c_int, C.c_int]
        L.cdc_extrapolate_turn.argtypes = [vp, C.c_int, vp, P(cdc_scan_params), C.c_int, vp, vp, vp]
        L.cdc_scan_seeds_split.argtypes = [vp, C.c_int, i64, vp, vp, vp, vp, P(cdc_scan_params), vp, vp, vp]
        L.cdc_common_hits.argtypes = [vp, C.c_int, vp, vp, vp, C.c_int, C.c_int, vp, vp]
        L.cdc_set_scan_config.argtypes = [vp, P(cdc_scan_config)]
        L.cdc_get_scan_config.argtypes = [vp, P(cdc_scan_config)]
        L.cdc_tune_scan.argtypes = [vp, C.c_int, vp, vp, vp, vp, P(cdc_scan_params), C.c_int, P(cdc_scan_config),
                                    vp, vp]
        L.cdc_fp32_peak.argtypes = [vp, C.c_int, P(C.c_double), P(C.c_double), vp]
        L.cdc_efficiency_purity.argtypes = [vp, C.c_int, vp, C.c_int, vp, vp, vp]
        for name in EXPORTS:
            if name not in ("cdc_destroy", "cdc_last_error"):
                getattr(L, name).restype = C.c_int
        _lib = L
    return _lib


class CdcError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


def _dev(t, dtype, name, device, nullable=False):
    """Device pointer of a torch tensor (contiguous, dtype, on the context's GPU)."""
    if t is None:
        if nullable:
            return None
        raise ValueError(f"{name} is required")
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA torch tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if t.device.index != device:
        raise ValueError(f"{name} is on cuda:{t.device.index}, the context on cuda:{device}")
    return t.data_ptr()


def _host(a, dtype):
    a = np.ascontiguousarray(a, dtype=dtype)
    return a, a.ctypes.data


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return int(getattr(stream, "cuda_stream", stream))


def scan_params(h=2.0, max_steps=1000, lam=4.0, max_partitions=1, direction=1, charge=-1.0, k=8, n_rounds=1,
                n_zoom=4, max_drift=8.0) -> cdc_scan_params:
    return cdc_scan_params(float(h), int(max_steps), float(lam), int(max_partitions), int(direction), float(charge),
                           int(k), int(n_rounds), int(n_zoom), float(max_drift))


def hough_params(n_bins=512, bin_um=2000, origin_um=-512000, n_r=32, r_min_um=200000, r_step_um=5000, n_phi=512,
                 target_um=100000, min_peak=8, max_cand=4, r_hist_half_um=2500, b_nominal=1.0, charge=-1.0,
                 grid_template=None) -> cdc_hough_params:
    p = cdc_hough_params(n_bins, bin_um, origin_um, n_r, r_min_um, r_step_um, n_phi, target_um, min_peak, max_cand,
                         r_hist_half_um, float(b_nominal), float(charge))
    if grid_template is not None:
        g = np.asarray(grid_template).view(GRID_DTYPE).reshape(-1)[0]
        p.grid_template.centre[:] = [float(x) for x in g["centre"]]
        p.grid_template.step[:] = [float(x) for x in g["step"]]
        p.grid_template.n[:] = [int(x) for x in g["n"]]
    return p


def refine_params(n_iter=5, sigma=0.2, scale=(1.0, 100.0, 10.0, 10.0, 10.0), checkpoint=128) -> cdc_refine_params:
    r = cdc_refine_params(int(n_iter), float(sigma))
    r.scale[:] = [float(s) for s in scale]
    r.checkpoint = int(checkpoint)
    return r


def grids_to_tensor(grids, device):
    """numpy GRID_DTYPE records -> CUDA uint8 tensor [n, 60] (the cdc_grid layout)."""
    import torch
    g = np.ascontiguousarray(np.asarray(grids, dtype=GRID_DTYPE).reshape(-1))
    return torch.from_numpy(g.view(np.uint8).reshape(-1, GRID_BYTES).copy()).to(device)


def tensor_to_grids(t):
    return np.ascontiguousarray(t.detach().cpu().numpy()).reshape(-1).view(GRID_DTYPE)


class Context:
    """One cdc_ctx on one CUDA device; methods carry the C entry-point names."""

    def __init__(self, device: int = 0):
        import torch
        self.L = lib()
        self.device = int(device)
        torch.cuda.init()
        h = C.c_void_p()
        rc = self.L.cdc_create(C.byref(h), self.device)
        if rc != 0:
            raise CdcError(rc, f"cdc_create(device={device}) failed")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.L.cdc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc):
        if rc != 0:
            raise CdcError(rc, self.L.cdc_last_error(self.h).decode())
        return rc

    # -------------------------------------------------------------- loading
    def cdc_load_geometry(self, R, alpha, N, phi_off, z_half, R0, R_out):
        R, pR = _host(R, np.float64)
        al, pa = _host(alpha, np.float64)
        n, pn = _host(N, np.int32)
        ph, pp = _host(phi_off, np.float64)
        return self._check(self.L.cdc_load_geometry(self.h, int(R.size), pR, pa, pn, pp, float(z_half), float(R0),
                                                    float(R_out)))

    def cdc_load_field(self, kind, b0, bz=None, br=None, nr=0, nz=0, r_min=0.0, z_min=0.0, dr=1.0, dz=1.0):
        if kind == 0:
            return self._check(self.L.cdc_load_field(self.h, 0, float(b0), None, None, 0, 0, 0.0, 0.0, 1.0, 1.0))
        bz, pz = _host(bz, np.float32)
        br, pr = _host(br, np.float32)
        return self._check(self.L.cdc_load_field(self.h, 1, float(b0), pz, pr, int(nr), int(nz), float(r_min),
                                                 float(z_min), float(dr), float(dz)))

    def cdc_reserve(self, max_events, max_seeds, max_hits):
        return self._check(self.L.cdc_reserve(self.h, int(max_events), int(max_seeds), int(max_hits)))

    # -------------------------------------------------------------- compute
    def cdc_hough_seeds(self, n_events, hit_off, wire_id, params, acc, cand, n_cand, grid_out, flags, stream=None):
        import torch
        d = self.device
        return self._check(self.L.cdc_hough_seeds(
            self.h, int(n_events), _dev(hit_off, torch.int32, "hit_off", d), _dev(wire_id, torch.int32, "wire_id", d),
            C.byref(params), _dev(acc, torch.int32, "acc", d), _dev(cand, torch.uint8, "cand", d),
            _dev(n_cand, torch.int32, "n_cand", d), _dev(grid_out, torch.uint8, "grid_out", d, True),
            _dev(flags, torch.int32, "flags", d), _stream(stream)))

    def cdc_candidate_grids(self, n_events, params, cand, n_cand, grids, stream=None):
        import torch
        d = self.device
        return self._check(self.L.cdc_candidate_grids(
            self.h, int(n_events), C.byref(params), _dev(cand, torch.uint8, "cand", d),
            _dev(n_cand, torch.int32, "n_cand", d), _dev(grids, torch.uint8, "grids", d), _stream(stream)))

    def cdc_scan_seeds(self, n_events, hit_off, wire_id, drift, grids, params, E, topk0, best_E, best_seed, hit_part,
                       hit_res2, zoom_grids, flags, steps, stream=None):
        import torch
        d = self.device
        return self._check(self.L.cdc_scan_seeds(
            self.h, int(n_events), _dev(hit_off, torch.int32, "hit_off", d), _dev(wire_id, torch.int32, "wire_id", d),
            _dev(drift, torch.float32, "drift", d), _dev(grids, torch.uint8, "grids", d), C.byref(params),
            _dev(E, torch.float32, "E", d, True), _dev(topk0, torch.int64, "topk0", d, True),
            _dev(best_E, torch.float32, "best_E", d), _dev(best_seed, torch.float32, "best_seed", d),
            _dev(hit_part, torch.int8, "hit_part", d, True), _dev(hit_res2, torch.float32, "hit_res2", d, True),
            _dev(zoom_grids, torch.uint8, "zoom_grids", d, True), _dev(flags, torch.int32, "flags", d),
            _dev(steps, torch.int64, "steps", d, True), _stream(stream)))

    def cdc_refine_seeds(self, n_seeds, seed_event, seeds, n_events, hit_off, wire_id, drift, scan, params,
                         seeds_out, chi2, grad, n_used, flags, stream=None):
        import torch
        d = self.device
        return self._check(self.L.cdc_refine_seeds(
            self.h, int(n_seeds), _dev(seed_event, torch.int32, "seed_event", d), _dev(seeds, torch.float32, "seeds", d),
            int(n_events), _dev(hit_off, torch.int32, "hit_off", d), _dev(wire_id, torch.int32, "wire_id", d),
            _dev(drift, torch.float32, "drift", d), C.byref(scan), C.byref(params),
            _dev(seeds_out, torch.float32, "seeds_out", d), _dev(chi2, torch.float64, "chi2", d),
            _dev(grad, torch.float32, "grad", d, True), _dev(n_used, torch.int32, "n_used", d, True),
            _dev(flags, torch.int32, "flags", d), _stream(stream)))

    def cdc_chi2_grad(self, n_seeds, seed_event, seeds, n_events, hit_off, wire_id, drift, scan, params, chi2, grad,
                      n_used, flags, stream=None):
        import torch
        d = self.device
        return self._check(self.L.cdc_chi2_grad(
            self.h, int(n_seeds), _dev(seed_event, torch.int32, "seed_event", d), _dev(seeds, torch.float32, "seeds", d),
            int(n_events), _dev(hit_off, torch.int32, "hit_off", d), _dev(wire_id, torch.int32, "wire_id", d),
            _dev(drift, torch.float32, "drift", d), C.byref(scan), C.byref(params),
            _dev(chi2, torch.float64, "chi2", d), _dev(grad, torch.float32, "grad", d, True),
            _dev(n_used, torch.int32, "n_used", d, True), _dev(flags, torch.int32, "flags", d), _stream(stream)))

    def cdc_scan_seeds_noalloc(self, n_events, n_seeds, hit_off, wire_id, drift, grids, params, E, topk0, best_E,
                               best_seed, hit_part, hit_res2, flags, steps, stream=None):
        """Single-round scan whose workspace is a fixed device array of the
        library (for callers that must not allocate device memory)."""
        import torch
        d = self.device
        return self._check(self.L.cdc_scan_seeds_noalloc(
            self.h, int(n_events), int(n_seeds), _dev(hit_off, torch.int32, "hit_off", d),
            _dev(wire_id, torch.int32, "wire_id", d), _dev(drift, torch.float32, "drift", d),
            _dev(grids, torch.uint8, "grids", d), C.byref(params), _dev(E, torch.float32, "E", d, True),
            _dev(topk0, torch.int64, "topk0", d, True), _dev(best_E, torch.float32, "best_E", d),
            _dev(best_seed, torch.float32, "best_seed", d), _dev(hit_part, torch.int8, "hit_part", d, True),
            _dev(hit_res2, torch.float32, "hit_res2", d, True), _dev(flags, torch.int32, "flags", d),
            _dev(steps, torch.int64, "steps", d, True), _stream(stream)))

    def cdc_classification_counts(self, n_events, hit_off, hit_part, truth_part, n_part, counts, stream=None):
        import torch
        d = self.device
        return self._check(self.L.cdc_classification_counts(
            self.h, int(n_events), _dev(hit_off, torch.int32, "hit_off", d), _dev(hit_part, torch.int8, "hit_part", d),
            _dev(truth_part, torch.int8, "truth_part", d), int(n_part), _dev(counts, torch.int32, "counts", d),
            _stream(stream)))

    def cdc_efficiency_purity(self, n_sets, counts, n_part, eff, pur, stream=None):
        import torch
        d = self.device
        return self._check(self.L.cdc_efficiency_purity(
            self.h, int(n_sets), _dev(counts, torch.int32, "counts", d), int(n_part),
            _dev(eff, torch.float32, "eff", d), _dev(pur, torch.float32, "pur", d), _stream(stream)))

    def cdc_extrapolate_turn(self, n_seeds, seeds, scan, direction, seeds_out, status, stream=None):
        import torch
        d = self.device
        return self._check(self.L.cdc_extrapolate_turn(
            self.h, int(n_seeds), _dev(seeds, torch.float32, "seeds", d), C.byref(scan), int(direction),
            _dev(seeds_out, torch.float32, "seeds_out", d), _dev(status, torch.int32, "status", d), _stream(stream)))

    def cdc_reserve_split(self, chunk, max_steps):
        return self._check(self.L.cdc_reserve_split(self.h, int(chunk), int(max_steps)))

    def cdc_scan_seeds_split(self, n_events, n_seeds, hit_off, wire_id, drift, grids, params, E, flags, stream=None):
        """The paper's two-kernel scan (record states, then DOCA per hit): scores only."""
        import torch
        d = self.device
        return self._check(self.L.cdc_scan_seeds_split(
            self.h, int(n_events), int(n_seeds), _dev(hit_off, torch.int32, "hit_off", d),
            _dev(wire_id, torch.int32, "wire_id", d), _dev(drift, torch.float32, "drift", d),
            _dev(grids, torch.uint8, "grids", d), C.byref(params), _dev(E, torch.float32, "E", d),
            _dev(flags, torch.int32, "flags", d), _stream(stream)))

    def cdc_common_hits(self, n_events, hit_off, part_a, part_b, pa, pb, n_common, stream=None):
        import torch
        d = self.device
        return self._check(self.L.cdc_common_hits(
            self.h, int(n_events), _dev(hit_off, torch.int32, "hit_off", d), _dev(part_a, torch.int8, "part_a", d),
            _dev(part_b, torch.int8, "part_b", d), int(pa), int(pb), _dev(n_common, torch.int32, "n_common", d),
            _stream(stream)))

    def cdc_set_scan_config(self, block, chunk, warp_seeds=None):
        """Launch shape of later scans; warp_seeds None keeps the current value."""
        if warp_seeds is None:
            warp_seeds = self.cdc_get_scan_config()[2]
        return self._check(self.L.cdc_set_scan_config(
            self.h, C.byref(cdc_scan_config(int(block), int(chunk), int(warp_seeds)))))

    def cdc_get_scan_config(self):
        """(block, chunk, warp_seeds) of later scans."""
        cfg = cdc_scan_config()
        self._check(self.L.cdc_get_scan_config(self.h, C.byref(cfg)))
        return cfg.block, cfg.chunk, cfg.warp_seeds

    def cdc_tune_scan(self, n_events, hit_off, wire_id, drift, grids, params, reps=3, stream=None):
        """Times the coarse round under every launch shape and keeps the fastest:
        ((block, chunk), [median ms per shape in SCAN_CONFIGS order])."""
        import torch
        d = self.device
        best = cdc_scan_config()
        ms = np.zeros(CDC_SCAN_CONFIGS, np.float32)
        self._check(self.L.cdc_tune_scan(
            self.h, int(n_events), _dev(hit_off, torch.int32, "hit_off", d), _dev(wire_id, torch.int32, "wire_id", d),
            _dev(drift, torch.float32, "drift", d), _dev(grids, torch.uint8, "grids", d), C.byref(params), int(reps),
            C.byref(best), ms.ctypes.data, _stream(stream)))
        return (best.block, best.chunk), [float(x) for x in ms]

    def cdc_kernel_timer(self, enable):
        """enable: False/0 off, True/1 on, 2 on for a scan captured into a CUDA graph."""
        return self._check(self.L.cdc_kernel_timer(self.h, int(enable)))

    def cdc_fp32_peak(self, iters=4096, stream=None):
        """(TFLOP/s, ms) of the FP32 FMA throughput kernel (synchronous)."""
        tf, ms = C.c_double(0), C.c_double(0)
        self._check(self.L.cdc_fp32_peak(self.h, int(iters), C.byref(tf), C.byref(ms), _stream(stream)))
        return tf.value, ms.value

    def cdc_kernel_time(self, cap=2048):
        """(summed device ms, launches, per-launch ms) of the timed scan-kernel launches."""
        ms, n = C.c_double(0), C.c_int64(0)
        per = np.zeros(cap, np.float32)
        self._check(self.L.cdc_kernel_time(self.h, C.byref(ms), C.byref(n), per.ctypes.data, int(cap)))
        return ms.value, n.value, per[:min(n.value, cap)].copy()

    def cdc_propagate(self, n_seeds, seeds, params, every, n_rec, precision, pos, n_steps, path, stream=None):
        import torch
        d = self.device
        return self._check(self.L.cdc_propagate(
            self.h, int(n_seeds), _dev(seeds, torch.float32, "seeds", d), C.byref(params), int(every), int(n_rec),
            int(precision), _dev(pos, torch.float64, "pos", d), _dev(n_steps, torch.int32, "n_steps", d),
            _dev(path, torch.float64, "path", d), _stream(stream)))
