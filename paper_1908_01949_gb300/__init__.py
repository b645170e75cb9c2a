"""GB300 seed-scanning track finder for a cylindrical drift chamber
(arXiv:1908.01949, "GPU Tracking in the COMET Phase-I Cylindrical Drift
Chamber").

The compute path is the CUDA library libcdc.so behind the C ABI of
include/cdc.h; `Context` exposes its entry points under the same names
(argument marshalling only) and `Tracker` adds output allocation around them.
PyTorch provides device memory, streams and autograd.
"""
from __future__ import annotations

import numpy as np

from ._lib import (CAND_DTYPE, CDC_MAX_K, CDC_MAX_ZOOM, EXPORTS, FLAG_BAD_HIT, FLAG_DOCA_ZERO, FLAG_EMPTY,
                   FLAG_FOUND_OVERFLOW, FLAG_LOST_HIT, FLAG_NOT_SPD, FLAG_STEP_CAP, GRID_BYTES, GRID_DTYPE, CdcError,
                   Context, grids_to_tensor, hough_params, lib, refine_params, scan_params, tensor_to_grids)

__all__ = ["Context", "Tracker", "CdcError", "chi2", "scan_params", "hough_params", "refine_params", "grids_to_tensor",
           "tensor_to_grids", "GRID_DTYPE", "CAND_DTYPE", "EXPORTS", "lib"]


class Tracker:
    """A loaded context plus output allocation for the five calls."""

    def __init__(self, geometry, field, device: int = 0, max_events: int = 1, max_seeds: int = 1 << 20,
                 max_hits: int = 1 << 16):
        import torch
        self.torch = torch
        self.device = device
        self.dev = torch.device("cuda", device)
        self.ctx = Context(device)
        g = geometry
        self.ctx.cdc_load_geometry(g.R, g.alpha, g.N, g.phi_off, g.z_half, g.R0, g.R_out)
        if field.kind == 0:
            self.ctx.cdc_load_field(0, field.B0)
        else:
            self.ctx.cdc_load_field(1, field.B0, field.bz, field.br, field.bz.shape[0], field.bz.shape[1],
                                    field.r_min, field.z_min, field.dr, field.dz)
        self.reserve(max_events, max_seeds, max_hits)

    def reserve(self, max_events, max_seeds, max_hits):
        self.ctx.cdc_reserve(max_events, max_seeds, max_hits)
        self.max_events = max_events

    def events_to_device(self, hit_off, wire_id, drift):
        t = self.torch
        return (t.as_tensor(np.asarray(hit_off, np.int32), device=self.dev),
                t.as_tensor(np.asarray(wire_id, np.int32), device=self.dev),
                t.as_tensor(np.asarray(drift, np.float32), device=self.dev))

    def hough(self, hit_off, wire_id, params, stream=None):
        """Circle Hough of every event (cdc_hough_seeds): accumulators, candidates,
        the top candidate's seed grid and flags.  The peak search uses this
        tracker's workspace, so the events may number at most its max_events."""
        t = self.torch
        ne = int(hit_off.numel()) - 1
        nb = params.n_bins
        out = dict(acc=t.empty((ne, nb, nb), dtype=t.int32, device=self.dev),
                   cand=t.empty((ne, params.max_cand, CAND_DTYPE.itemsize), dtype=t.uint8, device=self.dev),
                   n_cand=t.empty(ne, dtype=t.int32, device=self.dev),
                   grid=t.empty((ne, GRID_BYTES), dtype=t.uint8, device=self.dev),
                   flags=t.empty(ne, dtype=t.int32, device=self.dev))
        self.ctx.cdc_hough_seeds(ne, hit_off, wire_id, params, out["acc"], out["cand"], out["n_cand"], out["grid"],
                                 out["flags"], stream)
        return out

    def candidate_grids(self, hough_out, params, stream=None):
        """One seed grid per candidate slot of a hough() result: [n_events * max_cand]
        grid records (slot-major within each event; zero seeds past the event's
        candidates)."""
        ne = int(hough_out["n_cand"].numel())
        grids = self.torch.empty((ne * params.max_cand, GRID_BYTES), dtype=self.torch.uint8, device=self.dev)
        self.ctx.cdc_candidate_grids(ne, params, hough_out["cand"], hough_out["n_cand"], grids, stream)
        return grids

    def scan(self, hit_off, wire_id, drift, grids, params, want_E=False, want_topk0=True, want_hits=True,
             want_zoom_grids=False, n_seeds=None, stream=None):
        t = self.torch
        ne = int(hit_off.numel()) - 1
        K = params.k
        out = dict(best_E=t.empty((ne, K), dtype=t.float32, device=self.dev),
                   best_seed=t.empty((ne, K, 5), dtype=t.float32, device=self.dev),
                   flags=t.empty(ne, dtype=t.int32, device=self.dev),
                   steps=t.zeros(params.n_rounds, dtype=t.int64, device=self.dev))
        out["E"] = t.empty(int(n_seeds), dtype=t.float32, device=self.dev) if want_E else None
        out["topk0"] = t.empty((ne, K), dtype=t.int64, device=self.dev) if want_topk0 else None
        nh = int(wire_id.numel())
        out["hit_part"] = t.empty(max(nh, 1), dtype=t.int8, device=self.dev) if want_hits else None
        out["hit_res2"] = t.empty(max(nh, 1), dtype=t.float32, device=self.dev) if want_hits else None
        nz = params.n_zoom if params.n_rounds > 1 else 1
        out["zoom_grids"] = (t.empty((params.n_rounds, ne, nz, GRID_BYTES), dtype=t.uint8, device=self.dev)
                             if want_zoom_grids else None)
        self.ctx.cdc_scan_seeds(ne, hit_off, wire_id, drift, grids, params, out["E"], out["topk0"], out["best_E"],
                                out["best_seed"], out["hit_part"], out["hit_res2"], out["zoom_grids"], out["flags"],
                                out["steps"], stream)
        return out

    def tune(self, hit_off, wire_id, drift, grids, params, reps=3, stream=None):
        """Autotune the scan kernel's launch shape on these events (synchronous);
        later scans on this tracker use the fastest shape."""
        ne = int(hit_off.numel()) - 1
        return self.ctx.cdc_tune_scan(ne, hit_off, wire_id, drift, grids, params, reps, stream)

    def classification_counts(self, hit_off, hit_part, truth_part, n_part, stream=None):
        """Per-event counts [n_events, n_part + 1, n_part + 1] of (truth partition,
        classified partition) pairs, index 0 = -1 (sec. 3.1, Eqs. 2-3)."""
        t = self.torch
        ne = int(hit_off.numel()) - 1
        counts = t.empty((ne, n_part + 1, n_part + 1), dtype=t.int32, device=self.dev)
        self.ctx.cdc_classification_counts(ne, hit_off, hit_part, truth_part, n_part, counts, stream)
        return counts

    def efficiency_purity(self, counts, stream=None):
        """Eqs. 2-3 (sec. 3.1) from device counts [..., n+1, n+1] (as
        classification_counts writes them), summed over the leading axes:
        (eff [n], pur [n]) float32 device tensors, NaN for a zero denominator."""
        t = self.torch
        c = counts.reshape(-1, counts.shape[-2], counts.shape[-1]).contiguous()
        n = int(c.shape[-1]) - 1
        eff = t.empty(n, dtype=t.float32, device=self.dev)
        pur = t.empty(n, dtype=t.float32, device=self.dev)
        self.ctx.cdc_efficiency_purity(int(c.shape[0]), c, n, eff, pur, stream)
        return eff, pur

    def extrapolate_turn(self, seeds, params, direction, stream=None):
        """Seeds of the previous (-1) or next (+1) turn partition (sec. 2.3):
        (seeds [n, 5] float32, status [n] int32)."""
        t = self.torch
        n = int(seeds.shape[0])
        out = t.empty((n, 5), dtype=t.float32, device=self.dev)
        st = t.empty(n, dtype=t.int32, device=self.dev)
        self.ctx.cdc_extrapolate_turn(n, seeds, params, direction, out, st, stream)
        return out, st

    def common_hits(self, hit_off, part_a, part_b, pa=0, pb=0, stream=None):
        """N_c per event: hits classified pa by one scan and pb by the other
        (sec. 2.2, bidirectional scan)."""
        t = self.torch
        ne = int(hit_off.numel()) - 1
        n = t.empty(ne, dtype=t.int32, device=self.dev)
        self.ctx.cdc_common_hits(ne, hit_off, part_a, part_b, pa, pb, n, stream)
        return n

    def propagate(self, seeds, params, every, n_rec, precision=0, stream=None):
        t = self.torch
        n = int(seeds.shape[0])
        out = dict(pos=t.empty((n, n_rec, 3), dtype=t.float64, device=self.dev),
                   n_steps=t.empty(n, dtype=t.int32, device=self.dev),
                   path=t.empty(n, dtype=t.float64, device=self.dev))
        self.ctx.cdc_propagate(n, seeds, params, every, n_rec, precision, out["pos"], out["n_steps"], out["path"],
                               stream)
        return out

    def refine(self, seed_event, seeds, hit_off, wire_id, drift, scan, params, want_grad=True, stream=None):
        t = self.torch
        n = int(seeds.shape[0])
        out = dict(seeds=t.empty((n, 5), dtype=t.float32, device=self.dev),
                   chi2=t.empty(n, dtype=t.float64, device=self.dev),
                   grad=t.empty((n, 5), dtype=t.float32, device=self.dev) if want_grad else None,
                   n_used=t.empty(n, dtype=t.int32, device=self.dev),
                   flags=t.empty(n, dtype=t.int32, device=self.dev))
        self.ctx.cdc_refine_seeds(n, seed_event, seeds, int(hit_off.numel()) - 1, hit_off, wire_id, drift, scan,
                                  params, out["seeds"], out["chi2"], out["grad"], out["n_used"], out["flags"], stream)
        return out

    def chi2_grad(self, seed_event, seeds, hit_off, wire_id, drift, scan, params, want_grad=True, stream=None):
        t = self.torch
        n = int(seeds.shape[0])
        out = dict(chi2=t.empty(n, dtype=t.float64, device=self.dev),
                   grad=t.empty((n, 5), dtype=t.float32, device=self.dev) if want_grad else None,
                   n_used=t.empty(n, dtype=t.int32, device=self.dev),
                   flags=t.empty(n, dtype=t.int32, device=self.dev))
        self.ctx.cdc_chi2_grad(n, seed_event, seeds, int(hit_off.numel()) - 1, hit_off, wire_id, drift, scan, params,
                               out["chi2"], out["grad"], out["n_used"], out["flags"], stream)
        return out


_CHI2_FN = None


def _chi2_function():
    """torch.autograd.Function: chi^2 of the assigned hits' DOCA residuals of
    each seed (forward) and d chi^2 / d seed from the adjoint RKN kernel
    (backward), both from one cdc_chi2_grad call."""
    global _CHI2_FN
    if _CHI2_FN is None:
        import torch

        class Chi2(torch.autograd.Function):
            @staticmethod
            def forward(ctx, seeds, tracker, seed_event, hit_off, wire_id, drift, scan, params):
                out = tracker.chi2_grad(seed_event, seeds.detach().contiguous(), hit_off, wire_id, drift, scan,
                                        params, want_grad=True)
                ctx.save_for_backward(out["grad"])
                ctx.extra = (out["n_used"], out["flags"])
                return out["chi2"]

            @staticmethod
            def backward(ctx, g):
                (grad,) = ctx.saved_tensors
                return (g.to(grad.dtype)[:, None] * grad,) + (None,) * 7

        _CHI2_FN = Chi2
    return _CHI2_FN


def chi2(tracker, seed_event, seeds, hit_off, wire_id, drift, scan, params):
    """Differentiable chi^2 [n_seeds] (float64) of seeds [n_seeds, 5] (float32,
    may require grad); the hit assignment of each seed is taken at the seed
    itself, as in cdc_chi2_grad."""
    return _chi2_function().apply(seeds, tracker, seed_event, hit_off, wire_id, drift, scan, params)


def decode_candidates(t):
    return np.ascontiguousarray(t.detach().cpu().numpy()).reshape(-1).view(CAND_DTYPE)
