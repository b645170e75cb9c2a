"""The event loop over turn partitions (arXiv:1908.01949 sec. 2.3, Fig. 7).

A turn is found by a scan of the unclassified hits, its best seed refined by
Gauss-Newton (kept only where chi^2 decreases), and the seed of the
neighbouring turn predicted by extrapolating
the refined track to the neighbouring crossing of the R0 cylinder
(cdc_extrapolate_turn; the paper extrapolates backwards, here both ways, since
the first turn found need not be the last).  The neighbour is then scanned on
a grid around the prediction whose longitudinal span follows the resolution
the paper quotes for the predicted (z0, pz0), 2.6 cm and 1.7 MeV/c, over the
hits not yet classified; the loop ends when fewer than ten hits remain
unclassified, when a scan classifies fewer than ten, or when the track leaves
the chamber.  Every step runs in the library's kernels; the host only selects
the remaining hits between the calls.
"""
from __future__ import annotations

import numpy as np

from ._lib import GRID_DTYPE, grids_to_tensor, scan_params

SIGMA_Z0, SIGMA_PZ0 = 26.0, 1.7        # resolution of the predicted longitudinal seed [mm, MeV/c] (sec. 2.3)
MIN_HITS = 10                          # the loop stops below ten unclassified hits (sec. 2.3)
UNCLASSIFIED = -128


def neighbour_grid(seed, n=(5, 13, 5, 5, 13), transverse_step=(0.002, 0.5, 0.5)):
    """Seed grid around a predicted seed: (z0, pz0) over +-3 sigma in steps of
    sigma / 2, (theta0, px0, py0) over +-2 fine steps."""
    g = np.zeros(1, dtype=GRID_DTYPE)
    g["centre"][0] = np.asarray(seed, dtype=np.float64)
    g["step"][0] = (transverse_step[0], SIGMA_Z0 / 2, transverse_step[1], transverse_step[2], SIGMA_PZ0 / 2)
    g["n"][0] = n
    return g


def event_loop(tracker, wire_id, drift, first_grid, params, refine_params, max_turns=8, min_hits=MIN_HITS,
               grid_n=(5, 13, 5, 5, 13)):
    """Classify the hits of one event into turns.  Returns (labels, seeds):
    labels[h] = turn index relative to the first turn found (0; -1 the turn
    before it, +1 the one after) or UNCLASSIFIED; seeds[k] = refined seed
    (float32[5]) of turn k.  grid_n: points per axis of the neighbour grids."""
    torch = tracker.torch
    wid = np.asarray(wire_id, np.int32)
    dr = np.asarray(drift, np.float32)
    labels = np.full(wid.size, UNCLASSIFIED, np.int32)
    p1 = scan_params(h=params.h, max_steps=params.max_steps, lam=params.lambda_, max_partitions=1,
                     direction=params.direction, charge=params.charge, k=params.k, n_rounds=params.n_rounds,
                     n_zoom=params.n_zoom, max_drift=params.max_drift)

    def remaining():
        idx = np.flatnonzero(labels == UNCLASSIFIED)
        return idx, tracker.events_to_device([0, idx.size], wid[idx], dr[idx])

    def find_turn(grid):
        """Scan the unclassified hits; (hits of partition 0, refined seed) or None."""
        idx, (off, w, d) = remaining()
        if idx.size < min_hits:
            return None
        out = tracker.scan(off, w, d, grids_to_tensor(grid, tracker.dev), p1)
        hp = out["hit_part"][:idx.size].cpu().numpy()
        found = idx[hp == 0]
        if found.size < min_hits:
            return None
        best = out["best_seed"][0, :1].contiguous()
        if refine_params is None:
            return found, best
        se = torch.zeros(1, dtype=torch.int32, device=tracker.dev)
        r = tracker.refine(se, best, off, w, d, p1, refine_params, want_grad=False)
        c0 = tracker.chi2_grad(se, best, off, w, d, p1, refine_params, want_grad=False)["chi2"]
        # Gauss-Newton without a line search can overshoot along a weakly constrained
        # direction of one turn: keep the refined seed only where chi^2 went down
        ok = bool(torch.isfinite(r["seeds"]).all()) and float(r["chi2"][0]) < float(c0[0])
        return found, (r["seeds"] if ok else best)

    seeds = {}
    first = find_turn(first_grid)
    if first is None:
        return labels, seeds
    labels[first[0]] = 0
    seeds[0] = first[1]
    for direction in (-1, 1):
        cur, k = seeds[0], 0
        while abs(k) < max_turns:
            pred, status = tracker.extrapolate_turn(cur, p1, direction)
            if int(status[0]) != 0:
                break
            turn = find_turn(neighbour_grid(pred[0].cpu().numpy(), n=grid_n))
            if turn is None:
                break
            k += direction
            labels[turn[0]] = k
            seeds[k] = cur = turn[1]
    return labels, {k: v[0].cpu().numpy() for k, v in seeds.items()}


def findable_truth(truth_part, min_hits=MIN_HITS):
    """Truth turn labels with turns of fewer than min_hits hits (which the loop
    never takes as a turn) counted as noise, for Eqs. 2-3."""
    t = np.asarray(truth_part).astype(np.int64)
    n = np.bincount(t[t >= 0], minlength=1) if np.any(t >= 0) else np.zeros(1, np.int64)
    small = np.flatnonzero(n < min_hits)
    return np.where(np.isin(t, small), -1, t).astype(np.int8)


def align_to_truth(labels, truth_part):
    """Relative turn labels -> truth turn numbers: the first turn found is the
    truth turn most of its hits come from; unclassified hits -> -1."""
    lab = np.asarray(labels)
    truth = np.asarray(truth_part)
    first = truth[(lab == 0) & (truth >= 0)]
    if first.size == 0:
        return np.full(lab.size, -1, np.int8)
    t0 = int(np.bincount(first).argmax())
    out = np.where(lab == UNCLASSIFIED, -1, lab + t0)
    return np.where((out >= -1) & (out < 127), out, -1).astype(np.int8)
