"""Helpers of the GPU parity tests: run the CUDA path through the C ABI and
the FP64 oracle on the same seeded synthetic inputs."""
from __future__ import annotations

import numpy as np

import cdc_synth as S
import oracle as O

E_REL = 1e-3          # score tolerance (relative)
MARGIN = 1e-3         # mm: seeds/hits this close to a discrete decision are compared loosely


def tracker(g, f, max_events=8, max_seeds=1 << 18, max_hits=1 << 16):
    import paper_1908_01949_gb300 as cdc
    return cdc.Tracker(g, f, device=0, max_events=max_events, max_seeds=max_seeds, max_hits=max_hits)


def oracle_params(p):
    return O.scan_params(h=p.h, max_steps=p.max_steps, lam=p.lambda_, max_partitions=p.max_partitions,
                         direction=p.direction, charge=p.charge)


def compare_scores(E_gpu, ref, rel=E_REL, margin=MARGIN):
    """Element-wise E parity; seeds whose trace passes within `margin` mm of a
    stop/partition boundary (where FP32 and FP64 may take a different
    discrete decision) are excluded and counted."""
    E_gpu = np.asarray(E_gpu, np.float64)
    ok = ref["margin"] >= margin
    d = np.abs(E_gpu - ref["E"]) / np.maximum(ref["E"], 1e-30)
    bad = np.flatnonzero(ok & ~(d <= rel))
    return bad, int((~ok).sum()), float(d[ok].max()) if ok.any() else 0.0


def check_topk(idx_gpu, E_ref, k, rel=E_REL):
    """The GPU's top-k index set equals the oracle's up to seeds whose oracle
    score lies within `rel` of the k-th best score (ties within tolerance)."""
    order = O.topk(E_ref, k)
    kth = E_ref[order[-1]]
    a, b = set(int(i) for i in idx_gpu), set(int(i) for i in order)
    for i in a ^ b:
        if abs(E_ref[i] - kth) > rel * kth:
            return False, (sorted(a - b), sorted(b - a))
    return True, None


def keys_to_index(keys):
    k = np.asarray(keys).view(np.uint64)
    return (k & np.uint64(0xffffffff)).astype(np.int64), (k >> np.uint64(32)).astype(np.uint32).view(np.float32)
