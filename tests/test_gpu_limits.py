"""GPU behaviour at the scan's limits, against the FP64 oracle: the step cap,
the largest top-K list, and a seed that scores more wires than its record
holds."""
import numpy as np
import pytest

import cdc_synth as S
import oracle as O
from tests.gpu_util import check_topk, compare_scores, keys_to_index, oracle_params, tracker

CDC_MAX_FOUND = 128   # record entries of a seed (include/cdc.h)

pytestmark = pytest.mark.gpu


def _scan(tr, ev, grid, p):
    import torch
    import paper_1908_01949_gb300 as cdc
    n = int(np.prod(grid["n"][0]))
    off, wid, dr = tr.events_to_device([0, ev.wire_id.size], ev.wire_id, ev.drift)
    out = tr.scan(off, wid, dr, cdc.grids_to_tensor(grid, tr.dev), p, want_E=True, n_seeds=n)
    torch.cuda.synchronize()
    return out


def test_step_cap_is_flagged_and_scored_like_the_oracle():
    """max_steps = 100 stops every track early: the event carries the step-cap
    flag, every score follows the oracle with the same cap (the track end is a
    minimum where the distance still shrinks) and the step total is exact."""
    import paper_1908_01949_gb300 as cdc
    g, f, ev, grid = S.cfg1_case(5)
    n = int(np.prod(grid["n"][0]))
    tr = tracker(g, f)
    p = cdc.scan_params(h=2.0, max_steps=100, lam=4.0, max_partitions=1, k=8, n_rounds=1)
    out = _scan(tr, ev, grid, p)
    ref = O.scan(g, f, ev.wire_id, ev.drift.astype(np.float64), O.grid_values(grid), oracle_params(p))
    assert int(out["flags"][0]) & cdc.FLAG_STEP_CAP
    assert np.all(ref["n_steps"] <= 100) and int(out["steps"][0]) == int(ref["n_steps"].sum())
    bad, excluded, worst = compare_scores(out["E"].cpu().numpy(), ref)
    assert bad.size == 0, (bad[:10], worst)
    assert excluded < 0.02 * n


def test_largest_top_k_matches_oracle():
    """k = 64 (the largest list): the 64 best of 12600 seeds are the oracle's up
    to ties, in ascending order of the GPU's own scores."""
    import paper_1908_01949_gb300 as cdc
    g, f, ev, grid = S.cfg1_case(0)
    grid["n"][0] = (10, 5, 6, 6, 7)
    tr = tracker(g, f)
    p = cdc.scan_params(h=2.0, max_steps=1000, lam=4.0, max_partitions=1, k=cdc.CDC_MAX_K, n_rounds=1)
    out = _scan(tr, ev, grid, p)
    ref = O.scan(g, f, ev.wire_id, ev.drift.astype(np.float64), O.grid_values(grid), oracle_params(p))
    idx, Ek = keys_to_index(out["topk0"][0].cpu().numpy())
    assert idx.size == 64 and np.all(np.diff(Ek) >= 0)
    ok, diff = check_topk(idx, ref["E"], 64)
    assert ok, diff


def test_record_overflow_is_flagged():
    """Three turns of 137 signal hits at lambda = 9 mm^2: seeds near the truth
    score 133-137 wires below lambda, more than the 128 entries their record
    holds (one per wire with a pass closer than drift + sqrt(lambda)), and the
    event carries the overflow flag; followed over one turn only (about 65 such
    wires) the same seeds raise no flag and score like the oracle."""
    import paper_1908_01949_gb300 as cdc
    fm = S.solenoid_map()
    g, f, ev = S.cfg2_case(7, fm, occupancy=0.10)
    grid = S.make_grid(ev.truth_seeds[0], (0.001, 2.0, 0.2, 0.2, 0.2), (3, 1, 3, 3, 1))
    seeds = O.grid_values(grid)
    tr = tracker(g, f)
    for parts, overflow in ((3, True), (1, False)):
        p = cdc.scan_params(h=2.0, max_steps=3500, lam=9.0, max_partitions=parts, k=8, n_rounds=1)
        ref = O.scan(g, f, ev.wire_id, ev.drift.astype(np.float64), seeds, oracle_params(p), per_hit=True)
        below = ((ref["hit_res2"] < 9.0) & (ref["hit_part"] >= 0)).sum(1)
        assert (below.max() > CDC_MAX_FOUND) == overflow, below
        out = _scan(tr, ev, grid, p)
        flagged = bool(int(out["flags"][0]) & cdc.FLAG_FOUND_OVERFLOW)
        assert flagged == overflow
        if not overflow:
            bad, _, worst = compare_scores(out["E"].cpu().numpy(), ref)
            assert bad.size == 0, (bad[:10], worst)


def test_grids_beyond_the_reserved_capacity_scan_nothing():
    """Two events whose grids (2 x 4000 seeds) exceed a workspace reserved for
    3888 scores: without a caller score buffer the call scans nothing and flags
    both events empty (no best seed, no hit classes); with the caller's buffer
    for the coarse scores the same call scans normally and equals a tracker
    with room to spare, bit for bit."""
    import torch
    import paper_1908_01949_gb300 as cdc
    g, f, ev0, grid0 = S.cfg1_case(6)
    _, _, ev1, grid1 = S.cfg1_case(7)
    grids = np.concatenate([grid0, grid1])
    n = 2 * int(np.prod(grid0["n"][0]))
    off = np.array([0, ev0.wire_id.size, ev0.wire_id.size + ev1.wire_id.size])
    wid = np.concatenate([ev0.wire_id, ev1.wire_id])
    dr = np.concatenate([ev0.drift, ev1.drift])
    p = cdc.scan_params(h=2.0, max_steps=1000, lam=4.0, max_partitions=1, k=8, n_rounds=3, n_zoom=2)
    small = tracker(g, f, max_events=2, max_seeds=1000)
    big = tracker(g, f, max_events=2, max_seeds=n)
    outs = {}
    for name, tr, want_E in (("over", small, False), ("caller_E", small, True), ("big", big, True)):
        o, w, d = tr.events_to_device(off, wid, dr)
        outs[name] = tr.scan(o, w, d, cdc.grids_to_tensor(grids, tr.dev), p, want_E=want_E, n_seeds=n)
    torch.cuda.synchronize()
    over = outs["over"]
    assert np.all(over["flags"].cpu().numpy() & cdc.FLAG_EMPTY)
    assert np.all(np.isinf(over["best_E"].cpu().numpy()))
    assert np.all(np.isnan(over["best_seed"].cpu().numpy()))
    assert np.all(over["hit_part"].cpu().numpy() == -1)
    assert int(over["steps"].sum()) == 0
    for key in ("E", "topk0", "best_E", "best_seed", "hit_part", "hit_res2", "flags", "steps"):
        assert torch.equal(outs["caller_E"][key], outs["big"][key]), key
