"""GPU behaviour at the scan's limits, against the FP64 oracle: the step cap,
the largest top-K list, a seed whose record compacts its finished partitions,
and a seed that scores more wires than its record holds."""
import numpy as np
import pytest

import cdc_synth as S
import oracle as O
from tests.gpu_util import check_topk, compare_scores, keys_to_index, oracle_params, tracker

CDC_MAX_FOUND = 256   # record entries of a seed (include/cdc.h)

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


def _all_wires_event(seed_index=7):
    """Every wire fired (drift U[0, 2] mm) and seeds tangent-free near a slow
    (pz0 = 1 MeV/c) copy of a multi-turn signal, so that one seed passes
    hundreds of fired wires within drift + sqrt(lambda) over its turns."""
    fm = S.solenoid_map()
    g, f, ev = S.cfg2_case(seed_index, fm, occupancy=0.10)
    rng = np.random.default_rng(5)
    wid = np.arange(g.n_wires).astype(np.int32)
    dr = rng.uniform(0, 2, wid.size).astype(np.float32)
    c = ev.truth_seeds[0].copy()
    c[1], c[4] = 0.0, 1.0
    grid = S.make_grid(c, (0.001, 2.0, 0.2, 0.2, 0.2), (3, 1, 3, 1, 1))
    return g, f, S.Event(wire_id=wid, drift=dr, truth_part=np.full(wid.size, -1, np.int8),
                         truth_seeds=ev.truth_seeds, n_turns=ev.n_turns), grid


def test_record_compaction_and_overflow():
    """lambda = 90 mm^2 with every wire fired: over one turn a seed keeps ~75
    passes (no compaction); over three turns ~225, beyond the point where the
    record compacts its finished partitions, and the scores, best seed and hit
    classes still follow the oracle; over all its turns (~6) the seed scores
    ~290 distinct wires, more than the 256 entries a record can hold even
    compacted, and the event carries the overflow flag."""
    import paper_1908_01949_gb300 as cdc
    g, f, ev, grid = _all_wires_event()
    seeds = O.grid_values(grid)
    tr = tracker(g, f)
    for parts, overflow in ((1, False), (3, False), (16, True)):
        p = cdc.scan_params(h=2.0, max_steps=20000, lam=90.0, max_partitions=parts, k=8, n_rounds=1, max_drift=2.0)
        ref = O.scan(g, f, ev.wire_id, ev.drift.astype(np.float64), seeds, oracle_params(p), per_hit=True)
        below = ((ref["hit_res2"] < 90.0) & (ref["hit_part"] >= 0)).sum(1)
        assert (below.min() > CDC_MAX_FOUND) if overflow else (below.max() < CDC_MAX_FOUND), below
        out = _scan(tr, ev, grid, p)
        assert bool(int(out["flags"][0]) & cdc.FLAG_FOUND_OVERFLOW) == overflow
        if overflow:
            continue
        # E = H lambda + sum over the scored wires of (term - lambda): compare the scored part
        E = out["E"].cpu().numpy().astype(np.float64)
        Hl = ev.wire_id.size * 90.0
        ok = ref["margin"] >= 1e-3
        rel = np.abs(E - ref["E"]) / (Hl - ref["E"])
        assert ok.sum() >= 5 and np.all(rel[ok] <= 1e-3), (rel, ref["margin"])
        best = out["best_seed"][0, 0].cpu().numpy().astype(np.float64)
        rb = O.scan(g, f, ev.wire_id, ev.drift.astype(np.float64), best[None], oracle_params(p), per_hit=True)
        clear = rb["hit_margin"][0] >= 1e-3
        hp = out["hit_part"].cpu().numpy()
        assert np.mean(hp[clear] == rb["hit_part"][0][clear]) == 1.0


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
