"""GPU parity of the reversed scan (direction -1: seeds at the exit of a turn
partition) and of the bidirectional common-hit count N_c (sec. 2.2)."""
import numpy as np
import pytest

import cdc_synth as S
import oracle as O
from tests.gpu_util import check_topk, compare_scores, keys_to_index, oracle_params, tracker

pytestmark = pytest.mark.gpu


def test_reversed_scan_matches_oracle(field_map):
    """675 exit seeds of a multi-turn track in the solenoid map scanned with
    direction = -1: scores within 1e-3 relative of the oracle, top-K equal."""
    import torch
    import paper_1908_01949_gb300 as cdc
    g, f, ev = S.cfg2_case(1, field_map, occupancy=0.05)
    x = ev.exit_seeds[0]
    grid = S.make_grid(x + np.array([0.002, 6.0, -1.0, 1.0, 0.7]), (0.004, 12.0, 1.0, 1.0, 1.5), (3, 5, 3, 3, 5))
    n = int(np.prod(grid["n"][0]))
    tr = tracker(g, f)
    off, wid, dr = tr.events_to_device([0, ev.wire_id.size], ev.wire_id, ev.drift)
    p = cdc.scan_params(h=2.0, max_steps=3500, lam=4.0, max_partitions=2, direction=-1, k=8, n_rounds=1)
    out = tr.scan(off, wid, dr, cdc.grids_to_tensor(grid, tr.dev), p, want_E=True, n_seeds=n)
    torch.cuda.synchronize()
    ref = O.scan(g, f, ev.wire_id, ev.drift.astype(np.float64), O.grid_values(grid), oracle_params(p))
    bad, excluded, worst = compare_scores(out["E"].cpu().numpy(), ref)
    assert bad.size == 0, (bad[:10], worst)
    assert excluded < 0.02 * n
    idx, _ = keys_to_index(out["topk0"][0].cpu().numpy())
    ok, diff = check_topk(idx, ref["E"], 8)
    assert ok, diff


def test_bidirectional_common_hits(field_map):
    """Two events scanned from the entrance (direction +1) and from the exit
    (direction -1) of their first turn: N_c per event from the kernel equals the
    oracle's count on the same classifications, and both directions find the
    turn (N_c >= 20)."""
    import torch
    import paper_1908_01949_gb300 as cdc
    g = S.make_geometry()
    evs = [S.cfg2_case(i, field_map, occupancy=0.05)[2] for i in (0, 2)]
    step, n = (0.004, 12.0, 1.0, 1.0, 1.5), (3, 3, 3, 3, 3)
    ent = np.concatenate([S.make_grid(e.truth_seeds[0], step, n) for e in evs])
    ext = np.concatenate([S.make_grid(e.exit_seeds[0], step, n) for e in evs])
    off, wid, dr = S.pack_events(evs)
    tr = tracker(g, field_map)
    off_t, wid_t, dr_t = tr.events_to_device(off, wid, dr)
    outs = []
    for grids, direction in ((ent, 1), (ext, -1)):
        p = cdc.scan_params(h=2.0, max_steps=3500, lam=4.0, max_partitions=1, direction=direction, k=8, n_rounds=3,
                            n_zoom=4)
        outs.append(tr.scan(off_t, wid_t, dr_t, cdc.grids_to_tensor(grids, tr.dev), p))
    nc = tr.common_hits(off_t, outs[0]["hit_part"], outs[1]["hit_part"])
    torch.cuda.synchronize()
    pa, pb = outs[0]["hit_part"].cpu().numpy(), outs[1]["hit_part"].cpu().numpy()
    assert np.array_equal(nc.cpu().numpy(), O.common_hits(off, pa, pb))
    assert np.all(nc.cpu().numpy() >= 20)
