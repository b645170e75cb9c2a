"""The event loop over turn partitions (sec. 2.3, Fig. 7): from a scan of one
turn (the first, complete one: synthetic events have no trigger counter that
would single out the last), neighbouring turns are predicted by
extrapolation, scanned on narrow grids and classified until fewer than ten
hits remain."""
import numpy as np
import pytest

import cdc_synth as S
import oracle as O
from tests.gpu_util import tracker

pytestmark = pytest.mark.gpu


def test_extrapolated_seeds_match_oracle(field_map):
    import torch
    import paper_1908_01949_gb300 as cdc
    g, f, ev = S.cfg2_case(3, field_map, occupancy=0.05)
    tr = tracker(g, f)
    p = cdc.scan_params(h=2.0, max_steps=5000, lam=4.0, max_partitions=1)
    seeds = torch.as_tensor(ev.truth_seeds.astype(np.float32), device=tr.dev)
    for direction in (-1, 1):
        out, st = tr.extrapolate_turn(seeds, p, direction)
        torch.cuda.synchronize()
        out, st = out.cpu().numpy(), st.cpu().numpy()
        op = O.scan_params(h=2.0, max_steps=5000, lam=4.0, max_partitions=1)
        for i, sd in enumerate(ev.truth_seeds.astype(np.float32).astype(np.float64)):
            ref, rst = O.extrapolate_turn(g, f, sd, op, direction)
            assert st[i] == rst, (direction, i)
            if rst == 0:
                assert abs(out[i, 0] - ref[0]) < 2e-6 and abs(out[i, 1] - ref[1]) < 2e-3, (out[i], ref)
                assert np.all(np.abs(out[i, 2:] - ref[2:]) < 2e-4), (out[i], ref)


def test_event_loop_classifies_every_turn(field_map):
    """Three multi-turn events: the loop finds every truth turn of at least ten
    hits (smaller ones are never taken as a turn and count as noise) in at least
    two of them, and over the three the classification of each turn has
    efficiency and purity (Eqs. 2-3) of at least 0.7 (hits of another turn that
    pass within sqrt(lambda) of a wire are ambiguous by construction)."""
    import paper_1908_01949_gb300 as cdc
    from paper_1908_01949_gb300.event_loop import align_to_truth, event_loop, findable_truth
    g = S.make_geometry()
    tr = tracker(g, field_map, max_seeds=1 << 16)
    sp = cdc.scan_params(h=2.0, max_steps=3500, lam=4.0, max_partitions=1, k=8, n_rounds=6, n_zoom=4)
    rp = cdc.refine_params(n_iter=3, sigma=0.2, checkpoint=128)
    total = np.zeros((4, 4), np.int64)
    complete = 0
    for index in (0, 1, 2):
        ev = S.cfg2_case(index, field_map, occupancy=0.05)[2]
        grid = S.make_grid(ev.truth_seeds[0] + np.array([0.002, 5.0, 0.4, -0.4, 0.5]),
                           (0.004, 12.0, 1.0, 1.0, 1.5), (5, 7, 5, 5, 7))
        labels, seeds = event_loop(tr, ev.wire_id, ev.drift, grid, sp, rp)
        aligned = align_to_truth(labels, ev.truth_part)
        truth = findable_truth(ev.truth_part)
        c = O.classification_counts([0, ev.wire_id.size], aligned, truth, 3)[0]
        total += c
        complete += int(all(c[t + 1, t + 1] > 0 for t in range(ev.n_turns) if np.any(truth == t)))
    eps, pur = O.efficiency_purity(total)
    assert complete >= 2, (complete, total)
    ok = ~np.isnan(eps)
    assert np.all(eps[ok] >= 0.7) and np.all(pur[ok] >= 0.7), (eps, pur)


LOOP_GRID_N = (3, 7, 3, 3, 7)     # neighbour grids reduced so that the FP64 loop runs in seconds


@pytest.mark.parametrize("index", [0, 1, 2])
def test_event_loop_matches_the_fp64_oracle_loop(field_map, index):
    """The same loop in FP64 (oracle.event_loop: the oracle's repeated scan,
    classification, Gauss-Newton refinement and turn extrapolation, with the
    same rules and constants): the same turns, the same hit labels except for
    hits whose residual lies near a classification cut in the oracle's scan
    (the two best seeds of a turn agree only to the final zoom step, which
    moves a residual by up to ~0.02 mm), and refined seeds that agree to a
    fraction of the grid steps."""
    import paper_1908_01949_gb300 as cdc
    from paper_1908_01949_gb300.event_loop import event_loop
    g = S.make_geometry()
    tr = tracker(g, field_map, max_seeds=1 << 16)
    sp = cdc.scan_params(h=2.0, max_steps=3500, lam=4.0, max_partitions=1, k=8, n_rounds=10, n_zoom=2)
    rp = cdc.refine_params(n_iter=3, sigma=0.2, checkpoint=128)
    ev = S.cfg2_case(index, field_map, occupancy=0.05)[2]
    grid = S.make_grid(ev.truth_seeds[0] + np.array([0.002, 5.0, 0.4, -0.4, 0.5]),
                       (0.004, 12.0, 1.0, 1.0, 1.5), (3, 5, 3, 3, 5))
    labels, seeds = event_loop(tr, ev.wire_id, ev.drift, grid, sp, rp, grid_n=LOOP_GRID_N)
    op = O.scan_params(h=2.0, max_steps=3500, lam=4.0, max_partitions=1)
    rl, rs, margin = O.event_loop(g, field_map, ev.wire_id, ev.drift.astype(np.float64), grid, op, k=8, n_rounds=10,
                                  n_zoom=2, n_iter=3, grid_n=LOOP_GRID_N, return_margin=True)
    assert sorted(seeds) == sorted(rs), (sorted(seeds), sorted(rs))
    diff = np.flatnonzero(labels != rl)
    assert np.all(margin[diff] < 0.02), (diff, labels[diff], rl[diff], margin[diff])
    assert diff.size <= max(2, labels.size // 50)
    scale = np.array([1.0, 100.0, 10.0, 10.0, 10.0])
    for t in seeds:
        assert np.all(np.abs(seeds[t] - rs[t]) / scale < 2e-3), (t, seeds[t], rs[t])
