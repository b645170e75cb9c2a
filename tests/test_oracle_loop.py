"""Pins of the oracle's repeated scan (sec. 2.2: the scan repeated around its
best seeds) and of its event loop over turn partitions (sec. 2.3, Fig. 7),
against what the generator's truth fixes."""
import numpy as np

import cdc_synth as S
import oracle as O


def _clean_single_turn(index):
    g, f, ev, grid = S.cfg1_case(index)
    sig = ev.truth_part >= 0                      # the signal alone: no noise wires
    return g, f, ev.wire_id[sig], ev.drift[sig], ev.truth_seeds[0], grid


def test_one_round_is_the_plain_scan_top_k():
    g, f, wid, dr, truth, grid = _clean_single_turn(0)
    grid["n"][0] = (3, 3, 3, 3, 3)
    p = O.scan_params(max_steps=1000, lam=4.0)
    z = O.zoom_scan(g, f, wid, dr.astype(np.float64), grid, p, k=5, n_rounds=1)
    seeds = O.grid_values(grid)
    E = O.scan(g, f, wid, dr.astype(np.float64), seeds, p)["E"]
    order = O.topk(E, 5)
    assert np.array_equal(z["index"], order) and np.all(z["round"] == 0)
    assert np.array_equal(z["E"], E[order]) and np.array_equal(z["seeds"], seeds[order])


def test_rounds_close_in_on_the_truth_at_halved_steps():
    """Around a coarse grid whose steps are the paper's resolutions, ten rounds
    bring the best seed of a noiseless-geometry track to within a small part
    of the coarse step of the truth, every round's best no worse than the
    coarse best, and each reported score is the score of its seed."""
    g, f, wid, dr, truth, grid = _clean_single_turn(1)
    grid["n"][0] = (3, 3, 3, 3, 3)
    p = O.scan_params(max_steps=1000, lam=4.0)
    z = O.zoom_scan(g, f, wid, dr.astype(np.float64), grid, p, k=8, n_rounds=10, n_zoom=4)
    coarse = O.zoom_scan(g, f, wid, dr.astype(np.float64), grid, p, k=8, n_rounds=1)
    assert z["E"][0] <= coarse["E"][0]
    assert np.all(np.diff(z["E"]) >= 0)
    assert z["round"][0] > 0                        # a zoom round improved on the coarse grid
    step = np.asarray(grid["step"][0], np.float64)
    dev = np.abs(z["seeds"][0] - truth) / step
    assert np.all(dev[[0, 2, 3]] < 0.25), dev      # theta0, px0, py0
    again = O.scan(g, f, wid, dr.astype(np.float64), z["seeds"], p)["E"]
    assert np.allclose(again, z["E"], rtol=0, atol=1e-12)


def test_zoom_grids_are_centred_on_the_previous_best_at_halved_steps():
    """Round r's seeds are the 3^5 grids around round r-1's n_zoom best at the
    first grid's steps times 2^-r: the second round's best seed lies on such a
    grid around one of the first round's best seeds."""
    g, f, wid, dr, truth, grid = _clean_single_turn(2)
    grid["n"][0] = (3, 3, 3, 3, 3)
    p = O.scan_params(max_steps=1000, lam=4.0)
    r0 = O.zoom_scan(g, f, wid, dr.astype(np.float64), grid, p, k=2, n_rounds=1)
    z = O.zoom_scan(g, f, wid, dr.astype(np.float64), grid, p, k=200, n_rounds=2, n_zoom=2)
    r1 = z["seeds"][z["round"] == 1]
    step = np.asarray(grid["step"][0], np.float32) * np.float32(0.5)
    for s in r1:
        ok = False
        for c in r0["seeds"]:
            k = (s - c) / step.astype(np.float64)
            ok |= bool(np.all(np.abs(k - np.round(k)) < 1e-3) and np.all(np.abs(np.round(k)) <= 1))
        assert ok, s


def test_event_loop_finds_the_turns_of_a_clean_multi_turn_event(field_map):
    """A 2-3 turn signal with 5 % DIO-like noise: the loop, started on a grid
    around the first turn, labels each findable truth turn's hits with
    efficiency and purity (Eqs. 2-3) of at least 0.7, and its refined seeds lie
    near the generator's truth seeds."""
    g, f, ev = S.cfg2_case(0, field_map, occupancy=0.05)
    grid = S.make_grid(ev.truth_seeds[0] + np.array([0.002, 5.0, 0.4, -0.4, 0.5]), (0.004, 12.0, 1.0, 1.0, 1.5),
                       (3, 5, 3, 3, 5))
    p = O.scan_params(h=2.0, max_steps=3500, lam=4.0, max_partitions=1)
    labels, seeds = O.event_loop(g, f, ev.wire_id, ev.drift.astype(np.float64), grid, p, k=8, n_rounds=4, n_zoom=2,
                                 n_iter=3, grid_n=(3, 7, 3, 3, 7))
    assert sorted(seeds) == list(range(ev.n_turns))
    C = O.classification_counts([0, labels.size], np.where(labels == O.UNCLASSIFIED, -1, labels), ev.truth_part,
                                ev.n_turns)
    eps, pur = O.efficiency_purity(C)
    assert np.all(eps >= 0.7) and np.all(pur >= 0.7), (eps, pur)
    for t, s in seeds.items():
        d = np.abs(s - ev.truth_seeds[t])
        assert d[0] < 0.01 and d[2] < 2.0 and d[3] < 2.0, (t, s, ev.truth_seeds[t])


def test_event_loop_stops_below_ten_hits(field_map):
    g, f, ev = S.cfg2_case(0, field_map, occupancy=0.05)
    grid = S.make_grid(ev.truth_seeds[0], (0.004, 12.0, 1.0, 1.0, 1.5), (1, 1, 1, 1, 1))
    p = O.scan_params(h=2.0, max_steps=3500, lam=4.0, max_partitions=1)
    keep = np.arange(9)
    labels, seeds = O.event_loop(g, f, ev.wire_id[keep], ev.drift[keep].astype(np.float64), grid, p, n_rounds=1)
    assert seeds == {} and np.all(labels == O.UNCLASSIFIED)
