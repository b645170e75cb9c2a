"""Pins of the reversed scan and of the bidirectional common-hit count
(sec. 2.2: the scan runs from seeds at the entrance and at the exit of a turn
partition; N_c counts the hits both directions find)."""
import numpy as np

import cdc_synth as S
import oracle as O
from tests import helix_ref as HR


def test_reversed_scan_matches_dense_helix_enumerator():
    """direction = -1 (t -> -t, q -> -q): the oracle's E and per-hit classes
    equal the independent enumerator on the reversed closed-form helix."""
    rng = np.random.default_rng(S.BASE_SEED + 600)
    g = S.make_geometry()
    f = S.uniform_field(1.0)
    ev = S.make_event(g, f, rng, turns=(2,), noise="uniform", n_noise=40)
    sel = np.concatenate([np.flatnonzero(ev.truth_part == 0)[:16], np.flatnonzero(ev.truth_part < 0)[:8]])
    wid, drift = ev.wire_id[sel], ev.drift[sel].astype(np.float64)
    assert np.isfinite(ev.exit_seeds[0, 0])
    x = ev.exit_seeds[0]
    seeds = O.grid_values(S.make_grid(x, (0.004, 8.0, 1.0, 1.0, 0.8), (3, 1, 3, 1, 3)))
    P = O.scan_params(h=2.0, max_steps=1000, lam=4.0, max_partitions=1, direction=-1)
    out = O.scan(g, f, wid, drift, seeds, P, per_hit=True)
    wm, wd, _ = S.wire_lines(g)
    for i, sd in enumerate(seeds):
        E, r2, parts, n = HR.score(sd, 1.0, 2.0, 1000, 1, 4.0, (wm, wd), wid, drift, g.R0, g.R_out, g.z_half,
                                   direction=-1)
        assert out["n_steps"][i] == n
        assert abs(out["E"][i] - E) < 1e-6, (i, out["E"][i], E)
        clear = out["hit_margin"][i] > 1e-6
        assert np.array_equal(out["hit_part"][i][clear], parts[clear])


def test_entrance_and_exit_scans_share_the_turn():
    """The forward scan from a turn's entrance seed and the reversed scan from
    its exit seed classify the same signal hits into partition 0: N_c covers
    nearly all of the turn's hits (a wrong reversal would share almost none)."""
    fm = S.solenoid_map()
    for index in (0, 1):
        g, f, ev = S.cfg2_case(index, fm, occupancy=0.05)
        assert np.isfinite(ev.exit_seeds[0, 0])
        drift = ev.drift.astype(np.float64)
        fwd = O.scan(g, f, ev.wire_id, drift, ev.truth_seeds[:1], O.scan_params(
            h=2.0, max_steps=3500, lam=4.0, max_partitions=1, direction=1), per_hit=True)
        bwd = O.scan(g, f, ev.wire_id, drift, ev.exit_seeds[:1], O.scan_params(
            h=2.0, max_steps=3500, lam=4.0, max_partitions=1, direction=-1), per_hit=True)
        off = [0, ev.wire_id.size]
        nc = O.common_hits(off, fwd["hit_part"][0], bwd["hit_part"][0])[0]
        turn0 = int(np.sum(ev.truth_part == 0))
        assert nc >= 20 and nc >= 0.85 * turn0, (index, nc, turn0)
        wrong = O.scan(g, f, ev.wire_id, drift, ev.exit_seeds[:1], O.scan_params(
            h=2.0, max_steps=3500, lam=4.0, max_partitions=1, direction=1), per_hit=True)
        assert O.common_hits(off, fwd["hit_part"][0], wrong["hit_part"][0])[0] < 0.2 * turn0


def test_common_hits_counts():
    off = [0, 5, 5, 8]
    a = [0, 0, -1, 1, 0, 0, 0, 2]
    b = [0, 1, 0, 1, 0, -1, 0, 2]
    assert O.common_hits(off, a, b).tolist() == [2, 0, 1]
    assert O.common_hits(off, a, b, 1, 1).tolist() == [1, 0, 0]


def test_extrapolated_turns_reproduce_the_generator_seeds():
    """Sec. 2.3: the seed of the previous / next turn extrapolated by the oracle
    (RKN, h = 2 mm) equals the generator's truth seed of that turn (its own RK4
    at 1 mm, interpolated at the crossing) to 2e-3 mm in z0 and 1e-3 MeV/c."""
    fm = S.solenoid_map()
    P = O.scan_params(h=2.0, max_steps=5000)
    checked = 0
    for index in range(4):
        g, f, ev = S.cfg2_case(index, fm, occupancy=0.05)
        ts = ev.truth_seeds
        for k in range(len(ts)):
            for direction, j in ((-1, k - 1), (1, k + 1)):
                if 0 <= j < len(ts):
                    out, st = O.extrapolate_turn(g, f, ts[k], P, direction)
                    assert st == 0
                    assert abs(out[0] - ts[j][0]) < 1e-5 and abs(out[1] - ts[j][1]) < 2e-3, (out, ts[j])
                    assert np.all(np.abs(out[2:] - ts[j][2:]) < 1e-3), (out, ts[j])
                    checked += 1
    assert checked >= 10
