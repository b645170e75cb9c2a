"""Pins of the oracle's score (Eq. 1), hit classification and top-K."""
import math

import numpy as np
import pytest

import cdc_synth as S
import oracle as O
from tests import helix_ref as HR


def _tiny_case(index=0, n_signal=14, n_noise=6, turns=(1,), max_part=1):
    rng = np.random.default_rng(S.BASE_SEED + 500 + index)
    g = S.make_geometry()
    f = S.uniform_field(1.0)
    ev = S.make_event(g, f, rng, turns=turns, noise="uniform", n_noise=40)
    sig = np.flatnonzero(ev.truth_part >= 0)[:n_signal]
    noi = np.flatnonzero(ev.truth_part < 0)[:n_noise]
    sel = np.concatenate([sig, noi])
    step = (0.004, 8.0, 1.0, 1.0, 0.8)
    grid = S.make_grid(ev.truth_seeds[0], step, (3, 3, 3, 3, 3))
    return g, f, ev.wire_id[sel], ev.drift[sel].astype(np.float64), grid


@pytest.mark.parametrize("lam", [1.0, 4.0, 9.0])
def test_score_matches_dense_helix_enumerator(lam):
    """3^5 seeds x 20 hits: the oracle's E equals an independent dense-sampling
    enumerator on the closed-form helix to 1e-6 mm^2, per-hit classes equal."""
    g, f, wid, drift, grid = _tiny_case(0)
    P = O.scan_params(h=2.0, max_steps=1000, lam=lam, max_partitions=1)
    seeds = O.grid_values(grid)
    sub = seeds[::11]                                    # 23 of the 243 seeds
    out = O.scan(g, f, wid, drift, sub, P, per_hit=True)
    wm, wd, _ = S.wire_lines(g)
    for i, sd in enumerate(sub):
        E, r2, parts, n = HR.score(sd, 1.0, 2.0, 1000, 1, lam, (wm, wd), wid, drift, g.R0, g.R_out, g.z_half)
        assert out["n_steps"][i] == n
        assert abs(out["E"][i] - E) < 1e-6, (i, out["E"][i], E)
        fin = np.isfinite(r2) & (r2 < lam)
        assert np.allclose(out["hit_res2"][i][fin], r2[fin], atol=1e-6)
        clear = out["hit_margin"][i] > 1e-6
        assert np.array_equal(out["hit_part"][i][clear], parts[clear])


def test_score_multi_partition_matches_enumerator():
    """Two-turn track, max_partitions = 3: min over turns of Eq. 1 and the
    partition of each classified hit agree with the enumerator."""
    g, f, wid, drift, grid = _tiny_case(1, n_signal=30, n_noise=6, turns=(2,), max_part=3)
    P = O.scan_params(h=2.0, max_steps=3500, lam=4.0, max_partitions=3)
    seeds = O.grid_values(grid)[[0, 60, 121, 200, 242]]
    out = O.scan(g, f, wid, drift, seeds, P, per_hit=True)
    wm, wd, _ = S.wire_lines(g)
    for i, sd in enumerate(seeds):
        E, r2, parts, n = HR.score(sd, 1.0, 2.0, 3500, 3, 4.0, (wm, wd), wid, drift, g.R0, g.R_out, g.z_half)
        assert abs(out["E"][i] - E) < 1e-6
        clear = out["hit_margin"][i] > 1e-6
        assert np.array_equal(out["hit_part"][i][clear], parts[clear])
    assert (out["hit_part"] >= 1).any()          # the second turn classifies hits


def test_score_special_cases():
    """Eq. 1 limits: far from every wire E = H lambda; with huge lambda E is the
    plain sum of (|DCA| - drift)^2; the score never exceeds H lambda."""
    g, f, wid, drift, grid = _tiny_case(2)
    seeds = O.grid_values(grid)[:5]
    P = O.scan_params(lam=4.0)
    out = O.scan(g, f, wid, drift, seeds, P, per_hit=True)
    assert np.all(out["E"] <= wid.size * 4.0 + 1e-12)
    # a seed aimed inward never reaches a wire: every term is lambda
    inward = np.array([0.3, 0.0, -80.0 * math.cos(0.3), -80.0 * math.sin(0.3), 10.0])
    e = O.scan(g, f, wid, drift, inward[None], P)["E"][0]
    assert e == pytest.approx(wid.size * 4.0, abs=0)
    big = O.scan_params(lam=1e12)
    out2 = O.scan(g, f, wid, drift, seeds, big, per_hit=True)
    assert np.allclose(out2["E"], out2["hit_res2"].sum(1), rtol=1e-12)
    # drift = 0: terms become min(DCA^2, lambda); mirror points collapse onto the wire
    out3 = O.scan(g, f, wid, np.zeros_like(drift), seeds, P, per_hit=True)
    assert np.all(out3["hit_res2"] >= 0)


def test_truth_seed_classifies_signal_hits():
    """At the true seed of a clean single-turn event the signal hits are
    classified to partition 0 and noise hits are mostly not."""
    g, f, ev, grid = S.cfg1_case(3)
    P = O.scan_params(lam=4.0)
    out = O.scan(g, f, ev.wire_id, ev.drift, ev.truth_seeds[:1], P, per_hit=True)
    hp = out["hit_part"][0]
    sig = ev.truth_part >= 0
    assert (hp[sig] == 0).mean() > 0.9
    assert (hp[~sig] == -1).mean() > 0.8


def test_topk_order_and_ties():
    E = np.array([3.0, 1.0, 2.0, 1.0, 0.5, 2.0])
    assert list(O.topk(E, 4)) == [4, 1, 3, 2]


def test_grid_values_row_major_float32():
    grid = S.make_grid((0.1, 10.0, 50.0, -60.0, 20.0), (0.01, 5.0, 2.5, 2.5, 1.7), (2, 1, 3, 1, 2))
    v = O.grid_values(grid)
    assert v.shape == (12, 5)
    assert np.all(v == v.astype(np.float32).astype(np.float64))
    f32 = lambda x: float(np.float32(x))
    # one rounding of the exact value centre + k step from the float32 record
    assert v[0, 0] == f32(f32(0.1) - 0.5 * f32(0.01)) and v[-1, 0] == f32(f32(0.1) + 0.5 * f32(0.01))
    assert v[1, 4] == f32(20.0 + 0.5 * f32(1.7)) and v[2, 2] == 50.0 and v[4, 2] == 52.5
