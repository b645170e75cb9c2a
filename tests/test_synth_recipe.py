"""The seeded synthetic workload that stands in for the COMET Phase-I
simulation meets the recipe it states: one hit per wire, drifts clamped to
[0, 8] mm, a 104.97 MeV/c signal (sec. 1) from the target disk with the stated
turn counts, the stated noise counts and occupancies, and the stated grid
shapes and sizes."""
import numpy as np
import pytest

import cdc_synth as S

MAX_DRIFT = 8.0


@pytest.fixture(scope="module")
def field_map():
    return S.solenoid_map()


def _common(g, ev):
    wid = ev.wire_id
    assert np.unique(wid).size == wid.size                      # one hit per wire
    assert wid.min() >= 0 and wid.max() < g.n_wires
    assert np.all((ev.drift >= 0.0) & (ev.drift <= MAX_DRIFT))
    signal = ev.truth_part >= 0
    assert set(np.unique(ev.truth_part[signal])) == set(range(ev.n_turns))
    for sd in ev.truth_seeds:                                   # (theta0, z0, px0, py0, pz0) at r = R0
        assert abs(np.linalg.norm(sd[2:]) - S.SIGNAL_P) < 1e-9 * S.SIGNAL_P
        assert abs(sd[1]) <= g.z_half
    r0 = np.asarray(ev.signal_r0)
    assert np.hypot(r0[0], r0[1]) <= 100.0 and abs(r0[2]) <= 400.0      # start on the target disk
    return int(signal.sum()), int((~signal).sum())


def test_single_turn_case():
    for i in range(4):
        g, f, ev, grid = S.cfg1_case(i)
        assert f.B0 == 1.0 and ev.n_turns == 1
        n_sig, n_noise = _common(g, ev)
        assert n_noise == 40 and n_sig >= 20
        assert tuple(grid["n"][0]) == S.CFG1_N and np.allclose(grid["step"][0], S.CFG1_STEP)
        off = (grid["centre"][0] - ev.truth_seeds[0]) / grid["step"][0]
        assert np.all(np.abs(off) <= 0.5 + 1e-6)                  # random sub-step offset around the truth


def test_multi_turn_case_at_ten_percent_occupancy(field_map):
    tmpl = S.cfg2_grid_template()
    assert int(np.prod(tmpl["n"][0])) == 10 ** 6
    for i in range(3):
        g, f, ev = S.cfg2_case(i, field_map)
        assert ev.n_turns in (2, 3)
        n_sig, n_noise = _common(g, ev)
        assert n_noise == round(0.10 * g.n_wires) and n_sig >= 20


def test_batched_events(field_map):
    for i in range(6):
        ev, grid = S.cfg3_event(i, field_map)
        g = S.make_geometry()
        assert ev.n_turns in (1, 2, 3)
        n_sig, n_noise = _common(g, ev)
        assert 30 <= n_sig <= 200
        assert 0.05 * g.n_wires - 1 <= n_noise <= 0.20 * g.n_wires + 1
        n = int(np.prod(grid["n"][0]))
        assert 0.5 * S.CFG3_SEEDS[0] <= n <= 2.0 * S.CFG3_SEEDS[1]
        tmpl = S.cfg2_grid_template()
        span = grid["n"][0] * grid["step"][0]                   # counts scaled, spans kept
        assert np.allclose(span, tmpl["n"][0] * tmpl["step"][0], rtol=1e-5)


def test_sweep_events_at_thirty_percent_occupancy(field_map):
    for i in range(2):
        ev, grid = S.cfg5_event(i, field_map)
        g = S.make_geometry()
        n_sig, n_noise = _common(g, ev)
        assert n_noise == round(0.30 * g.n_wires)
        n = int(np.prod(grid["n"][0]))
        assert 0.5 * S.CFG5_SEEDS / S.CFG5_EVENTS <= n <= 2.0 * S.CFG5_SEEDS / S.CFG5_EVENTS
