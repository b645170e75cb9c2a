"""Oracle pins on a turn partition that passes fired wires more than once
(sec. 2.2, Eq. 1: the DCA of a partition is its closest approach).

The event of tests/double_pass.py keeps one partition over several
revolutions.  The oracle's per-hit term must equal the nearest pass of each
partition minus the drift, recomputed here from the passes' distances
(refined independently along the oracle's trace), and on that event the
other reading (the smallest residual over the passes) differs from it by far
more than the scan's score tolerance, so the GPU parity test on the same event
separates the two."""
import numpy as np

import oracle as O
from tests import double_pass as DP


def _setup():
    g, f, wid, dr = DP.setup()
    return g, f, wid, dr


def test_event_keeps_one_partition_over_several_revolutions():
    g, f, _, _ = _setup()
    st, flags, margin = O.propagate(g, f, DP.SEED, DP.scan_params())
    assert flags == 0 and np.all(st[:, 6] == 0)
    assert margin > 0.01                      # no stop or partition decision within 0.01 mm
    phi = np.unwrap(np.arctan2(st[:, 1] - 0.0, st[:, 0] - 633.0))   # azimuth about the circle's centre
    assert abs(phi[-1] - phi[0]) > 4 * 2 * np.pi
    assert abs(st[-1, 2]) > g.z_half          # leaves through the end plate


def test_every_trap_wire_is_passed_twice_within_reach():
    g, f, _, _ = _setup()
    for w, d in DP.TRAPS.items():
        ps = DP.passes(g, f, DP.SEED, w)
        near = [D for _, p, D in ps if p == 0 and D < d + np.sqrt(DP.LAM)]
        assert len(near) >= 2, (w, ps)


def test_oracle_term_is_the_nearest_pass_of_the_partition():
    g, f, wid, dr = _setup()
    ref = O.scan(g, f, wid, dr.astype(np.float64), DP.SEED[None], DP.scan_params(), per_hit=True)
    E = 0.0
    for i, (w, d) in enumerate(zip(wid, dr.astype(np.float64))):
        ps = DP.passes(g, f, DP.SEED, int(w))
        expect = DP.term_nearest_pass(ps, d)
        assert abs(min(ref["hit_res2"][0, i], DP.LAM) - expect) < 1e-6, (int(w), ref["hit_res2"][0, i], expect)
        E += expect
    assert abs(ref["E"][0] - E) < 1e-5


def test_the_two_readings_differ_on_every_trap():
    g, f, wid, dr = _setup()
    gap = 0.0
    for w, d in DP.TRAPS.items():
        ps = DP.passes(g, f, DP.SEED, w)
        a, b = DP.term_nearest_pass(ps, d), DP.term_smallest_residual(ps, d)
        assert a - b > 0.5, (w, a, b)
        gap += a - b
    for w, d in DP.SAME.items():
        ps = DP.passes(g, f, DP.SEED, w)
        assert abs(DP.term_nearest_pass(ps, d) - DP.term_smallest_residual(ps, d)) < 1e-9
    ref = O.scan(g, f, wid, dr.astype(np.float64), DP.SEED[None], DP.scan_params())
    assert gap > 100 * 1e-3 * ref["E"][0]     # far beyond the 1e-3 relative score tolerance


def test_classification_follows_the_nearest_pass():
    """Hits whose nearer pass lies beyond drift - sqrt(lambda) are not
    classified, though another pass of the same partition fits the drift."""
    g, f, wid, dr = _setup()
    ref = O.scan(g, f, wid, dr.astype(np.float64), DP.SEED[None], DP.scan_params(), per_hit=True)
    part = dict(zip(wid.tolist(), ref["hit_part"][0].tolist()))
    for w in (3, 1026, 145, 2376):
        assert part[w] == -1
    for w in (2, 154, 831):
        assert part[w] == 0
    for w in DP.CONTROLS:
        assert part[w] == 0
    for w in DP.FAR:
        assert part[w] == -1
