"""Pins to the numbers the paper prints (tests/golden/paper_constants.txt): the
synthetic workload and the event loop use them, and the oracle's trace of the
paper's signal electron in the paper's field has the closed-form radius and
pitch at those values."""
import math
import os

import numpy as np

import cdc_synth as S
import oracle as O

KAPPA = 0.299792458  # MeV/c per (T mm)


def _golden():
    path = os.path.join(os.path.dirname(__file__), "golden", "paper_constants.txt")
    out = {}
    for line in open(path):
        line = line.split("#")[0].strip()
        if line:
            name, value = line.split()[:2]
            out[name] = float(value)
    return out


def test_workload_uses_the_printed_constants():
    c = _golden()
    g = S.make_geometry()
    assert S.SIGNAL_P == c["signal_momentum"]
    assert g.n_layers == int(c["sense_layers"])
    assert g.R0 == c["seed_radius"]
    assert S.uniform_field().B0 == c["field"]
    tmpl = S.cfg2_grid_template()
    assert float(tmpl["step"][0][0]) == np.float32(c["hough_theta0_step"])
    assert float(tmpl["step"][0][2]) == float(tmpl["step"][0][3]) == c["hough_pxy_step"]
    assert S.CFG1_STEP[0] == c["hough_theta0_step"] and S.CFG1_STEP[2] == S.CFG1_STEP[3] == c["hough_pxy_step"]


def test_event_loop_uses_the_printed_resolutions_and_stop():
    from paper_1908_01949_gb300 import event_loop as E
    c = _golden()
    assert (E.SIGMA_Z0, E.SIGMA_PZ0, E.MIN_HITS) == (c["loop_z0_sigma"], c["loop_pz0_sigma"], int(c["loop_min_hits"]))
    g = E.neighbour_grid(np.zeros(5))
    assert float(g["step"][0][1]) == c["loop_z0_sigma"] / 2 and float(g["step"][0][4]) == np.float32(c["loop_pz0_sigma"] / 2)


def test_signal_electron_radius_and_pitch_at_the_printed_momentum_and_field():
    """The oracle's trace of a 104.97 MeV/c electron with pT = 90 MeV/c in 1 T
    closes on a circle of radius pT/(kappa B) = 300.2 mm and advances
    2 pi pz/(kappa B) in z per turn."""
    c = _golden()
    p, pt, B = c["signal_momentum"], 90.0, c["field"]
    pz = math.sqrt(p * p - pt * pt)
    rho = pt / (KAPPA * B)
    assert abs(rho - 300.2) < 0.05
    g = S.make_geometry()
    g.z_half, g.R_out = 1e9, 1e9
    P = O.scan_params(h=2.0, max_steps=2500, max_partitions=100)
    st, _, _ = O.propagate(g, S.uniform_field(B), np.array([0.0, 0.0, 0.0, pt, pz]), P)
    cen = np.array([c["seed_radius"] - rho, 0.0])           # e- in +Bz turns counter-clockwise
    assert np.abs(np.linalg.norm(st[:, :2] - cen, axis=1) - rho).max() < 1e-6
    s_turn = 2 * math.pi * rho * p / pt                     # arc length of one turn
    j = int(round(s_turn / 2.0))
    z_turn = st[j, 2] + (s_turn - 2.0 * j) * pz / p
    assert abs(z_turn - 2 * math.pi * pz / (KAPPA * B)) < 1e-6


def test_benchmark_uses_the_printed_round_count_and_common_hit_cut():
    import bench
    c = _golden()
    assert bench.N_ROUNDS == int(c["zoom_rounds"])
    assert bench.NC_CUT == int(c["common_hits_cut"])
