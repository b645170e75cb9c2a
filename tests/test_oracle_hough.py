"""Pins of the oracle's integer circle Hough transform (sec. 2.1, Fig. 4)."""
import math

import numpy as np

import cdc_synth as S
import oracle as O


def _wire_xy_um(g):
    wm, _, _ = S.wire_lines(g)
    return np.rint(wm[:, 0] * 1000).astype(np.int64), np.rint(wm[:, 1] * 1000).astype(np.int64)


def test_accumulator_equals_python_recount():
    """Every cell of a 3-hit accumulator equals a pure-Python integer recount."""
    g = S.make_geometry()
    H = O.hough_params()
    wid = np.array([5, 900, 3000])
    acc, _, _ = O.hough(g, H, wid)
    X, Y = _wire_xy_um(g)
    ref = {}
    for w in wid:
        for j in range(H.n_r):
            R = H.r_min_um + j * H.r_step_um
            for k in range(H.n_phi):
                ph = 2 * math.pi * k / H.n_phi
                cx = int(X[w]) + int(round(R * math.cos(ph)))
                cy = int(Y[w]) + int(round(R * math.sin(ph)))
                c2 = cx * cx + cy * cy
                if not ((R - H.target_um) ** 2 <= c2 <= (R + H.target_um) ** 2):
                    continue
                bx = (cx - H.origin_um) // H.bin_um
                by = (cy - H.origin_um) // H.bin_um
                if 0 <= bx < H.n_bins and 0 <= by < H.n_bins:
                    ref[(by, bx)] = ref.get((by, bx), 0) + 1
    dense = np.zeros_like(acc)
    for (by, bx), v in ref.items():
        dense[by, bx] = v
    assert np.array_equal(acc, dense)
    assert acc.sum() > 0


def test_total_votes_closed_count():
    """Without the target constraint and with every centre in range, each hit
    casts exactly n_r * n_phi votes."""
    g = S.make_geometry()
    H = O.hough_params(n_bins=1500, origin_um=-1500000, target_um=10**7, n_r=8, n_phi=64)
    wid = np.arange(0, 4050, 97)
    acc, _, _ = O.hough(g, H, wid)
    assert acc.sum() == wid.size * 8 * 64


def test_noiseless_circle_peak_at_true_centre():
    """Fine axial wires at all radii, hits = wires within 1 mm of a circle through the target:
    the top peak is within one bin of the true centre, the radius bin within one
    step, and the seed centre lies on the circle at r = R0 moving outward."""
    # fine axial cells at all radii, so that hits sample the whole circle
    g = S.make_geometry(n_layers=60, r_first=60.0, r_last=900.0, n_first=100, n_last=1500, stereo=0.0)
    X, Y = _wire_xy_um(g)
    H = O.hough_params(n_phi=2048)      # vote spacing finer than a bin
    rng = np.random.default_rng(7)
    for _ in range(5):
        R = 200.0 + 5.0 * rng.integers(12, 28)
        phc = rng.uniform(-math.pi, math.pi)
        d = R + rng.uniform(-80.0, 80.0)
        C = np.array([d * math.cos(phc), d * math.sin(phc)])
        dist = np.hypot(X / 1000.0 - C[0], Y / 1000.0 - C[1])
        wid = np.flatnonzero(np.abs(dist - R) < 1.0)
        assert wid.size >= 8
        acc, cand, cen = O.hough(g, H, wid)
        assert cand.shape[0] >= 1
        ix, iy, cnt, rb = cand[0]
        bc = (np.array([ix, iy]) + 0.5) * H.bin_um / 1000.0 + H.origin_um / 1000.0
        assert np.all(np.abs(bc - C) <= 1.5 * H.bin_um / 1000.0), (bc, C)
        assert abs((H.r_min_um + rb * H.r_step_um) / 1000.0 - R) <= H.r_step_um / 1000.0
        th, px, py = cen[0]
        P = 500.0 * np.array([math.cos(th), math.sin(th)])
        Rb = (H.r_min_um + rb * H.r_step_um) / 1000.0
        assert abs(np.linalg.norm(P - bc) - Rb) < 1e-9
        # e- in +Bz: counter-clockwise, tangent points outward at the seed
        t = np.array([px, py]) / math.hypot(px, py)
        assert t @ P > 0
        rv = P - bc
        assert rv[0] * t[1] - rv[1] * t[0] > 0.99 * Rb      # t = z x (P - C)/R
        assert abs(math.hypot(px, py) - 0.299792458 * Rb) < 1e-9


def test_peak_rules_threshold_ties_order():
    """Peak list: threshold max(min_peak, ceil(max/2)), strict 3x3 maxima with
    equal neighbours resolved to the lower index, ordered by (count desc,
    index asc) -- checked on the accumulator of a real signal event against a
    numpy re-evaluation of those rules."""
    g, f, ev, grid = S.cfg1_case(1)
    H = O.hough_params(max_cand=50)
    acc, cand, _ = O.hough(g, H, ev.wire_id)
    nb = H.n_bins
    thr = max(H.min_peak, (int(acc.max()) + 1) // 2)
    pad = np.full((nb + 2, nb + 2), -1, np.int64)
    pad[1:-1, 1:-1] = acc
    idx = np.arange(nb * nb).reshape(nb, nb)
    ipad = np.full((nb + 2, nb + 2), -1, np.int64)
    ipad[1:-1, 1:-1] = idx
    ok = acc >= thr
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            if dx == 0 and dy == 0:
                continue
            nv = pad[1 + dy:nb + 1 + dy, 1 + dx:nb + 1 + dx]
            ni = ipad[1 + dy:nb + 1 + dy, 1 + dx:nb + 1 + dx]
            ok &= (acc > nv) | ((acc == nv) & ((ni < 0) | (idx < ni)))
    ys, xs = np.nonzero(ok)
    order = np.lexsort((ys * nb + xs, -acc[ys, xs]))[:H.max_cand]
    assert np.array_equal(cand[:, 0], xs[order]) and np.array_equal(cand[:, 1], ys[order])
    assert np.array_equal(cand[:, 2], acc[ys, xs][order])


def test_signal_radius_window_finds_the_multi_turn_signal():
    """The multi-turn configuration's Hough votes only for radii a two- or
    three-turn 104.97 MeV/c signal can have (325-355 mm at 1 T), at 1024
    angles.  On the first twenty multi-turn events at 10 % DIO-like occupancy,
    the signal's first turn (theta0, px0, py0 within the half span of the
    configuration's grid) is among the four candidates in at least twelve
    events and the top candidate in at least six; over the library's default
    200-355 mm range at 512 angles, whose radii the noise tracks share, it is
    a candidate in at most two."""
    fm = S.solenoid_map()
    tmpl = S.cfg2_grid_template()[0]
    half = 0.5 * np.asarray(tmpl["step"], np.float64) * np.asarray(tmpl["n"], np.float64)

    def rank(ev, g, H):
        _, _, cen = O.hough(g, H, ev.wire_id)
        t = ev.truth_seeds[0]
        for r, c in enumerate(cen):
            dth = (c[0] - t[0] + math.pi) % (2 * math.pi) - math.pi
            if abs(dth) <= half[0] and abs(c[1] - t[2]) <= half[2] and abs(c[2] - t[3]) <= half[3]:
                return r
        return None

    win, full = O.hough_params(**S.CFG2_HOUGH), O.hough_params()
    rw, rf = [], []
    for i in range(20):
        g, _, ev = S.cfg2_case(i, fm, occupancy=0.10)
        rw.append(rank(ev, g, win))
        rf.append(rank(ev, g, full))
    assert sum(r is not None for r in rw) >= 12, rw
    assert sum(r == 0 for r in rw) >= 6, rw
    assert sum(r is not None for r in rf) <= 2, rf
