"""Pins of the FP64 oracle's propagation and field against closed forms."""
import math

import numpy as np
import pytest

import cdc_synth as S
import oracle as O

KAPPA = 0.299792458


def _helix_closed(r0, t0, w, s):
    # t_x = t_x0 cos ws + t_y0 sin ws, t_y = t_y0 cos ws - t_x0 sin ws (uniform Bz)
    x = r0[0] + (t0[0] * math.sin(w * s) + t0[1] * (1 - math.cos(w * s))) / w
    y = r0[1] + (t0[1] * math.sin(w * s) - t0[0] * (1 - math.cos(w * s))) / w
    z = r0[2] + t0[2] * s
    return np.array([x, y, z])


def _run_steps(f, lam, h, r, t, n):
    for _ in range(n):
        r, t = O.step(f, lam, h, r, t)
    return r, t


@pytest.mark.parametrize("p,pz", [(104.97, 20.0), (104.97, 60.0), (60.0, 10.0)])
def test_rkn_matches_closed_form_helix(p, pz):
    """Uniform 1 T: 3000 RKN steps of 2 mm (6 m) stay within 1e-6 mm of the helix."""
    f = S.uniform_field(1.0)
    pt = math.sqrt(p * p - pz * pz)
    t0 = np.array([pt / p, 0.0, pz / p])
    r0 = np.array([500.0, 0.0, -100.0])
    lam = -KAPPA / p
    w = lam * 1.0
    r, t = r0.copy(), t0.copy()
    worst = 0.0
    for blk in range(30):
        r, t = _run_steps(f, lam, 2.0, r, t, 100)
        ref = _helix_closed(r0, t0, w, 2.0 * 100 * (blk + 1))
        worst = max(worst, float(np.abs(r - ref).max()))
    assert worst < 1e-6, worst
    # radius of the projected circle = pT / (kappa B)
    assert abs(abs(1.0 / w) * pt / p - pt / KAPPA) < 1e-9


def test_helix_radius_and_pitch_from_trace():
    """Circle radius and pitch read off a propagated trace: pT/(kappa B), 2 pi pz/(kappa B)."""
    p, pz = 104.97, 30.0
    pt = math.sqrt(p * p - pz * pz)
    g = S.make_geometry()
    g.z_half, g.R_out = 1e9, 1e9
    P = O.scan_params(h=2.0, max_steps=4000, max_partitions=100)
    seed = np.array([0.0, 0.0, 0.0, pt, pz])   # at (R0, 0, 0) moving along +y
    st, fl, mg = O.propagate(g, S.uniform_field(1.0), seed, P)
    xy = st[:, :2]
    # centre: e- in +Bz turns counter-clockwise, so the centre is at -x of the start
    rho_c = pt / KAPPA
    cen = np.array([500.0 - rho_c, 0.0])
    dist = np.linalg.norm(xy - cen, axis=1)
    assert np.abs(dist - rho_c).max() < 1e-6
    period = 2 * math.pi * rho_c * p / pt              # arclength of one turn
    n = int(round(period / 2.0))
    dz = st[n, 2] - st[0, 2]
    assert abs(dz - 2 * math.pi * pz / KAPPA * (n * 2.0 / period)) < 1e-6


def test_momentum_magnitude_conserved():
    """|t| (so |p| = p |t|) drifts by < 1e-12 relative over 3500 steps at 104.97 MeV, 1 T."""
    f = S.uniform_field(1.0)
    p = 104.97
    t = np.array([0.6, 0.7, 0.0])
    t[2] = math.sqrt(1 - t[0] ** 2 - t[1] ** 2)
    r = np.array([500.0, 0.0, 0.0])
    r, t = _run_steps(f, -KAPPA / p, 2.0, r, t, 3500)
    assert abs(np.linalg.norm(t) - 1.0) < 1e-12


def test_fourth_order_convergence():
    """Halving h cuts the end-point error by ~16 (global order 4)."""
    f = S.uniform_field(1.0)
    p, pz = 104.97, 40.0
    pt = math.sqrt(p * p - pz * pz)
    t0 = np.array([0.0, pt / p, pz / p])
    r0 = np.array([500.0, 0.0, 0.0])
    lam = -KAPPA / p
    L = 1200.0
    errs = []
    for h in (40.0, 20.0, 10.0):
        r, t = _run_steps(f, lam, h, r0, t0, int(L / h))
        errs.append(np.linalg.norm(r - _helix_closed(r0, t0, lam, L)))
    assert 12.0 < errs[0] / errs[1] < 20.0
    assert 12.0 < errs[1] / errs[2] < 20.0


def test_field_map_on_axis_matches_textbook(field_map):
    """Synthetic map: on-axis Bz of a finite solenoid,
    (mu0 n I / 2) [(z+b)/sqrt((z+b)^2+a^2) - (z-b)/sqrt((z-b)^2+a^2)], scaled to 1 T at 0."""
    a, b = 1000.0, 1500.0
    z = field_map.z_min + field_map.dz * np.arange(field_map.nz)
    f = lambda z: (z + b) / np.sqrt((z + b) ** 2 + a * a) - (z - b) / np.sqrt((z - b) ** 2 + a * a)
    ref = f(z) / f(0.0)
    assert np.abs(field_map.bz[0] - ref).max() < 1e-6
    assert np.abs(field_map.br[0]).max() < 1e-7


def test_field_map_divergence_free_and_symmetric(field_map):
    """div B = (1/r) d(r Br)/dr + dBz/dz ~ 0 on the samples; Br(r,-z) = -Br(r,z)."""
    fm = field_map
    r = fm.r_min + fm.dr * np.arange(fm.nr)
    rb = r[:, None] * fm.br.astype(np.float64)
    div = (rb[2:, 1:-1] - rb[:-2, 1:-1]) / (2 * fm.dr) / r[1:-1, None] + \
          (fm.bz[1:-1, 2:].astype(np.float64) - fm.bz[1:-1, :-2]) / (2 * fm.dz)
    assert np.abs(div[10:]).max() < 2e-6
    assert np.abs(fm.br + fm.br[:, ::-1]).max() < 1e-6
    assert np.abs(fm.bz - fm.bz[:, ::-1]).max() < 1e-6


def test_oracle_field_interpolation_exact_on_bilinear():
    """The map lookup reproduces a field that is bilinear in (r, z) exactly,
    gives Bx, By = Br (x, y)/r, clamps outside the grid, and its gradient
    matches central differences."""
    nr, nz, dr, dz = 6, 7, 100.0, 200.0
    r = np.arange(nr) * dr
    z = -600.0 + np.arange(nz) * dz
    Rm, Zm = np.meshgrid(r, z, indexing="ij")
    bzf = lambda r, z: 1.0 + 1e-4 * r - 2e-4 * z + 3e-8 * r * z
    brf = lambda r, z: 2e-5 * r + 1e-8 * r * z
    f = S.Field(kind=1, B0=1.0, bz=bzf(Rm, Zm).astype(np.float32), br=brf(Rm, Zm).astype(np.float32),
                r_min=0.0, z_min=-600.0, dr=dr, dz=dz)
    rng = np.random.default_rng(3)
    for _ in range(50):
        x, y, zz = rng.uniform(-350, 350), rng.uniform(-350, 350), rng.uniform(-590, 590)
        rho = math.hypot(x, y)
        B, G = O.field_at(f, np.array([x, y, zz]))
        # samples are float32: compare with 1e-6 slack
        assert abs(B[2] - bzf(rho, zz)) < 1e-6
        assert abs(B[0] - brf(rho, zz) * x / rho) < 1e-6
        assert abs(B[1] - brf(rho, zz) * y / rho) < 1e-6
        for j in range(3):
            e = np.zeros(3)
            e[j] = 1e-3
            Bp, _ = O.field_at(f, np.array([x, y, zz]) + e)
            Bm, _ = O.field_at(f, np.array([x, y, zz]) - e)
            assert np.allclose((Bp - Bm) / 2e-3, G[:, j], atol=1e-9)
    B, _ = O.field_at(f, np.array([0.0, 0.0, 5000.0]))      # clamped to z_max
    assert abs(B[2] - bzf(0.0, 600.0)) < 1e-6


def test_straight_line_doca_is_textbook_line_distance():
    """B = 0: the track is a straight line and DCA = |(m - r0).(t x d)| / |t x d|."""
    g = S.make_geometry()
    wm, wd, _ = S.wire_lines(g)
    f = S.uniform_field(0.0)
    P = O.scan_params(h=2.0, max_steps=2000, lam=1e6, max_partitions=1)
    rng = np.random.default_rng(11)
    for _ in range(20):
        th = rng.uniform(-math.pi, math.pi)
        r0 = np.array([500 * math.cos(th), 500 * math.sin(th), rng.uniform(-200, 200)])
        out = np.array([math.cos(th), math.sin(th), 0.0])
        t = out + rng.uniform(-0.4, 0.4, 3)
        t[2] = rng.uniform(-0.3, 0.3)
        t /= np.linalg.norm(t)
        seed = np.array([th, r0[2], *(100.0 * t)])
        # pick the wire whose line passes closest to the ray, inside the layer band
        cr = np.cross(t, wd)
        dist = np.abs(((wm - r0) * cr).sum(1)) / np.linalg.norm(cr, axis=1)
        w0 = r0 - wm
        b = wd @ t
        s_star = (b * (w0 * wd).sum(1) - w0 @ t) / (1 - b * b)   # closest point on the ray
        pc = r0 + s_star[:, None] * t
        ok = (s_star > 5.0) & (np.hypot(pc[:, 0], pc[:, 1]) < 830) & (np.abs(pc[:, 2]) < 740)
        w = int(np.flatnonzero(ok)[np.argmin(dist[ok])])
        E = O.scan(g, f, [w], [0.0], seed[None], P)["E"][0]
        assert abs(math.sqrt(E) - dist[w]) < 1e-9
