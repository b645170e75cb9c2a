"""The scan's stepper takes the field of each step's end estimate as the next
step's first-stage field instead of evaluating the map again at the new
position.  The two points differ by h^2/6 (2 k3 - k1 - k2), of order h^3 /
rho^2, so the scheme stays within a small fraction of the 1e-4 mm per metre
propagation tolerance of the classical step.  This test bounds that difference
in FP64 on the solenoid map, with the FP64 oracle's field and classical step;
the reused-field step is restated here from its definition (no GPU code)."""
import numpy as np

import cdc_synth as S
import oracle as O

KAPPA = 0.299792458


def _reused_field_run(f, r, t, lam, h, n):
    B, _ = O.field_at(f, r)
    out = []
    for _ in range(n):
        k1 = lam * np.cross(t, B)
        Bm, _ = O.field_at(f, r + 0.5 * h * t + h * h / 8.0 * k1)
        k2 = lam * np.cross(t + 0.5 * h * k1, Bm)
        k3 = lam * np.cross(t + 0.5 * h * k2, Bm)
        B, _ = O.field_at(f, r + h * t + 0.5 * h * h * k3)   # serves as the next step's first stage
        k4 = lam * np.cross(t + h * k3, B)
        r = r + h * t + h * h / 6.0 * (k1 + k2 + k3)
        t = t + h / 6.0 * (k1 + 2.0 * k2 + 2.0 * k3 + k4)
        out.append(r)
    return np.array(out)


def _classical_run(f, r, t, lam, h, n):
    out = []
    for _ in range(n):
        r, t = O.step(f, lam, h, r, t)
        out.append(r)
    return np.array(out)


def test_reused_end_field_stays_within_1e_5_mm_over_6_m(field_map):
    """Two 105 MeV/c multi-turn tracks from r = 500 mm, 3000 steps of 2 mm:
    positions of the two schemes within 1e-5 mm at every step (1e-4 mm per
    metre would allow 6e-4 mm at 6 m)."""
    f = field_map
    for th, z0, pt, psi, pz in ((0.3, -300.0, 90.0, 0.2, 25.0), (2.5, 250.0, 95.0, -0.4, -40.0)):
        r = np.array([500.0 * np.cos(th), 500.0 * np.sin(th), z0])
        p = np.array([pt * np.cos(th + psi), pt * np.sin(th + psi), pz])
        pn = float(np.linalg.norm(p))
        t, lam = p / pn, -KAPPA / pn
        a = _classical_run(f, r.copy(), t.copy(), lam, 2.0, 3000)
        b = _reused_field_run(f, r.copy(), t.copy(), lam, 2.0, 3000)
        d = np.linalg.norm(a - b, axis=1)
        assert d.max() < 1e-5, d.max()
        # and the difference is not zero: the map's field does vary along the track
        assert d.max() > 1e-9


def test_uniform_field_reuse_is_the_classical_step():
    """In a uniform field the reused field is the field: identical states."""
    f = S.uniform_field(1.0)
    r = np.array([500.0, 0.0, 0.0])
    t = np.array([0.6, 0.7, 0.2])
    t = t / np.linalg.norm(t)
    a = _classical_run(f, r.copy(), t.copy(), -KAPPA / 104.97, 2.0, 200)
    b = _reused_field_run(f, r.copy(), t.copy(), -KAPPA / 104.97, 2.0, 200)
    assert np.abs(a - b).max() < 1e-9
