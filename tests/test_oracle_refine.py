"""Pins of the oracle's chi^2 gradient and Gauss-Newton refinement."""
import math

import numpy as np
import pytest

import cdc_synth as S
import oracle as O
from tests import helix_ref as HR

SCALE = np.array([1.0, 100.0, 10.0, 10.0, 10.0])


def _case(kind, index=0):
    if kind == "uniform":
        g, f, ev, grid = S.cfg1_case(index)
        P = O.scan_params(h=2.0, max_steps=1000, lam=4.0, max_partitions=1)
    else:
        g = S.make_geometry()
        f = S.solenoid_map(nr=226, nz=501, dr=4.0, dz=4.0)
        rng = np.random.default_rng(S.BASE_SEED + 77 + index)
        ev = S.make_event(g, f, rng, turns=(1,), noise="uniform", n_noise=10)
        P = O.scan_params(h=2.0, max_steps=1500, lam=4.0, max_partitions=1)
    seed = ev.truth_seeds[0] + np.array([0.002, 3.0, 0.8, -0.6, 0.5])
    part = O.scan(g, f, ev.wire_id, ev.drift, ev.truth_seeds[:1], P, per_hit=True)["hit_part"][0]
    return g, f, ev, P, seed, part


def _fd_grad(g, f, ev, P, part, seed):
    """Central differences at h_i = 1e-4 max(|x_i|, s_i) and h_i/2, combined by
    Richardson extrapolation (truncation error O(h^4))."""
    def cd(i, h):
        e = np.zeros(5)
        e[i] = h
        cp = O.chi2(g, f, P, ev.wire_id, ev.drift, part, seed + e)[0]
        cm = O.chi2(g, f, P, ev.wire_id, ev.drift, part, seed - e)[0]
        return (cp - cm) / (2 * h)

    fd = np.zeros(5)
    for i in range(5):
        h = 1e-4 * max(abs(seed[i]), SCALE[i])
        fd[i] = (4.0 * cd(i, 0.5 * h) - cd(i, h)) / 3.0
    return fd


@pytest.mark.parametrize("kind", ["uniform", "map"])
def test_tangent_gradient_matches_central_differences(kind):
    """d chi^2 / d seed from FP64 forward tangents equals central finite
    differences (h_i = 1e-4 max(|x_i|, s_i)) of the FP64 forward chi^2."""
    g, f, ev, P, seed, part = _case(kind)
    c2, grad, jtj, nu, fl = O.chi2(g, f, P, ev.wire_id, ev.drift, part, seed)
    assert nu >= 15 and fl == 0
    fd = _fd_grad(g, f, ev, P, part, seed)
    rel = np.linalg.norm((fd - grad) * SCALE) / np.linalg.norm(grad * SCALE)
    # the bilinear map has kinks at cell edges that the difference quotient straddles
    assert rel < (1e-6 if kind == "uniform" else 1e-4), (grad, fd)
    # Gauss-Newton matrix is the Gram matrix of J: symmetric positive semi-definite
    assert np.allclose(jtj, jtj.T) and np.linalg.eigvalsh(jtj).min() > -1e-9 * np.abs(jtj).max()


def test_gradient_matches_closed_form_helix():
    """Uniform field: central differences of chi^2 computed on the closed-form
    helix (independent enumerator) match the oracle's tangent gradient."""
    g, f, ev, P, seed, part = _case("uniform", 2)
    # |DCA| has a kink where the track crosses the wire: keep hits whose DCA is
    # far larger than the difference step's displacement (~0.15 mm)
    nocut = O.scan_params(h=2.0, max_steps=1000, lam=1e12, max_partitions=1)
    doca = np.sqrt(O.scan(g, f, ev.wire_id, np.zeros_like(ev.drift), seed[None], nocut,
                          per_hit=True)["hit_res2"][0])
    sel = np.flatnonzero((part >= 0) & (doca > 1.0))[:12]
    wid, dr, pt = ev.wire_id[sel], ev.drift[sel].astype(np.float64), part[sel]
    c2, grad, _, nu, fl = O.chi2(g, f, P, wid, dr, pt, seed)
    wm, wd, _ = S.wire_lines(g)

    def chi2_helix(s):
        n, labels = HR.trace_rule(s, 1.0, 2.0, 1000, 1, g.R0, g.R_out, g.z_half)
        tot = 0.0
        for w, d in zip(wid, dr):
            b = HR.doca_per_partition(s, 1.0, 2.0, n, labels, wm[w], wd[w], g.R0, 1, ds=0.05)
            tot += ((b[0] - d) / 0.2) ** 2
        return tot

    assert abs(chi2_helix(seed) - c2) < 1e-6 * max(1.0, c2)
    fd = np.zeros(5)
    for i in range(5):
        h = 1e-4 * max(abs(seed[i]), SCALE[i])
        e = np.zeros(5)
        e[i] = h
        fd[i] = (chi2_helix(seed + e) - chi2_helix(seed - e)) / (2 * h)
    rel = np.linalg.norm((fd - grad) * SCALE) / np.linalg.norm(grad * SCALE)
    assert rel < 1e-4, (grad, fd)


def test_gauss_newton_recovers_noiseless_truth():
    """With drifts equal to the true DCAs (no smearing), five Gauss-Newton
    iterations from a displaced seed return to the truth: chi^2 ~ 0."""
    g, f, ev, grid = S.cfg1_case(4)
    P = O.scan_params(h=2.0, max_steps=1000, lam=4.0, max_partitions=1)
    truth = ev.truth_seeds[0]
    nocut = O.scan_params(h=2.0, max_steps=1000, lam=1e12, max_partitions=1)
    out = O.scan(g, f, ev.wire_id, np.zeros_like(ev.drift), truth[None], nocut, per_hit=True)
    sig = ev.truth_part >= 0
    drift = np.where(sig, np.sqrt(out["hit_res2"][0]), ev.drift).astype(np.float64)
    part = np.where(sig, 0, -1)
    start = truth + 0.3 * np.array([0.0005, 0.6, 0.2, -0.2, 0.15])
    so, c2, grad, nu, fl = O.refine(g, f, P, ev.wire_id, drift, part, start, n_iter=5)
    assert c2 < 1e-10
    assert np.all(np.abs((so - truth) / SCALE) < 1e-7)
    c0 = O.chi2(g, f, P, ev.wire_id, drift, part, start)[0]
    assert c0 > 50.0


def test_no_classified_hit_leaves_the_seed_and_flags_the_system():
    """An event without hits: chi^2 is an empty sum (0), its gradient is zero,
    the 5x5 normal matrix is zero (not positive definite, flagged) and the
    seed stays where it was."""
    g, f, ev, _ = S.cfg1_case(7)
    P = O.scan_params(h=2.0, max_steps=1000, lam=4.0, max_partitions=1)
    sd = ev.truth_seeds[0].astype(np.float64)
    none_i, none_f = np.zeros(0, np.int32), np.zeros(0)
    so, c2, gr, nu, fl = O.refine(g, f, P, none_i, none_f, none_i, sd, n_iter=3)
    assert c2 == 0.0 and nu == 0 and np.all(gr == 0.0)
    assert np.array_equal(so, sd)
    assert fl & 8
    c2b, grb = O.chi2(g, f, P, none_i, none_f, none_i, sd)[:2]
    assert c2b == 0.0 and np.all(grb == 0.0)
