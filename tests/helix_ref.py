"""Second, independent enumerator for the oracle pins (uniform field only).

It never calls the oracle: positions come from the closed-form helix, the
distance of closest approach from dense sampling of that helix refined with
scipy's bounded scalar minimiser, and Eq. 1 is summed directly.  The discrete
stop and partition rules (the same reading the oracle implements) are applied
to helix points at s = j h."""
from __future__ import annotations

import math

import numpy as np
from scipy.optimize import minimize_scalar

KAPPA = 0.299792458


def helix(seed, B0, s, R0, charge=-1.0, direction=1):
    """Closed-form helix point(s) and direction(s) at arclength s from a seed."""
    th, z0, px, py, pz = seed
    p = math.sqrt(px * px + py * py + pz * pz)
    dirn = -1.0 if direction < 0 else 1.0
    t0 = dirn * np.array([px, py, pz]) / p
    w = dirn * charge * KAPPA * B0 / p
    s = np.asarray(s, dtype=np.float64)
    cw, sw = np.cos(w * s), np.sin(w * s)
    x = R0 * math.cos(th) + (t0[0] * sw + t0[1] * (1 - cw)) / w
    y = R0 * math.sin(th) + (t0[1] * sw - t0[0] * (1 - cw)) / w
    z = z0 + t0[2] * s
    tx = t0[0] * cw + t0[1] * sw
    ty = t0[1] * cw - t0[0] * sw
    return np.stack([x, y, z], -1), np.stack([tx, ty, np.full_like(s, t0[2])], -1)


def trace_rule(seed, B0, h, max_steps, max_partitions, R0, R_out, z_half, charge=-1.0, direction=1):
    """Number of steps n and the partition label of states 0..n (stop rules of
    the scan: inward R0 crossing ends a partition; |z| > z_half or rho > R_out
    ends the track; at most max_steps steps)."""
    labels = [0]
    part, outside = 0, True
    n = 0
    while n < max_steps:
        n += 1
        pos, _ = helix(seed, B0, n * h, R0, charge, direction)
        rho = math.hypot(pos[0], pos[1])
        now_out = rho >= R0
        stop = False
        if outside and not now_out:
            part += 1
            stop = part >= max_partitions
        outside = now_out
        if abs(pos[2]) > z_half or rho > R_out:
            stop = True
        labels.append(part)
        if stop:
            break
    return n, np.array(labels)


def line_dist(P, m, d):
    w = P - m
    wd = w @ d
    q = w - np.outer(wd, d) if w.ndim == 2 else w - wd * d
    return np.sqrt((q * q).sum(-1))


def doca_per_partition(seed, B0, h, n, labels, m, d, R0, max_partitions, charge=-1.0, direction=1, ds=0.02):
    s_end = n * h
    s = np.linspace(0.0, s_end, int(math.ceil(s_end / ds)) + 1)
    P, _ = helix(seed, B0, s, R0, charge, direction)
    D = line_dist(P, m, d)
    best = [math.inf] * max_partitions
    idx = [i for i in range(len(s))
           if (i == 0 or D[i] <= D[i - 1]) and (i == len(s) - 1 or D[i] < D[i + 1])]
    for i in idx:
        lo, hi = s[max(i - 1, 0)], s[min(i + 1, len(s) - 1)]
        f = lambda u: float(line_dist(helix(seed, B0, u, R0, charge, direction)[0], m, d))
        if hi > lo:
            r = minimize_scalar(f, bounds=(lo, hi), method="bounded", options={"xatol": 1e-12})
            sv, dv = float(r.x), float(r.fun)
            for e in (lo, hi):
                fe = f(e)
                if fe < dv:
                    sv, dv = e, fe
        else:
            sv, dv = lo, f(lo)
        k = int(labels[min(int(sv // h), n)])
        if k < max_partitions and dv < best[k]:
            best[k] = dv
    return best


def score(seed, B0, h, max_steps, max_partitions, lam, geom_lines, wire_id, drift, R0, R_out, z_half,
          charge=-1.0, direction=1):
    """Eq. 1 with per-hit best squared residual and partition."""
    wm, wd = geom_lines
    n, labels = trace_rule(seed, B0, h, max_steps, max_partitions, R0, R_out, z_half, charge, direction)
    E = 0.0
    res2, parts = [], []
    for w, dr in zip(wire_id, drift):
        best = doca_per_partition(seed, B0, h, n, labels, wm[w], wd[w], R0, max_partitions, charge, direction)
        r2 = [(b - dr) ** 2 if math.isfinite(b) else math.inf for b in best]
        k = int(np.argmin(r2))
        E += min(r2[k], lam)
        res2.append(r2[k])
        parts.append(k if r2[k] < lam else -1)
    return E, np.array(res2), np.array(parts), n
