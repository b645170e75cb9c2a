"""Seeded synthetic inputs for the COMET CDC seed-scanning track finder.

This module builds *inputs only*: the drift-chamber geometry parameters, the
magnetic-field samples and simulated events (fired wires with drift distances)
shaped like the workloads of the paper (sec. 1: 18 stereo sense layers, 1 T
solenoid, 104.97 MeV signal electrons from an aluminium target; sec. 2.1:
seeds defined at R0 = 50 cm).  It holds none of the track finder's arithmetic:
the truth tracks are made with the closed-form helix (uniform field) or a
classical 6-D Runge-Kutta simulation (field map; a small C loop in _sim.c,
built with gcc on first use), and the hits with a plain dense-sampling
distance search.  Both the FP64 oracle and the CUDA library
consume what it returns; neither is imported here.

Units: mm, MeV/c, T, rad.  Electron charge q = -1.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

KAPPA = 0.299792458          # MeV/c per (T mm): rho[mm] = pT / (KAPPA * B)
SIGNAL_P = 104.97            # MeV/c, mu -> e conversion on Al (sec. 1)
BASE_SEED = 1908_01949


# ---------------------------------------------------------------- geometry
@dataclass
class Geometry:
    """Sense-layer parameters of a stereo drift chamber (sec. 1: 18 layers)."""
    R: np.ndarray          # float64[L] waist radius at z = 0 [mm]
    alpha: np.ndarray      # float64[L] stereo angle [rad]
    N: np.ndarray          # int32[L] wires per layer
    phi_off: np.ndarray    # float64[L] azimuth of wire 0 [rad]
    z_half: float = 750.0  # active half length [mm]
    R0: float = 500.0      # seed cylinder (sec. 2.1: 50 cm)
    R_out: float = 840.0   # outer stop radius [mm]

    @property
    def n_layers(self) -> int:
        return int(self.R.shape[0])

    @property
    def n_wires(self) -> int:
        return int(self.N.sum())

    @property
    def base(self) -> np.ndarray:
        return np.concatenate([[0], np.cumsum(self.N)[:-1]]).astype(np.int64)


def make_geometry(n_layers: int = 18, r_first: float = 530.0, r_last: float = 820.0,
                  n_first: int = 150, n_last: int = 300, stereo: float = 0.070) -> Geometry:
    """18 alternating-stereo layers, 530-820 mm, 150-300 wires (4050 total)."""
    l = np.arange(n_layers)
    R = r_first + l * (r_last - r_first) / (n_layers - 1)
    N = np.array([n_first + int(round((n_last - n_first) * i / (n_layers - 1))) for i in l],
                 dtype=np.int32)
    alpha = np.where(l % 2 == 0, stereo, -stereo).astype(np.float64)
    phi_off = (l % 2) * np.pi / N
    return Geometry(R=R.astype(np.float64), alpha=alpha, N=N, phi_off=phi_off.astype(np.float64))


def wire_lines(g: Geometry):
    """Per-wire midpoint m (z = 0) and unit direction d, float64 [W,3] each.

    Wire i of layer l sits at azimuth phi = phi_off + 2 pi i / N at z = 0 and
    is tilted by the stereo angle alpha in the azimuthal direction."""
    ms, ds, lay = [], [], []
    for li in range(g.n_layers):
        phi = g.phi_off[li] + 2.0 * np.pi * np.arange(g.N[li]) / g.N[li]
        c, s = np.cos(phi), np.sin(phi)
        sa, ca = math.sin(g.alpha[li]), math.cos(g.alpha[li])
        ms.append(np.stack([g.R[li] * c, g.R[li] * s, np.zeros_like(c)], 1))
        ds.append(np.stack([-sa * s, sa * c, np.full_like(c, ca)], 1))
        lay.append(np.full(g.N[li], li, dtype=np.int32))
    return np.concatenate(ms), np.concatenate(ds), np.concatenate(lay)


# ------------------------------------------------------------------- field
@dataclass
class Field:
    kind: int                      # 0 uniform Bz, 1 axisymmetric (r,z) map
    B0: float = 1.0
    bz: np.ndarray | None = None   # float32[nr, nz]
    br: np.ndarray | None = None
    r_min: float = 0.0
    z_min: float = 0.0
    dr: float = 1.0
    dz: float = 1.0

    @property
    def nr(self) -> int:
        return 0 if self.bz is None else int(self.bz.shape[0])

    @property
    def nz(self) -> int:
        return 0 if self.bz is None else int(self.bz.shape[1])


def uniform_field(B0: float = 1.0) -> Field:
    return Field(kind=0, B0=float(B0))


def cel(kc, p, c, s, iters: int = 40):
    """Bulirsch's general complete elliptic integral (Numer. Math. 13, 1969),
    cel(kc,p,c,s) = int_0^{pi/2} (c cos^2 + s sin^2) /
                    ((cos^2 + p sin^2) sqrt(cos^2 + kc^2 sin^2)) dphi,
    evaluated with the published Gauss-type iteration (vectorised, p > 0 only)."""
    kc = np.abs(np.asarray(kc, dtype=np.float64))
    p = np.asarray(p, dtype=np.float64) * np.ones_like(kc)
    c = np.asarray(c, dtype=np.float64) * np.ones_like(kc)
    s = np.asarray(s, dtype=np.float64) * np.ones_like(kc)
    if np.any(p <= 0):
        raise ValueError("cel: this restatement needs p > 0")
    em = np.ones_like(kc)
    pp = np.sqrt(p)
    ss = s / pp
    f = c.copy()
    cc = c + ss / pp
    g = kc / pp
    ss = 2.0 * (ss + f * g)
    pp = g + pp
    g = em.copy()
    em = kc + em
    kk = kc.copy()
    k = kc.copy()
    for _ in range(iters):
        done = np.abs(g - k) <= g * 1e-15
        if np.all(done):
            break
        k = 2.0 * np.sqrt(kk)
        kk = k * em
        f = cc
        cc = cc + ss / pp
        g = kk / pp
        ss = 2.0 * (ss + f * g)
        pp = g + pp
        g = em
        em = k + em
    return 0.5 * np.pi * (ss + cc * em) / (em * (em + pp))


def solenoid_field_rz(rho, z, a: float, b: float):
    """Field of an ideal finite current sheet (radius a, half-length b) in units
    of mu0 n I, closed form of Derby & Olbert, Am. J. Phys. 78 (2010) 229.
    Returns (Bz, Br) float64 arrays."""
    rho = np.asarray(rho, dtype=np.float64)
    z = np.asarray(z, dtype=np.float64)
    bz = np.zeros(np.broadcast(rho, z).shape)
    br = np.zeros_like(bz)
    rho_b = np.broadcast_to(rho, bz.shape)
    z_b = np.broadcast_to(z, bz.shape)
    gamma = (a - rho_b) / (a + rho_b)
    for sign in (+1.0, -1.0):
        zs = z_b + sign * b
        den = np.sqrt(zs * zs + (rho_b + a) ** 2)
        alpha = a / den
        beta = zs / den
        k = np.sqrt((zs * zs + (a - rho_b) ** 2) / (zs * zs + (a + rho_b) ** 2))
        k = np.maximum(k, 1e-300)
        br += sign * alpha * cel(k, 1.0, 1.0, -1.0)
        bz += sign * (a / (a + rho_b)) * beta * cel(k, gamma * gamma, 1.0, gamma)
    # B0 = mu0 n I / pi
    return bz / np.pi, br / np.pi


def solenoid_map(nr: int = 451, nz: int = 1001, r_min: float = 0.0, z_min: float = -1000.0,
                 dr: float = 2.0, dz: float = 2.0, a: float = 1000.0, b: float = 1500.0,
                 b_centre: float = 1.0) -> Field:
    """(Bz, Br) of a finite solenoid sampled to FP32 on an (r, z) grid, scaled so
    that Bz(0, 0) = b_centre tesla."""
    r = r_min + dr * np.arange(nr)
    zz = z_min + dz * np.arange(nz)
    R, Z = np.meshgrid(r, zz, indexing="ij")
    bz, br = solenoid_field_rz(R, Z, a, b)
    bz0, _ = solenoid_field_rz(np.array([0.0]), np.array([0.0]), a, b)
    scale = b_centre / float(bz0[0])
    return Field(kind=1, B0=b_centre, bz=(bz * scale).astype(np.float32),
                 br=(br * scale).astype(np.float32), r_min=r_min, z_min=z_min, dr=dr, dz=dz)


# -------------------------------------------------------- truth simulation
_HERE = os.path.dirname(os.path.abspath(__file__))
_SIM_SRC = os.path.join(_HERE, "_sim.c")
_SIM_LIB = os.path.join(_HERE, "_build", "libsynth.so")
_sim = None
_sim_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile the field-map truth simulator (_sim.c) with gcc, no FMA
    contraction, so every machine produces the same events."""
    os.makedirs(os.path.dirname(_SIM_LIB), exist_ok=True)
    if force or not os.path.exists(_SIM_LIB) or os.path.getmtime(_SIM_LIB) < os.path.getmtime(_SIM_SRC):
        tmp = _SIM_LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-o", tmp,
                               _SIM_SRC, "-lm"])
        os.replace(tmp, _SIM_LIB)
    return _SIM_LIB


def _sim_lib():
    global _sim
    with _sim_lock:
        if _sim is None:
            L = ctypes.CDLL(build())
            d, i, pd, pf = ctypes.c_double, ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_float)
            L.synth_track_map.argtypes = [pf, pf, i, i, d, d, d, d, d, pd, pd, d, i, d, d, pd, pd]
            L.synth_track_map.restype = i
            _sim = L
    return _sim


def _map_track(f: "Field", r0, t0, lam, ds, n, z_stop, r_stop):
    bz = np.ascontiguousarray(f.bz, dtype=np.float32)
    br = np.ascontiguousarray(f.br, dtype=np.float32)
    r0 = np.ascontiguousarray(r0, dtype=np.float64)
    t0 = np.ascontiguousarray(t0, dtype=np.float64)
    pos = np.empty((n, 3))
    dirs = np.empty((n, 3))
    pf, pd = ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_double)
    m = _sim_lib().synth_track_map(bz.ctypes.data_as(pf), br.ctypes.data_as(pf), f.nr, f.nz, f.r_min, f.z_min, f.dr,
                                   f.dz, lam, r0.ctypes.data_as(pd), t0.ctypes.data_as(pd), ds, n, z_stop, r_stop,
                                   pos.ctypes.data_as(pd), dirs.ctypes.data_as(pd))
    return pos[:m], dirs[:m]


def simulate_track(f: Field, r0, p0, q: float = -1.0, max_len: float = 8000.0,
                   ds: float = 1.0, z_stop: float = 800.0, r_stop: float = 900.0):
    """Truth trajectory sampled every ds mm: returns (pos [n,3], dir [n,3]).

    Uniform field: closed-form helix.  Map: classical RK4 on (r, t) with step ds
    (_sim.c).  Stops once |z| > z_stop or rho > r_stop or after max_len."""
    r0 = np.asarray(r0, dtype=np.float64)
    p0 = np.asarray(p0, dtype=np.float64)
    p = float(np.linalg.norm(p0))
    t0 = p0 / p
    n = int(max_len / ds) + 1
    if f.kind == 0:
        w = q * KAPPA * f.B0 / p
        s = ds * np.arange(n)
        cw, sw = np.cos(w * s), np.sin(w * s)
        pos = np.stack([r0[0] + (t0[0] * sw + t0[1] * (1 - cw)) / w,
                        r0[1] + (t0[1] * sw - t0[0] * (1 - cw)) / w,
                        r0[2] + t0[2] * s], 1)
        dirs = np.stack([t0[0] * cw + t0[1] * sw, t0[1] * cw - t0[0] * sw,
                         np.full_like(s, t0[2])], 1)
    else:
        pos, dirs = _map_track(f, r0, t0, q * KAPPA / p, ds, n, z_stop, r_stop)
    rho = np.hypot(pos[:, 0], pos[:, 1])
    out = np.nonzero((np.abs(pos[:, 2]) > z_stop) | (rho > r_stop))[0]
    if out.size:
        pos, dirs = pos[: out[0] + 1], dirs[: out[0] + 1]
    return pos, dirs


def turn_labels(pos: np.ndarray, R0: float):
    """Partition label per sample: number of outward R0 crossings so far - 1."""
    rho = np.hypot(pos[:, 0], pos[:, 1])
    outward = (rho[1:] >= R0) & (rho[:-1] < R0)
    lab = np.concatenate([[0], np.cumsum(outward)]) - 1
    return lab, np.nonzero(outward)[0]


def inward_crossings(pos: np.ndarray, R0: float):
    """Sample indices i with an inward R0 crossing between samples i and i + 1."""
    rho = np.hypot(pos[:, 0], pos[:, 1])
    return np.nonzero((rho[1:] < R0) & (rho[:-1] >= R0))[0]


def exit_seeds(pos, dirs, outward, R0, p):
    """Per turn (started at the outward crossings `outward`), the state at the
    first inward R0 crossing after its start, or NaN."""
    inw = inward_crossings(pos, R0)
    out = np.full((len(outward), 5), np.nan)
    for k, c in enumerate(outward):
        after = inw[inw > c]
        end = outward[k + 1] if k + 1 < len(outward) else len(pos)
        if after.size and after[0] < end:
            out[k] = crossing_seed(pos, dirs, int(after[0]), R0, p)
    return out


def crossing_seed(pos, dirs, i, R0, p):
    """Truth seed (theta0, z0, px0, py0, pz0) at the R0 crossing in (i, i+1)."""
    r1 = math.hypot(pos[i, 0], pos[i, 1])
    r2 = math.hypot(pos[i + 1, 0], pos[i + 1, 1])
    w = (R0 - r1) / (r2 - r1)
    P = pos[i] + w * (pos[i + 1] - pos[i])
    T = dirs[i] + w * (dirs[i + 1] - dirs[i])
    T /= np.linalg.norm(T)
    P[:2] *= R0 / math.hypot(P[0], P[1])
    return np.array([math.atan2(P[1], P[0]), P[2], p * T[0], p * T[1], p * T[2]])


def track_hits(g: Geometry, wm, wd, pos: np.ndarray, labels: np.ndarray):
    """Fired wires of one simulated track: per wire its true distance of closest
    approach (dense samples, each refined on its chord) if it is within half a
    cell width and inside the active length.  Returns dict wire -> (doca, label)."""
    rho = np.hypot(pos[:, 0], pos[:, 1])
    res = {}
    base = g.base
    spacing = np.min(np.diff(g.R)) if g.n_layers > 1 else 20.0
    inside = (np.abs(pos[:, 2]) <= g.z_half) & (labels >= 0)
    for li in range(g.n_layers):
        rl = np.sqrt(g.R[li] ** 2 + (pos[:, 2] * math.tan(g.alpha[li])) ** 2)
        sel = np.nonzero(inside & (np.abs(rho - rl) < 0.5 * spacing + 2.0))[0]
        if sel.size == 0:
            continue
        N = int(g.N[li])
        phi = np.arctan2(pos[sel, 1], pos[sel, 0])
        twist = np.arctan(pos[sel, 2] * math.tan(g.alpha[li]) / g.R[li])
        c = (phi - twist - g.phi_off[li]) * N / (2 * np.pi)
        half_cell = math.pi * g.R[li] / N
        for off in (-1, 0, 1):
            i = (np.floor(c + 0.5).astype(np.int64) + off) % N
            w = base[li] + i
            d = _seg_line_dist(pos, sel, wm[w], wd[w])
            for wid in np.unique(w):
                m = w == wid
                k = np.argmin(d[m])
                dmin = float(d[m][k])
                if dmin <= half_cell:
                    lab = int(labels[sel[m][k]])
                    old = res.get(int(wid))
                    if old is None or dmin < old[0]:
                        res[int(wid)] = (dmin, lab)
    return res


def _seg_line_dist(pos, sel, m, d):
    """Distance from the chords (pos[j], pos[j+1]), j in sel, to the lines (m, d)."""
    j = np.minimum(sel, len(pos) - 2)
    a = pos[j] - m
    b = pos[j + 1] - pos[j]
    # minimise |(a + u b) x d| over u in [0, 1]
    ap = a - (a * d).sum(1, keepdims=True) * d
    bp = b - (b * d).sum(1, keepdims=True) * d
    bb = (bp * bp).sum(1)
    u = np.clip(-(ap * bp).sum(1) / np.maximum(bb, 1e-300), 0.0, 1.0)
    v = ap + u[:, None] * bp
    return np.sqrt((v * v).sum(1))


# ------------------------------------------------------------------ events
@dataclass
class Event:
    wire_id: np.ndarray            # int32[H]
    drift: np.ndarray              # float32[H] mm
    truth_part: np.ndarray         # int8[H]: signal partition, -1 noise
    truth_seeds: np.ndarray        # float64[n_turns, 5] at each outward R0 crossing
    n_turns: int
    signal_p0: np.ndarray = field(default_factory=lambda: np.zeros(3))
    signal_r0: np.ndarray = field(default_factory=lambda: np.zeros(3))
    # float64[n_turns, 5]: state at the inward R0 crossing that ends each turn
    # (momentum along the motion; NaN for a turn that leaves through an end
    # plate), the seed of the reversed scan of that turn
    exit_seeds: np.ndarray = field(default_factory=lambda: np.zeros((0, 5)))


def _iso_dir(rng):
    while True:
        v = rng.uniform(-1, 1, 3)
        n = float(v @ v)
        if 1e-6 < n <= 1.0:
            return v / math.sqrt(n)


def _target_point(rng, z_range=(-400.0, 400.0), r_target=100.0):
    r = r_target * math.sqrt(rng.uniform())
    ph = rng.uniform(0, 2 * math.pi)
    return np.array([r * math.cos(ph), r * math.sin(ph), rng.uniform(*z_range)])


def _signal(g, f, rng, turns, max_tries=20000, min_hits=20, p=SIGNAL_P, max_hits=None):
    """Draw a signal e- from the target that reaches layer >= 4, leaves through
    |z| > z_half between R0 and R_out and makes the requested number of turns."""
    wm, wd, _ = wire_lines(g)
    uf = uniform_field(f.B0)
    for _ in range(max_tries):
        r0 = _target_point(rng)
        t = _iso_dir(rng)
        pt = p * math.hypot(t[0], t[1])
        if pt < KAPPA * f.B0 * 0.5 * (g.R[4] - 100.0):
            continue   # max radius <= 2 rho + 100 mm cannot reach layer 4
        if f.kind != 0:
            # cheap pre-selection in the nominal uniform field
            pos, _ = simulate_track(uf, r0, p * t, max_len=8000.0, ds=4.0,
                                    z_stop=g.z_half, r_stop=g.R_out)
            _, cr = turn_labels(pos, g.R0)
            if len(cr) < max(1, min(turns) - 1) or len(cr) > max(turns) + 1:
                continue
        pos, dirs = simulate_track(f, r0, p * t, max_len=8000.0, ds=1.0,
                                   z_stop=g.z_half, r_stop=g.R_out)
        lab, cr = turn_labels(pos, g.R0)
        rho = np.hypot(pos[:, 0], pos[:, 1])
        if len(cr) not in turns or rho.max() < g.R[4]:
            continue
        if not (abs(pos[-1, 2]) > g.z_half and g.R0 <= rho[-1] <= g.R_out):
            continue
        hits = track_hits(g, wm, wd, pos, lab)
        if len(hits) < min_hits or (max_hits is not None and len(hits) > max_hits):
            continue
        seeds = np.array([crossing_seed(pos, dirs, i, g.R0, p) for i in cr])
        return hits, seeds, len(cr), r0, p * t, exit_seeds(pos, dirs, cr, g.R0, p)
    raise RuntimeError("signal generation failed")


def _dio_hits(g, f, rng, target_wires, taken, wm, wd):
    """DIO-like e- (p uniform 40-100 MeV/c) from the target, nominal-field helix,
    until the requested number of distinct wires has fired."""
    uf = uniform_field(f.B0)
    out = {}
    tries = 0
    while len(out) < target_wires and tries < 200000:
        tries += 1
        p = rng.uniform(40.0, 100.0)
        t = _iso_dir(rng)
        pos, dirs = simulate_track(uf, _target_point(rng), p * t, max_len=6000.0, ds=1.0,
                                   z_stop=g.z_half + 2.0, r_stop=g.R_out + 20)
        lab, _ = turn_labels(pos, g.R0)
        if np.hypot(pos[:, 0], pos[:, 1]).max() < g.R[0] - 10:
            continue
        for w, (d, _) in track_hits(g, wm, wd, pos, lab).items():
            if w in taken or w in out:
                continue
            out[w] = d
            if len(out) >= target_wires:
                break
    return out


def make_event(g: Geometry, f: Field, rng: np.random.Generator, turns=(1,),
               noise: str = "uniform", n_noise: int = 40, occupancy: float = 0.0,
               sigma: float = 0.2, max_drift: float = 8.0, min_hits: int = 20, max_hits=None) -> Event:
    """One event: a signal e- plus noise.  noise='uniform': n_noise random wires
    with drift U[0, max_drift]; noise='dio': DIO-like tracks up to `occupancy`
    of all wires."""
    wm, wd, _ = wire_lines(g)
    hits, seeds, nt, r0, p0, xseeds = _signal(g, f, rng, turns, min_hits=min_hits, max_hits=max_hits)
    wires = sorted(hits)
    drift = [min(max(hits[w][0] + rng.normal(0.0, sigma), 0.0), max_drift) for w in wires]
    part = [hits[w][1] for w in wires]
    taken = set(wires)
    if noise == "uniform" and n_noise > 0:
        free = np.array([w for w in range(g.n_wires) if w not in taken])
        pick = rng.choice(free, size=min(n_noise, free.size), replace=False)
        for w in pick:
            wires.append(int(w))
            drift.append(float(rng.uniform(0.0, max_drift)))
            part.append(-1)
    elif noise == "dio" and occupancy > 0:
        target = int(round(occupancy * g.n_wires))
        for w, d in _dio_hits(g, f, rng, target, taken, wm, wd).items():
            wires.append(int(w))
            drift.append(min(max(d + rng.normal(0.0, sigma), 0.0), max_drift))
            part.append(-1)
    order = rng.permutation(len(wires))
    return Event(wire_id=np.asarray(wires, dtype=np.int32)[order],
                 drift=np.asarray(drift, dtype=np.float32)[order],
                 truth_part=np.asarray(part, dtype=np.int8)[order],
                 truth_seeds=seeds, n_turns=nt, signal_p0=np.asarray(p0), signal_r0=np.asarray(r0),
                 exit_seeds=xseeds)


def pack_events(events):
    """CSR packing: (hit_off int32[E+1], wire_id int32[H], drift float32[H])."""
    off = np.zeros(len(events) + 1, dtype=np.int32)
    off[1:] = np.cumsum([e.wire_id.size for e in events])
    if not events:
        return off, np.zeros(0, np.int32), np.zeros(0, np.float32)
    return (off, np.concatenate([e.wire_id for e in events]).astype(np.int32),
            np.concatenate([e.drift for e in events]).astype(np.float32))


# ------------------------------------------------------------------- grids
GRID_DTYPE = np.dtype([("centre", np.float32, 5), ("step", np.float32, 5), ("n", np.int32, 5)])


def make_grid(centre, step, n) -> np.ndarray:
    """One seed grid record: values centre + (i - (n-1)/2) * step per axis over
    (theta0, z0, px0, py0, pz0); seeds enumerated row-major in that order."""
    g = np.zeros(1, dtype=GRID_DTYPE)
    g["centre"][0] = centre
    g["step"][0] = step
    g["n"][0] = n
    return g


# Config-shaped workloads (sec. 2.1 resolutions: 0.01 rad, 2.5 MeV; sec. 2.3: 2.6 cm, 1.7 MeV)
CFG1_STEP = (0.01, 26.0, 2.5, 2.5, 1.7)
CFG1_N = (8, 4, 5, 5, 5)


def cfg1_case(index: int = 0):
    """Single-turn 104.97 MeV e- in a uniform 1 T field, 40 uniform noise wires,
    a 4000-seed grid around the truth (random sub-step offset per axis)."""
    rng = np.random.default_rng(BASE_SEED + index)
    g = make_geometry()
    f = uniform_field(1.0)
    ev = make_event(g, f, rng, turns=(1,), noise="uniform", n_noise=40)
    off = rng.uniform(-0.5, 0.5, 5) * np.asarray(CFG1_STEP)
    grid = make_grid(ev.truth_seeds[0] + off, CFG1_STEP, CFG1_N)
    return g, f, ev, grid


# Radii and angles of the multi-turn configuration's circle Hough: a 104.97 MeV/c electron that makes
# two or three turns before leaving |z| <= 750 mm has |pz| below ~30 MeV/c, so p_T >= ~97.4 MeV/c and a
# transverse radius of at least 325 mm at 1 T; the window R_j = 325 + 5 j mm, j < 7, reaches 355 mm
# (p_T = 106 MeV/c).  1024 vote angles keep consecutive votes of a hit 2.2 mm apart at 355 mm, about a
# 2 mm bin, where 512 would skip every other bin.
CFG2_HOUGH = {"n_r": 7, "r_min_um": 325000, "r_step_um": 5000, "n_phi": 1024}


def cfg2_grid_template():
    """(z0, pz0) ranges of the multi-turn single-event workload: 40 x 25 points,
    35 mm and 4 MeV/c steps, centred at 0; (theta0, px0, py0) 10 x 10 x 10 at
    0.01 rad, 2.5, 2.5 MeV/c around the circle-Hough output."""
    return make_grid((0.0, 0.0, 0.0, 0.0, 0.0), (0.01, 35.0, 2.5, 2.5, 4.0), (10, 40, 10, 10, 25))


def cfg2_case(index: int = 0, field_map: Field | None = None, occupancy: float = 0.10):
    """Multi-turn (2-3 turns) e- in the solenoid map with DIO-like noise."""
    rng = np.random.default_rng(BASE_SEED + 1000 + index)
    g = make_geometry()
    f = field_map if field_map is not None else solenoid_map()
    ev = make_event(g, f, rng, turns=(2, 3), noise="dio", occupancy=occupancy)
    return g, f, ev


# ------------------------------------------------------------ batched events
CFG3_EVENTS = 256
CFG3_SEEDS = (1.0e4, 1.0e6)


def scaled_grid(truth_seed, n_seeds: float, rng: np.random.Generator) -> np.ndarray:
    """The multi-turn grid with every axis count scaled by f = (n_seeds / 10^6)^(1/5)
    (steps scaled by the inverse ratio, so each axis keeps its span): (theta0,
    px0, py0) around the truth plus a random sub-step offset, (z0, pz0) around 0."""
    tmpl = cfg2_grid_template()
    n0 = tmpl["n"][0].astype(np.float64)
    s0 = tmpl["step"][0].astype(np.float64)
    f = (float(n_seeds) / float(np.prod(n0))) ** 0.2
    n = np.maximum(1, np.round(n0 * f)).astype(np.int32)
    step = s0 * n0 / n
    centre = np.array([truth_seed[0], 0.0, truth_seed[2], truth_seed[3], 0.0])
    off = rng.uniform(-0.5, 0.5, 5) * step
    off[[1, 4]] = 0.0
    return make_grid(centre + off, step, n)


def cfg3_event(index: int, field_map: Field | None = None, seeds=CFG3_SEEDS):
    """One event of the batched workload: a signal e- of 1-3 turns with 30-200
    hits, DIO-like noise at an occupancy uniform in 5-20 %, and a seed grid whose
    size is log-uniform in `seeds` (the multi-turn grid scaled, see scaled_grid)."""
    rng = np.random.default_rng(BASE_SEED + 2000 + index)
    g = make_geometry()
    f = field_map if field_map is not None else solenoid_map()
    occ = rng.uniform(0.05, 0.20)
    n_seeds = math.exp(rng.uniform(math.log(seeds[0]), math.log(seeds[1])))
    ev = make_event(g, f, rng, turns=(1, 2, 3), noise="dio", occupancy=occ, min_hits=30, max_hits=200)
    return ev, scaled_grid(ev.truth_seeds[0], n_seeds, rng)


def cfg3_case(n_events: int = CFG3_EVENTS, field_map: Field | None = None, seeds=CFG3_SEEDS, first: int = 0):
    """Batched workload: geometry, field, events and grids [n_events]."""
    f = field_map if field_map is not None else solenoid_map()
    out = [cfg3_event(first + i, f, seeds) for i in range(n_events)]
    grids = np.concatenate([gr for _, gr in out])
    return make_geometry(), f, [ev for ev, _ in out], grids


CFG4_EVENTS = 1024


def cfg4_event(index: int, field_map: Field | None = None, n_seeds: float = 2.0e4):
    """One event of the differentiable-refine workload: a 3-turn e- with DIO-like
    noise at 10 % occupancy, and a scaled multi-turn grid of ~n_seeds seeds
    around its first turn from which a scan selects the seeds to refine."""
    rng = np.random.default_rng(BASE_SEED + 4000 + index)
    g = make_geometry()
    f = field_map if field_map is not None else solenoid_map()
    ev = make_event(g, f, rng, turns=(3,), noise="dio", occupancy=0.10)
    return ev, scaled_grid(ev.truth_seeds[0], n_seeds, rng)


CFG5_EVENTS = 64
CFG5_SEEDS = 1.0e7


def cfg5_event(index: int, field_map: Field | None = None, n_seeds: float = CFG5_SEEDS / CFG5_EVENTS):
    """One event of the precision/scale sweep: a 1-3 turn signal and DIO-like
    noise at 30 % occupancy, with a scaled multi-turn grid of ~n_seeds seeds."""
    rng = np.random.default_rng(BASE_SEED + 3000 + index)
    g = make_geometry()
    f = field_map if field_map is not None else solenoid_map()
    ev = make_event(g, f, rng, turns=(1, 2, 3), noise="dio", occupancy=0.30)
    return ev, scaled_grid(ev.truth_seeds[0], n_seeds, rng)


def sweep_geometry(g: Geometry) -> Geometry:
    """The chamber without its stop surfaces (|z| and rho limits far outside), for
    fixed-length propagation of the precision sweep."""
    return Geometry(R=g.R, alpha=g.alpha, N=g.N, phi_off=g.phi_off, z_half=5000.0, R0=g.R0, R_out=980.0)
