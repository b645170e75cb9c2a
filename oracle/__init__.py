"""FP64 CPU oracle of the seed-scanning track finder (arXiv:1908.01949).

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the benchmark's
CPU-baseline leg and reference arm are the only users.  The arithmetic lives in oracle.c
(plain C, double precision); this module builds it with gcc, marshals numpy
arrays through ctypes, and adds the steps that are library primitives (sort
for the top-K) or plain control flow over the C routines: the repeated scan
around the best seeds (zoom_scan, sec. 2.2) and the event loop over turn
partitions (event_loop, sec. 2.3, Fig. 7).
It imports nothing from the CUDA package.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_OUT = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None
_lock = threading.Lock()

FLAG_STEP_CAP = 1
FLAG_NOT_SPD = 8
FLAG_DOCA_ZERO = 16
FLAG_LOST_HIT = 32


def build(force: bool = False) -> str:
    """Compile oracle.c into _build/liboracle.so (gcc -O2, no fast-math)."""
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    if force or not os.path.exists(_OUT) or os.path.getmtime(_OUT) < os.path.getmtime(_SRC):
        tmp = _OUT + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _OUT)
    return _OUT


class Geometry(C.Structure):
    _fields_ = [("n_layers", C.c_int), ("R", C.POINTER(C.c_double)), ("alpha", C.POINTER(C.c_double)),
                ("N", C.POINTER(C.c_int)), ("phi_off", C.POINTER(C.c_double)),
                ("z_half", C.c_double), ("R0", C.c_double), ("R_out", C.c_double)]


class Field(C.Structure):
    _fields_ = [("kind", C.c_int), ("B0", C.c_double), ("nr", C.c_int), ("nz", C.c_int),
                ("r_min", C.c_double), ("z_min", C.c_double), ("dr", C.c_double), ("dz", C.c_double),
                ("bz", C.POINTER(C.c_float)), ("br", C.POINTER(C.c_float))]


class ScanParams(C.Structure):
    _fields_ = [("h", C.c_double), ("max_steps", C.c_int), ("lam", C.c_double),
                ("max_partitions", C.c_int), ("direction", C.c_int), ("charge", C.c_double)]


class HoughParams(C.Structure):
    _fields_ = [("n_bins", C.c_int), ("bin_um", C.c_int), ("origin_um", C.c_int), ("n_r", C.c_int),
                ("r_min_um", C.c_int), ("r_step_um", C.c_int), ("n_phi", C.c_int), ("target_um", C.c_int),
                ("min_peak", C.c_int), ("max_cand", C.c_int), ("r_hist_half_um", C.c_int),
                ("b_nominal", C.c_double), ("charge", C.c_double), ("R0", C.c_double)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = C.CDLL(build())
            P = C.POINTER
            dp, ip, fp = P(C.c_double), P(C.c_int), P(C.c_int32)
            _lib.orc_scan.argtypes = [P(Geometry), P(Field), P(ScanParams), C.c_int, ip, dp, C.c_int, dp, dp,
                                      ip, ip, dp, dp, ip, dp]
            _lib.orc_propagate.argtypes = [P(Geometry), P(Field), P(ScanParams), dp, C.c_int, dp, ip, dp]
            _lib.orc_step.argtypes = [P(Field), C.c_double, C.c_double, dp, dp, dp, dp]
            _lib.orc_step.restype = None
            _lib.orc_field_at.argtypes = [P(Field), dp, dp, dp]
            _lib.orc_field_at.restype = None
            _lib.orc_hough_vote.argtypes = [P(Geometry), P(HoughParams), C.c_int, ip, fp]
            _lib.orc_hough_peaks.argtypes = [P(Geometry), P(HoughParams), C.c_int, ip, fp, fp, dp]
            _lib.orc_refine.argtypes = [P(Geometry), P(Field), P(ScanParams), C.c_int, C.c_double, dp, C.c_int,
                                        ip, dp, ip, dp, dp, dp, dp, ip, ip]
            _lib.orc_extrapolate_turn.argtypes = [P(Geometry), P(Field), P(ScanParams), dp, C.c_int, dp]
            _lib.orc_chi2.argtypes = [P(Geometry), P(Field), P(ScanParams), C.c_double, C.c_int, ip, dp, ip, dp,
                                      dp, dp, dp, ip, ip]
        return _lib


def _p(a, t):
    return a.ctypes.data_as(C.POINTER(t)) if a is not None else None


class _Keep:
    """Holds the numpy buffers a ctypes struct points into."""

    def __init__(self):
        self.refs = []

    def arr(self, a, dtype):
        a = np.ascontiguousarray(a, dtype=dtype)
        self.refs.append(a)
        return a


def _geom(g, keep):
    R = keep.arr(g.R, np.float64)
    al = keep.arr(g.alpha, np.float64)
    N = keep.arr(g.N, np.intc)
    ph = keep.arr(g.phi_off, np.float64)
    return Geometry(int(R.size), _p(R, C.c_double), _p(al, C.c_double), _p(N, C.c_int), _p(ph, C.c_double),
                    float(g.z_half), float(g.R0), float(g.R_out))


def _field(f, keep):
    if f.kind == 0:
        return Field(0, float(f.B0), 0, 0, 0.0, 0.0, 1.0, 1.0, None, None)
    bz = keep.arr(f.bz, np.float32)
    br = keep.arr(f.br, np.float32)
    return Field(1, float(f.B0), int(bz.shape[0]), int(bz.shape[1]), float(f.r_min), float(f.z_min),
                 float(f.dr), float(f.dz), _p(bz, C.c_float), _p(br, C.c_float))


def scan_params(h=2.0, max_steps=1000, lam=4.0, max_partitions=1, direction=1, charge=-1.0):
    return ScanParams(float(h), int(max_steps), float(lam), int(max_partitions), int(direction), float(charge))


# ------------------------------------------------------------------- seeds
def grid_values(grid) -> np.ndarray:
    """Seeds of one grid record, row-major over (theta0, z0, px0, py0, pz0).
    Axis value = centre + (i - (n-1)/2) * step, rounded once to float32 (the
    grid record is float32; the seed is the float32 nearest the exact value)."""
    c = np.asarray(grid["centre"], dtype=np.float32).reshape(5).astype(np.float64)
    s = np.asarray(grid["step"], dtype=np.float32).reshape(5).astype(np.float64)
    n = np.asarray(grid["n"]).reshape(5).astype(np.int64)
    axes = [(c[a] + (np.arange(n[a]) - (n[a] - 1) * 0.5) * s[a]).astype(np.float32) for a in range(5)]
    mesh = np.meshgrid(*axes, indexing="ij")
    return np.stack([m.reshape(-1) for m in mesh], 1).astype(np.float64)


# -------------------------------------------------------------------- scan
def scan(g, f, wire_id, drift, seeds, params: ScanParams, per_hit=False, threads=None):
    """Eq. 1 score of every seed (float64 [n,5]) by brute force; seeds are split
    across host threads (each thread runs the same C routine on its share)."""
    L = lib()
    keep = _Keep()
    G, F = _geom(g, keep), _field(f, keep)
    wid = keep.arr(wire_id, np.intc)
    dr = keep.arr(drift, np.float64)
    seeds = keep.arr(seeds, np.float64).reshape(-1, 5)
    n = seeds.shape[0]
    H = wid.size
    E = np.zeros(n)
    ns = np.zeros(n, np.intc)
    fl = np.zeros(n, np.intc)
    mg = np.zeros(n)
    hr = np.zeros((n, H)) if per_hit else None
    hp = np.zeros((n, H), np.intc) if per_hit else None
    hm = np.zeros((n, H)) if per_hit else None
    threads = threads or os.cpu_count() or 1
    chunks = np.array_split(np.arange(n), max(1, min(threads, n)))

    def run(idx):
        if idx.size == 0:
            return 0
        a = int(idx[0])
        m = int(idx.size)
        return L.orc_scan(C.byref(G), C.byref(F), C.byref(params), H, _p(wid, C.c_int), _p(dr, C.c_double), m,
                          _p(seeds[a:], C.c_double), _p(E[a:], C.c_double), _p(ns[a:], C.c_int),
                          _p(fl[a:], C.c_int), _p(mg[a:], C.c_double),
                          _p(hr[a:] if per_hit else None, C.c_double), _p(hp[a:] if per_hit else None, C.c_int),
                          _p(hm[a:] if per_hit else None, C.c_double))

    if len(chunks) == 1:
        rc = [run(chunks[0])]
    else:
        with ThreadPoolExecutor(len(chunks)) as ex:
            rc = list(ex.map(run, chunks))
    if any(rc):
        raise RuntimeError("orc_scan failed")
    out = dict(E=E, n_steps=ns, flags=fl, margin=mg)
    if per_hit:
        out.update(hit_res2=hr, hit_part=hp, hit_margin=hm)
    return out


def propagate(g, f, seed, params: ScanParams):
    """Recorded states (x,y,z,tx,ty,tz,partition) of one seed."""
    L = lib()
    keep = _Keep()
    G, F = _geom(g, keep), _field(f, keep)
    s = keep.arr(seed, np.float64)
    cap = params.max_steps + 1
    st = np.zeros((cap, 7))
    fl = C.c_int(0)
    mg = C.c_double(0)
    n = L.orc_propagate(C.byref(G), C.byref(F), C.byref(params), _p(s, C.c_double), cap, _p(st, C.c_double),
                        C.byref(fl), C.byref(mg))
    return st[:n], fl.value, mg.value


def step(f, lam, h, r, t):
    keep = _Keep()
    F = _field(f, keep)
    r = keep.arr(r, np.float64)
    t = keep.arr(t, np.float64)
    ro, to = np.zeros(3), np.zeros(3)
    lib().orc_step(C.byref(F), float(lam), float(h), _p(r, C.c_double), _p(t, C.c_double), _p(ro, C.c_double),
                   _p(to, C.c_double))
    return ro, to


def field_at(f, r):
    keep = _Keep()
    F = _field(f, keep)
    r = keep.arr(r, np.float64)
    B, G = np.zeros(3), np.zeros(9)
    lib().orc_field_at(C.byref(F), _p(r, C.c_double), _p(B, C.c_double), _p(G, C.c_double))
    return B, G.reshape(3, 3)


# ------------------------------------------------------------------- top-K
def topk(E, k):
    """Indices of the k lowest scores, ordered by (E asc, index asc)."""
    E = np.asarray(E)
    order = np.lexsort((np.arange(E.size), E))
    return order[:k]


# ------------------------------------------------------------------- Hough
def hough_params(n_bins=512, bin_um=2000, origin_um=-512000, n_r=32, r_min_um=200000, r_step_um=5000,
                 n_phi=512, target_um=100000, min_peak=8, max_cand=4, r_hist_half_um=2500, b_nominal=1.0,
                 charge=-1.0, R0=500.0):
    return HoughParams(n_bins, bin_um, origin_um, n_r, r_min_um, r_step_um, n_phi, target_um, min_peak, max_cand,
                       r_hist_half_um, float(b_nominal), float(charge), float(R0))


def hough(g, H: HoughParams, wire_id):
    """Accumulator int32[n_bins, n_bins] (row = y bin), candidates
    int32[n,4] (ix, iy, count, r_bin) and seed centres float64[n,3]."""
    L = lib()
    keep = _Keep()
    G = _geom(g, keep)
    wid = keep.arr(wire_id, np.intc)
    acc = np.zeros((H.n_bins, H.n_bins), np.int32)
    L.orc_hough_vote(C.byref(G), C.byref(H), wid.size, _p(wid, C.c_int), _p(acc, C.c_int32))
    cand = np.zeros((H.max_cand, 4), np.int32)
    cen = np.zeros((H.max_cand, 3))
    nc = L.orc_hough_peaks(C.byref(G), C.byref(H), wid.size, _p(wid, C.c_int), _p(acc, C.c_int32),
                           _p(cand, C.c_int32), _p(cen, C.c_double))
    return acc, cand[:nc], cen[:nc]


# ------------------------------------------------------------------ refine
SCALE = np.array([1.0, 100.0, 10.0, 10.0, 10.0])


def refine(g, f, params, wire_id, drift, part, seed, n_iter=5, sigma=0.2, scale=SCALE):
    """Gauss-Newton refinement of one seed: (seed_out, chi2, grad, n_used, flags)."""
    L = lib()
    keep = _Keep()
    G, F = _geom(g, keep), _field(f, keep)
    wid = keep.arr(wire_id, np.intc)
    dr = keep.arr(drift, np.float64)
    pt = keep.arr(part, np.intc)
    sc = keep.arr(scale, np.float64)
    s = keep.arr(seed, np.float64)
    so, gr = np.zeros(5), np.zeros(5)
    c2 = C.c_double(0)
    nu, fl = C.c_int(0), C.c_int(0)
    rc = L.orc_refine(C.byref(G), C.byref(F), C.byref(params), int(n_iter), float(sigma), _p(sc, C.c_double),
                      wid.size, _p(wid, C.c_int), _p(dr, C.c_double), _p(pt, C.c_int), _p(s, C.c_double),
                      _p(so, C.c_double), C.byref(c2), _p(gr, C.c_double), C.byref(nu), C.byref(fl))
    if rc:
        raise RuntimeError("orc_refine failed")
    return so, c2.value, gr, nu.value, fl.value


def chi2(g, f, params, wire_id, drift, part, seed, sigma=0.2):
    """chi^2, its gradient and J^T J at a fixed seed: (chi2, grad, JtJ, n_used, flags)."""
    L = lib()
    keep = _Keep()
    G, F = _geom(g, keep), _field(f, keep)
    wid = keep.arr(wire_id, np.intc)
    dr = keep.arr(drift, np.float64)
    pt = keep.arr(part, np.intc)
    s = keep.arr(seed, np.float64)
    gr, jtj = np.zeros(5), np.zeros(25)
    c2 = C.c_double(0)
    nu, fl = C.c_int(0), C.c_int(0)
    rc = L.orc_chi2(C.byref(G), C.byref(F), C.byref(params), float(sigma), wid.size, _p(wid, C.c_int),
                    _p(dr, C.c_double), _p(pt, C.c_int), _p(s, C.c_double), C.byref(c2), _p(gr, C.c_double),
                    _p(jtj, C.c_double), C.byref(nu), C.byref(fl))
    if rc:
        raise RuntimeError("orc_chi2 failed")
    return c2.value, gr, jtj.reshape(5, 5), nu.value, fl.value


# ------------------------------------------------- classification quality
def classification_counts(hit_off, hit_part, truth_part, n_part):
    """Sec. 3.1: C[e, i + 1, j + 1] = number of hits of event e whose truth
    partition is i and whose classified partition is j (i, j in -1 .. n_part-1;
    -1 = noise / not classified; labels outside the range count as -1)."""
    ne = len(hit_off) - 1
    C = np.zeros((ne, n_part + 1, n_part + 1), np.int64)
    for e in range(ne):
        for h in range(hit_off[e], hit_off[e + 1]):
            i, j = int(truth_part[h]), int(hit_part[h])
            i = i + 1 if 0 <= i < n_part else 0
            j = j + 1 if 0 <= j < n_part else 0
            C[e, i, j] += 1
    return C


def efficiency_purity(C):
    """Eq. 2, eps_n' = C_{n'->n'} / C_{n'} (C_{n'}: all hits of truth partition
    n'), and Eq. 3, pi_n' = C_{n'->n'} / sum_{i=1..n} C_{i->n'} (over the
    signal's partitions only), from counts C [..., n+1, n+1] summed over the
    leading axes; NaN where the denominator is 0."""
    C = np.asarray(C).reshape(-1, np.shape(C)[-2], np.shape(C)[-1]).sum(0)
    n = C.shape[0] - 1
    eps = np.full(n, np.nan)
    pur = np.full(n, np.nan)
    for k in range(n):
        c_k = sum(C[k + 1, j] for j in range(n + 1))
        to_k = sum(C[i + 1, k + 1] for i in range(n))
        if c_k:
            eps[k] = C[k + 1, k + 1] / c_k
        if to_k:
            pur[k] = C[k + 1, k + 1] / to_k
    return eps, pur


def common_hits(hit_off, part_a, part_b, pa=0, pb=0):
    """Sec. 2.2 (bidirectional scan): per event the number of hits classified
    pa by the scan in one direction and pb by the scan in the other."""
    return np.array([sum(1 for h in range(hit_off[e], hit_off[e + 1]) if part_a[h] == pa and part_b[h] == pb)
                     for e in range(len(hit_off) - 1)], np.int64)


# ------------------------------------------------------- neighbouring turn
def extrapolate_turn(g, f, seed, params: ScanParams, direction):
    """Sec. 2.3: seed of the previous (direction -1) or next (+1) turn partition
    from the seed of a turn: (seed float64[5], status 0 found / 1 left the
    chamber / 2 step limit)."""
    L = lib()
    keep = _Keep()
    G, F = _geom(g, keep), _field(f, keep)
    s = keep.arr(seed, np.float64)
    out = np.zeros(5)
    st = L.orc_extrapolate_turn(C.byref(G), C.byref(F), C.byref(params), _p(s, C.c_double), int(direction),
                                _p(out, C.c_double))
    return out, int(st)


# ----------------------------------------------------------- repeated scan
_GRID = np.dtype([("centre", np.float32, 5), ("step", np.float32, 5), ("n", np.int32, 5)])


def _grid(centre, step, n):
    g = np.zeros(1, dtype=_GRID)
    g["centre"][0] = centre
    g["step"][0] = step
    g["n"][0] = n
    return g


def zoom_scan(g, f, wire_id, drift, grid, params: ScanParams, k=8, n_rounds=10, n_zoom=4, threads=None):
    """Sec. 2.2: the scan repeated around its best seeds ("repeated ten times").
    Round 0 scores every seed of `grid`.  Round r = 1 .. n_rounds-1 takes the
    n_zoom best seeds of round r-1 (order (E, index)) and scores, around each,
    a 3^5 grid with the first grid's steps times 2^-r; the round's seeds are
    numbered grid after grid in candidate order, row-major within a grid, and
    every value is rounded once to float32 like any grid seed.  A seed met
    again is scored again.  Returns the k best of all rounds in the order
    (E, round, index): dict(seeds [k,5], E [k], round [k], index [k])."""
    step0 = np.asarray(grid["step"], np.float32).reshape(5)
    seeds = grid_values(grid)
    E = scan(g, f, wire_id, drift, seeds, params, threads=threads)["E"]
    best = [(E[i], 0, int(i), seeds[i]) for i in topk(E, k)]
    for r in range(1, n_rounds):
        step = (step0 * np.float32(2.0 ** -r)).astype(np.float32)
        cand = topk(E, n_zoom)
        seeds = np.concatenate([grid_values(_grid(seeds[c].astype(np.float32), step, (3, 3, 3, 3, 3)))
                                for c in cand]) if len(cand) else np.zeros((0, 5))
        E = scan(g, f, wire_id, drift, seeds, params, threads=threads)["E"] if len(seeds) else np.zeros(0)
        best += [(E[i], r, int(i), seeds[i]) for i in topk(E, k)]
    best.sort(key=lambda t: (t[0], t[1], t[2]))
    best = best[:k]
    return dict(seeds=np.array([b[3] for b in best]).reshape(-1, 5), E=np.array([b[0] for b in best]),
                round=np.array([b[1] for b in best], np.int64), index=np.array([b[2] for b in best], np.int64))


# --------------------------------------------------------------- event loop
LOOP_SIGMA_Z0, LOOP_SIGMA_PZ0 = 26.0, 1.7   # resolution of the predicted (z0, pz0) [mm, MeV/c] (sec. 2.3)
LOOP_MIN_HITS = 10                          # the loop stops below ten unclassified hits (sec. 2.3)
LOOP_GRID_N = (5, 13, 5, 5, 13)             # neighbour grid: (z0, pz0) over +-3 sigma in sigma/2 steps,
LOOP_TRANSVERSE_STEP = (0.002, 0.5, 0.5)    # (theta0, px0, py0) over +-2 fine steps
UNCLASSIFIED = -128


def neighbour_grid(seed, n=LOOP_GRID_N):
    """Grid around a predicted seed of the neighbouring turn (sec. 2.3): n
    points per axis at steps (0.002 rad, sigma_z0 / 2, 0.5, 0.5 MeV/c,
    sigma_pz0 / 2)."""
    return _grid(np.asarray(seed, np.float64).astype(np.float32),
                 (LOOP_TRANSVERSE_STEP[0], LOOP_SIGMA_Z0 / 2, LOOP_TRANSVERSE_STEP[1], LOOP_TRANSVERSE_STEP[2],
                  LOOP_SIGMA_PZ0 / 2), n)


def event_loop(g, f, wire_id, drift, first_grid, params: ScanParams, k=8, n_rounds=10, n_zoom=4, n_iter=5,
               sigma=0.2, max_turns=8, min_hits=LOOP_MIN_HITS, grid_n=LOOP_GRID_N, threads=None,
               return_margin=False):
    """Sec. 2.3, Fig. 7: the hits of one event classified into turns, in FP64.
    A turn is found by the repeated scan (zoom_scan, one partition) of the hits
    not yet classified; its hits are those the best seed classifies into
    partition 0 (at least min_hits, else no turn).  The best seed is refined by
    Gauss-Newton (n_iter iterations, the classification at the best seed held)
    and the refined seed kept only where chi^2 went down.  From a turn's seed
    the neighbouring turn's seed is predicted (extrapolate_turn) backwards
    (-1) and forwards (+1) and searched on neighbour_grid (grid_n points per
    axis); each direction
    stops when the prediction leaves the chamber, when fewer than min_hits
    hits remain or a scan classifies fewer, or after max_turns turns.
    Returns (labels int32[H]: turn relative to the first one found, or
    UNCLASSIFIED; seeds: turn -> float64[5]), and with return_margin the
    smallest distance [mm] of each hit's |residual| to a classification cut
    over the turn scans that classified it (inf if none did)."""
    wid = np.asarray(wire_id, np.int32)
    dr = np.asarray(drift, np.float64)
    labels = np.full(wid.size, UNCLASSIFIED, np.int32)
    margin = np.full(wid.size, np.inf)
    p1 = ScanParams(params.h, params.max_steps, params.lam, 1, params.direction, params.charge)

    def find_turn(grid):
        idx = np.flatnonzero(labels == UNCLASSIFIED)
        if idx.size < min_hits:
            return None
        w, d = wid[idx], dr[idx]
        z = zoom_scan(g, f, w, d, grid, p1, k=k, n_rounds=n_rounds, n_zoom=n_zoom, threads=threads)
        if z["E"].size == 0:
            return None
        best = z["seeds"][0]
        cls = scan(g, f, w, d, best[None], p1, per_hit=True, threads=1)
        part = cls["hit_part"][0]
        margin[idx] = np.minimum(margin[idx], cls["hit_margin"][0])
        found = idx[part == 0]
        if found.size < min_hits:
            return None
        c0 = chi2(g, f, p1, w, d, part, best, sigma=sigma)[0]
        so, c1, _, _, _ = refine(g, f, p1, w, d, part, best, n_iter=n_iter, sigma=sigma)
        keep = bool(np.all(np.isfinite(so))) and c1 < c0
        return found, (so if keep else best)

    seeds = {}
    first = find_turn(first_grid)
    if first is None:
        return (labels, seeds, margin) if return_margin else (labels, seeds)
    labels[first[0]] = 0
    seeds[0] = first[1]
    for direction in (-1, 1):
        cur, t = seeds[0], 0
        while abs(t) < max_turns:
            pred, status = extrapolate_turn(g, f, cur, p1, direction)
            if status != 0:
                break
            turn = find_turn(neighbour_grid(pred, grid_n))
            if turn is None:
                break
            t += direction
            labels[turn[0]] = t
            seeds[t] = cur = turn[1]
    return (labels, seeds, margin) if return_margin else (labels, seeds)
