"""GPU parity on a turn partition that passes fired wires more than once (sec.
2.2, Eq. 1): the partition's DCA is its nearest pass, in every kernel that
scores or classifies hits.  The event (tests/double_pass.py) keeps one
partition over several revolutions; on it, scoring each wire by its smallest
residual over the passes instead misses the oracle by far more than the score
tolerance (tests/test_oracle_double_pass.py)."""
import numpy as np
import pytest

import oracle as O
from tests import double_pass as DP
from tests.gpu_util import E_REL, MARGIN, check_topk, compare_scores, keys_to_index, oracle_params, tracker

pytestmark = pytest.mark.gpu


def _grid(centre, step, n):
    import cdc_synth as S
    return S.make_grid(np.asarray(centre, np.float64), step, n)


def _run(grid, p, n_seeds, want_E=True):
    import torch
    import paper_1908_01949_gb300 as cdc
    g, f, wid, dr = DP.setup()
    tr = tracker(g, f)
    off, w, d = tr.events_to_device([0, wid.size], wid, dr)
    out = tr.scan(off, w, d, cdc.grids_to_tensor(grid, tr.dev), p, want_E=want_E, n_seeds=n_seeds)
    torch.cuda.synchronize()
    return g, f, wid, dr, tr, (off, w, d), out


def _check_hits(g, f, wid, dr, out, p):
    best = out["best_seed"][0, 0].cpu().numpy().astype(np.float64)
    ref = O.scan(g, f, wid, dr.astype(np.float64), best[None], oracle_params(p), per_hit=True)
    hp = out["hit_part"].cpu().numpy()
    r2 = out["hit_res2"].cpu().numpy()
    clear = ref["hit_margin"][0] >= MARGIN
    assert clear[: len(DP.TRAPS)].all()
    assert np.array_equal(hp[clear], ref["hit_part"][0][clear]), (hp, ref["hit_part"][0])
    assert np.allclose(r2, np.minimum(ref["hit_res2"][0], DP.LAM), atol=2e-3), (r2, ref["hit_res2"][0])
    return ref


def test_lane_scan_scores_and_classifies_by_the_nearest_pass():
    """Thread-per-seed scan of nine seeds around the hand-placed one (z0, pz0
    varied, the seed stays tangent to R0): every score equals the oracle's,
    and the best seed's hit classes (traced again by the warp tracer) too."""
    import paper_1908_01949_gb300 as cdc
    grid = _grid(DP.SEED, (1e-7, 10.0, 1e-5, 1e-5, 0.5), (1, 3, 1, 1, 3))
    p = cdc.scan_params(h=2.0, max_steps=3500, lam=DP.LAM, max_partitions=3, k=4, n_rounds=1)
    g, f, wid, dr, tr, _, out = _run(grid, p, 9)
    seeds = O.grid_values(grid)
    ref = O.scan(g, f, wid, dr.astype(np.float64), seeds, oracle_params(p))
    assert ref["margin"][4] >= MARGIN           # the centre seed is compared without exclusion
    bad, excluded, worst = compare_scores(out["E"].cpu().numpy(), ref)
    assert bad.size == 0, (bad, worst, out["E"].cpu().numpy(), ref["E"])
    assert excluded <= 2
    idx, _ = keys_to_index(out["topk0"][0].cpu().numpy())
    ok, diff = check_topk(idx, ref["E"], 4)
    assert ok, diff
    _check_hits(g, f, wid, dr, out, p)


def test_warp_scan_zoom_round_scores_and_keeps_the_nearest_pass():
    """One coarse seed 0.3 MeV/c off the hand-placed one and one zoom round
    around it (3^5 seeds at half the step; warp-per-seed kernel): the best
    seed comes from the zoom round, its score and the K best scores equal the
    oracle's, and the hit classes come from the zoom round's kept record."""
    import paper_1908_01949_gb300 as cdc
    centre = DP.SEED + np.array([0.0, 0.0, 0.0, 0.0, 0.3])
    grid = _grid(centre, (2e-7, 2e-4, 2e-5, 2e-5, 0.6), (1, 1, 1, 1, 1))
    p = cdc.scan_params(h=2.0, max_steps=3500, lam=DP.LAM, max_partitions=3, k=8, n_rounds=2, n_zoom=1)
    g, f, wid, dr, tr, _, out = _run(grid, p, 1)
    op = oracle_params(p)
    coarse = O.scan(g, f, wid, dr.astype(np.float64), O.grid_values(grid), op)
    bE = out["best_E"][0].cpu().numpy().astype(np.float64)
    bs = out["best_seed"][0].cpu().numpy().astype(np.float64)
    assert bE[0] < coarse["E"][0] * (1 - 10 * E_REL)  # a zoom-round seed won
    ref = O.scan(g, f, wid, dr.astype(np.float64), bs, op)
    ok = ref["margin"] >= MARGIN
    assert ok[0]
    rel = np.abs(bE - ref["E"]) / ref["E"]
    assert np.all(rel[ok] <= E_REL), (rel, bE, ref["E"])
    _check_hits(g, f, wid, dr, out, p)


def test_split_scan_takes_the_nearest_pass():
    """The two-kernel scan (recorded states, then a thread per hit) on the
    nine seeds: per partition the nearest pass, like the oracle."""
    import torch
    import paper_1908_01949_gb300 as cdc
    grid = _grid(DP.SEED, (1e-7, 10.0, 1e-5, 1e-5, 0.5), (1, 3, 1, 1, 3))
    p = cdc.scan_params(h=2.0, max_steps=3500, lam=DP.LAM, max_partitions=3, k=4, n_rounds=1)
    g, f, wid, dr = DP.setup()
    tr = tracker(g, f, max_seeds=9)
    tr.ctx.cdc_reserve_split(16, p.max_steps)
    off, w, d = tr.events_to_device([0, wid.size], wid, dr)
    E = torch.full((9,), float("nan"), dtype=torch.float32, device=tr.dev)
    flags = torch.empty(1, dtype=torch.int32, device=tr.dev)
    tr.ctx.cdc_scan_seeds_split(1, 9, off, w, d, cdc.grids_to_tensor(grid, tr.dev), p, E, flags)
    torch.cuda.synchronize()
    ref = O.scan(g, f, wid, dr.astype(np.float64), O.grid_values(grid), oracle_params(p))
    bad, excluded, worst = compare_scores(E.cpu().numpy(), ref)
    assert bad.size == 0 and excluded <= 2, (bad, worst)


def test_refine_classifies_by_the_nearest_pass():
    """chi^2 and its adjoint gradient at the hand-placed seed use the hits the
    nearest pass classifies: the same hits, chi^2 and gradient as the oracle."""
    import torch
    import paper_1908_01949_gb300 as cdc
    g, f, wid, dr = DP.setup()
    tr = tracker(g, f)
    off, w, d = tr.events_to_device([0, wid.size], wid, dr)
    sp = cdc.scan_params(h=2.0, max_steps=3500, lam=DP.LAM, max_partitions=3)
    rp = cdc.refine_params(n_iter=0, sigma=0.2, checkpoint=128)
    seed = DP.SEED.astype(np.float32)[None]
    out = tr.chi2_grad(torch.zeros(1, dtype=torch.int32, device=tr.dev), torch.as_tensor(seed, device=tr.dev),
                       off, w, d, sp, rp)
    torch.cuda.synchronize()
    op = oracle_params(sp)
    sd = seed[0].astype(np.float64)
    ref = O.scan(g, f, wid, dr.astype(np.float64), sd[None], op, per_hit=True)
    assert (ref["hit_margin"][0] >= MARGIN).all()
    rc2, rg, _, rnu, _ = O.chi2(g, f, op, wid, dr.astype(np.float64), ref["hit_part"][0], sd)
    assert int(out["n_used"][0]) == rnu
    assert abs(float(out["chi2"][0]) - rc2) <= 1e-4 * rc2
    scale = np.array([1.0, 100.0, 10.0, 10.0, 10.0])
    g_rel = np.linalg.norm((out["grad"][0].cpu().numpy() - rg) * scale) / np.linalg.norm(rg * scale)
    assert g_rel <= 1e-3, (out["grad"][0].cpu().numpy(), rg)
