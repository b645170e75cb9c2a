"""GPU parity of the Gauss-Newton refinement and of the adjoint-RKN chi^2
gradient against the FP64 oracle (tangent gradient), through the C ABI."""
import numpy as np
import pytest

import cdc_synth as S
import oracle as O
from tests.gpu_util import oracle_params, tracker

pytestmark = pytest.mark.gpu
SCALE = np.array([1.0, 100.0, 10.0, 10.0, 10.0])


def _cases(kind, field_map=None):
    if kind == "uniform":
        g, f, ev, grid = S.cfg1_case(7)
        mp, ms = 1, 1000
    else:
        g = S.make_geometry()
        f = field_map
        ev = S.cfg2_case(2, field_map, occupancy=0.05)[2]
        mp, ms = 3, 3500
    rng = np.random.default_rng(11)
    truth = ev.truth_seeds[0]          # first turn: the map case follows 2-3 turns
    sig = np.array([3e-4, 0.4, 0.15, 0.15, 0.1]) * (1.0 if kind == "uniform" else 0.3)
    seeds = [truth + rng.normal(0, 1, 5) * sig for _ in range(8)]
    return g, f, ev, np.asarray(seeds, np.float32), mp, ms


def _oracle_part(g, f, ev, seed, op):
    out = O.scan(g, f, ev.wire_id, ev.drift.astype(np.float64), seed[None], op, per_hit=True)
    return out["hit_part"][0], out["hit_margin"][0]


@pytest.mark.parametrize("kind", ["uniform", "map"])
def test_adjoint_gradient_matches_fp64_oracle(kind, field_map):
    """chi^2 within 1e-4 relative and d chi^2/d seed (adjoint RKN, FP32) within
    1e-4 relative (scaled parameters) of the FP64 forward-tangent gradient."""
    import torch
    import paper_1908_01949_gb300 as cdc
    g, f, ev, seeds, mp, ms = _cases(kind, field_map)
    tr = tracker(g, f)
    off, wid, dr = tr.events_to_device([0, ev.wire_id.size], ev.wire_id, ev.drift)
    sp = cdc.scan_params(h=2.0, max_steps=ms, lam=4.0, max_partitions=mp)
    rp = cdc.refine_params(n_iter=0, sigma=0.2, checkpoint=128)
    se = torch.zeros(len(seeds), dtype=torch.int32, device=tr.dev)
    out = tr.chi2_grad(se, torch.as_tensor(seeds, device=tr.dev), off, wid, dr, sp, rp)
    torch.cuda.synchronize()
    c2 = out["chi2"].cpu().numpy()
    gr = out["grad"].cpu().numpy()
    nu = out["n_used"].cpu().numpy()
    op = oracle_params(sp)
    checked = 0
    for i, sd in enumerate(seeds.astype(np.float64)):
        part, margin = _oracle_part(g, f, ev, sd, op)
        if (margin < 1e-3).any():
            continue                      # a hit at a classification cut: the two sides may classify differently
        rc2, rg, _, rnu, rfl = O.chi2(g, f, op, ev.wire_id, ev.drift.astype(np.float64), part, sd)
        assert nu[i] == rnu
        assert abs(c2[i] - rc2) <= 1e-4 * rc2, (i, c2[i], rc2)
        rel = np.linalg.norm((gr[i] - rg) * SCALE) / np.linalg.norm(rg * SCALE)
        assert rel <= 1e-4, (i, rel, gr[i], rg)
        checked += 1
    assert checked >= 4


@pytest.mark.parametrize("kind", ["uniform", "map"])
def test_gauss_newton_refine_matches_oracle(kind, field_map):
    """Five Gauss-Newton iterations from the same starting seeds land on the
    same refined seeds as the FP64 oracle, with the same chi^2."""
    import torch
    import paper_1908_01949_gb300 as cdc
    g, f, ev, seeds, mp, ms = _cases(kind, field_map)
    tr = tracker(g, f)
    off, wid, dr = tr.events_to_device([0, ev.wire_id.size], ev.wire_id, ev.drift)
    sp = cdc.scan_params(h=2.0, max_steps=ms, lam=4.0, max_partitions=mp)
    rp = cdc.refine_params(n_iter=5, sigma=0.2, checkpoint=128)
    se = torch.zeros(len(seeds), dtype=torch.int32, device=tr.dev)
    out = tr.refine(se, torch.as_tensor(seeds, device=tr.dev), off, wid, dr, sp, rp)
    torch.cuda.synchronize()
    so = out["seeds"].cpu().numpy().astype(np.float64)
    c2 = out["chi2"].cpu().numpy()
    op = oracle_params(sp)
    checked = 0
    for i, sd in enumerate(seeds.astype(np.float64)):
        part, margin = _oracle_part(g, f, ev, sd, op)
        if (margin < 1e-3).any():
            continue
        rso, rc2, rg, rnu, rfl = O.refine(g, f, op, ev.wire_id, ev.drift.astype(np.float64), part, sd, n_iter=5)
        c0 = O.chi2(g, f, op, ev.wire_id, ev.drift.astype(np.float64), part, sd)[0]
        if not rc2 < c0:
            continue                      # the start lies outside the Gauss-Newton basin: no unique answer
        assert abs(c2[i] - rc2) <= 1e-3 * max(rc2, 1.0), (i, c2[i], rc2)
        assert np.all(np.abs((so[i] - rso) / SCALE) < 2e-4), (i, so[i], rso)
        checked += 1
    assert checked >= 4


def test_seed_event_out_of_range_is_flagged():
    import torch
    import paper_1908_01949_gb300 as cdc
    g, f, ev, seeds, mp, ms = _cases("uniform")
    tr = tracker(g, f)
    off, wid, dr = tr.events_to_device([0, ev.wire_id.size], ev.wire_id, ev.drift)
    sp = cdc.scan_params(h=2.0, max_steps=ms, lam=4.0, max_partitions=mp)
    rp = cdc.refine_params(n_iter=1)
    se = torch.tensor([0, 5], dtype=torch.int32, device=tr.dev)
    out = tr.refine(se, torch.as_tensor(seeds[:2], device=tr.dev), off, wid, dr, sp, rp)
    torch.cuda.synchronize()
    fl = out["flags"].cpu().numpy()
    assert fl[1] & cdc.FLAG_BAD_HIT and np.isnan(out["chi2"][1].item())
    assert not (fl[0] & cdc.FLAG_BAD_HIT)


def test_autograd_function_backward_is_the_adjoint_gradient():
    """cdc.chi2 as a torch.autograd.Function: backward of sum(w * chi2) gives
    w_i * d chi2_i / d seed_i, the adjoint gradient of cdc_chi2_grad."""
    import torch
    import paper_1908_01949_gb300 as cdc
    g, f, ev, seeds, mp, ms = _cases("uniform")
    tr = tracker(g, f)
    off, wid, dr = tr.events_to_device([0, ev.wire_id.size], ev.wire_id, ev.drift)
    sp = cdc.scan_params(h=2.0, max_steps=ms, lam=4.0, max_partitions=mp)
    rp = cdc.refine_params(n_iter=0, sigma=0.2, checkpoint=128)
    se = torch.zeros(len(seeds), dtype=torch.int32, device=tr.dev)
    x = torch.as_tensor(seeds, device=tr.dev).clone().requires_grad_(True)
    c = cdc.chi2(tr, se, x, off, wid, dr, sp, rp)
    w = torch.arange(1, len(seeds) + 1, dtype=torch.float64, device=tr.dev)
    (w * c).sum().backward()
    ref = tr.chi2_grad(se, torch.as_tensor(seeds, device=tr.dev), off, wid, dr, sp, rp)
    torch.cuda.synchronize()
    assert torch.equal(c.detach(), ref["chi2"])
    expect = (w.float()[:, None] * ref["grad"]).cpu().numpy()
    assert np.allclose(x.grad.cpu().numpy(), expect, rtol=1e-6, atol=0)


def test_empty_call_and_a_seed_whose_event_has_no_hits():
    """n_seeds = 0 is a no-op.  A seed of an event without hits classifies no
    hit: chi^2 = 0, no hit used, zero gradient, the normal matrix flagged and
    the seed left where it was.  A seed's outputs do not depend on the other
    seeds of the launch: refined beside the empty event's seed, the seed of the
    event with hits gives the bits it gives alone."""
    import torch
    import paper_1908_01949_gb300 as cdc
    g, f, ev, seeds, mp, ms = _cases("uniform")
    tr = tracker(g, f)
    n = ev.wire_id.size
    off, wid, dr = tr.events_to_device([0, n, n], ev.wire_id, ev.drift)     # event 1 has no hits
    sp = cdc.scan_params(h=2.0, max_steps=ms, lam=4.0, max_partitions=mp)
    rp = cdc.refine_params(n_iter=3, sigma=0.2, checkpoint=128)
    x = torch.as_tensor(seeds[:2], device=tr.dev)
    none = tr.refine(torch.zeros(0, dtype=torch.int32, device=tr.dev), x[:0], off, wid, dr, sp, rp)
    assert none["seeds"].shape == (0, 5) and none["chi2"].shape == (0,)
    both = tr.refine(torch.tensor([1, 0], dtype=torch.int32, device=tr.dev), x, off, wid, dr, sp, rp)
    alone = tr.refine(torch.tensor([0], dtype=torch.int32, device=tr.dev), x[1:].contiguous(), off, wid, dr, sp, rp)
    torch.cuda.synchronize()
    assert float(both["chi2"][0]) == 0.0 and int(both["n_used"][0]) == 0
    assert torch.all(both["grad"][0] == 0)
    assert torch.equal(both["seeds"][0], x[0])
    assert int(both["flags"][0]) & cdc.FLAG_NOT_SPD
    assert int(both["n_used"][1]) > 0 and float(both["chi2"][1]) > 0.0
    for k in ("seeds", "chi2", "grad", "n_used", "flags"):
        assert torch.equal(both[k][1:], alone[k]), k


@pytest.mark.parametrize("spread", [1.0, 0.1])
def test_three_turn_seed_with_more_than_128_classified_hits(field_map, spread):
    """A three-turn signal classifies up to ~150 hits (the refine workload's
    events); every one of them enters chi^2: n_used and chi^2 follow the oracle,
    with no overflow flag, and so does the adjoint gradient.  At seeds one
    spread (3e-4 rad, 0.4 mm, 0.15, 0.15, 0.1 MeV/c) from the truth the gradient
    is within 1e-4 relative.  Within a tenth of that spread the seeds sit near
    the chi^2 minimum, where the gradient is a cancellation of per-hit terms 30
    to 70 times its own size; there the FP32 error is bounded against the size
    of those terms, 2 sqrt(chi^2 tr(S J^T J S)) in the scaled parameters S
    (the Cauchy-Schwarz bound of sum_i 2 r_i |J_i|): within 2e-5 of it."""
    import torch
    import paper_1908_01949_gb300 as cdc
    g = S.make_geometry()
    ev = S.cfg4_event(1, field_map)[0]
    tr = tracker(g, field_map)
    off, wid, dr = tr.events_to_device([0, ev.wire_id.size], ev.wire_id, ev.drift)
    sp = cdc.scan_params(h=2.0, max_steps=3500, lam=4.0, max_partitions=3)
    rp = cdc.refine_params(n_iter=0, sigma=0.2, checkpoint=128)
    rng = np.random.default_rng(5)
    sig = np.array([3e-4, 0.4, 0.15, 0.15, 0.1]) * spread
    seeds = np.asarray([ev.truth_seeds[0] + rng.normal(0, 1, 5) * sig for _ in range(4)], np.float32)
    se = torch.zeros(len(seeds), dtype=torch.int32, device=tr.dev)
    out = tr.chi2_grad(se, torch.as_tensor(seeds, device=tr.dev), off, wid, dr, sp, rp)
    torch.cuda.synchronize()
    c2, gr = out["chi2"].cpu().numpy(), out["grad"].cpu().numpy()
    nu, fl = out["n_used"].cpu().numpy(), out["flags"].cpu().numpy()
    op = oracle_params(sp)
    checked = 0
    for i, sd in enumerate(seeds.astype(np.float64)):
        part, margin = _oracle_part(g, field_map, ev, sd, op)
        if (margin < 1e-3).any():
            continue
        rc2, rg, jtj, rnu, _ = O.chi2(g, field_map, op, ev.wire_id, ev.drift.astype(np.float64), part, sd)
        assert rnu > 128, rnu                 # the case this test is about
        assert not (fl[i] & cdc.FLAG_FOUND_OVERFLOW)
        assert nu[i] == rnu
        assert abs(c2[i] - rc2) <= 1e-4 * rc2, (i, c2[i], rc2)
        err = np.linalg.norm((gr[i] - rg) * SCALE)
        if spread >= 1.0:
            rel = err / np.linalg.norm(rg * SCALE)
            assert rel <= 1e-4, (i, rel, gr[i], rg)
        else:
            terms = 2.0 * np.sqrt(rc2 * np.trace(np.diag(SCALE) @ jtj @ np.diag(SCALE)))
            assert err <= 2e-5 * terms, (i, err / terms, gr[i], rg)
        checked += 1
    assert checked >= 2
