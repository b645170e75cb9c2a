"""Precision/scale sweep on events at 30 % occupancy: Hough accumulators
bit-exact for every event, and propagated positions of seeds drawn from the
events' grids against the FP64 oracle at every 0.5 m up to 6 m, for the FP32
scan stepper, the FP32 refine stepper and the FP64 GPU stepper."""
import numpy as np
import pytest

import cdc_synth as S
import oracle as O
from tests.gpu_util import tracker

pytestmark = pytest.mark.gpu

N_EVENTS = 6
N_SEEDS = 240          # subsample propagated by both sides
EVERY, N_REC = 250, 12  # 0.5 m records up to 6 m


@pytest.fixture(scope="module")
def sweep_events(field_map):
    out = [S.cfg5_event(i, field_map, n_seeds=2.0e4) for i in range(N_EVENTS)]
    return [e for e, _ in out], np.concatenate([g for _, g in out])


def test_hough_bit_exact_at_30_percent_occupancy(field_map, sweep_events):
    import torch
    import paper_1908_01949_gb300 as cdc
    g = S.make_geometry()
    evs, _ = sweep_events
    off, wid, dr = S.pack_events(evs)
    tr = tracker(g, field_map)
    doff, dwid, _ = tr.events_to_device(off, wid, dr)
    out = tr.hough(doff, dwid, cdc.hough_params(grid_template=S.cfg2_grid_template()))
    torch.cuda.synchronize()
    acc = out["acc"].cpu().numpy()
    OH = O.hough_params()
    for e, ev in enumerate(evs):
        assert ev.wire_id.size >= 0.29 * g.n_wires
        racc, rc, _ = O.hough(g, OH, ev.wire_id)
        assert np.array_equal(acc[e], racc), e
        assert int(out["n_cand"][e]) == rc.shape[0]


@pytest.mark.parametrize("precision,tol", [(0, 1e-4), (2, 1e-4), (1, 1e-9)])
def test_position_error_per_metre_up_to_6m(field_map, sweep_events, precision, tol):
    import torch
    import paper_1908_01949_gb300 as cdc
    g = S.sweep_geometry(S.make_geometry())
    _, grids = sweep_events
    rng = np.random.default_rng(7)
    seeds = np.concatenate([O.grid_values(grids[e:e + 1])[rng.choice(int(np.prod(grids[e]["n"])),
                                                                     N_SEEDS // N_EVENTS, replace=False)]
                            for e in range(N_EVENTS)]).astype(np.float32)
    tr = tracker(g, field_map)
    p = cdc.scan_params(h=2.0, max_steps=EVERY * N_REC, lam=4.0, max_partitions=16)
    out = tr.propagate(torch.as_tensor(seeds, device=tr.dev), p, every=EVERY, n_rec=N_REC, precision=precision)
    torch.cuda.synchronize()
    pos = out["pos"].cpu().numpy()
    op = O.scan_params(h=2.0, max_steps=EVERY * N_REC, lam=4.0, max_partitions=16)
    worst, compared = 0.0, 0
    for i, sd in enumerate(seeds.astype(np.float64)):
        st, _, _ = O.propagate(g, field_map, sd, op)
        for r in range(N_REC):
            j = EVERY * (r + 1)
            if j >= len(st) or not np.isfinite(pos[i, r, 0]):
                continue
            worst = max(worst, np.linalg.norm(pos[i, r] - st[j, :3]) / (j * 2.0e-3))
            compared += 1
    assert compared > N_SEEDS * 4
    assert worst < tol, worst
