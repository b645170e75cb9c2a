"""The paper's two-kernel scan (record states, then DOCA per hit) against the
fused scan and the FP64 oracle on the same seeds."""
import numpy as np
import pytest

import cdc_synth as S
import oracle as O
from tests.gpu_util import compare_scores, oracle_params, tracker

pytestmark = pytest.mark.gpu


def _split_and_fused(g, f, ev, grid, p, chunk):
    import torch
    import paper_1908_01949_gb300 as cdc
    n = int(np.prod(grid["n"][0]))
    tr = tracker(g, f, max_seeds=n)
    tr.ctx.cdc_reserve_split(chunk, p.max_steps)
    off, wid, dr = tr.events_to_device([0, ev.wire_id.size], ev.wire_id, ev.drift)
    gt = cdc.grids_to_tensor(grid, tr.dev)
    fused = tr.scan(off, wid, dr, gt, p, want_E=True, n_seeds=n)
    E = torch.full((n,), float("nan"), dtype=torch.float32, device=tr.dev)
    flags = torch.empty(1, dtype=torch.int32, device=tr.dev)
    tr.ctx.cdc_scan_seeds_split(1, n, off, wid, dr, gt, p, E, flags)
    torch.cuda.synchronize()
    return E.cpu().numpy(), fused["E"].cpu().numpy(), int(flags[0])


@pytest.mark.parametrize("case", ["uniform", "map"])
def test_split_scan_equals_fused_scan_and_oracle(case, field_map):
    import paper_1908_01949_gb300 as cdc
    if case == "uniform":
        g, f, ev, grid = S.cfg1_case(3)
        grid["n"][0] = (6, 4, 5, 5, 6)       # 3600 seeds in chunks of 1000: a ragged last chunk
        p = cdc.scan_params(h=2.0, max_steps=1000, lam=4.0, max_partitions=1, k=8, n_rounds=1)
    else:
        g, f, ev = S.cfg2_case(0, field_map, occupancy=0.05)
        grid = S.make_grid(ev.truth_seeds[-1] + np.array([0.003, 10.0, 1.0, -1.0, 1.0]),
                           (0.004, 12.0, 1.0, 1.0, 1.5), (3, 5, 3, 3, 5))
        p = cdc.scan_params(h=2.0, max_steps=3500, lam=4.0, max_partitions=3, k=8, n_rounds=1)
    Es, Ef, fl = _split_and_fused(g, f, ev, grid, p, chunk=1000)
    assert fl == 0 and np.all(np.isfinite(Es))
    assert np.allclose(Es, Ef, rtol=1e-5, atol=1e-5), float(np.max(np.abs(Es - Ef) / np.maximum(Ef, 1e-30)))
    ref = O.scan(g, f, ev.wire_id, ev.drift.astype(np.float64), O.grid_values(grid), oracle_params(p))
    bad, excluded, worst = compare_scores(Es, ref)
    assert bad.size == 0, (bad[:10], worst)


def test_split_scan_argument_errors():
    """Missing parameters, a missing split workspace and a step limit above
    the reserved one are status codes, not crashes."""
    import torch
    import paper_1908_01949_gb300 as cdc
    g, f, ev, grid = S.cfg1_case(3)
    n = int(np.prod(grid["n"][0]))
    tr = tracker(g, f, max_seeds=n)
    off, wid, dr = tr.events_to_device([0, ev.wire_id.size], ev.wire_id, ev.drift)
    gt = cdc.grids_to_tensor(grid, tr.dev)
    E = torch.empty(n, dtype=torch.float32, device=tr.dev)
    flags = torch.empty(1, dtype=torch.int32, device=tr.dev)
    ptr = [t.data_ptr() for t in (off, wid, dr, gt, E, flags)]
    L = tr.ctx.L
    assert L.cdc_scan_seeds_split(tr.ctx.h, 1, n, ptr[0], ptr[1], ptr[2], ptr[3], None, ptr[4], ptr[5], None) == -1
    p = cdc.scan_params(h=2.0, max_steps=1000, lam=4.0, max_partitions=1, k=8, n_rounds=1)
    with pytest.raises(cdc.CdcError):                      # no split workspace reserved yet
        tr.ctx.cdc_scan_seeds_split(1, n, off, wid, dr, gt, p, E, flags)
    tr.ctx.cdc_reserve_split(1000, 500)
    with pytest.raises(cdc.CdcError):                      # max_steps above the reserve
        tr.ctx.cdc_scan_seeds_split(1, n, off, wid, dr, gt, p, E, flags)
    with pytest.raises(cdc.CdcError):
        tr.ctx.cdc_reserve_split(0, 500)
