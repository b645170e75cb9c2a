"""The allocation-free scan entry point, cdc_scan_seeds_noalloc.

It serves callers that must not allocate device memory at call time (for
example code running inside an allocator callback, or a process whose device
memory is owned by another framework's caching allocator).  Its results must
equal those of cdc_scan_seeds, which takes its workspace from cdc_reserve.
This file is collected last on purpose: a failure here stops a -x run only
after every other test has run."""
import numpy as np
import pytest

import cdc_synth as S
from tests.gpu_util import E_REL

pytestmark = pytest.mark.gpu


def _run_both(tr, ev, grid, lam):
    import torch
    import paper_1908_01949_gb300 as cdc
    n = int(np.prod(grid["n"][0]))
    off, wid, dr = tr.events_to_device([0, ev.wire_id.size], ev.wire_id, ev.drift)
    dg = cdc.grids_to_tensor(grid, tr.dev)
    p = cdc.scan_params(h=2.0, max_steps=1000, lam=lam, max_partitions=1, k=8, n_rounds=1)
    ref = tr.scan(off, wid, dr, dg, p, want_E=True, n_seeds=n)
    t = torch
    out = dict(E=t.empty(n, dtype=t.float32, device=tr.dev), topk0=t.empty((1, 8), dtype=t.int64, device=tr.dev),
               best_E=t.empty((1, 8), dtype=t.float32, device=tr.dev),
               best_seed=t.empty((1, 8, 5), dtype=t.float32, device=tr.dev),
               hit_part=t.empty(ev.wire_id.size, dtype=t.int8, device=tr.dev),
               hit_res2=t.empty(ev.wire_id.size, dtype=t.float32, device=tr.dev),
               flags=t.empty(1, dtype=t.int32, device=tr.dev), steps=t.zeros(1, dtype=t.int64, device=tr.dev))
    tr.ctx.cdc_scan_seeds_noalloc(1, n, off, wid, dr, dg, p, out["E"], out["topk0"], out["best_E"], out["best_seed"],
                                  out["hit_part"], out["hit_res2"], out["flags"], out["steps"])
    torch.cuda.synchronize()
    return ref, out


def test_noalloc_scan_matches_reserved_scan_twice():
    """Two calls in a row (different events, seed counts and cutoffs) give the
    scores, top-K, best seed and hit classes of the workspace-backed scan, bit
    for bit: the reserved scan takes the (z0, pz0) blocks longest estimated
    track first, the allocation-free one in their natural order, and the
    order in which seeds are processed changes no score."""
    import paper_1908_01949_gb300 as cdc
    from tests.gpu_util import tracker
    g, f, ev1, grid1 = S.cfg1_case(8)
    _, _, ev2, grid2 = S.cfg1_case(9)
    grid2["n"][0] = (9, 5, 6, 6, 7)           # 11340 seeds: several top-K segments
    tr = tracker(g, f)
    for ev, grid, lam in ((ev1, grid1, 4.0), (ev2, grid2, 9.0)):
        ref, out = _run_both(tr, ev, grid, lam)
        Er, Eo = ref["E"].cpu().numpy(), out["E"].cpu().numpy()
        assert np.array_equal(Eo, Er)
        assert np.array_equal(out["topk0"].cpu().numpy(), ref["topk0"].cpu().numpy())
        assert np.allclose(out["best_E"].cpu().numpy(), ref["best_E"].cpu().numpy(), rtol=E_REL)
        assert np.array_equal(out["best_seed"].cpu().numpy(), ref["best_seed"].cpu().numpy())
        assert np.array_equal(out["hit_part"].cpu().numpy(), ref["hit_part"].cpu().numpy())
        assert int(out["flags"][0]) == int(ref["flags"][0]) == 0
        assert int(out["steps"][0]) == int(ref["steps"][0])


def test_noalloc_scan_rejects_sizes_beyond_its_array():
    import torch
    import paper_1908_01949_gb300 as cdc
    from tests.gpu_util import tracker
    g, f, ev, grid = S.cfg1_case(8)
    tr = tracker(g, f)
    off, wid, dr = tr.events_to_device([0, ev.wire_id.size], ev.wire_id, ev.drift)
    dg = cdc.grids_to_tensor(grid, tr.dev)
    t = torch
    be, bs = t.empty((9, 8), device=tr.dev), t.empty((9, 8, 5), device=tr.dev)
    fl = t.empty(9, dtype=t.int32, device=tr.dev)
    p = cdc.scan_params(k=8, n_rounds=1)
    with pytest.raises(cdc.CdcError, match="CDC_NOALLOC_MAX_SEEDS"):
        tr.ctx.cdc_scan_seeds_noalloc(1, 65537, off, wid, dr, dg, p, None, None, be, bs, None, None, fl, None)
    with pytest.raises(cdc.CdcError, match="CDC_NOALLOC_MAX_EVENTS"):
        tr.ctx.cdc_scan_seeds_noalloc(9, 10, off, wid, dr, dg, p, None, None, be, bs, None, None, fl, None)
    with pytest.raises(cdc.CdcError, match="n_rounds"):
        tr.ctx.cdc_scan_seeds_noalloc(1, 10, off, wid, dr, dg, cdc.scan_params(k=8, n_rounds=2), None, None, be, bs,
                                      None, None, fl, None)


def test_noalloc_scan_without_E_and_grids_beyond_the_stated_count():
    """Without E the scores stay in the library's array: top-K, best seeds and
    hit classes still equal the reserved scan's.  A second call takes no
    device memory.  Grids holding more seeds than the caller states scan
    nothing and flag the event empty, with or without E, and leave E as it
    was."""
    import torch
    import paper_1908_01949_gb300 as cdc
    from tests.gpu_util import tracker
    g, f, ev, grid = S.cfg1_case(10)
    n = int(np.prod(grid["n"][0]))
    tr = tracker(g, f)
    ref, _ = _run_both(tr, ev, grid, 4.0)
    off, wid, dr = tr.events_to_device([0, ev.wire_id.size], ev.wire_id, ev.drift)
    dg = cdc.grids_to_tensor(grid, tr.dev)
    p = cdc.scan_params(h=2.0, max_steps=1000, lam=4.0, max_partitions=1, k=8, n_rounds=1)
    t = torch
    out = dict(topk0=t.empty((1, 8), dtype=t.int64, device=tr.dev),
               best_E=t.empty((1, 8), dtype=t.float32, device=tr.dev),
               best_seed=t.empty((1, 8, 5), dtype=t.float32, device=tr.dev),
               hit_part=t.empty(ev.wire_id.size, dtype=t.int8, device=tr.dev),
               hit_res2=t.empty(ev.wire_id.size, dtype=t.float32, device=tr.dev),
               flags=t.empty(1, dtype=t.int32, device=tr.dev), steps=t.zeros(1, dtype=t.int64, device=tr.dev))

    def call(n_stated, E=None):
        out["steps"].zero_()                  # the call adds its step count to the counter
        tr.ctx.cdc_scan_seeds_noalloc(1, n_stated, off, wid, dr, dg, p, E, out["topk0"], out["best_E"],
                                      out["best_seed"], out["hit_part"], out["hit_res2"], out["flags"], out["steps"])

    call(n)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info(tr.dev)[0]
    call(n)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info(tr.dev)[0] == free0
    for key in ("topk0", "best_E", "best_seed", "hit_part", "hit_res2", "flags"):
        assert torch.equal(out[key], ref[key]), key
    assert int(out["steps"][0]) == int(ref["steps"][0])
    for with_E in (False, True):
        E = torch.full((n,), -1.0, dtype=torch.float32, device=tr.dev) if with_E else None
        call(n - 1, E)
        torch.cuda.synchronize()
        assert int(out["flags"][0]) & cdc.FLAG_EMPTY
        assert int(out["steps"][0]) == 0
        assert np.all(np.isinf(out["best_E"].cpu().numpy()))
        if with_E:
            assert torch.all(E == -1.0)
