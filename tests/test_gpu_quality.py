"""GPU classification counts (sec. 3.1, Eqs. 2-3) against the oracle's
definition: bit-exact on random labels and on a scan's classification."""
import numpy as np
import pytest

import cdc_synth as S
import oracle as O
from tests.gpu_util import tracker

pytestmark = pytest.mark.gpu


def test_counts_bit_exact_on_random_labels():
    import torch
    rng = np.random.default_rng(3)
    sizes = [0, 57, 1, 300, 1024]
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int32)
    truth = rng.integers(-3, 5, off[-1]).astype(np.int8)     # includes labels outside -1..n_part-1
    cls = rng.integers(-2, 5, off[-1]).astype(np.int8)
    g, f = S.make_geometry(), S.uniform_field(1.0)
    tr = tracker(g, f)
    d = tr.dev
    out = tr.classification_counts(torch.as_tensor(off, device=d), torch.as_tensor(cls, device=d),
                                   torch.as_tensor(truth, device=d), 3)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), O.classification_counts(off, cls, truth, 3))


def test_scan_classification_efficiency_and_purity():
    """Counts of a scan's classification (truth-centred single-turn grids of
    three events) equal the oracle's; the best seed classifies most signal hits
    into partition 0 and few noise hits."""
    import torch
    import paper_1908_01949_gb300 as cdc
    cases = [S.cfg1_case(i) for i in (0, 1, 2)]
    g, f = cases[0][0], cases[0][1]
    evs = [c[2] for c in cases]
    grids = np.concatenate([c[3] for c in cases])
    off, wid, dr = S.pack_events(evs)
    truth = np.concatenate([e.truth_part for e in evs]).astype(np.int8)
    tr = tracker(g, f)
    off_t, wid_t, dr_t = tr.events_to_device(off, wid, dr)
    p = cdc.scan_params(h=2.0, max_steps=1000, lam=4.0, max_partitions=1, k=8, n_rounds=3, n_zoom=4)
    out = tr.scan(off_t, wid_t, dr_t, cdc.grids_to_tensor(grids, tr.dev), p)
    counts = tr.classification_counts(off_t, out["hit_part"], torch.as_tensor(truth, device=tr.dev), 1)
    torch.cuda.synchronize()
    hp = out["hit_part"].cpu().numpy()
    assert np.array_equal(counts.cpu().numpy(), O.classification_counts(off, hp, truth, 1))
    eps, pur = (x.cpu().numpy() for x in tr.efficiency_purity(counts))
    assert eps[0] > 0.8 and pur[0] == 1.0


def test_efficiency_and_purity_follow_the_oracle_formula():
    """cdc_efficiency_purity (Eqs. 2-3 on the device, counts summed over the
    events) against the oracle's formula on random counts, with empty rows and
    columns giving NaN."""
    import torch
    rng = np.random.default_rng(1)
    C = rng.integers(0, 9, (5, 4, 4)).astype(np.int32)
    C[:, 2, :] = 0                                    # truth partition 1 absent: eps NaN
    C[:, 1:, 3] = 0                                   # nothing classified 2: pur NaN
    g, f = S.make_geometry(), S.uniform_field(1.0)
    tr = tracker(g, f)
    eps, pur = tr.efficiency_purity(torch.as_tensor(C, device=tr.dev))
    torch.cuda.synchronize()
    e0, p0 = O.efficiency_purity(C)
    assert np.allclose(eps.cpu().numpy(), e0, rtol=1e-6, equal_nan=True)
    assert np.allclose(pur.cpu().numpy(), p0, rtol=1e-6, equal_nan=True)
    assert np.isnan(e0[1]) and np.isnan(p0[2])
