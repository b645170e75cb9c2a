"""Pins of the classification efficiency and purity (sec. 3.1, Eqs. 2-3)."""
import numpy as np

import oracle as O


def test_hand_worked_efficiency_and_purity():
    # one event: truth turns 0,0,0,1,1 and two noise hits; classified 0,0,1,1,-,0,-
    off = [0, 7]
    truth = [0, 0, 0, 1, 1, -1, -1]
    cls = [0, 0, 1, 1, -1, 0, -1]
    C = O.classification_counts(off, cls, truth, 2)
    assert C[0].tolist() == [[1, 1, 0], [0, 2, 1], [1, 0, 1]]
    eps, pur = O.efficiency_purity(C)
    # eps_0 = 2/3 (one of three turn-0 hits went to turn 1), eps_1 = 1/2 (one unclassified);
    # pi_0 = 2/2 (the noise hit classified as 0 is not in Eq. 3's sum), pi_1 = 1/2
    assert np.allclose(eps, [2 / 3, 1 / 2]) and np.allclose(pur, [1.0, 0.5])


def test_perfect_classification_and_event_sums():
    rng = np.random.default_rng(0)
    off = [0, 40, 40, 100]                      # includes an event without hits
    truth = rng.integers(-1, 3, 100)
    C = O.classification_counts(off, truth, truth, 3)
    eps, pur = O.efficiency_purity(C)
    assert np.all(eps == 1.0) and np.all(pur == 1.0)
    assert C[1].sum() == 0 and C.sum() == 100
    # labels beyond n_part count as -1
    C2 = O.classification_counts([0, 3], [5, 0, -7], [0, 0, 0], 1)
    assert C2[0].tolist() == [[0, 0], [2, 1]]
