"""Host logic of the learned scheduler (no GPU): queue order, list-scheduling
makespan, panel binning and the padded-work ratio, checked on hand-worked
cases and against brute force."""
import itertools

import numpy as np

from paper_1402_7285_gb300 import scheduler


def test_longest_first_is_a_stable_descending_order():
    pred = np.array([3.0, 1.0, 3.0, 7.0, 0.5])
    order = scheduler.longest_first(pred)
    assert order.tolist() == [3, 0, 2, 1, 4]          # ties keep the given order
    assert order.dtype == np.int64


def test_greedy_makespan_hand_cases():
    # two workers, costs 5, 4, 3, 3, 3: given order -> {5+3, 4+3+3} = 10; longest first is the same here
    assert scheduler.greedy_makespan([5, 4, 3, 3, 3], range(5), 2) == 10.0
    # one long job last in the given order: plain 1+1+9 on one worker vs 9 | 1+1 longest first
    costs = [1.0, 1.0, 9.0]
    assert scheduler.greedy_makespan(costs, [0, 1, 2], 2) == 10.0
    assert scheduler.greedy_makespan(costs, scheduler.longest_first(costs), 2) == 9.0
    # more workers than jobs: the longest job
    assert scheduler.greedy_makespan([2.0, 7.0], [0, 1], 5) == 7.0


def test_longest_first_meets_the_list_scheduling_bound():
    """Longest-first list scheduling is within 4/3 of the optimal makespan
    (Graham's bound); checked against brute force on small instances."""
    rng = np.random.default_rng(0)
    for _ in range(30):
        costs = rng.integers(1, 20, size=7).astype(float)
        workers = int(rng.integers(2, 4))
        best = min(scheduler.greedy_makespan(costs, perm, workers)
                   for perm in itertools.permutations(range(len(costs))))
        lpt = scheduler.greedy_makespan(costs, scheduler.longest_first(costs), workers)
        assert best <= lpt <= (4.0 / 3.0) * best + 1e-12


def test_padded_work_hand_cases():
    iters = np.array([1.0, 4.0, 2.0, 3.0])
    # panels of two in the given order: (1,4), (2,3) -> 2*4 + 2*3 = 14 over 10
    assert abs(scheduler.padded_work(iters, np.arange(4), 2) - 1.4) < 1e-15
    # binned by (here exact) prediction: (4,3), (2,1) -> 2*4 + 2*2 = 12 over 10
    order = scheduler.panels_by_prediction(iters, 2)
    assert abs(scheduler.padded_work(iters, order, 2) - 1.2) < 1e-15
    # a ragged last panel counts its full width
    assert abs(scheduler.padded_work(np.array([2.0, 2.0, 2.0]), np.arange(3), 2) - (2 * 2 + 2 * 2) / 6) < 1e-15


def test_sorting_minimises_padded_work():
    """Binning columns of similar length (sorted order) never pads more than
    any other order; checked against all orders of small instances."""
    rng = np.random.default_rng(1)
    for _ in range(20):
        iters = rng.integers(1, 50, size=6).astype(float)
        sorted_pad = scheduler.padded_work(iters, scheduler.panels_by_prediction(iters, 2), 2)
        best = min(scheduler.padded_work(iters, np.array(p), 2) for p in itertools.permutations(range(6)))
        assert abs(sorted_pad - best) < 1e-12


def test_predictor_normalisation_round_trip():
    X = np.arange(12, dtype=np.float32).reshape(3, 4)
    p = scheduler.Predictor(np.zeros(1, np.float32), X.mean(axis=0), X.std(axis=0) + 1, 0.0, 1.0)
    Xn = p.normalise(X)
    assert Xn.dtype == np.float32
    assert np.allclose(Xn * p.x_std + p.x_mean, X)
