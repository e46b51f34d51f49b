"""Host-side scheduling of hicu_reconstruct_batched: the start order (no GPU needed)."""
import ctypes

import pytest


@pytest.fixture(scope="module")
def hicu():
    from paper_2004_08962_gb300 import build, hicu
    build.build()
    return hicu


def _problem(hicu, n, C, k, rank, stages):
    pr = hicu.hicu_problem()
    pr.geom = hicu.make_geom((n, n, 1), C, (k, k, 1))
    pr.params = hicu.make_params(rank, stages)
    pr._keep = pr.params
    return pr


def test_longest_first_with_stable_ties(hicu):
    full = lambda n, it, gd, p: ((0, 0, 0), (n, n, 1), it, gd, p)
    probs = [
        _problem(hicu, 128, 4, 5, 37, [full(128, 2, 10, 8)]),     # 0: small
        _problem(hicu, 320, 16, 5, 150, [full(320, 2, 10, 32)]),  # 1: largest
        _problem(hicu, 128, 4, 5, 37, [full(128, 2, 10, 8)]),     # 2: tie with 0
        _problem(hicu, 256, 8, 5, 75, [full(256, 2, 10, 32)]),    # 3
        _problem(hicu, 256, 8, 5, 75, [full(256, 4, 10, 32)]),    # 4: twice the iterations of 3
    ]
    order, cost = hicu.hicu_batch_order(probs)
    assert sorted(order) == list(range(5))
    assert order == [1, 4, 3, 0, 2]
    assert cost[4] == pytest.approx(2 * cost[3])
    assert cost[0] == cost[2] > 0
    # every term grows with the work: more coils, larger matrix, more descent steps
    bigger = [_problem(hicu, 128, 8, 5, 37, [full(128, 2, 10, 8)]),
              _problem(hicu, 192, 4, 5, 37, [full(192, 2, 10, 8)]),
              _problem(hicu, 128, 4, 5, 37, [full(128, 2, 20, 8)])]
    _, cb = hicu.hicu_batch_order(bigger)
    assert all(c > cost[0] for c in cb)


def test_empty_and_bad_arguments(hicu):
    assert hicu.hicu_batch_order([]) == ([], [])
    L = hicu.lib()
    assert L.hicu_batch_order(-1, None, None, None) == 1          # HICU_ERR_ARG
    order = (ctypes.c_int32 * 1)()
    assert L.hicu_batch_order(1, None, order, None) == 1
