"""Host logic of the learned order (no GPU): the work a single walker spends
before the first solution-bearing subtree, the geometric-mean summary of two
orders, and the scorer's initial parameters."""
import numpy as np

from paper_2508_08702_gb300 import learn


def test_work_before_first():
    nodes = np.array([5, 3, 7, 2])
    sols = np.array([0, 0, 1, 1])
    assert learn._work_before_first(nodes, sols, np.arange(4)) == (8, 2)
    assert learn._work_before_first(nodes, sols, np.array([3, 2, 1, 0])) == (0, 0)
    assert learn._work_before_first(nodes, sols, np.array([1, 0, 3, 2])) == (8, 2)
    assert learn._work_before_first(nodes, np.zeros(4, int), np.arange(4)) == (17, 4)


def test_ratios_are_geometric_means_over_solved_instances():
    w = learn.OrderWork(plain=[99, 3, 50], learned=[9, 3, 1], plain_rank=[9, 1, 4], learned_rank=[0, 1, 4],
                        prefixes=[10, 10, 4])
    work, rank = w.ratios()
    # the third instance has no solution-bearing subtree (rank == prefixes): left out
    assert np.isclose(work, np.sqrt((10 / 100) * (4 / 4)))
    assert np.isclose(rank, np.sqrt((1 / 10) * (2 / 2)))


def test_initial_parameters():
    a, b = learn.init_params(0), learn.init_params(0)
    assert np.array_equal(a, b) and a.dtype == np.float32
    n1, n2, n3 = learn.IN * learn.HID, learn.HID * learn.HID, learn.HID * learn.OUT
    assert a.size == n1 + learn.HID + n2 + learn.HID + n3 + learn.OUT
    w1 = a[:n1]
    b1 = a[n1:n1 + learn.HID]
    assert not b1.any()
    assert abs(w1.std() - np.sqrt(2.0 / learn.IN)) < 0.1 * np.sqrt(2.0 / learn.IN)
    assert not np.array_equal(learn.init_params(1), a)
