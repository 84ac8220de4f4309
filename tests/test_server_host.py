"""Host-side logic of the request server: the device-footprint estimate used
for admission and the first-come admission rule (no GPU needed)."""
import pytest

from paper_2609_18841_b300 import lindtebd as lt


def test_context_bytes_scales_with_the_ensemble():
    base = dict(precision=lt.LT_MIXED, num_sms=148)
    b1 = lt.lt_context_bytes(64, 64, 16, **base)
    b2 = lt.lt_context_bytes(64, 64, 32, **base)
    # the site tensors dominate: 2 chi^2 complex64 per site and trajectory
    tensors = 64 * 2 * 64 * 64 * 8
    assert b2 - b1 >= 16 * tensors
    assert b1 >= 16 * tensors
    assert lt.lt_context_bytes(64, 64, 16, precision=lt.LT_FP64, num_sms=148) > b1
    assert lt.lt_context_bytes(32, 64, 16, **base) < b1
    assert lt.lt_context_bytes(64, 32, 16, **base) < b1
    with pytest.raises(lt.LtError):
        lt.lt_context_bytes(64, 257, 16, **base)


def test_context_bytes_of_a_vectorised_density_matrix():
    # four local values per site: the site tensors are twice as large
    base = dict(precision=lt.LT_MIXED, num_sms=148)
    traj = lt.lt_context_bytes(32, 64, 8, **base)
    rho = lt.lt_context_bytes(32, 64, 8, method=lt.LT_MPDO, **base)
    assert rho - traj >= 8 * 32 * 2 * 64 * 64 * 8


@pytest.mark.parametrize("budget,used,max_active,n_active,queue,want", [
    (100, 0, 8, 0, [30, 30, 30, 30], 3),     # budget stops the fourth
    (100, 50, 8, 1, [30, 10], 2),            # both fit in order (80, then 90)
    (100, 50, 8, 1, [60, 10], 0),            # head of line: 60 does not fit, 10 waits behind it
    (100, 0, 2, 1, [10, 10, 10], 1),         # active cap
    (100, 0, 8, 0, [200, 10], 0),            # the head does not fit: nothing passes it
    (100, 0, 8, 0, [], 0),
    (100, 100, 8, 3, [0], 1),                # an empty request always fits
])
def test_admission_is_first_come_under_budget_and_cap(budget, used, max_active, n_active, queue, want):
    assert lt.lt_admit_plan(budget, used, max_active, n_active, queue) == want
