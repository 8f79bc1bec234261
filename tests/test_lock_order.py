"""The host-side lock-order checker (agile_lock_order_check), which stands in for the
paper's debug lock chain (Sec. 3.5): it reports an order in which threads can wait for
each other forever.  Checked on textbook cases and on the library's own orders."""
import pytest

import paper_2504_19365_gb300 as ag

A, R, T = ag.AGILE_LOCK_ACQUIRE, ag.AGILE_LOCK_RELEASE, ag.AGILE_LOCK_TRY


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2504_19365_gb300 import build
    build.build()


def test_abba_is_a_cycle():
    ev = [(0, A, 1), (0, A, 2), (0, R, 2), (0, R, 1),
          (1, A, 2), (1, A, 1), (1, R, 1), (1, R, 2)]
    n, cyc = ag.agile_lock_order_check(ev)
    assert n == 1 and sorted(cyc) == [1, 2]


def test_three_lock_cycle_and_consistent_order():
    ev = [(0, A, 10), (0, A, 11), (0, R, 11), (0, R, 10),
          (1, A, 11), (1, A, 12), (1, R, 12), (1, R, 11)]
    assert ag.agile_lock_order_check(ev)[0] == 0          # 10 < 11 < 12: consistent
    n, cyc = ag.agile_lock_order_check(ev + [(2, A, 12), (2, A, 10)])
    assert n == 1 and sorted(cyc) == [10, 11, 12]


def test_reacquiring_a_held_lock_is_a_cycle_of_one():
    n, cyc = ag.agile_lock_order_check([(0, A, 7), (0, A, 7)])
    assert n == 1 and cyc == [7]


def test_try_acquire_never_waits():
    # thread 0 holds 1 and only tries 2; thread 1 takes 2 then 1: no wait cycle
    ev = [(0, A, 1), (0, T, 2), (0, R, 2), (0, R, 1), (1, A, 2), (1, A, 1), (1, R, 1), (1, R, 2)]
    assert ag.agile_lock_order_check(ev)[0] == 0


def test_the_library_orders_are_consistent():
    # The orders the library takes its exclusive resources in, per path (numbers name
    # the resource kinds of one page p / line l / queue q):
    #   share entry(p) -> in-flight entry(p) -> line pin(l) -> doorbell lock(q) (tried)
    #   in-flight entry(p) -> victim's in-flight entry(v) -> line claim(l) -> doorbell (tried)
    #   closing share entry(p) -> in-flight entry(p) -> line claim(l)
    # and no path waits for a completion while it holds a line (a waiter holds nothing).
    SH, FL, LN, DB, VF = 1, 2, 3, 4, 5
    paths = [[(A, SH), (A, FL), (A, LN), (T, DB)],
             [(A, FL), (A, VF), (A, LN), (T, DB)],
             [(A, SH), (A, FL), (A, LN)],
             [(A, FL), (A, LN), (T, DB)]]
    ev = []
    for t, path in enumerate(paths):
        ev += [(t, op, lk) for op, lk in path] + [(t, R, lk) for _, lk in reversed(path)]
    assert ag.agile_lock_order_check(ev)[0] == 0
    # taking a line and then blocking on a page's in-flight entry would close a cycle
    assert ag.agile_lock_order_check(ev + [(9, A, LN), (9, A, FL)])[0] == 1


def test_bad_op_is_rejected():
    with pytest.raises(ag.AgileError):
        ag.agile_lock_order_check([(0, 9, 1)])
