"""The serving loop's host logic (admission by memory budget, continuous
batching, ordering, timeouts, back-pressure) in dry-run mode: no GPU work,
each launch completes a fixed time after it starts."""
import time

import pytest

import paper_2210_06438_gb300 as hydro
from paper_2210_06438_gb300 import _build

MS = 1_000_000


@pytest.fixture(scope="module", autouse=True)
def lib():
    _build.build()
    hydro.load()


def task(n, N=8, F=6):
    return hydro.descriptors([(4096 * (i + 1), 0.1, N, F) for i in range(n)])


def task_bytes(n, N=8, F=6, ghost=3):
    G = N + 2 * ghost
    return n * ((G ** 3 + N ** 3) * F * 8 + 8)


FAKE_OUT, FAKE_AMAX = 1 << 20, 1 << 21


def test_tasks_arriving_during_a_launch_join_the_next_one():
    s = hydro.Server(n_streams=1, max_batch=1000, dry_run_ns=40 * MS)
    rc, a = s.submit(task(3), FAKE_OUT, FAKE_AMAX)
    assert rc == hydro.HYDRO_OK
    time.sleep(0.005)  # a is running
    ts = [s.submit(task(k), FAKE_OUT, FAKE_AMAX)[1] for k in (2, 5, 4)]
    for t in [a] + ts:
        assert s.wait(t) == hydro.HYDRO_OK
    st = s.stats()
    assert st["launches"] == 2 and st["max_subgrids_per_launch"] == 11
    assert st["completed"] == 4 and st["subgrids_launched"] == 14
    ta = s.times(a)
    tb = s.times(ts[0])
    assert ta[0] <= ta[1] <= ta[2] <= tb[1] <= tb[2]
    s.close()


def test_budget_bounds_bytes_in_flight():
    budget = task_bytes(8)
    s = hydro.Server(n_streams=4, max_batch=1000, budget_bytes=budget, dry_run_ns=5 * MS)
    ts = [s.submit(task(3), FAKE_OUT, FAKE_AMAX)[1] for _ in range(12)]
    for t in ts:
        assert s.wait(t, 5_000 * MS) == hydro.HYDRO_OK
    st = s.stats()
    assert st["peak_bytes_in_flight"] <= budget
    assert st["completed"] == 12 and st["bytes_in_flight"] == 0
    s.close()


def test_task_larger_than_budget_is_rejected():
    s = hydro.Server(budget_bytes=task_bytes(4), dry_run_ns=MS)
    rc, _ = s.submit(task(5), FAKE_OUT, FAKE_AMAX)
    assert rc == hydro.HYDRO_EBUDGET
    rc, t = s.submit(task(4), FAKE_OUT, FAKE_AMAX)
    assert rc == hydro.HYDRO_OK and s.wait(t) == hydro.HYDRO_OK
    assert s.stats()["rejected"] == 1
    s.close()


def test_full_queue_pushes_back():
    s = hydro.Server(n_streams=1, queue_capacity=2, dry_run_ns=200 * MS)
    rcs = []
    for _ in range(4):
        rcs.append(s.submit(task(1), FAKE_OUT, FAKE_AMAX)[0])
        time.sleep(0.002)
    assert hydro.HYDRO_EBUSY in rcs
    s.close()


def test_wait_deadline_is_host_side():
    s = hydro.Server(n_streams=1, dry_run_ns=100 * MS)
    rc, t = s.submit(task(1), FAKE_OUT, FAKE_AMAX)
    assert s.wait(t, 1 * MS) == hydro.HYDRO_ETIMEDOUT
    assert s.poll(t) == hydro.HYDRO_EBUSY
    assert s.wait(t) == hydro.HYDRO_OK and s.poll(t) == hydro.HYDRO_OK
    assert s.poll(10 ** 9) == hydro.HYDRO_EINVAL
    s.close()


def test_per_task_mode_never_aggregates_and_max_batch_caps_launches():
    s = hydro.Server(n_streams=1, per_task=True, dry_run_ns=5 * MS)
    ts = [s.submit(task(2), FAKE_OUT, FAKE_AMAX)[1] for _ in range(5)]
    for t in ts:
        s.wait(t)
    assert s.stats()["launches"] == 5
    s.close()
    s = hydro.Server(n_streams=1, max_batch=4, dry_run_ns=5 * MS)
    ts = [s.submit(task(3), FAKE_OUT, FAKE_AMAX)[1] for _ in range(6)]
    ts.append(s.submit(task(9), FAKE_OUT, FAKE_AMAX)[1])  # larger than max_batch: alone
    for t in ts:
        s.wait(t)
    st = s.stats()
    assert st["max_subgrids_per_launch"] == 9 and st["launches"] == 7
    s.close()


def test_invalid_submissions():
    s = hydro.Server(dry_run_ns=MS)
    for bad in (hydro.descriptors([(0, 0.1, 8, 6)]), hydro.descriptors([(8, 0.1, 8, 4)])):
        with pytest.raises(hydro.HydroError):
            s.submit(bad, FAKE_OUT, FAKE_AMAX)
    with pytest.raises(hydro.HydroError):
        s.submit(task(1), 0, FAKE_AMAX)
    s.close()
