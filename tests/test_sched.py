"""The serving loop's admission policy (host logic, no device): FIFO under a
byte budget and a slot limit, through the C ABI's hz_sched_* calls.  Checked
against a plain model of the rule on scripted and random event sequences."""
import numpy as np
import pytest

from paper_2511_16808_gb300 import hz


def test_fifo_budget_and_slots():
    s = hz.hz_sched_create(100, 2)
    assert hz.hz_sched_offer(s, 1, 60)
    assert hz.hz_sched_offer(s, 2, 50)
    assert hz.hz_sched_offer(s, 3, 10)
    assert not hz.hz_sched_offer(s, 4, 101)          # larger than the whole budget: refused
    assert hz.hz_sched_next(s) == 1
    assert hz.hz_sched_next(s) is None               # 60 + 50 > 100: the head waits ...
    st = hz.hz_sched_state(s)
    assert st == {"in_use": 60, "peak": 60, "active": 1, "queued": 2}   # ... and 3 does not overtake it
    hz.hz_sched_release(s, 60)
    assert hz.hz_sched_next(s) == 2
    assert hz.hz_sched_next(s) == 3
    assert hz.hz_sched_state(s)["active"] == 2
    assert hz.hz_sched_offer(s, 5, 5)
    assert hz.hz_sched_next(s) is None               # both slots taken
    hz.hz_sched_release(s, 10)
    assert hz.hz_sched_next(s) == 5
    st = hz.hz_sched_state(s)
    assert st["in_use"] == 55 and st["peak"] == 60 and st["queued"] == 0
    hz.hz_sched_destroy(s)


def test_exact_fit_admits():
    s = hz.hz_sched_create(100, 4)
    assert hz.hz_sched_offer(s, 7, 100)
    assert hz.hz_sched_next(s) == 7
    assert hz.hz_sched_state(s)["in_use"] == 100
    hz.hz_sched_destroy(s)


@pytest.mark.parametrize("seed", range(5))
def test_random_sequences_follow_the_rule(seed):
    """Random offers / admissions / releases against a plain model: admission
    in arrival order, never above the budget or the slot limit, and an
    admission happens whenever the head fits."""
    rng = np.random.default_rng(seed)
    budget, slots = int(rng.integers(50, 200)), int(rng.integers(1, 5))
    s = hz.hz_sched_create(budget, slots)
    queue, active, in_use, peak, order, admitted, t = [], {}, 0, 0, [], [], 0
    for _ in range(400):
        op = rng.integers(3)
        if op == 0:
            t += 1
            b = int(rng.integers(1, budget + 20))
            ok = hz.hz_sched_offer(s, t, b)
            assert ok == (b <= budget)
            if ok:
                queue.append((t, b))
                order.append(t)
        elif op == 1:
            got = hz.hz_sched_next(s)
            fits = bool(queue) and len(active) < slots and in_use + queue[0][1] <= budget
            if fits:
                assert got == queue[0][0]
                tt, b = queue.pop(0)
                active[tt] = b
                in_use += b
                peak = max(peak, in_use)
                admitted.append(tt)
            else:
                assert got is None
        elif active:
            tt = list(active)[int(rng.integers(len(active)))]
            b = active.pop(tt)
            in_use -= b
            hz.hz_sched_release(s, b)
        st = hz.hz_sched_state(s)
        assert st == {"in_use": in_use, "peak": peak, "active": len(active), "queued": len(queue)}
        assert in_use <= budget and len(active) <= slots
    assert admitted == order[:len(admitted)]
    hz.hz_sched_destroy(s)
