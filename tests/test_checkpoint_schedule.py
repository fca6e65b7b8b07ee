"""Host-side check of the binomial checkpoint schedule (no GPU): simulating the actions
must reverse every step exactly once in order N-1..0 with the right state current,
evaluate the objective once at X_N before the first adjoint step, never use more slots
than given, and recompute at most t forward sweeps with t minimal for
C(s + t, s) >= N (Griewank-Walther binomial bound)."""
from math import comb

import pytest

from paper_2506_14792_gb300 import build, spadj


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if build.stale():
        build.build()


def simulate(n, slots, host_slots=0):
    ops = spadj.checkpoint_schedule(n, slots, host_slots)
    store = {}
    cur = 0
    adjoint_order = []
    advances = 0
    objective_at = None
    for typ, a, b, sl in ops:
        if typ == spadj.CK_STORE:
            assert cur == a
            assert 0 <= sl < min(slots, n + 1) or slots <= sl < slots + host_slots
            assert sl not in store
            store[sl] = a
        elif typ == spadj.CK_RESTORE:
            assert store.get(sl) == a
            cur = a
        elif typ == spadj.CK_ADVANCE:
            assert cur == a and b > a
            advances += b - a
            cur = b
        elif typ == spadj.CK_OBJECTIVE:
            assert cur == n and objective_at is None and not adjoint_order
            objective_at = a
        elif typ == spadj.CK_ADJOINT:
            assert cur == a and objective_at == n
            adjoint_order.append(a)
        elif typ == spadj.CK_FREE:
            assert store.get(sl) == a
            del store[sl]
    assert adjoint_order == list(range(n - 1, -1, -1))
    return advances


@pytest.mark.parametrize("n", [1, 2, 7, 30, 200, 2000])
@pytest.mark.parametrize("slots", [1, 2, 3, 16, 64, 100000])
def test_schedule_valid_and_binomial(n, slots):
    if n >= 2000 and slots <= 2:
        pytest.skip("quadratic schedule, covered at smaller n")
    adv = simulate(n, slots)
    s = min(slots, n + 1) - 1
    if s >= n:
        assert adv == n  # store-all: one forward sweep
        return
    if s == 0:
        assert adv == n * (n + 1) // 2
        return
    t = 1
    while comb(s + t, s) < n:
        t += 1
    assert adv <= t * n + n


def test_rejects_bad_arguments():
    with pytest.raises(spadj.SpadjError):
        spadj.checkpoint_schedule(0, 4)


@pytest.mark.parametrize("n,slots,host", [(1, 1, 1), (7, 1, 3), (30, 2, 4), (200, 3, 10), (2000, 16, 40),
                                          (2000, 4, 2000), (13, 100, 5)])
def test_two_level_schedule(n, slots, host):
    """Device + host schedule: valid (every step reversed once in order, objective first, no slot
    reused before it is freed, host slots in their own range); the host holds one state per
    segment, stored during the single first sweep; each segment is then reversed within the
    binomial bound on the device slots."""
    ops = spadj.checkpoint_schedule(n, slots, host)
    K = -(-n // host)
    nseg = -(-n // K)
    host_stores = [a for typ, a, b, sl in ops if typ == spadj.CK_STORE and sl >= slots]
    assert host_stores == [j * K for j in range(nseg)]
    adv = simulate(n, slots, host)
    s = min(slots, K + 1) - 1
    first = (nseg - 1) * K
    if s >= K:  # store-all inside each segment: L - 1 advances per segment, one more for the objective
        assert adv == first + (n - nseg) + 1
    else:
        t = 1
        while s > 0 and comb(s + t, s) < K:
            t += 1
        bound = K * (K + 1) // 2 if s == 0 else t * K + K
        assert adv <= first + nseg * bound
