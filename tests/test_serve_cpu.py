"""Host-side pieces of the server: arrival process, image bytes and the
admission policy (with a stand-in footprint: the tile's bytes plus 2 B per
pixel of scratch, and 128 MiB of fixed state per slot)."""
import numpy as np

from paper_2108_12050_gb300 import serve


def test_poisson_arrivals_rate_and_determinism():
    a = serve.poisson_arrivals(500, 4.0, seed=5)
    b = serve.poisson_arrivals(500, 4.0, seed=5)
    assert a == b and all(x < y for x, y in zip(a, a[1:]))
    assert 1800 < len(a) < 2200          # 500/s over 4 s, within ~4.5 sigma
    gaps = np.diff([0.0] + a)
    assert abs(gaps.mean() - 1 / 500) < 2e-4


def test_image_bytes_grow_with_pixels_and_dtype():
    f8 = serve.image_bytes((1024, 1024), np.uint8)
    f16 = serve.image_bytes((1024, 1024), np.uint16)
    assert f16 - f8 == 1024 * 1024
    assert serve.image_bytes((2048, 2048), np.uint8) == 4 * f8
    assert serve.image_bytes((3, 5), np.float32) == 60


F = 128 << 20


def _footprint(shape, dtype):
    return serve.image_bytes(shape, dtype) + 2 * shape[0] * shape[1]


def test_admission_prefers_the_slot_that_needs_least_growth():
    # slot 1 already holds scratch for a large tile: no growth needed there
    act, k = serve.plan_admission([0, 1, 2], {0: 500, 1: 0, 2: 500},
                                  {0: F, 1: F + 800, 2: F}, used=3 * F + 800, budget=10 * F,
                                  fixed=F)
    assert (act, k) == ("admit", 1)
    # ties go to the first free slot
    assert serve.plan_admission([2, 0], {0: 7, 2: 7}, {0: F, 2: F}, 0, 10 * F, F) == ("admit", 2)


def test_admission_releases_the_biggest_grown_slot_when_the_budget_is_short():
    budget = 4 * F
    used = 2 * F + 3 * F // 4           # slot 0 grown by F/4, slot 1 by F/2
    resident = {0: F + F // 4, 1: F + F // 2}
    act, k = serve.plan_admission([0, 1], {0: F // 2, 1: F // 4}, resident, used, budget, F)
    assert (act, k) == ("admit", 1)      # still fits by growing slot 1 a little
    act, k = serve.plan_admission([0, 1], {0: F + F, 1: F + F // 2}, resident, used, budget, F)
    assert (act, k) == ("reset", 1)      # nothing fits: give back the larger scratch


def test_admission_waits_when_nothing_can_be_released():
    assert serve.plan_admission([0], {0: 5 * F}, {0: F}, 2 * F, 4 * F, F) == ("wait", None)
    assert serve.plan_admission([], {}, {}, 0, 4 * F, F) == ("wait", None)


def _simulate(sizes, durations, n_slots, budget):
    """The server's admission loop as a discrete-event simulation: slots grow
    their resident scratch to the largest tile they served and give it back
    only when the head of the queue does not fit otherwise."""
    import collections
    fp = [_footprint(s, np.uint16) for s in sizes]
    resident = [F] * n_slots
    busy = [None] * n_slots
    used = F * n_slots
    queue = collections.deque(range(len(sizes)))
    t, order, peak = 0.0, [], used
    while queue or any(b is not None for b in busy):
        while queue:
            r = queue[0]
            free = [k for k in range(n_slots) if busy[k] is None]
            need = {k: max(0, F + fp[r] - resident[k]) for k in free}
            act, k = serve.plan_admission(free, need, {k: resident[k] for k in free}, used, budget,
                                          F)
            if act == "wait":
                break
            if act == "reset":
                used -= resident[k] - F
                resident[k] = F
                continue
            queue.popleft()
            resident[k] += need[k]
            used += need[k]
            busy[k] = (t + durations[r], r)
            order.append(r)
            assert used == sum(resident) and used <= budget
            peak = max(peak, used)
        running = [(b, k) for k, b in enumerate(busy) if b is not None]
        assert running, "queue stalled with every slot free"
        (t, _), k = min(running)
        busy[k] = None
    return order, peak


def test_admission_never_exceeds_the_budget_and_keeps_arrival_order():
    rng = np.random.default_rng(3)
    sides = [256, 512, 1024, 2048, 4096, 8192]
    for trial in range(20):
        n = int(rng.integers(20, 80))
        sizes = [(int(rng.choice(sides)), int(rng.choice(sides))) for _ in range(n)]
        durations = rng.exponential(1.0, n)
        n_slots = int(rng.integers(1, 9))
        biggest = max(_footprint(s, np.uint16) for s in sizes)
        # every request fits alone next to all slots' fixed state (what
        # submit() checks); some budgets leave room for one large tile only
        budget = F * n_slots + biggest + int(rng.integers(0, 3)) * biggest // 2
        order, peak = _simulate(sizes, durations, n_slots, budget)
        assert order == list(range(n)), trial
        assert peak <= budget
