"""A model of the split-call schedule of the persistent kernels, on the CPU:
P slots (resident replica groups) take work units in queue order; unit u is
part u // R of replica u % R and may start only when unit u - R (the same
replica's previous part) has finished. With R > P, the model checks the
argument behind the bounded wait in the kernels. Every unit finishes (no
deadlock), parts of a replica run in order, and a wait, when one happens, is
shorter than one part's duration. It also checks that splitting removes the
idle last round: the makespan approaches R * K / P part durations instead of
ceil(R / P) whole calls."""

import heapq
import math
import random

import pytest


def simulate(P, R, K, jitter, seed=0):
    rng = random.Random(seed)
    finish = {}
    free = [(0.0, s) for s in range(P)]  # (time the slot is free, slot)
    heapq.heapify(free)
    waits = []
    order = {}
    for u in range(R * K):
        t_free, s = heapq.heappop(free)
        start = t_free
        if u >= R:
            prev = finish[u - R]  # taken R units earlier: already scheduled
            if prev > start:
                waits.append(prev - start)
                start = prev
        dur = 1.0 + rng.uniform(-jitter, jitter)
        finish[u] = start + dur
        order.setdefault(u % R, []).append((u // R, start, finish[u]))
        heapq.heappush(free, (finish[u], s))
    return max(finish.values()), waits, order


@pytest.mark.parametrize("P,R,K", [(2432, 4096, 16), (2432, 3648, 16), (760, 4096, 16), (5, 7, 4), (3, 4, 8)])
def test_parts_complete_in_order_with_short_waits(P, R, K):
    span, waits, order = simulate(P, R, K, jitter=0.2)
    for parts in order.values():
        assert [k for k, _, _ in parts] == list(range(K))
        for (_, _, f0), (_, s1, _) in zip(parts, parts[1:]):
            assert s1 >= f0  # part k + 1 after part k
    assert all(w < 1.2 for w in waits)  # below one part's duration


def test_parts_remove_the_idle_last_round():
    # n100: 4096 replicas, 2432 slots. Whole calls: two rounds of one call
    # each (16 parts' worth of time per round); 16 parts: close to the
    # fluid bound R * K / P.
    P, R, K = 2432, 4096, 16
    whole, _, _ = simulate(P, R, 1, jitter=0.0)
    parts, _, _ = simulate(P, R, K, jitter=0.05)
    assert whole == math.ceil(R / P)  # in units of one whole call
    fluid = R * K / P / K  # in whole-call units
    assert parts / K < fluid * 1.08
    assert parts / K < whole * 0.9
