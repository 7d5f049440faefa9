"""The fused kernel's work split, restated on the CPU: the batch's iterations
laid end to end (candidate j has max(K_j, 1) units), CTA m takes units
[m cap, (m+1) cap) with cap = max(ceil(units / slots), longest candidate), and
walks its candidates in descending order.  These checks pin the properties the
kernel relies on: every unit runs exactly once, a candidate is cut into at
most two parts on neighbouring CTAs, the first part is the first thing its CTA
runs and the second part the last thing the next CTA runs (so the only wait,
second part on first part, can always be satisfied), and no CTA exceeds cap."""
import random

import pytest


def split(lengths_K, slots):
    B = len(lengths_K)
    L = [max(k, 1) for k in lengths_K]
    start = [0]
    for l in L:
        start.append(start[-1] + l)
    units = start[-1]
    cap = max((units + slots - 1) // slots, max(L))
    grid = (units + cap - 1) // cap

    def job_of(x):  # largest j with start[j] <= x (binary search, as the kernel)
        lo, hi = 0, B - 1
        while lo < hi:
            mid = (lo + hi + 1) >> 1
            if start[mid] <= x:
                lo = mid
            else:
                hi = mid - 1
        return lo

    runs = []
    for m in range(grid):
        m0, m1 = m * cap, min(m * cap + cap, units)
        seq = []
        for j in range(job_of(m1 - 1), job_of(m0) - 1, -1):
            u0, u1 = max(m0 - start[j], 0), min(m1 - start[j], L[j])
            seq.append((j, u0, u1))
        runs.append(seq)
    return runs, L, cap, grid


@pytest.mark.parametrize("trial", range(400))
def test_split_invariants(trial):
    rng = random.Random(trial)
    B, slots = rng.randint(1, 600), rng.randint(1, 460)
    Ks = [rng.randint(0, 100)] * B if trial % 2 else [rng.randint(0, 80) for _ in range(B)]
    runs, L, cap, grid = split(Ks, slots)
    assert grid <= slots
    cover = [[0] * l for l in L]
    where = {}
    for m, seq in enumerate(runs):
        assert sum(u1 - u0 for _, u0, u1 in seq) <= cap
        for pos, (j, u0, u1) in enumerate(seq):
            assert u0 < u1
            for u in range(u0, u1):
                cover[j][u] += 1
            where.setdefault(j, []).append((m, pos, u0, u1))
    assert all(c == 1 for row in cover for c in row)
    for j, parts in where.items():
        assert len(parts) <= 2
        if len(parts) == 2:
            (ma, pa, a0, a1), (mb, pb, b0, b1) = sorted(parts)
            assert mb == ma + 1 and a0 == 0 and b1 == L[j] and a1 == b0
            assert pa == 0, "first part runs first on its CTA"
            assert pb == len(runs[mb]) - 1, "second part runs last on the next CTA"


def test_benchmark_batch_split():
    runs, L, cap, grid = split([50] * 256, 152)
    assert (cap, grid) == (85, 151)  # vs 2 rounds x 50 without the split
