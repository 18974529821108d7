"""The schedule of the band route's pipelined bulge chase, checked on the host.

Step t of sweep i (c0 = i + 1 + 8t, c1 = min(c0 + 7, n - 1), row = i for t = 0
else c0 - 8) applies a right reflector to rows row .. row+15 over columns
c0 .. c1 and a left reflector to rows c0 .. c1 over columns c0 .. c0+15, on the
band window of offsets c - r in [-7, 15].  Sweep i's step t starts once sweep
i-1 has finished step t+3 (or all its steps); by induction sweep i-d has then
finished step t+3d.  The steps that can run meanwhile are therefore those
(i-d, t') with t' >= t+3d; the test checks that no such step touches an entry
that step (i, t) touches, which makes the pipelined order give the
sequential chase's result.  It also checks the step count each sweep stores
reflectors for against the sweep loop.
"""
import pytest

B = 8
LAG = 3


def sweep_steps(i, n):
    m = n - 2 - i
    return (m + B - 1) // B if m > 0 else 0


def sweep_loop_steps(i, n):
    c0, c1, t = i + 1, min(i + B, n - 1), 0
    while c1 > c0:
        t += 1
        c0 += B
        c1 = min(c1 + B, n - 1)
    return t


def touched(i, t, n):
    c0 = i + 1 + B * t
    c1 = min(c0 + B - 1, n - 1)
    row = i if t == 0 else c0 - B
    out = set()
    for r in range(row, min(row + 16, n)):            # right reflector
        for c in range(c0, c1 + 1):
            if -7 <= c - r <= 15:
                out.add((r, c))
    for r in range(c0, c1 + 1):                       # left reflector
        for c in range(c0, min(c0 + 16, n)):
            if -7 <= c - r <= 15:
                out.add((r, c))
    return out


@pytest.mark.parametrize("n", [16, 24, 64, 136])
def test_step_counts(n):
    assert [sweep_steps(i, n) for i in range(n - 1)] == [sweep_loop_steps(i, n) for i in range(n - 1)]


@pytest.mark.parametrize("n", [40, 64, 72, 136])
def test_concurrent_steps_touch_disjoint_entries(n):
    regions = {(i, t): touched(i, t, n) for i in range(n - 1) for t in range(sweep_steps(i, n))}
    rows = {k: (min(r for r, _ in v), max(r for r, _ in v)) for k, v in regions.items() if v}
    pairs = 0
    for (i, t), reg in regions.items():
        if not reg:
            continue
        lo, hi = rows[(i, t)]
        for d in range(1, i + 1):
            for tp in range(t + LAG * d, sweep_steps(i - d, n)):
                pairs += 1
                other = rows.get((i - d, tp))
                if other is None or other[1] < lo or other[0] > hi:
                    continue                          # rows apart: disjoint
                assert not (reg & regions[(i - d, tp)]), (i, t, i - d, tp)
    assert pairs > 0


def test_a_lag_of_two_would_overlap():
    # the margin is needed: with sweep i two steps behind sweep i-1, some steps share entries
    n = 64
    clash = any(touched(i, t, n) & touched(i - 1, t + 2, n)
                for i in range(1, n - 1) for t in range(sweep_steps(i, n)) if t + 2 < sweep_steps(i - 1, n))
    assert clash
