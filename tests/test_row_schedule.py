"""Host model of the row aggregation kernel's walk schedule (`agg_rows`, one direction per lane
group): the chain walks the W pixels of a row, computing the path term L_r of Eq. sgm_path
(Sec. 2.1.2) step by step, with the costs of step t + U loaded into a U-deep register ring while
step t is computed.

The kernel takes blocks of U steps whose steps and refills all lie inside the row (t0 + 2U < W)
on a loop without end-of-row tests, adding through a running pointer, and the last blocks on the
tested loop. This module restates both loops (the same cursor arithmetic) and checks, for every
row length up to 299 and both ring depths, that together they issue exactly the loads and adds of
the tested loop alone, and that every load reads a pixel of the row."""
import pytest


def _tested(W, U):
    ev, cp = [], 0
    for u in range(U):
        if u < W:
            ev.append(("load", u, cp))
        if u + 1 < W:
            cp += 1
    t0 = 0
    while t0 < W:
        for u in range(U):
            t = t0 + u
            if t >= W:
                break
            if t + U < W:
                ev.append(("load", t + U, cp))
            if t + U + 1 < W:
                cp += 1
            ev.append(("add", t, t))
        t0 += U
    return ev


def _split(W, U):
    ev, cp = [], 0
    for u in range(U):
        if u < W:
            ev.append(("load", u, cp))
        if u + 1 < W:
            cp += 1
    t0, e = 0, 0
    while t0 + 2 * U < W:          # blocks inside the row: no tests
        sp = e
        for u in range(U):
            ev.append(("load", t0 + u + U, cp))
            cp += 1
            ev.append(("add", t0 + u, sp))
            sp += 1
        e += U
        t0 += U
        assert cp <= W - 1         # the cost pointer never leaves the row, not even unused
    while t0 < W:                  # the last blocks: tested
        for u in range(U):
            t = t0 + u
            if t >= W:
                break
            if t + U < W:
                ev.append(("load", t + U, cp))
            if t + U + 1 < W:
                cp += 1
            ev.append(("add", t, e))
            e += 1
        t0 += U
    return ev


@pytest.mark.parametrize("U", [8, 16])
def test_split_loop_issues_the_tested_loops_loads_and_adds(U):
    for W in range(1, 300):
        ev = _split(W, U)
        assert ev == _tested(W, U), W
        for kind, step, ptr in ev:
            assert ptr == step and 0 <= step < W       # the pointer sits on the step's pixel
        assert sorted(s for k, s, _ in ev if k == "add") == list(range(W))
        assert sorted(s for k, s, _ in ev if k == "load") == list(range(W))
