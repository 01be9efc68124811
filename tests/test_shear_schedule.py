"""Host model of the sheared-column aggregation kernel's walk schedule, checked against the
definition of its chains.

The kernel (`agg_shear_t`) walks the column and diagonal paths of the SGM recurrence (the path
term L_r of Eq. sgm_path, Sec. 2.1.2, computed along independent path lines as in Sec. 2.2.2) as
sheared chains: chain j of a kind with shear s visits
pixel x = (j + s y) mod W of every row, top-down or bottom-up, and restarts where x wraps around
the image edge, because a new line of the path enters there. A warp owns n adjacent chains. Each
step copies the costs of its run 6 steps ahead into an 8-slot ring and adds the step's sums into
S with one bulk reduction, or two where the run wraps. Pairs of steps for which no step involved
meets an event (a wrapping run, a restart, a cursor wrap, the last rows) take a fast path that
tests for none of them; the other steps take the general path.

This module restates that schedule (the same cursor arithmetic and fast-pair conditions as the
kernel) and checks, for widths, heights, disparity counts, chain counts, all six kinds and first
and last warp items:
- every copy reads the right pixel of the right row, in bounds, into the step's ring slot;
- every bulk add covers exactly the run's pixels;
- every chain restart falls on a general step;
- every row is copied exactly once.
The GPU parity tests check the kernel's results; this checks the schedule's index arithmetic on
the CPU, including shapes too many to run on the GPU."""
import pytest

KS = 8  # steps in the cost ring


def walk(W, H, D, CH, kind, j0, BPE=2):
    n = min(CH, W - j0)
    SH0 = kind < 2
    sh = 0 if SH0 else (1 if kind < 4 else -1)
    back = (kind & 1) != 0
    dy = -1 if back else 1
    dx = -sh if back else sh
    ystart = H - 1 if back else 0
    xs = (j0 + sh * ystart) % W
    PP = D // 16
    slot_bytes = CH * D
    cstride = (dy * W + dx) * D
    astride = cstride * BPE
    cwrap = W * D
    awrap = cwrap * BPE
    crun = (ystart * W + xs) * D
    xc = xs
    arun = (ystart * W + xs) * D * BPE
    NCP = (CH * D) // 512 if CH * D >= 512 else 1
    pieces = [(p // PP, p % PP) for p in range(32 * NCP)]
    copies = {}
    restarts = {}
    edge = 0 if dx > 0 else W - 1

    def y_of(t):
        return ystart + dy * t

    def x0_of(t):
        return (j0 + sh * y_of(t)) % W

    def slot_of(t):
        return (t & (KS - 1)) * slot_bytes

    def copy_step(tc):
        nonlocal crun, xc
        if tc >= H:
            return
        lst = []
        if SH0 or xc + n <= W:
            lst = [(slot_of(tc), pc, pi, crun + 16 * i)
                   for i, (pc, pi) in enumerate(pieces) if pc < n]
        else:
            for i, (pc, pi) in enumerate(pieces):
                if pc < n:
                    back_w = W if xc + pc >= W else 0
                    lst.append((slot_of(tc), pc, pi, crun + (pc - back_w) * D + pi * 16))
        assert tc not in copies
        copies[tc] = lst
        crun += cstride
        if not SH0:
            xc += dx
            if xc >= W:
                xc -= W
                crun -= cwrap
            elif xc < 0:
                xc += W
                crun += cwrap

    def copy_two(tc):
        nonlocal crun, xc
        for k in range(2):
            assert tc + k not in copies and tc + k < H
            copies[tc + k] = [(slot_of(tc + k), pc, pi, crun + k * cstride + 16 * i)
                              for i, (pc, pi) in enumerate(pieces) if pc < n]
        crun += 2 * cstride
        if not SH0:
            xc += 2 * dx

    def fast_pairs(t):
        qh = H - KS - t
        if qh < 0:
            return 0
        q = qh >> 1
        if not SH0:
            if dx > 0:
                lim = min(W - n, W - 2) - (KS - 1)
                if xs < 1 or xs > lim:
                    return 0
                q = min(q, (lim - xs) >> 1)
            else:
                if xs < KS or xs > W - n - 1:
                    return 0
                q = min(q, (xs - KS) >> 1)
        return q + 1

    def check_step(t, n1):
        y, x0 = y_of(t), x0_of(t)
        assert x0 == xs
        lst = copies[t]
        assert len(lst) == n * PP
        for slot, pc, pi, off in lst:
            assert slot == slot_of(t)
            assert off == (y * W + (x0 + pc) % W) * D + pi * 16
            assert 0 <= off and off + 16 <= W * H * D
        ranges = [(arun, n1)]
        if not SH0 and n1 < n:
            ranges.append((arun - xs * D * BPE, n - n1))
        covered = [a + k * D * BPE for a, m in ranges for k in range(m)]
        assert all(m > 0 for _, m in ranges)
        assert covered == [(y * W + (x0 + c) % W) * D * BPE for c in range(n)]

    nfast = 0
    for s in range(0, KS - 2, 2):
        copy_step(s)
        copy_step(s + 1)
    t = 0
    while t < H:
        np_ = 0 if (t & 1) else fast_pairs(t)
        while np_ > 0:
            for u in range(2):
                if u == 0:
                    copy_two(t + u + KS - 2)
                if not SH0 and t + u > 0:
                    assert all((xs + c) % W != edge for c in range(n)), "restart on a fast step"
                check_step(t + u, n)
                nfast += 1
                arun += astride
                if not SH0:
                    xs += dx
                    assert 0 <= xs < W
            np_ -= 1
            t += 2
        if t >= H:
            break
        if (t & 1) == 0:
            copy_step(t + KS - 2)
            copy_step(t + KS - 1)
        if not SH0 and t > 0:
            restarts[t] = [c for c in range(CH) if (xs + c) % W == edge]
        check_step(t, (W - xs) if (not SH0 and xs + n > W) else n)
        arun += astride
        if not SH0:
            xs += dx
            if xs >= W:
                xs -= W
                arun -= awrap
            elif xs < 0:
                xs += W
                arun += awrap
        t += 1
    if not SH0:
        for tt in range(1, H):
            due = [c for c in range(n) if (x0_of(tt) + c) % W == edge]
            if due:
                assert tt in restarts and set(due) <= set(restarts[tt]), (tt, due)
    assert set(copies) == set(range(H))
    return nfast


@pytest.mark.parametrize("W", [1, 2, 5, 8, 9, 16, 17, 40, 97, 311])
def test_schedule_matches_chain_definition(W):
    for H in [1, 2, 7, 8, 9, 16, 33, 100]:
        for D, CH in [(16, 32), (32, 16), (64, 8), (128, 4), (128, 8), (256, 2), (256, 4)]:
            G = (W + CH - 1) // CH
            for kind in range(6):
                for j0 in sorted({0, CH * (G // 2), CH * (G - 1)}):
                    walk(W, H, D, CH, kind, j0)


def test_fast_path_share_on_a_large_frame():
    # 1242 x 375 at D = 128 with 8 chains per warp: every warp item takes most of its steps on the
    # fast path (only the window around the edge column and the last rows are general).
    worst = min(walk(1242, 375, 128, 8, kind, j0) / 375
                for kind in range(6) for j0 in range(0, 1242, 8 * 7))
    assert worst > 0.9
