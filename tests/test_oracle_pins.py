"""Pins of the CPU oracle to what the paper and the mathematics fix, independent of the oracle.

Each test derives its expected values from something other than the oracle's own code: closed
forms, brute-force enumeration over tiny inputs, the paper's worked examples (tests/golden/),
invariants and independent numpy restatements. A dropped term, a flipped sign or direction, a
transposed index or a wrong tie-break in the oracle fails at least one of them.
"""
import itertools
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_golden(name):
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, v = line.split(":", 1)
            out[k.strip()] = v.split()
    return out


# ----------------------------------------------------------------------------- census (Sec. 2.1.1)
@pytest.mark.parametrize("cw,ch", [(5, 5), (9, 7), (3, 3)])
def test_census_raster_gradient_closed_form(cw, ch):
    # Intensities rise strictly in raster order, so exactly the neighbours that precede the
    # centre in row-major order are darker: the low B/2 bits are set, the high B/2 are clear.
    img = (1 + np.arange(cw * ch)).reshape(ch, cw).astype(np.uint8)
    ct = oracle.census(img, cw, ch)
    B = cw * ch - 1
    assert int(ct[ch // 2, cw // 2]) == (1 << (B // 2)) - 1
    # reversed gradient: the complement within B bits
    ct2 = oracle.census(img[::-1, ::-1].copy(), cw, ch)
    assert int(ct2[ch // 2, cw // 2]) == ((1 << B) - 1) ^ ((1 << (B // 2)) - 1)


@pytest.mark.parametrize("cw,ch", [(5, 5), (9, 7)])
def test_census_zero_margin_at_corner(cw, ch):
    # Constant image c > 0: inside neighbours are equal (bit 0); outside neighbours read 0 < c
    # (bit 1). At the top-left corner (rx+1)(ry+1) window cells lie inside the image.
    img = np.full((ch + 2, cw + 2), 77, np.uint8)
    ct = oracle.census(img, cw, ch)
    rx, ry = cw // 2, ch // 2
    assert bin(int(ct[0, 0])).count("1") == cw * ch - (rx + 1) * (ry + 1)
    # the bit of the neighbour at offset (-1, -1) (outside) is set, the one at (+1, +1) is not
    k_out = (ry - 1) * cw + (rx - 1)
    k_in = (ry + 1) * cw + (rx + 1) - 1  # minus one: the centre is skipped
    assert (int(ct[0, 0]) >> k_out) & 1 == 1
    assert (int(ct[0, 0]) >> k_in) & 1 == 0
    assert int(oracle.census(np.zeros((9, 9), np.uint8), cw, ch).max()) == 0


def test_census_invariant_under_monotone_map():
    # The census is non-parametric (Zabih & Woodfill): a strictly increasing f with f(0) = 0
    # leaves every descriptor unchanged, border pixels included (the margin stays 0).
    rng = np.random.default_rng(3)
    img = rng.integers(0, 81, (23, 31)).astype(np.uint8)
    f = lambda v: 2 * v + (v * v) // 128  # strictly increasing on 0..80, f(0) = 0, max 210
    img2 = f(img.astype(np.int64)).astype(np.uint8)
    for cw, ch in ((5, 5), (9, 7)):
        assert np.array_equal(oracle.census(img, cw, ch), oracle.census(img2, cw, ch))
    # ... but not under a map with f(0) != 0 at the border
    img3 = (img.astype(np.int64) + 10).astype(np.uint8)
    assert not np.array_equal(oracle.census(img, 5, 5), oracle.census(img3, 5, 5))
    # interior descriptors survive any strictly increasing map
    assert np.array_equal(oracle.census(img, 5, 5)[2:-2, 2:-2],
                          oracle.census(img3, 5, 5)[2:-2, 2:-2])


@pytest.mark.parametrize("cw,ch", [(5, 5), (9, 7)])
def test_census_bits_within_window(cw, ch):
    rng = np.random.default_rng(4)
    img = rng.integers(0, 256, (17, 19)).astype(np.uint8)
    ct = oracle.census(img, cw, ch)
    B = cw * ch - 1
    if B < 64:
        assert int(ct.max()) < (1 << B)
    # the centre pixel is the strict maximum of a 1-hot image: every in-image bit is 0 except
    # none; with the single bright pixel, all its (in-image) neighbours are darker
    one = np.zeros((ch, cw), np.uint8)
    one[ch // 2, cw // 2] = 9
    assert int(oracle.census(one, cw, ch)[ch // 2, cw // 2]) == (1 << B) - 1


# ------------------------------------------------------------------------- cost (Eq. image_matching)
def test_cost_zero_at_true_shift_and_outside_value():
    rng = np.random.default_rng(5)
    W, H, D, s = 40, 12, 16, 6
    L = rng.integers(0, 256, (H, W)).astype(np.uint8)
    R = rng.integers(0, 256, (H, W)).astype(np.uint8)
    R[:, :W - s] = L[:, s:]  # R(x) = L(x + s)  =>  L(x) = R(x - s)
    for cw, ch in ((5, 5), (9, 7)):
        rx, ry = cw // 2, ch // 2
        C = oracle.cost(oracle.census(L, cw, ch), oracle.census(R, cw, ch), D)
        inner = C[ry:H - ry, s + rx:W - rx, s]
        assert inner.size > 0 and int(inner.max()) == 0
        # Hamming distance of the descriptors, independently with numpy bit counting
        ctl, ctr = oracle.census(L, cw, ch), oracle.census(R, cw, ch)
        y, x, d = 3, 20, 9
        assert C[y, x, d] == bin(int(ctl[y, x]) ^ int(ctr[y, x - d])).count("1")
        # matching pixel left of the image: 0xFF
        for x in range(D):
            assert np.all(C[:, x, x + 1:] == 255)
            assert np.all(C[:, x, :x + 1] <= cw * ch - 1)


# ------------------------------------------------------------------------ SGM paths (Eq. sgm_path)
def _V(a, b, P1, P2):
    return 0 if a == b else (P1 if abs(a - b) == 1 else P2)


def _chain_energy_min(costs, d_end, P1, P2):
    """min over labelings l_0..l_k with l_k = d_end of sum C(p_i,l_i) + sum V(l_i, l_{i+1}):
    the energy the 1-D dynamic programme minimises exactly, by exhaustive enumeration."""
    k = len(costs)
    D = len(costs[0])
    best = None
    for labels in itertools.product(range(D), repeat=k - 1):
        lab = list(labels) + [d_end]
        e = sum(int(costs[i][lab[i]]) for i in range(k))
        e += sum(_V(lab[i], lab[i + 1], P1, P2) for i in range(k - 1))
        best = e if best is None else min(best, e)
    return best


@pytest.mark.parametrize("seed", range(4))
def test_path_equals_bruteforce_chain_energy(seed):
    # Literal Eq. (sgm_path): L_eq(p,d) = C(p,d) + min_d' (L_eq(p-r,d') + V(d,d')) is the minimal
    # chain energy of the path ending at p with label d. The normalised form subtracts
    # m = min_k L_eq(p-r,k) at every step, so L(p,d) = L_eq(p,d) - min_k L_eq(p-r,k).
    rng = np.random.default_rng(seed)
    W, H, D = 5, 4, 3
    cost_vol = rng.integers(0, 64, (H, W, D)).astype(np.uint8)
    cost_vol[rng.random((H, W, D)) < 0.15] = 255
    P1 = int(rng.integers(0, 20))
    P2 = int(rng.integers(P1, 60))
    for r in oracle.DIRECTIONS:
        Lr = oracle.path(cost_vol, r, P1, P2)
        for y in range(H):
            for x in range(W):
                chain = []
                cx, cy = x, y
                while 0 <= cx < W and 0 <= cy < H:
                    chain.append(cost_vol[cy, cx])
                    cx, cy = cx - r[0], cy - r[1]
                chain = chain[::-1]  # from the line's entry pixel to p
                eq_p = [_chain_energy_min(chain, d, P1, P2) for d in range(D)]
                if len(chain) == 1:
                    expect = eq_p
                else:
                    eq_q = [_chain_energy_min(chain[:-1], d, P1, P2) for d in range(D)]
                    expect = [e - min(eq_q) for e in eq_p]
                assert list(Lr[y, x]) == expect, (r, x, y)


@pytest.mark.parametrize("R", [4, 8])
def test_zero_penalties_reduce_to_cost_sum(R):
    # P1 = P2 = 0: min(L(q,d), L(q,d+-1), m) - m = 0, so every L_r = C and S = R * C.
    rng = np.random.default_rng(7)
    cost_vol = rng.integers(0, 256, (9, 11, 8)).astype(np.uint8)
    S = oracle.aggregate(cost_vol, R, 0, 0)
    assert np.array_equal(S, np.minimum(R * cost_vol.astype(np.int64), 65535))


def _steps_from_entry(W, H, r):
    """Number of pixels on the path of direction r from its entry pixel to p, inclusive."""
    n = np.zeros((H, W), np.int64)
    for y in range(H):
        for x in range(W):
            k, cx, cy = 0, x, y
            while 0 <= cx < W and 0 <= cy < H:
                k += 1
                cx, cy = cx - r[0], cy - r[1]
            n[y, x] = k
    return n


@pytest.mark.parametrize("R,P2", [(4, 400), (8, 400), (8, 16384)])
def test_aggregate_closed_form_and_saturation(R, P2):
    # Cost 0 at d = 0 and 255 elsewhere, P1 = P2: along every path L(p,0) = 0 and, for d >= 1,
    # L(p,d) = min(255 * n_r(p), 255 + P2) with n_r(p) the pixels walked from the entry.
    # S = min(65535, sum_r L_r): with P2 = 16384 the centre saturates (8 * 16639 > 65535).
    W, H, D = 80, 72, 4
    cost_vol = np.full((H, W, D), 255, np.uint8)
    cost_vol[:, :, 0] = 0
    S = oracle.aggregate(cost_vol, R, P2, P2)
    total = np.zeros((H, W), np.int64)
    for r in oracle.DIRECTIONS[:R]:
        total += np.minimum(255 * _steps_from_entry(W, H, r), 255 + P2)
    expect = np.minimum(total, 65535)
    assert np.all(S[:, :, 0] == 0)
    for d in range(1, D):
        assert np.array_equal(S[:, :, d].astype(np.int64), expect)
    if P2 == 16384:
        assert int(S[H // 2, W // 2, 1]) == 65535


# ------------------------------------------------------------------------------- WTA (Eq. wta)
def test_wta_map_reduce_worked_example():
    g = _read_golden("map_reduce_min.txt")
    costs = [int(v) for v in g["costs"]]
    disps = [int(v) for v in g["disparities"]]
    S = np.array(costs, np.uint16).reshape(1, 1, -1)
    # the oracle's 0-based disparity of the minimum equals the figure's 1-based label 05
    best = oracle.wta(S)[0, 0]
    assert disps[best] == int(g["step3"][0].split("@")[1])
    assert costs[best] == int(g["step3"][0].split("@")[0])
    # the figure's halving pairing (i with i + n/2), restated here, reproduces every step
    vals = list(zip(costs, disps))
    for step in ("step1", "step2", "step3"):
        n = len(vals) // 2
        vals = [min(vals[i], vals[i + n]) for i in range(n)]
        assert [f"{c}@{d}" for c, d in vals] == g[step]


def test_wta_tie_takes_smallest_disparity():
    S = np.array([[[9, 3, 7, 3, 3]]], np.uint16)
    assert oracle.wta(S)[0, 0] == 1
    rng = np.random.default_rng(8)
    S = rng.integers(0, 6, (7, 9, 16)).astype(np.uint16)  # many ties
    assert np.array_equal(oracle.wta(S), np.argmin(S, axis=2))


# --------------------------------------------------------------- right disparity (Eq. right_disp.)
def test_right_disparity_bruteforce():
    rng = np.random.default_rng(9)
    H, W, D = 6, 13, 8
    S = rng.integers(0, 20, (H, W, D)).astype(np.uint16)
    DR = oracle.right_disparity(S)
    for y in range(H):
        for x in range(W):
            cand = [S[y, x + d, d] for d in range(min(D, W - x))]
            assert DR[y, x] == int(np.argmin(cand))


# ------------------------------------------------------------------------ LR check (Eq. LR_check)
def test_lr_check_definition_cases():
    DL = np.array([[0, 1, 3, 2, 2, 0]], np.uint16)
    DR = np.array([[0, 1, 5, 0, 3, 1]], np.uint16)
    D, mask = oracle.lr_check(DL, DR, 1)
    # x=0: DR[0]=0 ok; x=1: DR[0]=0, |1-0|<=1 ok; x=2: 2-3<0 invalid;
    # x=3: DR[1]=1, |2-1|=1 ok; x=4: DR[2]=5, |2-5|=3 invalid; x=5: DR[5]=1, |0-1|=1 ok
    assert list(mask[0]) == [1, 1, 0, 1, 0, 1]
    assert list(D[0]) == [0, 1, 0xFFFF, 2, 0xFFFF, 0]
    D0, mask0 = oracle.lr_check(DL, DR, 0)
    assert list(mask0[0]) == [1, 0, 0, 0, 0, 0]


# ---------------------------------------------------------------------------- median (Sec. 2.1.3)
def test_median_sorting_network_worked_example():
    g = _read_golden("sorting_network_median.txt")
    vals = [int(v) for v in g["input"]]
    img = np.array(vals, np.uint16).reshape(3, 3)
    out = oracle.median3x3(img)
    assert out[1, 1] == int(g["median"][0])
    assert sorted(vals) == [int(v) for v in g["sorted"]]
    # a bubble-sort network of five passes, restated here: each pass carries the largest
    # remaining value down to the lowest open wire (the smaller value stays on the upper wire),
    # so after the fifth pass wires 8..4 hold the five largest values in order and wire 4 is
    # the median
    w = list(vals)
    for p in range(5):
        for i in range(0, 8 - p):
            if w[i] > w[i + 1]:
                w[i], w[i + 1] = w[i + 1], w[i]
    assert w[4:] == [int(v) for v in g["sorted"]][4:]
    assert w[4] == int(g["median"][0])


def test_median_borders_and_invalid():
    rng = np.random.default_rng(10)
    Din = rng.integers(0, 50, (8, 9)).astype(np.uint16)
    Din[rng.random(Din.shape) < 0.3] = 0xFFFF
    out = oracle.median3x3(Din)
    P = np.pad(Din.astype(np.int64), 1, constant_values=0xFFFF)
    for y in range(8):
        for x in range(9):
            if Din[y, x] == 0xFFFF:
                assert out[y, x] == 0xFFFF
            else:
                assert out[y, x] == np.sort(P[y:y + 3, x:x + 3].ravel())[4]


# ----------------------------------------------------------------------------------- end to end
@pytest.mark.parametrize("cw,ch,R", [(5, 5, 4), (9, 7, 8)])
def test_constant_shift_recovered(cw, ch, R):
    rng = np.random.default_rng(11)
    W, H, D, s = 96, 40, 32, 7
    from paper_2106_07927_gb300 import scenes
    L = scenes._to_u8(scenes._blur(rng.random((H, W)), 1.0))
    R_img = rng.integers(0, 256, (H, W)).astype(np.uint8)
    R_img[:, :W - s] = L[:, s:]
    disp, dbg = oracle.sgm(L, R_img, D, cw, ch, 10, 120, R, oracle.FLAG_LR_CHECK, debug=True)
    rx = cw // 2
    inner = dbg["dl"][:, s + rx:W - D]
    assert np.all(inner == s)
    # the left-right check keeps the interior. Near the left border the approximate D^R of
    # Eq. (right_disparity) is biased (paths entering there have summed fewer pixels), so the
    # check is asserted from x = 3 s on.
    assert np.all(disp[:, 3 * s:W - D] == s)


def test_occluded_band_is_invalidated():
    # Background at d = 4, a foreground box at d = 20: the background strip just left of the
    # box is hidden in the right image (occlusion), so the LR check must drop most of it while
    # keeping nearly all visible background pixels.
    rng = np.random.default_rng(12)
    W, H, D = 160, 48, 32
    from paper_2106_07927_gb300 import scenes
    L = scenes._to_u8(scenes._blur(rng.random((H, W)), 1.0))
    disp = np.full((H, W), 4, np.int32)
    x1, x2 = 90, 130
    disp[:, x1:x2] = 20
    R_img = scenes.forward_warp(rng, L, disp)
    out, dbg = oracle.sgm(L, R_img, D, 9, 7, 10, 120, 8, oracle.FLAG_LR_CHECK, debug=True)
    occl = dbg["mask"][8:H - 8, x1 - 14:x1 - 2]
    vis = dbg["mask"][8:H - 8, 40:x1 - 20]
    assert occl.mean() < 0.2
    assert vis.mean() > 0.95
    assert np.all(out[8:H - 8, 40:x1 - 20][vis.astype(bool)] == 4)


# ------------------------------------------------------------------ sub-pixel refinement (Sec. 2.1.3)
def _parabola_volume(rng, H, W, D):
    """S(p, d) = A (d - d*)^2 + B with d* = k + j/4: integral at integer d when 16 | A, so the
    parabola through any three samples is the generating one and its minimum lies at d*."""
    k = rng.integers(1, D - 1, size=(H, W))
    j = rng.integers(-1, 2, size=(H, W))          # d* - k in {-1/4, 0, 1/4}
    A = 16 * rng.integers(1, 4, size=(H, W))
    B = rng.integers(0, 200, size=(H, W))
    d = np.arange(D)[None, None, :]
    dstar4 = 4 * k + j                             # 4 d*
    S4 = A[..., None] * (4 * d - dstar4[..., None]) ** 2  # 16 A (d - d*)^2
    S = S4 // 16 + B[..., None]
    assert np.all(S4 % 16 == 0) and S.max() < 65535
    return S.astype(np.uint16), dstar4 / 4.0


def test_subpixel_recovers_parabola_vertex():
    rng = np.random.default_rng(11)
    S, dstar = _parabola_volume(rng, 6, 9, 32)
    DL = oracle.wta(S)
    assert np.array_equal(DL, np.round(dstar).astype(np.uint16))
    ref = oracle.subpixel(S, DL)
    assert np.array_equal(ref, dstar)  # exact: a sign or index error moves it by 1/2


def test_subpixel_half_pixel_tie_and_edges():
    D = 8
    S = np.full((1, 5, D), 500, np.uint16)
    S[0, 0, :] = [9, 5, 5, 9, 20, 30, 40, 50]       # tie d = 1, 2: WTA takes 1, vertex at 1.5
    S[0, 1, :] = [3, 8, 9, 9, 9, 9, 9, 9]           # D^L = 0: stays integral
    S[0, 2, :] = [9, 9, 9, 9, 9, 9, 8, 3]           # D^L = D - 1: stays integral
    S[0, 3, :] = [65535, 0, 65535, 1, 1, 1, 1, 1]   # saturated neighbours: symmetric, delta 0
    S[0, 4, :] = [100, 10, 40, 60, 70, 80, 90, 95]  # a = 90, b = 30: delta = 60 / 240
    DL = oracle.wta(S)
    ref = oracle.subpixel(S, DL)
    assert list(DL[0]) == [1, 0, 7, 1, 1]
    assert list(ref[0]) == [1.5, 0.0, 7.0, 1.0, 1.25]


def test_subpixel_invariant_under_offset_and_scale():
    rng = np.random.default_rng(5)
    S = rng.integers(0, 3000, size=(4, 7, 24)).astype(np.int64)
    DL = oracle.wta(S.astype(np.uint16))
    base = oracle.subpixel(S.astype(np.uint16), DL)
    for a, b in ((1, 77), (3, 0), (5, 1000)):
        T = (a * S + b).astype(np.uint16)
        assert np.array_equal(oracle.wta(T), DL)
        assert np.allclose(oracle.subpixel(T, DL), base, rtol=0, atol=1e-12)
    assert np.all(np.abs(base - DL) <= 0.5)


def test_median_f64_matches_integer_median_and_sort():
    rng = np.random.default_rng(3)
    for _ in range(4):
        H, W = rng.integers(1, 9, size=2)
        Din = rng.integers(0, 40, size=(H, W)).astype(np.uint16)
        Din[rng.random((H, W)) < 0.3] = oracle.INVALID
        F = np.where(Din == oracle.INVALID, np.inf, Din.astype(np.float64))
        want = oracle.median3x3(Din)
        got = oracle.median3x3_f64(F)
        assert np.array_equal(np.where(want == oracle.INVALID, np.inf, want), got)
        # non-integral values: element [4] of the sorted 9-neighbourhood (numpy sort)
        G = np.where(np.isinf(F), np.inf, F + rng.random((H, W)) * 0.9)
        pad = np.pad(G, 1, constant_values=np.inf)
        got = oracle.median3x3_f64(G)
        for y in range(H):
            for x in range(W):
                want_v = np.inf if np.isinf(G[y, x]) else np.sort(pad[y:y + 3, x:x + 3].ravel())[4]
                assert got[y, x] == want_v


@pytest.mark.parametrize("flags", [0, 1, 3])
def test_sgm_subpixel_within_half_pixel_of_integer_pipeline(flags):
    from paper_2106_07927_gb300 import scenes
    L, R, _, prm = scenes.single_pair("320x240_d64_ct5x5_r4", 1)
    L, R = L[:60, :120], R[:60, :120]
    D = prm["max_disp"]
    integer = oracle.sgm(L, R, D, 5, 5, 10, 120, 4, flags)
    sub, ref = oracle.sgm_subpixel(L, R, D, 5, 5, 10, 120, 4, flags)
    inv = integer == oracle.INVALID
    assert np.array_equal(inv, np.isinf(sub))  # validity is decided on the integer maps
    # every refined value lies within 1/2 of its integer one; the median is 1-Lipschitz
    assert np.all(np.abs(sub[~inv] - integer[~inv]) <= 0.5)
    _, dbg = oracle.sgm(L, R, D, 5, 5, 10, 120, 4, flags, debug=True)
    assert np.all(np.abs(ref - dbg["dl"]) <= 0.5)
    assert np.array_equal(ref, oracle.subpixel(dbg["agg"], dbg["dl"]))


# ------------------------------------------------------- exact consistency check (Sec. 3.2.3)
@pytest.mark.parametrize("cw,ch,R,seed", [(5, 5, 4, 0), (9, 7, 8, 1), (9, 7, 4, 2)])
def test_exact_right_disparity_equals_swap_and_flip(cw, ch, R, seed):
    # The paper builds the exact D^R by swapping the images, mirroring both and matching again.
    # The oracle computes it from the right-reference cost directly; the two must agree.
    rng = np.random.default_rng(40 + seed)
    H, W, D = 23, 57, 32
    L = rng.integers(0, 256, (H, W)).astype(np.uint8)
    R_img = rng.integers(0, 256, (H, W)).astype(np.uint8)
    flags = oracle.FLAG_LR_CHECK | oracle.FLAG_EXACT_CC
    _, dbg = oracle.sgm(L, R_img, D, cw, ch, 10, 120, R, flags, debug=True)
    dflip = oracle.sgm(R_img[:, ::-1], L[:, ::-1], D, cw, ch, 10, 120, R, 0)
    assert np.array_equal(dbg["dr"], dflip[:, ::-1])
    # and the cost it starts from is the definition: CT_R(x) against CT_L(x + d), 255 outside
    ctl, ctr = oracle.census(L, cw, ch), oracle.census(R_img, cw, ch)
    cr = oracle.cost_right(ctl, ctr, D)
    x, d = 11, 5
    assert cr[3, x, d] == bin(int(ctr[3, x]) ^ int(ctl[3, x + d])).count("1")
    assert np.all(cr[:, W - 1, 1:] == 255) and np.all(cr[:, W - D:, :][:, :, -1][:, 1:] == 255)


@pytest.mark.parametrize("cw,ch,R", [(5, 5, 4), (9, 7, 8)])
def test_exact_check_keeps_constant_shift_to_the_border(cw, ch, R):
    # R(x) = L(x + s): the exact D^R is s wherever x + s stays inside and the window sees the
    # same texture, so the check keeps D^L = s from x = s + rx on, where the approximate D^R of
    # Eq. (right_disparity) is still biased (see the test above it)
    rng = np.random.default_rng(11)
    W, H, D, s = 96, 40, 32, 7
    from paper_2106_07927_gb300 import scenes
    L = scenes._to_u8(scenes._blur(rng.random((H, W)), 1.0))
    R_img = rng.integers(0, 256, (H, W)).astype(np.uint8)
    R_img[:, :W - s] = L[:, s:]
    flags = oracle.FLAG_LR_CHECK | oracle.FLAG_EXACT_CC
    disp, dbg = oracle.sgm(L, R_img, D, cw, ch, 10, 120, R, flags, debug=True)
    rx = cw // 2
    assert np.all(dbg["dr"][:, rx:W - D] == s)
    assert np.all(disp[:, s + rx:W - D] == s)


# -------------------------------------------- NCC matching cost (Sec. 2.1.1, Sec. 2.2.1 "NCC")
def _ncc_expected(L, R, x, y, d, n):
    """255 - round(255 max(0, Phi)) with Phi from numpy's corrcoef on zero-padded patches;
    None when 255 Phi lies within 1e-3 of a rounding boundary (fp32 may go either way)."""
    r = n // 2
    Lp = np.pad(L.astype(np.float64), r)
    Rp = np.pad(R.astype(np.float64), r)
    a = Lp[y:y + n, x:x + n].ravel()
    b = Rp[y:y + n, x - d:x - d + n].ravel()
    if a.std() == 0 or b.std() == 0:
        return 255
    phi = np.corrcoef(a, b)[0, 1]
    v = 255 * max(0.0, phi)
    if abs(v - np.floor(v) - 0.5) < 1e-3:
        return None
    return 255 - int(np.floor(v + 0.5))


@pytest.mark.parametrize("n", [5, 9])
def test_ncc_cost_matches_numpy_corrcoef(n):
    rng = np.random.default_rng(70 + n)
    H, W, D = 17, 29, 16
    L = rng.integers(0, 256, (H, W)).astype(np.uint8)
    R = np.clip(L.astype(int) + rng.integers(-40, 41, (H, W)), 0, 255).astype(np.uint8)
    R[5:9, 3:12] = 77  # a constant area: zero variance somewhere
    C = oracle.ncc_cost(L, R, D, n)
    checked = 0
    for y in range(H):
        for x in range(W):
            for d in range(D):
                if x - d < 0:
                    assert C[y, x, d] == 255
                    continue
                want = _ncc_expected(L, R, x, y, d, n)
                if want is not None:
                    assert C[y, x, d] == want, (y, x, d)
                    checked += 1
    assert checked > 0.95 * H * W * D / 2


def _k_decimal(cov, va, vb):
    """round(255 max(0, cov / sqrt(va vb))), ties to even, in 80-digit decimal arithmetic: an
    independent statement of the NCC cost's scaling (exact where sqrt(va vb) is an integer, and
    80 digits resolve every other case)."""
    import decimal
    if cov <= 0 or va <= 0 or vb <= 0:
        return 0
    ctx = decimal.Context(prec=80, rounding=decimal.ROUND_HALF_EVEN)
    x = ctx.divide(ctx.multiply(decimal.Decimal(255), decimal.Decimal(cov)),
                   ctx.sqrt(decimal.Decimal(va) * decimal.Decimal(vb)))
    return int(x.quantize(decimal.Decimal(1), rounding=decimal.ROUND_HALF_EVEN, context=ctx))


def test_ncc_round_exact_ties_go_to_even():
    # Phi = (2m - 1) / 510 exactly puts 255 Phi on m - 1/2: the even one of m - 1 and m wins
    for m in range(1, 256):
        for s, t in ((1, 1), (7, 1), (3, 5), (101, 2)):
            va, vb, cov = 510 * s * t * t, 510 * s, (2 * m - 1) * s * t
            want = m - 1 if (m - 1) % 2 == 0 else m
            assert oracle.ncc_round(cov, va, vb) == want == _k_decimal(cov, va, vb), (m, s, t)
    # the end points and the truncation
    assert oracle.ncc_round(1, 510 * 510, 1) == 0 and _k_decimal(1, 510 * 510, 1) == 0  # 1/2
    assert oracle.ncc_round(3, 510 * 510, 1) == 2 and _k_decimal(3, 510 * 510, 1) == 2  # 3/2
    assert oracle.ncc_round(0, 5, 7) == 0 and oracle.ncc_round(-9, 5, 7) == 0
    assert oracle.ncc_round(5, 0, 7) == 0 and oracle.ncc_round(5, 7, 0) == 0
    assert oracle.ncc_round(12345, 12345, 12345) == 255


def test_ncc_round_near_ties_against_decimal():
    # (cov, vA, vB) in the ranges of 9 x 9 patches (< 2^27) with 255 Phi within about 1e-9 of
    # k + 1/2, on both sides
    rng = np.random.default_rng(5)
    checked = 0
    for _ in range(3000):
        va, vb = (int(v) for v in rng.integers(1, 1 << 27, 2))
        k = int(rng.integers(0, 255))
        cov = int(round((k + 0.5) * (va * vb) ** 0.5 / 255))
        for c in (cov - 1, cov, cov + 1):
            if 0 < c and c * c <= va * vb:
                assert oracle.ncc_round(c, va, vb) == _k_decimal(c, va, vb), (c, va, vb)
                checked += 1
    assert checked > 5000


def _near_tie_patch_pairs(n, seed, tol=1e-6, want=8):
    """Seeded n x n patch pairs (a, b) whose 255 Phi lies within tol of some k + 1/2: random pairs,
    with one pixel of b swept over 0..255, screened in float64 (exact enough to select)."""
    rng = np.random.default_rng(seed)
    N = n * n
    v = np.arange(256)
    found = []
    for _ in range(200):
        K = 4096
        a = rng.integers(0, 256, (K, N)).astype(np.int64)
        b = np.clip(a + rng.integers(-60, 61, (K, N)), 0, 255).astype(np.int64)
        sA, sAA = a.sum(1), (a * a).sum(1)
        sB = b[:, 1:].sum(1)[:, None] + v
        sBB = (b[:, 1:] ** 2).sum(1)[:, None] + v * v
        sAB = (a[:, 1:] * b[:, 1:]).sum(1)[:, None] + a[:, :1] * v
        vA = (N * sAA - sA * sA)[:, None]
        vB = N * sBB - sB * sB
        cov = N * sAB - sA[:, None] * sB
        ok = (cov > 0) & (vB > 0) & (vA > 0)
        with np.errstate(divide="ignore", invalid="ignore"):
            x = 255.0 * cov / np.sqrt(vA.astype(np.float64) * vB)
        dist = np.abs(x - np.floor(x) - 0.5)
        for i, j in np.argwhere(ok & (dist < tol)):
            bb = b[i].copy()
            bb[0] = j
            found.append((a[i].copy(), bb))
        if len(found) >= want:
            break
    return found[:want]


@pytest.mark.parametrize("n", [5, 9])
def test_ncc_cost_near_tie_patches_against_exact_rationals(n):
    """Patch pairs within 1e-6 of a rounding boundary: the oracle's cost equals 255 - k with k
    from exact arithmetic; the two fp32 evaluation orders ((cov iA) iB) 255 and (cov iA)(255 iB)
    disagree on some of them and each misses k on some, so this pin separates the integer
    definition from either."""
    pairs = _near_tie_patch_pairs(n, 600 + n, want=24)
    assert len(pairs) >= 20
    r, N = n // 2, n * n
    f32 = np.float32
    disagree = miss0 = miss1 = 0
    for a, b in pairs:
        sA, sB = int(a.sum()), int(b.sum())
        va = N * int((a * a).sum()) - sA * sA
        vb = N * int((b * b).sum()) - sB * sB
        cov = N * int((a * b).sum()) - sA * sB
        k = _k_decimal(cov, va, vb)
        L = a.reshape(n, n).astype(np.uint8)
        R = b.reshape(n, n).astype(np.uint8)
        assert oracle.ncc_cost(L, R, 1, n)[r, r, 0] == 255 - k
        ia = f32(1) / np.sqrt(f32(va))
        ib = f32(1) / np.sqrt(f32(vb))
        q0 = ((f32(cov) * ia) * ib) * f32(255)
        q1 = (f32(cov) * ia) * (f32(255) * ib)
        disagree += int(np.rint(q0) != np.rint(q1))
        miss0 += int(np.rint(q0) != k)
        miss1 += int(np.rint(q1) != k)
    assert disagree >= 1 and miss0 >= 1 and miss1 >= 1


@pytest.mark.parametrize("n", [5, 9])
def test_ncc_cost_special_cases(n):
    rng = np.random.default_rng(80 + n)
    H, W, D, s = 24, 60, 16, 6
    r = n // 2
    L = rng.integers(0, 200, (H, W)).astype(np.uint8)
    inner = (slice(r, H - r), slice(s + r, W - r))
    # right = left shifted by s: Phi = 1 at d = s away from the borders
    R = np.zeros_like(L)
    R[:, :W - s] = L[:, s:]
    C = oracle.ncc_cost(L, R, D, n)
    assert np.all(C[:, :, s][inner][:, :W - s - 2 * r - s] == 0)
    # a brightness offset keeps Phi = 1; an inverted image gives Phi = -1, cost 255
    C = oracle.ncc_cost(L, (L + 40).astype(np.uint8), D, n)
    assert np.all(C[r:H - r, r:W - r, 0] == 0)
    C = oracle.ncc_cost(L, (255 - L).astype(np.uint8), D, n)
    assert np.all(C[r:H - r, r:W - r, 0] == 255)
    # a constant reference patch (window inside the image) has no variance: cost 255
    C = oracle.ncc_cost(np.full((H, W), 9, np.uint8), L, D, n)
    assert np.all(C[r:H - r, r:W - r] == 255)


@pytest.mark.parametrize("n,R", [(5, 4), (9, 8)])
def test_ncc_exact_right_equals_swap_and_flip(n, R):
    rng = np.random.default_rng(90 + n)
    H, W, D = 19, 41, 16
    L = rng.integers(0, 256, (H, W)).astype(np.uint8)
    R_img = rng.integers(0, 256, (H, W)).astype(np.uint8)
    flags = oracle.FLAG_LR_CHECK | oracle.FLAG_EXACT_CC | oracle.FLAG_NCC
    _, dbg = oracle.sgm(L, R_img, D, n, n, 90, 880, R, flags, debug=True)
    dflip = oracle.sgm(R_img[:, ::-1], L[:, ::-1], D, n, n, 90, 880, R, oracle.FLAG_NCC)
    assert np.array_equal(dbg["dr"], dflip[:, ::-1])
    assert np.array_equal(dbg["cost"], oracle.ncc_cost(L, R_img, D, n))


def test_ncc_pipeline_recovers_constant_shift():
    rng = np.random.default_rng(13)
    W, H, D, s = 96, 40, 32, 7
    from paper_2106_07927_gb300 import scenes
    L = scenes._to_u8(scenes._blur(rng.random((H, W)), 1.0))
    R_img = rng.integers(0, 256, (H, W)).astype(np.uint8)
    R_img[:, :W - s] = L[:, s:]
    _, dbg = oracle.sgm(L, R_img, D, 5, 5, 90, 880, 8, oracle.FLAG_NCC, debug=True)
    assert np.all(dbg["dl"][:, s + 2:W - D] == s)


# ------------------------------------------------------- rectification (Sec. 2.1.1, resampling)
def test_rectify_identity_shift_and_half_pixel():
    rng = np.random.default_rng(21)
    raw = rng.integers(0, 256, (13, 17)).astype(np.uint8)
    y, x = np.mgrid[0:13, 0:17].astype(np.float32)
    assert np.array_equal(oracle.rectify(raw, x, y), raw)
    out = oracle.rectify(raw, x + 3, y - 2)  # integer shift, zeros from outside
    want = np.zeros_like(raw)
    want[2:, :14] = raw[:11, 3:]
    assert np.array_equal(out, want)
    out = oracle.rectify(raw, x + 0.5, y)  # half-pixel: (a + b + 1) >> 1
    nxt = np.concatenate([raw[:, 1:], np.zeros((13, 1), np.uint8)], axis=1).astype(int)
    assert np.array_equal(out, (raw.astype(int) + nxt + 1) >> 1)
    # non-finite or huge coordinates read 0
    x2 = x.copy()
    x2[0, 0], x2[0, 1], x2[0, 2] = np.nan, np.inf, 1e9
    assert list(oracle.rectify(raw, x2, y)[0, :3]) == [0, 0, 0]


def test_rectify_matches_scipy_bilinear_on_the_grid():
    ndimage = pytest.importorskip("scipy.ndimage")
    from paper_2106_07927_gb300 import scenes
    rng = np.random.default_rng(22)
    H, W = 40, 64
    raw = rng.integers(0, 256, (H + 6, W + 4)).astype(np.uint8)
    mapx, mapy = scenes.rectification_maps(3, W, H, W + 4, H + 6, strength=3.0)
    mapx[5, 5], mapy[7, 9] = -0.7, H + 5.6  # samples straddling the border
    out = oracle.rectify(raw, mapx, mapy)
    # the 1/32 grid the definition puts coordinates on, then scipy's exact bilinear value
    gx = np.rint(mapx.astype(np.float32) * np.float32(32)).astype(np.float64) / 32
    gy = np.rint(mapy.astype(np.float32) * np.float32(32)).astype(np.float64) / 32
    ref = ndimage.map_coordinates(raw.astype(np.float64), [gy, gx], order=1,
                                  mode="grid-constant", cval=0.0)
    assert np.array_equal(out, np.floor(ref + 0.5).astype(np.uint8))


# ------------------------------------------------- sums at single pixels (sampled full-size checks)
@pytest.mark.parametrize("cw,ch,R,flags,P2", [(5, 5, 4, 0, 120), (9, 7, 8, 0, 120),
                                              (5, 5, 8, 8, 880), (9, 7, 8, 0, 16384)])
def test_s_at_equals_full_aggregation(cw, ch, R, flags, P2):
    rng = np.random.default_rng(33)
    H, W, D = 13, 29, 32
    L = rng.integers(0, 256, (H, W)).astype(np.uint8)
    Rm = rng.integers(0, 256, (H, W)).astype(np.uint8)
    _, dbg = oracle.sgm(L, Rm, D, cw, ch, 10, P2, R, flags, debug=True)
    for y in range(H):
        for x in range(W):
            assert np.array_equal(oracle.s_at(L, Rm, D, cw, ch, 10, P2, R, flags, x, y),
                                  dbg["agg"][y, x]), (x, y)
