"""GPU path vs the CPU oracle, bit-exact on every intermediate (cost, aggregated volume, D^L,
D^R, LR mask) and on the final map. All arithmetic of the method is integer, so the bar is
equality, not a tolerance."""
import itertools

import numpy as np
import pytest

import oracle
from paper_2106_07927_gb300 import binding, scenes

pytestmark = pytest.mark.gpu

KEYS = ("cost", "agg", "dl", "dr", "mask")


def _gpu(left, right, prm, in_pad=0, out_pad=0, tuning=None):
    import torch
    H, W = left.shape
    st = binding.Stereo(prm)
    if tuning is not None:
        binding.res2tac_set_tuning(st.handle, tuning)
    Lb = torch.zeros((H, W + in_pad), dtype=torch.uint8, device="cuda")
    Rb = torch.zeros((H, W + in_pad), dtype=torch.uint8, device="cuda")
    Lb[:, :W] = torch.from_numpy(left).cuda()
    Rb[:, :W] = torch.from_numpy(right).cuda()
    outb = torch.full((H, W + out_pad), 0x1234, dtype=torch.int16, device="cuda")
    binding.res2tac_compute(st.handle, Lb.data_ptr(), Rb.data_ptr(), W + in_pad, outb.data_ptr(),
                            2 * (W + out_pad), torch.cuda.current_stream().cuda_stream)
    dbg = st.debug_outputs()
    torch.cuda.synchronize()
    out = binding.u16(outb)
    if out_pad:
        assert np.all(out[:, W:] == 0x1234), "wrote outside the row"
    got = {"cost": dbg["cost"].cpu().numpy(), "agg": binding.u16(dbg["agg"]),
           "dl": binding.u16(dbg["dl"]), "dr": binding.u16(dbg["dr"]),
           "mask": dbg["mask"].cpu().numpy()}
    st.close()
    return out[:, :W], got


def _oracle(left, right, prm):
    return oracle.sgm(left, right, prm["max_disp"], prm["census_w"], prm["census_h"], prm["p1"],
                      prm["p2"], prm["num_paths"], prm["flags"], prm["lr_threshold"], debug=True)


def _assert_same(left, right, prm, **kw):
    out, got = _gpu(left, right, prm, **kw)
    ref, rdbg = _oracle(left, right, prm)
    for k in KEYS:
        if not np.array_equal(got[k], rdbg[k]):
            bad = np.argwhere(got[k] != rdbg[k])
            raise AssertionError(f"{k}: {len(bad)} mismatches, first at {bad[0].tolist()}: "
                                 f"gpu {got[k][tuple(bad[0])]} oracle {rdbg[k][tuple(bad[0])]}")
    assert np.array_equal(out, ref), "final map"
    return out, ref


@pytest.mark.parametrize("name", list(scenes.SINGLE))
def test_single_pair_workloads_full_size(name):
    left, right, _, prm = scenes.single_pair(name, 0)
    _assert_same(left, right, prm)


@pytest.mark.parametrize("seed", range(12))
def test_tiny_random_shapes(seed):
    rng = np.random.default_rng(100 + seed)
    W = int(rng.integers(1, 70))
    H = int(rng.integers(1, 40))
    D = int(rng.choice([16, 32, 48, 64, 80, 128, 144, 256]))
    cw, ch = ((5, 5), (9, 7))[seed % 2]
    R = (4, 8)[(seed // 2) % 2]
    flags = seed % 4
    left = rng.integers(0, 256, (H, W)).astype(np.uint8)
    right = rng.integers(0, 256, (H, W)).astype(np.uint8)
    P1 = int(rng.integers(0, 30))
    P2 = int(rng.integers(P1, 300))
    prm = scenes.params(W, H, D, cw, ch, P1, P2, R, flags, int(rng.integers(0, 3)))
    _assert_same(left, right, prm)


@pytest.mark.parametrize("W,H,D", [(200, 3, 64), (3, 150, 32), (97, 61, 128), (257, 33, 256)])
def test_ragged_tiles(W, H, D):
    left, right, _ = scenes.make_scene("road", W + H, W, H, D)
    prm = scenes.params(W, H, D, 9, 7, 10, 120, 8, 3)
    _assert_same(left, right, prm)


def test_wide_sums_saturate_exactly():
    # P2 = 16384 with 8 paths: sums can exceed 65535, so the library keeps uint32 sums and
    # saturates them; the oracle saturates the exact sum.
    # Near the left border, large d cost 255 at every step of the vertical paths and of the paths
    # arriving from the right, so their L reach 255 + P2 and the sum passes 65535.
    rng = np.random.default_rng(5)
    W, H, D = 300, 200, 128
    left = rng.integers(0, 256, (H, W)).astype(np.uint8)
    right = rng.integers(0, 256, (H, W)).astype(np.uint8)
    prm = scenes.params(W, H, D, 5, 5, 100, 16384, 8, 3)
    ref, rdbg = _oracle(left, right, prm)
    assert (rdbg["agg"] == 65535).any(), "test input must reach saturation"
    _assert_same(left, right, prm)


def test_padded_pitches():
    left, right, _ = scenes.make_scene("nadir", 3, 130, 70, 64)
    prm = scenes.params(130, 70, 64, 9, 7, 8, 96, 8, 3)
    _assert_same(left, right, prm, in_pad=14, out_pad=6)


def test_every_tuning_is_bit_identical():
    left, right, _ = scenes.make_scene("road", 11, 300, 120, 128)
    prm = scenes.params(300, 120, 128, 9, 7, 10, 120, 8, 3)
    ref, rdbg = _oracle(left, right, prm)
    n = 0
    for dpl, warps, chunk, sdpl, mode, cpl in itertools.product((4, 8), (1, 4, 8), (64, 256),
                                                                (8, 16, 32), (1, 2), (1, 2)):
        t = binding.res2tac_tuning(dpl, warps, chunk, sdpl, mode, cpl)
        out, got = _gpu(left, right, prm, tuning=t)
        assert np.array_equal(out, ref), (dpl, warps, chunk, sdpl, mode, cpl)
        assert np.array_equal(got["agg"], rdbg["agg"])
        n += 1
    assert n == 144


# The cost volume on the tensor cores (tuning cost_mode 2): the same integers as the
# population counts, on shapes with one and several tiles per row, a ragged last tile, images
# narrower than a tile, padded pitches, wide sums and the exact check; 5 x 5 and D = 256 fall back
# to the population-count kernel.
TC = dict(cost_mode=2)


@pytest.mark.parametrize("W,H,D,cw,ch,p2,flags,pads", [
    (1242, 60, 128, 9, 7, 120, 3, (0, 0)),
    (300, 40, 64, 9, 7, 120, 3, (13, 3)),
    (1, 1, 64, 9, 7, 120, 0, (0, 0)),
    (5, 3, 128, 9, 7, 120, 3, (0, 0)),
    (127, 17, 128, 9, 7, 120, 2, (1, 1)),
    (257, 33, 128, 9, 7, 16384, 3, (0, 0)),
    (200, 30, 64, 9, 7, 120, 3 | 4, (0, 0)),  # exact consistency check
    (97, 21, 256, 9, 7, 120, 3, (0, 0)),
    (130, 20, 128, 5, 5, 120, 3, (0, 0)),
])
def test_tensor_core_cost_is_bit_exact(W, H, D, cw, ch, p2, flags, pads):
    left, right, _ = scenes.make_scene("road", W + 7 * H, W, H, D)
    prm = scenes.params(W, H, D, cw, ch, 10, p2, 8, flags)
    t = binding.res2tac_tuning(cost_mode=2)
    _assert_same(left, right, prm, tuning=t, in_pad=pads[0], out_pad=pads[1])


# The row kernel recomputing its costs from the census descriptors (tuning row_cost 2): every
# D it covers (agg_dpl 2, 4, 8 with 32 lanes), images narrower than its 8-step prefetch, both
# census windows, wide sums, the exact check (its flipped pass recomputes from the flipped
# pair's descriptors) and padded pitches; other settings and the NCC cost read the volume.
@pytest.mark.parametrize("W,H,D,dpl,cw,ch,p2,flags", [
    (300, 40, 128, 4, 9, 7, 120, 3),
    (257, 21, 64, 2, 9, 7, 120, 3),
    (97, 13, 256, 8, 9, 7, 120, 3),
    (5, 9, 64, 2, 9, 7, 120, 3),
    (1, 3, 128, 4, 9, 7, 120, 0),
    (200, 30, 128, 4, 5, 5, 120, 3 | 4),
    (150, 40, 128, 4, 5, 5, 16384, 3),
    (130, 20, 128, 8, 9, 7, 120, 3),
])
def test_row_recompute_is_bit_exact(W, H, D, dpl, cw, ch, p2, flags):
    left, right, _ = scenes.make_scene("road", W + 3 * H, W, H, D)
    prm = scenes.params(W, H, D, cw, ch, 10, p2, 8, flags)
    t = binding.res2tac_tuning(agg_dpl=dpl, row_mode=2, row_cost=2)
    _assert_same(left, right, prm, tuning=t, in_pad=3, out_pad=1)


def test_tensor_core_cost_setting_and_autotune():
    import torch
    left, right, _ = scenes.make_scene("road", 5, 160, 48, 64)
    prm = scenes.params(160, 48, 64, 9, 7, 10, 120, 8, 3)
    st = binding.Stereo(prm)
    assert binding.res2tac_get_tuning(st.handle).cost_mode == 1  # population counts by default
    assert binding.res2tac_get_tuning(st.handle).row_cost == 1  # the row kernel reads the volume
    with pytest.raises(binding.Res2tacError):
        binding.res2tac_set_tuning(st.handle, binding.res2tac_tuning(cost_mode=3))
    with pytest.raises(binding.Res2tacError):
        binding.res2tac_set_tuning(st.handle, binding.res2tac_tuning(row_cost=3))
    L, R = torch.from_numpy(left).cuda(), torch.from_numpy(right).cuda()
    o = torch.empty((48, 160), dtype=torch.int16, device="cuda")
    best = binding.res2tac_autotune(st.handle, L.data_ptr(), R.data_ptr(), 160, o.data_ptr(),
                                    320, torch.cuda.current_stream().cuda_stream)
    assert best.cost_mode in (1, 2) and best.row_cost in (1, 2)
    out = st.compute(L, R)
    assert np.array_equal(binding.u16(out), oracle.sgm(left, right, 64, 9, 7, 10, 120, 8, 3))
    st.close()


@pytest.mark.parametrize("D", [48, 80, 96, 144, 160, 256])
def test_partial_lane_groups_every_mode(D):
    # D that leaves lanes of a group without disparities, in both row modes and both sheared
    # widths the D allows
    rng = np.random.default_rng(D)
    W, H = 97, 45
    left = rng.integers(0, 256, (H, W)).astype(np.uint8)
    right = np.roll(left, -5, axis=1)
    prm = scenes.params(W, H, D, 9, 7, 7, 90, 8, 3)
    ref, rdbg = _oracle(left, right, prm)
    for sdpl, mode, cpl in itertools.product((8, 16, 32), (1, 2), (1, 2)):
        if D % sdpl:
            continue
        t = binding.res2tac_tuning(0, 0, 0, sdpl, mode, cpl)
        out, got = _gpu(left, right, prm, tuning=t)
        assert np.array_equal(got["agg"], rdbg["agg"]), (sdpl, mode, cpl)
        assert np.array_equal(out, ref), (sdpl, mode, cpl)


def test_repeatable_and_host_path():
    import torch
    left, right, _, prm = scenes.single_pair("320x240_d64_ct5x5_r4", 3)
    st = binding.Stereo(prm)
    a = st.compute(torch.from_numpy(left).cuda(), torch.from_numpy(right).cuda()).clone()
    b = st.compute(torch.from_numpy(left).cuda(), torch.from_numpy(right).cuda())
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    host_out = np.zeros((prm["height"], prm["width"]), np.uint16)
    binding.res2tac_compute_host(st.handle, left.ctypes.data, right.ctypes.data, prm["width"],
                                 host_out.ctypes.data, 2 * prm["width"], 0)
    assert np.array_equal(host_out, binding.u16(a))
    assert binding.res2tac_last_launch_count(st.handle) == 6
    # pinned host buffers: read and written in place by the kernels
    hl = torch.from_numpy(left).pin_memory()
    hr = torch.from_numpy(right).pin_memory()
    ho = torch.full((prm["height"], prm["width"]), 0x4321, dtype=torch.int16).pin_memory()
    binding.res2tac_compute_host(st.handle, hl.data_ptr(), hr.data_ptr(), prm["width"],
                                 ho.data_ptr(), 2 * prm["width"], 0)
    assert np.array_equal(ho.numpy().view(np.uint16), binding.u16(a))
    assert binding.res2tac_last_launch_count(st.handle) == 6
    st.close()


def test_invalid_pointers_and_pitch_rejected():
    import torch
    prm = scenes.params(64, 32, 32, 5, 5, 10, 120, 4, 0)
    st = binding.Stereo(prm)
    x = torch.zeros((32, 64), dtype=torch.uint8, device="cuda")
    out = torch.zeros((32, 64), dtype=torch.int16, device="cuda")
    with pytest.raises(binding.Res2tacError):
        binding.res2tac_compute(st.handle, x.data_ptr(), x.data_ptr(), 63, out.data_ptr(), 128, 0)
    with pytest.raises(binding.Res2tacError):
        binding.res2tac_compute(st.handle, x.data_ptr(), 0, 64, out.data_ptr(), 128, 0)
    with pytest.raises(binding.Res2tacError):
        binding.res2tac_compute(st.handle, x.data_ptr(), x.data_ptr(), 64, out.data_ptr(), 127, 0)
    st.close()


# ------------------------------------------------------- exact consistency check (Sec. 3.2.3)
EXACT = scenes.FLAG_LR_CHECK | 4


@pytest.mark.parametrize("name", list(scenes.SINGLE))
def test_exact_check_full_size_workloads(name):
    left, right, _, prm = scenes.single_pair(name, 0)
    prm = dict(prm, flags=prm["flags"] | EXACT)
    _assert_same(left, right, prm)


@pytest.mark.parametrize("seed", range(6))
def test_exact_check_tiny_random_shapes(seed):
    rng = np.random.default_rng(500 + seed)
    W = int(rng.integers(1, 70))
    H = int(rng.integers(1, 40))
    D = int(rng.choice([16, 32, 64, 128, 256]))
    cw, ch = ((5, 5), (9, 7))[seed % 2]
    R = (4, 8)[(seed // 2) % 2]
    left = rng.integers(0, 256, (H, W)).astype(np.uint8)
    right = rng.integers(0, 256, (H, W)).astype(np.uint8)
    prm = scenes.params(W, H, D, cw, ch, 10, 120, R, EXACT | (seed % 2) * 2, seed % 3)
    _assert_same(left, right, prm)


def test_exact_check_saturated_sums_padded_pitches():
    rng = np.random.default_rng(6)
    W, H, D = 150, 90, 128
    left = rng.integers(0, 256, (H, W)).astype(np.uint8)
    right = rng.integers(0, 256, (H, W)).astype(np.uint8)
    _assert_same(left, right, scenes.params(W, H, D, 5, 5, 100, 16384, 8, EXACT | 2), in_pad=9,
                 out_pad=3)


def test_exact_check_launches_stages_and_batch_rejection():
    import torch
    left, right, _, prm = scenes.single_pair("320x240_d64_ct5x5_r4", 0)
    prm = dict(prm, flags=EXACT | 2)
    st = binding.Stereo(prm)
    binding.res2tac_set_profiling(st.handle, True)
    L, R = torch.from_numpy(left).cuda(), torch.from_numpy(right).cuda()
    st.compute(L, R)
    times = binding.res2tac_stage_times(st.handle)
    assert binding.res2tac_last_launch_count(st.handle) == 12
    assert all(v > 0 for v in times.values())
    o = torch.empty_like(L, dtype=torch.int16)
    pair = binding.res2tac_pair(L.data_ptr(), R.data_ptr(), L.shape[1], o.data_ptr(),
                                2 * L.shape[1], L.shape[1], L.shape[0], prm["max_disp"], 0)
    with pytest.raises(binding.Res2tacError):
        binding.res2tac_compute_batch(st.handle, [pair], 0)
    st.close()


# ------------------------------------------------------------------------- NCC matching cost
NCC = 8


@pytest.mark.parametrize("n", [5, 9])
def test_ncc_full_size_road_pair(n):
    # the 1242 x 375 workload with the paper's NCC penalties (P1 = 90, P2 = 880)
    left, right, _, prm = scenes.single_pair("1242x375_d128_ct9x7_r8", 0)
    if n == 9:
        left, right = left[:160], right[:160]
    prm = dict(prm, census_w=n, census_h=n, p1=90, p2=880, flags=prm["flags"] | NCC,
               height=left.shape[0])
    _assert_same(left, right, prm)


@pytest.mark.parametrize("seed", range(8))
def test_ncc_tiny_random_shapes(seed):
    rng = np.random.default_rng(700 + seed)
    W = int(rng.integers(1, 90))
    H = int(rng.integers(1, 50))
    D = int(rng.choice([16, 32, 48, 64, 80, 128, 256]))
    n = (5, 9)[seed % 2]
    R = (4, 8)[(seed // 2) % 2]
    left = rng.integers(0, 256, (H, W)).astype(np.uint8)
    right = np.clip(left.astype(int) + rng.integers(-30, 31, (H, W)), 0, 255).astype(np.uint8)
    if seed % 3 == 0:
        right[: H // 2] = 128  # constant region: zero variance
    flags = NCC | (seed % 4) | (4 if seed >= 6 else 0)
    prm = scenes.params(W, H, D, n, n, int(rng.integers(0, 100)), 880, R, flags, seed % 3)
    _assert_same(left, right, prm)


@pytest.mark.parametrize("W,H,D,n", [(200, 37, 64, 5), (97, 61, 128, 9), (130, 33, 256, 9)])
def test_ncc_ragged_tiles(W, H, D, n):
    left, right, _ = scenes.make_scene("road", W + H + n, W, H, D)
    _assert_same(left, right, scenes.params(W, H, D, n, n, 90, 880, 8, 3 | NCC))


@pytest.mark.parametrize("n", [5, 9])
def test_ncc_near_tie_patches(n):
    """Patch pairs whose 255 Phi lies within 1e-6 of k + 1/2, side by side in one n-row image
    (pair i in columns [i n, (i + 1) n), so the patch at its centre is exactly that pair): the
    kernel's fp32 estimate cannot tell those roundings apart and must settle them on integers.
    Cost volume, sums and maps bit-exact against the oracle; the centre costs against exact
    decimal arithmetic."""
    from test_oracle_pins import _k_decimal, _near_tie_patch_pairs
    pairs = _near_tie_patch_pairs(n, 600 + n, want=24)
    left = np.concatenate([a.reshape(n, n) for a, _ in pairs], axis=1).astype(np.uint8)
    right = np.concatenate([b.reshape(n, n) for _, b in pairs], axis=1).astype(np.uint8)
    H, W = left.shape
    prm = scenes.params(W, H, 16, n, n, 90, 880, 8, 3 | NCC)
    _, got = _gpu(left, right, prm)
    r, N = n // 2, n * n
    for i, (a, b) in enumerate(pairs):
        sA, sB = int(a.sum()), int(b.sum())
        k = _k_decimal(N * int((a * b).sum()) - sA * sB, N * int((a * a).sum()) - sA * sA,
                       N * int((b * b).sum()) - sB * sB)
        assert got["cost"][r, i * n + r, 0] == 255 - k, i
    _assert_same(left, right, prm)


def test_ncc_saturated_sums_exact_check_padded_pitches():
    rng = np.random.default_rng(8)
    W, H, D = 140, 70, 64
    left = rng.integers(0, 256, (H, W)).astype(np.uint8)
    right = rng.integers(0, 256, (H, W)).astype(np.uint8)
    _assert_same(left, right, scenes.params(W, H, D, 5, 5, 100, 16384, 8, 3 | 4 | NCC),
                 in_pad=5, out_pad=2)


def test_ncc_launches_and_rejections():
    import torch
    left, right, _, prm = scenes.single_pair("320x240_d64_ct5x5_r4", 0)
    st = binding.Stereo(dict(prm, flags=3 | NCC))
    L, R = torch.from_numpy(left).cuda(), torch.from_numpy(right).cuda()
    st.compute(L, R)
    assert binding.res2tac_last_launch_count(st.handle) == 7
    o = torch.empty_like(L, dtype=torch.int16)
    pair = binding.res2tac_pair(L.data_ptr(), R.data_ptr(), L.shape[1], o.data_ptr(),
                                2 * L.shape[1], L.shape[1], L.shape[0], prm["max_disp"], 0)
    with pytest.raises(binding.Res2tacError):
        binding.res2tac_compute_batch(st.handle, [pair], 0)
    st.close()
    with pytest.raises(binding.Res2tacError):  # 9 x 7 is a census window, not an NCC patch
        binding.Stereo(dict(prm, census_w=9, census_h=7, flags=NCC))


# ----------------------------------------------------------------------------- maximum sizes
@pytest.mark.parametrize("W,H", [(16384, 12), (12, 16384)])
def test_maximum_width_and_height(W, H):
    rng = np.random.default_rng(W + H)
    left = rng.integers(0, 256, (H, W)).astype(np.uint8)
    right = np.roll(left, 9, axis=1)
    right[:, :9] = rng.integers(0, 256, (H, 9))
    _assert_same(left, right, scenes.params(W, H, 64, 5, 5, 10, 120, 8, 3))


def test_3840x2160_d256_sampled_sums():
    # the largest pair of the serving workload: the aggregated sums at sampled pixels (corners,
    # borders, interior) from the oracle's walk along the 8 path lines through each of them
    import torch
    W, H, D = 3840, 2160, 256
    left, right, _ = scenes.make_scene("road", 5, W, H, D)
    prm = scenes.params(W, H, D, 9, 7, 10, 120, 8, 3)
    st = binding.Stereo(prm)
    st.compute(torch.from_numpy(left).cuda(), torch.from_numpy(right).cuda())
    dbg = st.debug_outputs()
    rng = np.random.default_rng(6)
    pts = [(0, 0), (W - 1, 0), (0, H - 1), (W - 1, H - 1), (W // 2, H // 2), (D - 1, 7)]
    pts += [(int(rng.integers(0, W)), int(rng.integers(0, H))) for _ in range(10)]
    xs = torch.tensor([p[0] for p in pts], device="cuda")
    ys = torch.tensor([p[1] for p in pts], device="cuda")
    agg = binding.u16(dbg["agg"][ys, xs])
    dl = binding.u16(dbg["dl"][ys, xs])
    del dbg
    st.close()
    for i, (x, y) in enumerate(pts):
        want = oracle.s_at(left, right, D, 9, 7, 10, 120, 8, 0, x, y)
        assert np.array_equal(agg[i], want), (x, y)
        assert dl[i] == int(np.argmin(want)), (x, y)
