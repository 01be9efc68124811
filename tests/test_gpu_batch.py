"""Batch engine: uneven pairs in persistent kernels under a CUDA graph give, per pair, the same
bits as a single-pair call and as the oracle."""
import itertools

import numpy as np
import pytest

import oracle
from paper_2106_07927_gb300 import binding, scenes

pytestmark = pytest.mark.gpu


def _run_batch(h, tensors, shapes):
    import torch
    pairs = []
    outs = []
    for (L, R), (W, H, D) in zip(tensors, shapes):
        out = torch.full((H, W), -1, dtype=torch.int16, device="cuda")
        outs.append(out)
        pairs.append(binding.res2tac_pair(L.data_ptr(), R.data_ptr(), L.stride(0), out.data_ptr(),
                                          out.stride(0) * 2, W, H, D, 0))
    binding.res2tac_compute_batch(h, pairs, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return [binding.u16(o) for o in outs]


def _small_batch(seed, n):
    rng = np.random.default_rng(seed)
    items = []
    for i in range(n):
        W = int(rng.choice([40, 96, 160, 233]))
        H = int(rng.choice([24, 60, 97]))
        D = int(rng.choice([16, 64, 128, 256]))
        kind = ("road", "nadir")[i % 2]
        L, R, _ = scenes.make_scene(kind, seed * 31 + i, W, H, D)
        items.append((L, R, (W, H, D)))
    return items


@pytest.mark.parametrize("flags", [3, 0])
def test_batch_matches_oracle_and_single(flags):
    import torch
    items = _small_batch(1, 10)
    prm = scenes.params(64, 64, 64, 9, 7, 10, 120, 8, flags)
    ctx = binding.Stereo(prm)
    tensors = [(torch.from_numpy(L).cuda(), torch.from_numpy(R).cuda()) for L, R, _ in items]
    shapes = [s for _, _, s in items]
    outs = _run_batch(ctx.handle, tensors, shapes)
    for (L, R, (W, H, D)), got in zip(items, outs):
        ref = oracle.sgm(L, R, D, 9, 7, 10, 120, 8, flags)
        assert np.array_equal(got, ref), (W, H, D)
        single = binding.Stereo(scenes.params(W, H, D, 9, 7, 10, 120, 8, flags))
        s_out = single.compute(torch.from_numpy(L).cuda(), torch.from_numpy(R).cuda())
        torch.cuda.synchronize()
        assert np.array_equal(binding.u16(s_out), got)
        single.close()
    # replay of the captured graph with other pairs of the same layout, then a larger batch
    items2 = _small_batch(2, 10)
    for i in range(10):
        W, H, D = shapes[i]
        L, R, _ = scenes.make_scene("road", 500 + i, W, H, D)
        items2[i] = (L, R, (W, H, D))
    tensors2 = [(torch.from_numpy(L).cuda(), torch.from_numpy(R).cuda()) for L, R, _ in items2]
    outs2 = _run_batch(ctx.handle, tensors2, shapes)
    for (L, R, (W, H, D)), got in zip(items2, outs2):
        assert np.array_equal(got, oracle.sgm(L, R, D, 9, 7, 10, 120, 8, flags))
    items3 = _small_batch(3, 17)
    tensors3 = [(torch.from_numpy(L).cuda(), torch.from_numpy(R).cuda()) for L, R, _ in items3]
    outs3 = _run_batch(ctx.handle, tensors3, [s for _, _, s in items3])
    for (L, R, (W, H, D)), got in zip(items3, outs3):
        assert np.array_equal(got, oracle.sgm(L, R, D, 9, 7, 10, 120, 8, flags))
    ctx.close()


def test_batch_wide_and_four_paths():
    import torch
    items = _small_batch(4, 6)
    for (R_, P2) in ((4, 120), (8, 16384)):
        prm = scenes.params(64, 64, 64, 5, 5, 10, P2, R_, 3)
        ctx = binding.Stereo(prm)
        tensors = [(torch.from_numpy(L).cuda(), torch.from_numpy(R).cuda()) for L, R, _ in items]
        outs = _run_batch(ctx.handle, tensors, [s for _, _, s in items])
        for (L, R, (W, H, D)), got in zip(items, outs):
            assert np.array_equal(got, oracle.sgm(L, R, D, 5, 5, 10, P2, R_, 3))
        ctx.close()


LIMIT_DE = 1242 * 375 * 128  # pairs up to this size are compared with the full oracle


def _batch64_inputs():
    """The 64 uneven pairs of the batch workload (sizes from scenes.batch_specs(0, 64)), each
    cropped from one 1920 x 1080 scene per (kind, D), as the benchmark makes them."""
    specs = scenes.batch_specs(0, 64)
    masters, items = {}, []
    for s in specs:
        p = s["prm"]
        key = (s["kind"], p["max_disp"])
        if key not in masters:
            masters[key] = scenes.make_scene(s["kind"], 17 + len(masters), 1920, 1080,
                                             p["max_disp"])[:2]
        L, R = masters[key]
        W, H, D = p["width"], p["height"], p["max_disp"]
        items.append((np.ascontiguousarray(L[:H, :W]), np.ascontiguousarray(R[:H, :W]), (W, H, D)))
    return items


def _sample_points(W, H, D, rng, n=32):
    pts = [(0, 0), (W - 1, 0), (0, H - 1), (W - 1, H - 1), (W // 2, 0), (W // 2, H - 1),
           (0, H // 2), (W - 1, H // 2), (min(D, W) - 1, H // 3), (W // 2, H // 2)]
    while len(pts) < n:
        pts.append((int(rng.integers(0, W)), int(rng.integers(0, H))))
    return pts


def test_batch_of_64_uneven_pairs_against_oracle():
    """The 64-pair batch workload (W up to 1920, H up to 1080, D up to 256, D > W allowed) in one
    batch call, LR check and median on: every pair equal to its single-pair launch, every pair
    of at most 1242 x 375 x 128 disparity estimates equal to the full oracle. Then the same batch
    with WTA only: D^L of every D = 256 pair and of the 1920 x 1080 pairs at 32 sampled pixels
    (corners, borders, interior) equal to the argmin of the oracle's sums there."""
    import concurrent.futures
    import torch
    items = _batch64_inputs()
    shapes = [s for _, _, s in items]
    tensors = [(torch.from_numpy(L).cuda(), torch.from_numpy(R).cuda()) for L, R, _ in items]
    oracle._load()
    pool = concurrent.futures.ThreadPoolExecutor(16)  # the oracle releases the GIL in C
    small = [i for i, (W, H, D) in enumerate(shapes) if W * H * D <= LIMIT_DE]
    assert len(small) >= 8
    assert any(D == 256 for i in small for (_, _, D) in [shapes[i]])
    refs = {i: pool.submit(oracle.sgm, items[i][0], items[i][1], shapes[i][2], 9, 7, 10, 120, 8,
                           3) for i in small}
    ctx = binding.Stereo(scenes.params(64, 64, 64, 9, 7, 10, 120, 8, 3))
    outs = _run_batch(ctx.handle, tensors, shapes)
    for i, ((L, R), (W, H, D)) in enumerate(zip(tensors, shapes)):
        single = binding.Stereo(scenes.params(W, H, D, 9, 7, 10, 120, 8, 3))
        s_out = single.compute(L, R)
        torch.cuda.synchronize()
        assert np.array_equal(binding.u16(s_out), outs[i]), (i, W, H, D)
        single.close()
    for i in small:
        assert np.array_equal(outs[i], refs[i].result()), (i, shapes[i])
    ctx.close()

    # WTA only: the map is D^L, checked at sampled pixels of the large pairs
    big = [i for i, (W, H, D) in enumerate(shapes) if D == 256 or (W, H) == (1920, 1080)]
    assert any((W, H) == (1920, 1080) for (W, H, _) in (shapes[i] for i in big))
    assert any(W == 320 and D == 256 for (W, _, D) in (shapes[i] for i in big))
    ctx = binding.Stereo(scenes.params(64, 64, 64, 9, 7, 10, 120, 8, 0))
    outs = _run_batch(ctx.handle, tensors, shapes)
    ctx.close()
    rng = np.random.default_rng(11)
    jobs = []
    for i in big:
        W, H, D = shapes[i]
        for (x, y) in _sample_points(W, H, D, rng):
            jobs.append((i, x, y, pool.submit(oracle.s_at, items[i][0], items[i][1], D, 9, 7, 10,
                                              120, 8, 0, x, y)))
    for i, x, y, f in jobs:
        assert outs[i][y, x] == int(np.argmin(f.result())), (i, shapes[i], x, y)
    pool.shutdown()


def test_every_batch_tuning_candidate_matches_oracle():
    """Every setting the batch autotuner may pick (row disparities per lane, sheared disparities
    and chains per lane, WTA tile), applied to every bucket of a small uneven batch (D from 32 to
    256, both size classes), gives the oracle's maps; then the autotuner itself runs on that
    batch, reports a table of valid entries and leaves maps that still match."""
    import torch
    rng = np.random.default_rng(21)
    shapes = [(96, 40, 32), (130, 33, 64), (512, 520, 64), (200, 61, 128), (77, 50, 256),
              (160, 45, 144)]
    items = []
    for i, (W, H, D) in enumerate(shapes):
        L, R, _ = scenes.make_scene(("road", "nadir")[i % 2], 40 + i, W, H, D)
        items.append((L, R, (W, H, D)))
    refs = [oracle.sgm(L, R, D, 9, 7, 10, 120, 8, 3) for L, R, (W, H, D) in items]
    tensors = [(torch.from_numpy(L).cuda(), torch.from_numpy(R).cuda()) for L, R, _ in items]
    ctx = binding.Stereo(scenes.params(64, 64, 64, 9, 7, 10, 120, 8, 3))
    buckets = sorted({(D, int(W * H >= (1 << 18))) for W, H, D in shapes})
    tried = 0
    for row, (sd, sc), wpx in itertools.product((2, 4, 8), ((16, 1), (16, 2)), (64, 128, 256)):
        entries = [binding.res2tac_batch_tuning(D, lg, row, sd, sc, wpx) for D, lg in buckets
                   if D % row == 0 and D // row <= 32 and D % sd == 0]
        if not entries:
            continue
        binding.res2tac_set_batch_tuning(ctx.handle, entries)
        outs = _run_batch(ctx.handle, tensors, [s for _, _, s in items])
        for got, ref, (_, _, shp) in zip(outs, refs, items):
            assert np.array_equal(got, ref), (row, sd, sc, wpx, shp)
        tried += 1
    assert tried >= 18
    pairs, outs = [], []
    for (L, R), (W, H, D) in zip(tensors, [s for _, _, s in items]):
        o = torch.full((H, W), -1, dtype=torch.int16, device="cuda")
        outs.append(o)
        pairs.append(binding.res2tac_pair(L.data_ptr(), R.data_ptr(), L.stride(0), o.data_ptr(),
                                          2 * W, W, H, D, 0))
    table, ms0, ms1 = binding.res2tac_autotune_batch(ctx.handle, pairs,
                                                     torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert len(table) == len(buckets) and 0 < ms1 <= ms0
    for e in table:
        assert (e.max_disp, e.large) in buckets and e.max_disp % e.shear_dpl == 0
        got = binding.res2tac_get_batch_tuning(ctx.handle, e.max_disp, e.large)
        assert got.as_dict() == e.as_dict()
    for o, ref in zip(outs, refs):
        assert np.array_equal(binding.u16(o), ref)
    with pytest.raises(binding.Res2tacError):  # 8 disparities per sheared lane: not a setting
        binding.res2tac_set_batch_tuning(ctx.handle, [binding.res2tac_batch_tuning(64, 0, 2, 8,
                                                                                   1, 128)])
    ctx.close()
