"""Batch engine: uneven pairs in persistent kernels under a CUDA graph give, per pair, the same
bits as a single-pair call and as the oracle."""
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
