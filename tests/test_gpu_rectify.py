"""Rectification (Sec. 2.1.1) on the GPU vs the CPU oracle: bit-exact (integer arithmetic after
the 1/32-pixel grid step, which both sides take with the same exact float product and rint)."""
import numpy as np
import pytest

import oracle
from paper_2106_07927_gb300 import binding, scenes

pytestmark = pytest.mark.gpu


def _rectify_gpu(raw, mapx, mapy, raw_pad=0, out_pad=0, map_pad=0):
    import torch
    rh, rw = raw.shape
    H, W = mapx.shape
    rb = torch.zeros((rh, rw + raw_pad), dtype=torch.uint8, device="cuda")
    rb[:, :rw] = torch.from_numpy(raw).cuda()
    mx = torch.zeros((H, W + map_pad), dtype=torch.float32, device="cuda")
    my = torch.zeros((H, W + map_pad), dtype=torch.float32, device="cuda")
    mx[:, :W] = torch.from_numpy(mapx).cuda()
    my[:, :W] = torch.from_numpy(mapy).cuda()
    ob = torch.full((H, W + out_pad), 77, dtype=torch.uint8, device="cuda")
    binding.res2tac_rectify(rb.data_ptr(), rw + raw_pad, rw, rh, mx.data_ptr(), my.data_ptr(),
                            4 * (W + map_pad), ob.data_ptr(), W + out_pad, W, H,
                            torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    out = ob.cpu().numpy()
    if out_pad:
        assert np.all(out[:, W:] == 77), "wrote outside the row"
    return out[:, :W]


@pytest.mark.parametrize("W,H,rw,rh,strength,seed", [
    (1242, 375, 1242, 375, 1.0, 0), (640, 480, 700, 520, 2.0, 1), (97, 61, 80, 50, 4.0, 2),
    (1, 1, 3, 3, 1.0, 3), (300, 7, 300, 7, 6.0, 4)])
def test_rectify_matches_oracle(W, H, rw, rh, strength, seed):
    rng = np.random.default_rng(seed)
    raw = rng.integers(0, 256, (rh, rw)).astype(np.uint8)
    mapx, mapy = scenes.rectification_maps(seed, W, H, rw, rh, strength)
    # coordinates at and beyond the borders, and ones that are not finite or far outside
    mapx[0, 0], mapy[-1, -1] = -0.49, rh - 0.51
    if W > 4:
        mapx[0, 1], mapx[0, 2], mapy[0, 3], mapx[0, 4] = np.nan, np.inf, -np.inf, 3e8
    want = oracle.rectify(raw, mapx, mapy)
    got = _rectify_gpu(raw, mapx, mapy, raw_pad=3, out_pad=5, map_pad=2)
    assert np.array_equal(got, want)


def test_compute_raw_matches_oracle_chain():
    import torch
    left, right, _, prm = scenes.single_pair("320x240_d64_ct5x5_r4", 2)
    prm = dict(prm, flags=3)
    W, H = prm["width"], prm["height"]
    mlx, mly = scenes.rectification_maps(10, W, H)
    mrx, mry = scenes.rectification_maps(11, W, H)
    want = oracle.sgm(oracle.rectify(left, mlx, mly), oracle.rectify(right, mrx, mry),
                      prm["max_disp"], prm["census_w"], prm["census_h"], prm["p1"], prm["p2"],
                      prm["num_paths"], prm["flags"], prm["lr_threshold"])
    st = binding.Stereo(prm)
    maps = [torch.from_numpy(m).cuda() for m in (mlx, mly, mrx, mry)]
    s = torch.cuda.current_stream().cuda_stream
    with pytest.raises(binding.Res2tacError):  # no maps yet
        binding.res2tac_compute_raw(st.handle, 1, 1, W, 1, 2 * W, s)
    binding.res2tac_set_rectification(st.handle, *[m.data_ptr() for m in maps], 4 * W, W, H, s)
    L, R = torch.from_numpy(left).cuda(), torch.from_numpy(right).cuda()
    out = torch.empty((H, W), dtype=torch.int16, device="cuda")
    binding.res2tac_compute_raw(st.handle, L.data_ptr(), R.data_ptr(), W, out.data_ptr(), 2 * W, s)
    torch.cuda.synchronize()
    assert np.array_equal(binding.u16(out), want)
    assert binding.res2tac_last_launch_count(st.handle) == 7
    st.close()


def test_rectify_rejects_bad_arguments():
    import torch
    x = torch.zeros((8, 8), dtype=torch.uint8, device="cuda")
    m = torch.zeros((8, 8), dtype=torch.float32, device="cuda")
    with pytest.raises(binding.Res2tacError):  # map pitch below 4 W
        binding.res2tac_rectify(x.data_ptr(), 8, 8, 8, m.data_ptr(), m.data_ptr(), 28,
                                x.data_ptr(), 8, 8, 8, 0)
    with pytest.raises(binding.Res2tacError):  # misaligned map
        binding.res2tac_rectify(x.data_ptr(), 8, 8, 8, m.data_ptr() + 2, m.data_ptr(), 32,
                                x.data_ptr(), 8, 8, 8, 0)
    with pytest.raises(binding.Res2tacError):
        binding.res2tac_rectify(x.data_ptr(), 8, 8, 8, 0, m.data_ptr(), 32, x.data_ptr(), 8, 8,
                                8, 0)
