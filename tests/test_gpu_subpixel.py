"""Sub-pixel refinement (Sec. 2.1.3) on the GPU vs the fp64 CPU oracle.

The library refines in fp32 with a correctly rounded division and addition; the oracle solves the
parabola in fp64. For an integer D^L = d < 256 and |delta| <= 1/2 the fp32 result
fl(d + fl(delta)) is off by at most 2^-25 (rounding of delta) + 2^-16 (rounding of the sum, half
an ulp at [128, 256)), so the bar is TOL below. Validity (the left-right check, the median's
invalid count) is decided on integers and must match exactly: +inf on both sides.
"""
import numpy as np
import pytest

import oracle
from paper_2106_07927_gb300 import binding, scenes

pytestmark = pytest.mark.gpu

TOL = 2.0 ** -16 + 2.0 ** -25 + 1e-12


def _gpu_sub(left, right, prm, out_pad=0):
    import torch
    H, W = left.shape
    st = binding.Stereo(prm)
    L = torch.from_numpy(left).cuda()
    R = torch.from_numpy(right).cuda()
    outb = torch.full((H, W + out_pad), -7.0, dtype=torch.float32, device="cuda")
    binding.res2tac_compute_subpixel(st.handle, L.data_ptr(), R.data_ptr(), W, outb.data_ptr(),
                                     4 * (W + out_pad), torch.cuda.current_stream().cuda_stream)
    ref = st.debug_subpixel()
    launches = binding.res2tac_last_launch_count(st.handle)
    integer = st.compute(L, R)
    torch.cuda.synchronize()
    out = outb.cpu().numpy()
    if out_pad:
        assert np.all(out[:, W:] == -7.0), "wrote outside the row"
    res = out[:, :W].astype(np.float64), ref.cpu().numpy().astype(np.float64), binding.u16(integer)
    st.close()
    return res, launches


def _check(left, right, prm, **kw):
    (out, ref, integer), launches = _gpu_sub(left, right, prm, **kw)
    want, want_ref = oracle.sgm_subpixel(left, right, prm["max_disp"], prm["census_w"],
                                         prm["census_h"], prm["p1"], prm["p2"], prm["num_paths"],
                                         prm["flags"], prm["lr_threshold"])
    assert launches == (12 if prm["flags"] & 4 else 6)
    err = np.abs(ref - want_ref)
    assert err.max() <= TOL, f"refined D^L: max error {err.max()} at {np.argmax(err)}"
    inv = np.isinf(want)
    assert np.array_equal(np.isinf(out), inv), "invalid pixels differ"
    assert np.all(out[inv] > 0)
    if (~inv).any():
        e = np.abs(out[~inv] - want[~inv])
        assert e.max() <= TOL, f"final map: max error {e.max()}"
    # the same context's integer map agrees on validity and lies within 1/2 of the refined one
    assert np.array_equal(integer == binding.RES2TAC_INVALID, inv)
    assert np.all(np.abs(out[~inv] - integer[~inv]) <= 0.5)
    return out, want


@pytest.mark.parametrize("name", list(scenes.SINGLE))
def test_subpixel_full_size_workloads(name):
    left, right, _, prm = scenes.single_pair(name, 0)
    out, _ = _check(left, right, prm)
    frac = np.abs(out[np.isfinite(out)] % 1.0)
    assert (frac > 0).mean() > 0.1, "refinement left (nearly) every pixel integral"


@pytest.mark.parametrize("seed", range(8))
def test_subpixel_tiny_random_shapes(seed):
    rng = np.random.default_rng(300 + seed)
    W = int(rng.integers(1, 70))
    H = int(rng.integers(1, 40))
    D = int(rng.choice([16, 32, 48, 64, 128, 256]))
    cw, ch = ((5, 5), (9, 7))[seed % 2]
    R = (4, 8)[(seed // 2) % 2]
    flags = seed % 4
    left = rng.integers(0, 256, (H, W)).astype(np.uint8)
    right = rng.integers(0, 256, (H, W)).astype(np.uint8)
    P1 = int(rng.integers(0, 30))
    P2 = int(rng.integers(P1, 300))
    prm = scenes.params(W, H, D, cw, ch, P1, P2, R, flags, int(rng.integers(0, 3)))
    _check(left, right, prm)


@pytest.mark.parametrize("W,H,D", [(200, 3, 64), (97, 61, 128), (257, 33, 256)])
def test_subpixel_ragged_tiles(W, H, D):
    left, right, _ = scenes.make_scene("road", W + H, W, H, D)
    _check(left, right, scenes.params(W, H, D, 9, 7, 10, 120, 8, 3))


def test_subpixel_saturated_sums_and_padded_output():
    # P2 = 16384 with 8 paths: the uint32 sums saturate to 65535 before the parabola fit
    rng = np.random.default_rng(5)
    W, H, D = 300, 120, 128
    left = rng.integers(0, 256, (H, W)).astype(np.uint8)
    right = rng.integers(0, 256, (H, W)).astype(np.uint8)
    _check(left, right, scenes.params(W, H, D, 5, 5, 100, 16384, 8, 3), out_pad=5)


def test_subpixel_with_exact_check():
    left, right, _ = scenes.make_scene("road", 21, 240, 96, 128)
    _check(left, right, scenes.params(240, 96, 128, 9, 7, 10, 120, 8, 3 | 4))


def test_subpixel_invalid_pitch_and_alignment_rejected():
    import torch
    prm = scenes.params(64, 32, 32, 5, 5, 10, 120, 4, 0)
    st = binding.Stereo(prm)
    x = torch.zeros((32, 64), dtype=torch.uint8, device="cuda")
    out = torch.zeros((32, 65), dtype=torch.float32, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    with pytest.raises(binding.Res2tacError):  # pitch below 4 W
        binding.res2tac_compute_subpixel(st.handle, x.data_ptr(), x.data_ptr(), 64,
                                         out.data_ptr(), 4 * 63, s)
    with pytest.raises(binding.Res2tacError):  # pitch not a multiple of 4
        binding.res2tac_compute_subpixel(st.handle, x.data_ptr(), x.data_ptr(), 64,
                                         out.data_ptr(), 4 * 64 + 2, s)
    with pytest.raises(binding.Res2tacError):  # misaligned output
        binding.res2tac_compute_subpixel(st.handle, x.data_ptr(), x.data_ptr(), 64,
                                         out.data_ptr() + 2, 4 * 65, s)
    st.close()
