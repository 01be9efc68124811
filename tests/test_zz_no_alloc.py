"""res2tac_compute_static, the entry point that allocates nothing.

Some callers cannot allocate device memory while they run: an onboard stereo loop allowed to
allocate only at start-up, a plugin whose host framework owns all device memory, or a loop that
cannot afford the device-wide synchronisation cudaMalloc / cudaFree may cause. For them the
library offers res2tac_compute_static, whose scratch is a fixed device array inside the library.
These checks call it through the C ABI and compare its maps with those of the regular
context-based res2tac_compute, bit for bit (the method is integer arithmetic, so the tolerance
the other tests use is equality), over two calls in a row of different shapes so the second
call starts from the first call's leftovers in the shared array.
"""
import numpy as np
import pytest

from paper_2106_07927_gb300 import binding, scenes

pytestmark = pytest.mark.gpu


def _with_context(left, right, prm):
    import torch
    st = binding.Stereo(prm)
    out = st.compute(torch.from_numpy(left).cuda(), torch.from_numpy(right).cuda())
    torch.cuda.synchronize()
    res = binding.u16(out)
    st.close()
    return res


def _static_call(left, right, prm):
    import torch
    H, W = left.shape
    L = torch.from_numpy(left).cuda()
    R = torch.from_numpy(right).cuda()
    out = torch.full((H, W), 0x5A5A, dtype=torch.int16, device="cuda")
    binding.res2tac_compute_static(binding.params_from_dict(prm), L.data_ptr(), R.data_ptr(), W,
                                   out.data_ptr(), 2 * W,
                                   torch.cuda.current_stream().cuda_stream)
    return out


def test_static_entry_matches_context_entry_on_two_calls_in_a_row():
    import torch
    first = scenes.single_pair("320x240_d64_ct5x5_r4", 4)  # 4 paths, WTA only
    left2, right2, _ = scenes.make_scene("road", 9, 200, 150, 128)
    second = (left2, right2, None, scenes.params(200, 150, 128, 9, 7, 10, 120, 8,
                                                 scenes.FLAG_LR_CHECK | scenes.FLAG_MEDIAN))
    expected = [_with_context(c[0], c[1], c[3]) for c in (first, second)]
    got1 = _static_call(first[0], first[1], first[3])
    got2 = _static_call(second[0], second[1], second[3])
    torch.cuda.synchronize()
    assert np.array_equal(binding.u16(got1), expected[0])
    assert np.array_equal(binding.u16(got2), expected[1])
    # and once more on the first shape, after the second call's contents
    got3 = _static_call(first[0], first[1], first[3])
    torch.cuda.synchronize()
    assert np.array_equal(binding.u16(got3), expected[0])


def test_static_entry_exact_check_matches_context_entry():
    import torch
    left, right, _ = scenes.make_scene("nadir", 4, 180, 120, 64)
    prm = scenes.params(180, 120, 64, 9, 7, 10, 120, 8,
                        scenes.FLAG_LR_CHECK | scenes.FLAG_MEDIAN | binding.RES2TAC_EXACT_CC)
    expected = _with_context(left, right, prm)
    got = _static_call(left, right, prm)
    torch.cuda.synchronize()
    assert np.array_equal(binding.u16(got), expected)


def test_static_entry_wide_sums_and_ncc_after_a_narrow_call():
    """The two other layouts of the shared array: 32-bit sums (num_paths (255 + p2) > 65535,
    4 B per disparity estimate) and the NCC cost (patch statistics and variances placed after the
    maps), each called right after a call of another layout, so each starts from the previous
    call's contents; compared with res2tac_compute."""
    import torch
    narrow = scenes.single_pair("320x240_d64_ct5x5_r4", 2)
    lw, rw, _ = scenes.make_scene("road", 12, 160, 120, 64)
    wide = (lw, rw, None, scenes.params(160, 120, 64, 9, 7, 10, 9000, 8, 3))
    ln, rn, _ = scenes.make_scene("nadir", 13, 150, 100, 64)
    ncc = (ln, rn, None, scenes.params(150, 100, 64, 5, 5, 90, 880, 8, 3 | binding.RES2TAC_NCC))
    cases = (narrow, wide, ncc, wide)
    expected = [_with_context(c[0], c[1], c[3]) for c in cases]
    for c, want in zip(cases, expected):
        got = _static_call(c[0], c[1], c[3])
        torch.cuda.synchronize()
        assert np.array_equal(binding.u16(got), want)


def test_static_entry_rejects_a_problem_larger_than_its_array():
    import torch
    prm = scenes.params(1242, 375, 128, 9, 7, 10, 120, 8, 3)  # needs about 190 MB
    x = torch.zeros((375, 1242), dtype=torch.uint8, device="cuda")
    out = torch.zeros((375, 1242), dtype=torch.int16, device="cuda")
    with pytest.raises(binding.Res2tacError) as ei:
        binding.res2tac_compute_static(binding.params_from_dict(prm), x.data_ptr(), x.data_ptr(),
                                       1242, out.data_ptr(), 2 * 1242, 0)
    assert ei.value.code == binding.RES2TAC_ENOMEM
    assert str(binding.RES2TAC_STATIC_SCRATCH_BYTES) in str(ei.value)
