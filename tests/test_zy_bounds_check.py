"""The debug build with range checks (RES2TAC_CHECK_BOUNDS): every checked global access of the
aggregation and WTA kernels stays inside its buffer on tiny and ragged shapes, every tuning and
both sum widths, and the maps still equal the oracle's. A failing check records its site and
skips the access (no trap), so a failure here shows as a nonzero site."""
import itertools

import numpy as np
import pytest

import oracle
from paper_2106_07927_gb300 import binding, scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def check_lib():
    yield binding.use_check_library(True)
    binding.use_check_library(False)


def test_range_checks_pass_on_tiny_shapes(check_lib):
    import torch
    rng = np.random.default_rng(77)
    cases = [(1, 1, 16), (5, 3, 16), (17, 9, 32), (33, 20, 48), (70, 13, 64), (9, 40, 128),
             (130, 7, 144), (40, 31, 256)]
    for (W, H, D), (p2, paths) in zip(cases, itertools.cycle(((120, 8), (16384, 8), (90, 4)))):
        left = rng.integers(0, 256, (H, W)).astype(np.uint8)
        right = rng.integers(0, 256, (H, W)).astype(np.uint8)
        prm = scenes.params(W, H, D, 9, 7, 10, p2, paths, 3)
        st = binding.Stereo(prm)
        assert binding.res2tac_bounds_status(st.handle)[0] == 1  # the debug build
        L, R = torch.from_numpy(left).cuda(), torch.from_numpy(right).cuda()
        ref = oracle.sgm(left, right, D, 9, 7, 10, p2, paths, 3)
        for sdpl, mode, cpl in itertools.product((8, 16, 32), (1, 2), (1, 2)):
            if D % sdpl:
                continue
            binding.res2tac_set_tuning(st.handle, binding.res2tac_tuning(0, 0, 0, sdpl, mode, cpl))
            out = st.compute(L, R)
            torch.cuda.synchronize()
            checked, site, off = binding.res2tac_bounds_status(st.handle)
            assert site == 0, (W, H, D, sdpl, mode, cpl, site, off)
            assert np.array_equal(binding.u16(out), ref), (W, H, D, sdpl, mode, cpl)
        st.close()
