"""The C-ABI library loads without a GPU, exports every declared symbol and validates input."""
import os
import re

import pytest

from paper_2106_07927_gb300 import binding

INCLUDE = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")


def _declared(header="res2tac.h"):
    src = open(os.path.join(INCLUDE, header)).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(res2tac_\w+)\s*\(", src)))


def test_header_declarations_match_binding(cuda_lib):
    assert _declared() == sorted(binding.EXPORTS)
    assert _declared("res2tac_measure.h") == sorted(binding.MEASURE_EXPORTS)
    assert sorted(os.listdir(INCLUDE)) == ["res2tac.h", "res2tac_measure.h"]


def test_library_exports_every_declared_symbol(cuda_lib):
    for name in _declared() + _declared("res2tac_measure.h"):
        assert hasattr(cuda_lib, name), name


@pytest.mark.parametrize("bad", [
    dict(width=0), dict(height=16385), dict(max_disp=8), dict(max_disp=264), dict(max_disp=40),
    dict(census_w=7), dict(p1=20, p2=10), dict(p2=20000), dict(num_paths=6), dict(flags=16),
    dict(flags=8, census_w=9, census_h=7), dict(census_w=9, census_h=9), dict(lr_threshold=-1),
])
def test_invalid_params_rejected(cuda_lib, bad):
    d = dict(width=64, height=32, max_disp=32, census_w=9, census_h=7, p1=10, p2=120,
             num_paths=8, flags=3, lr_threshold=1)
    d.update(bad)
    p = binding.params_from_dict(d)
    assert binding.res2tac_workspace_bytes(p) == 0
    with pytest.raises(binding.Res2tacError) as ei:
        binding.res2tac_create(p)
    assert ei.value.code == binding.RES2TAC_EINVAL


def test_workspace_bytes_scale(cuda_lib):
    p = binding.make_params(1242, 375, 128)
    n = 1242 * 375
    ws = binding.res2tac_workspace_bytes(p)
    # census maps 16 B/px, cost 1 B/DE, aggregated volume 2 B/DE, maps and staging ~11 B/px
    assert 3 * n * 128 < ws < 3 * n * 128 + 40 * n
    wide = binding.make_params(1242, 375, 128, p2=16384)
    assert binding.res2tac_workspace_bytes(wide) > ws + n * 128


def test_null_handle_rejected(cuda_lib):
    assert cuda_lib.res2tac_compute(None, None, None, 0, None, 0, None) == binding.RES2TAC_EINVAL
    assert cuda_lib.res2tac_last_launch_count(None) == 0
    cuda_lib.res2tac_destroy(None)
    assert binding.res2tac_strerror(binding.RES2TAC_ETIMEOUT)
