"""The seeded input generators are deterministic and shaped like the listed workloads."""
import numpy as np

from paper_2106_07927_gb300 import scenes


def test_single_pairs_deterministic_and_shaped():
    for name in scenes.SINGLE:
        a = scenes.single_pair(name, 1)
        b = scenes.single_pair(name, 1)
        p = a[3]
        assert a[0].shape == (p["height"], p["width"]) and a[0].dtype == np.uint8
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
        assert 0 <= a[2].min() and a[2].max() < p["max_disp"]
    assert not np.array_equal(scenes.single_pair("320x240_d64_ct5x5_r4", 1)[0],
                              scenes.single_pair("320x240_d64_ct5x5_r4", 2)[0])


def test_batch_specs_cover_listed_sets():
    specs = scenes.batch_specs(0, 64)
    assert len(specs) == 64
    for s in specs:
        p = s["prm"]
        assert p["width"] in scenes.BATCH_WIDTHS and p["height"] in scenes.BATCH_HEIGHTS
        assert p["max_disp"] in scenes.BATCH_DISPS
    assert {s["kind"] for s in specs} == {"road", "nadir"}
    big = scenes.batch_specs(1, 400, big_fraction=0.05)
    nbig = sum(s["prm"]["width"] == 3840 for s in big)
    assert 5 <= nbig <= 40


def test_forward_warp_z_order():
    rng = np.random.default_rng(0)
    L = np.arange(10, dtype=np.uint8)[None, :].repeat(2, 0)
    disp = np.zeros((2, 10), np.int32)
    disp[:, 6] = 3  # pixel 6 lands on 3 and hides pixel 3 (d = 0)
    R = scenes.forward_warp(rng, L, disp)
    assert R[0, 3] == 6 and R[0, 5] == 5
