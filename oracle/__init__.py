"""Plain CPU oracle of the ReS2tAC SGM stereo path: test infrastructure, not the product.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import
this package. It wraps ``sgm_oracle.c`` (single-threaded C, int32 arithmetic) through ctypes and
shares no code with the CUDA library. Every function returns numpy arrays; the arithmetic and the
passage of the paper each step follows are documented in ``sgm_oracle.c``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sgm_oracle.c")
_LIB_PATH = os.path.join(_HERE, "libres2tac_oracle.so")
_lock = threading.Lock()
_lib = None

# Path directions (dx, dy): LR, RL, TB, BT, TLBR, TRBL, BLTR, BRTL (Sec. 2.3.3).
DIRECTIONS = ((1, 0), (-1, 0), (0, 1), (0, -1), (1, 1), (-1, 1), (1, -1), (-1, -1))
INVALID = 0xFFFF
FLAG_LR_CHECK = 1
FLAG_MEDIAN = 2
FLAG_EXACT_CC = 4
FLAG_NCC = 8


def build(force: bool = False) -> str:
    """Compile sgm_oracle.c into a shared library next to it (plain gcc, -O2, no SIMD flags)."""
    with _lock:
        stale = (not os.path.exists(_LIB_PATH)) or (
            os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC))
        if force or stale:
            tmp = _LIB_PATH + f".tmp{os.getpid()}"
            subprocess.check_call(
                ["gcc", "-O2", "-std=c99", "-shared", "-fPIC", _SRC, "-o", tmp, "-lm"])
            os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        P = ctypes.c_void_p
        I = ctypes.c_int
        I64 = ctypes.c_int64
        lib.r2o_census.argtypes = [P, I64, I, I, I, I, P]
        lib.r2o_cost.argtypes = [P, P, I, I, I, P]
        lib.r2o_path.argtypes = [P, I, I, I, I, I, I, I, P]
        lib.r2o_aggregate.argtypes = [P, I, I, I, I, I, I, P]
        lib.r2o_wta.argtypes = [P, I, I, I, P]
        lib.r2o_right_disparity.argtypes = [P, I, I, I, P]
        lib.r2o_lr_check.argtypes = [P, P, I, I, I, P, P]
        lib.r2o_median3x3.argtypes = [P, I, I, P]
        lib.r2o_sgm.argtypes = [P, P, I64, I, I, I, I, I, I, I, I, I, I, P, P, P, P, P, P]
        lib.r2o_subpixel.argtypes = [P, P, I, I, I, P]
        lib.r2o_cost_right.argtypes = [P, P, I, I, I, P]
        lib.r2o_ncc_cost.argtypes = [P, P, I64, I, I, I, I, P]
        lib.r2o_rectify.argtypes = [P, I64, I, I, P, P, I64, I, I, P, I64]
        lib.r2o_s_at.argtypes = [P, P, I64, I, I, I, I, I, I, I, I, I, I, I, P]
        lib.r2o_ncc_cost_right.argtypes = [P, P, I64, I, I, I, I, P]
        lib.r2o_median3x3_f64.argtypes = [P, I, I, P]
        lib.r2o_sgm_subpixel.argtypes = [P, P, I64, I, I, I, I, I, I, I, I, I, I, P, P]
        lib.r2o_ncc_round.argtypes = [I64, I64, I64]
        lib.r2o_ncc_round.restype = ctypes.c_int
        for f in (lib.r2o_census, lib.r2o_cost, lib.r2o_path, lib.r2o_aggregate, lib.r2o_wta,
                  lib.r2o_right_disparity, lib.r2o_lr_check, lib.r2o_median3x3, lib.r2o_sgm,
                  lib.r2o_subpixel, lib.r2o_median3x3_f64, lib.r2o_sgm_subpixel,
                  lib.r2o_cost_right, lib.r2o_ncc_cost, lib.r2o_ncc_cost_right, lib.r2o_rectify,
                  lib.r2o_s_at):
            f.restype = ctypes.c_int
        _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


def _check(rc: int, what: str):
    if rc != 0:
        raise ValueError(f"oracle {what} rejected its arguments (rc={rc})")


def census(img: np.ndarray, cw: int, ch: int) -> np.ndarray:
    img = np.ascontiguousarray(img, dtype=np.uint8)
    H, W = img.shape
    out = np.empty((H, W), np.uint64)
    _check(_load().r2o_census(_ptr(img), W, W, H, cw, ch, _ptr(out)), "census")
    return out


def cost(ctl: np.ndarray, ctr: np.ndarray, D: int) -> np.ndarray:
    ctl = np.ascontiguousarray(ctl, dtype=np.uint64)
    ctr = np.ascontiguousarray(ctr, dtype=np.uint64)
    H, W = ctl.shape
    out = np.empty((H, W, D), np.uint8)
    _check(_load().r2o_cost(_ptr(ctl), _ptr(ctr), W, H, D, _ptr(out)), "cost")
    return out


def cost_right(ctl: np.ndarray, ctr: np.ndarray, D: int) -> np.ndarray:
    """Right-reference cost C^R(x, y, d) = popcount(CT_R(x, y) ^ CT_L(x + d, y)), 255 outside."""
    ctl = np.ascontiguousarray(ctl, dtype=np.uint64)
    ctr = np.ascontiguousarray(ctr, dtype=np.uint64)
    H, W = ctl.shape
    out = np.empty((H, W, D), np.uint8)
    _check(_load().r2o_cost_right(_ptr(ctl), _ptr(ctr), W, H, D, _ptr(out)), "cost_right")
    return out


def ncc_round(cov: int, va: int, vb: int) -> int:
    """k = round(255 max(0, cov / sqrt(va vb))), ties to even, decided on integers (the scaling
    of the NCC cost; the cost is 255 - k)."""
    return int(_load().r2o_ncc_round(int(cov), int(va), int(vb)))


def ncc_cost(left: np.ndarray, right: np.ndarray, D: int, n: int,
             right_reference: bool = False) -> np.ndarray:
    """Inverted, truncated NCC cost on 0..255 over n x n patches (left image as reference, or
    the right one for the exact consistency check)."""
    left = np.ascontiguousarray(left, dtype=np.uint8)
    right = np.ascontiguousarray(right, dtype=np.uint8)
    H, W = left.shape
    out = np.empty((H, W, D), np.uint8)
    f = _load().r2o_ncc_cost_right if right_reference else _load().r2o_ncc_cost
    _check(f(_ptr(left), _ptr(right), W, W, H, D, n, _ptr(out)), "ncc_cost")
    return out


def path(cost_vol: np.ndarray, direction, P1: int, P2: int) -> np.ndarray:
    cost_vol = np.ascontiguousarray(cost_vol, dtype=np.uint8)
    H, W, D = cost_vol.shape
    out = np.empty((H, W, D), np.uint16)
    dx, dy = direction
    _check(_load().r2o_path(_ptr(cost_vol), W, H, D, dx, dy, P1, P2, _ptr(out)), "path")
    return out


def aggregate(cost_vol: np.ndarray, R: int, P1: int, P2: int) -> np.ndarray:
    cost_vol = np.ascontiguousarray(cost_vol, dtype=np.uint8)
    H, W, D = cost_vol.shape
    out = np.empty((H, W, D), np.uint16)
    _check(_load().r2o_aggregate(_ptr(cost_vol), W, H, D, R, P1, P2, _ptr(out)), "aggregate")
    return out


def wta(S: np.ndarray) -> np.ndarray:
    S = np.ascontiguousarray(S, dtype=np.uint16)
    H, W, D = S.shape
    out = np.empty((H, W), np.uint16)
    _check(_load().r2o_wta(_ptr(S), W, H, D, _ptr(out)), "wta")
    return out


def right_disparity(S: np.ndarray) -> np.ndarray:
    S = np.ascontiguousarray(S, dtype=np.uint16)
    H, W, D = S.shape
    out = np.empty((H, W), np.uint16)
    _check(_load().r2o_right_disparity(_ptr(S), W, H, D, _ptr(out)), "right_disparity")
    return out


def lr_check(DL: np.ndarray, DR: np.ndarray, threshold: int = 1):
    DL = np.ascontiguousarray(DL, dtype=np.uint16)
    DR = np.ascontiguousarray(DR, dtype=np.uint16)
    H, W = DL.shape
    out = np.empty((H, W), np.uint16)
    mask = np.empty((H, W), np.uint8)
    _check(_load().r2o_lr_check(_ptr(DL), _ptr(DR), W, H, threshold, _ptr(out), _ptr(mask)),
           "lr_check")
    return out, mask


def median3x3(Din: np.ndarray) -> np.ndarray:
    Din = np.ascontiguousarray(Din, dtype=np.uint16)
    H, W = Din.shape
    out = np.empty((H, W), np.uint16)
    _check(_load().r2o_median3x3(_ptr(Din), W, H, _ptr(out)), "median3x3")
    return out


def sgm(left: np.ndarray, right: np.ndarray, D: int, census_w: int, census_h: int, P1: int,
        P2: int, num_paths: int, flags: int, lr_threshold: int = 1, debug: bool = False):
    """Whole pipeline. Returns the final map, or (map, dict of intermediates) when debug."""
    left = np.ascontiguousarray(left, dtype=np.uint8)
    right = np.ascontiguousarray(right, dtype=np.uint8)
    H, W = left.shape
    disp = np.empty((H, W), np.uint16)
    null = ctypes.c_void_p(None)
    if debug:
        dbg = {
            "cost": np.empty((H, W, D), np.uint8),
            "agg": np.empty((H, W, D), np.uint16),
            "dl": np.empty((H, W), np.uint16),
            "dr": np.empty((H, W), np.uint16),
            "mask": np.empty((H, W), np.uint8),
        }
        ptrs = [_ptr(dbg[k]) for k in ("cost", "agg", "dl", "dr", "mask")]
    else:
        ptrs = [null] * 5
    rc = _load().r2o_sgm(_ptr(left), _ptr(right), W, W, H, D, census_w, census_h, P1, P2,
                         num_paths, flags, lr_threshold, _ptr(disp), *ptrs)
    _check(rc, "sgm")
    return (disp, dbg) if debug else disp


def subpixel(S: np.ndarray, DL: np.ndarray) -> np.ndarray:
    """Sub-pixel D^L (float64) from the aggregated volume and the integer D^L (Sec. 2.1.3)."""
    S = np.ascontiguousarray(S, dtype=np.uint16)
    DL = np.ascontiguousarray(DL, dtype=np.uint16)
    H, W, D = S.shape
    out = np.empty((H, W), np.float64)
    _check(_load().r2o_subpixel(_ptr(S), _ptr(DL), W, H, D, _ptr(out)), "subpixel")
    return out


def median3x3_f64(Din: np.ndarray) -> np.ndarray:
    Din = np.ascontiguousarray(Din, dtype=np.float64)
    H, W = Din.shape
    out = np.empty((H, W), np.float64)
    _check(_load().r2o_median3x3_f64(_ptr(Din), W, H, _ptr(out)), "median3x3_f64")
    return out


def sgm_subpixel(left: np.ndarray, right: np.ndarray, D: int, census_w: int, census_h: int,
                 P1: int, P2: int, num_paths: int, flags: int, lr_threshold: int = 1):
    """Whole pipeline with the sub-pixel refinement. Returns (final map, refined D^L), float64,
    +inf where invalid."""
    left = np.ascontiguousarray(left, dtype=np.uint8)
    right = np.ascontiguousarray(right, dtype=np.uint8)
    H, W = left.shape
    disp = np.empty((H, W), np.float64)
    ref = np.empty((H, W), np.float64)
    rc = _load().r2o_sgm_subpixel(_ptr(left), _ptr(right), W, W, H, D, census_w, census_h, P1,
                                  P2, num_paths, flags, lr_threshold, _ptr(disp), _ptr(ref))
    _check(rc, "sgm_subpixel")
    return disp, ref


def rectify(raw: np.ndarray, mapx: np.ndarray, mapy: np.ndarray) -> np.ndarray:
    """Rectified image [H, W] from a raw image and float32 maps [H, W] of source coordinates."""
    raw = np.ascontiguousarray(raw, dtype=np.uint8)
    mapx = np.ascontiguousarray(mapx, dtype=np.float32)
    mapy = np.ascontiguousarray(mapy, dtype=np.float32)
    rh, rw = raw.shape
    H, W = mapx.shape
    out = np.empty((H, W), np.uint8)
    _check(_load().r2o_rectify(_ptr(raw), rw, rw, rh, _ptr(mapx), _ptr(mapy), 4 * W, W, H,
                               _ptr(out), W), "rectify")
    return out


def s_at(left: np.ndarray, right: np.ndarray, D: int, census_w: int, census_h: int, P1: int,
         P2: int, num_paths: int, flags: int, x: int, y: int) -> np.ndarray:
    """S(x, y, .) (uint16, saturated) from the path lines through one pixel."""
    left = np.ascontiguousarray(left, dtype=np.uint8)
    right = np.ascontiguousarray(right, dtype=np.uint8)
    H, W = left.shape
    out = np.empty(D, np.uint16)
    _check(_load().r2o_s_at(_ptr(left), _ptr(right), W, W, H, D, census_w, census_h, P1, P2,
                            num_paths, flags, x, y, _ptr(out)), "s_at")
    return out
