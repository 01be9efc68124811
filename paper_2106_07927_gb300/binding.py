"""Thin ctypes binding of libres2tac.so (include/res2tac.h), argument marshalling only.

Every compute call goes through the CUDA library; there is no Python or CPU fallback. If the
library is not built this module raises at load time. Functions keep the C names; device
buffers are passed as integer device pointers (e.g. ``tensor.data_ptr()``) and streams as
integer ``cudaStream_t`` handles (e.g. ``torch.cuda.current_stream().cuda_stream``).
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

RES2TAC_OK = 0
RES2TAC_EINVAL = -1
RES2TAC_ENOMEM = -2
RES2TAC_ECUDA = -3
RES2TAC_ETIMEOUT = -4
RES2TAC_LR_CHECK = 1
RES2TAC_MEDIAN = 2
RES2TAC_EXACT_CC = 4
RES2TAC_NCC = 8
RES2TAC_INVALID = 0xFFFF

# Every symbol include/res2tac.h declares (checked by the tests).
EXPORTS = (
    "res2tac_create", "res2tac_compute", "res2tac_compute_host", "res2tac_compute_batch",
    "res2tac_debug_outputs", "res2tac_workspace_bytes", "res2tac_batch_workspace_bytes",
    "res2tac_get_tuning", "res2tac_set_tuning", "res2tac_autotune", "res2tac_last_launch_count",
    "res2tac_destroy", "res2tac_strerror", "res2tac_last_error", "res2tac_set_profiling",
    "res2tac_stage_times",
    "res2tac_batch_reserve",
    "res2tac_compute_static",
    "res2tac_compute_subpixel", "res2tac_debug_subpixel",
    "res2tac_rectify", "res2tac_set_rectification", "res2tac_compute_raw",
    "res2tac_set_batch_tuning", "res2tac_get_batch_tuning", "res2tac_autotune_batch",
)
# Every symbol include/res2tac_measure.h declares (measurement aids of the benchmark).
MEASURE_EXPORTS = ("res2tac_probe_int_peak", "res2tac_probe_red_peak", "res2tac_probe_popc_rate",
                   "res2tac_bounds_status")
RES2TAC_STATIC_SCRATCH_BYTES = 80 << 20
STAGES = ("census_cost", "aggregate", "wta_dr", "lr_median")


class res2tac_params(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int32) for n in (
        "width", "height", "max_disp", "census_w", "census_h", "p1", "p2", "num_paths", "flags",
        "lr_threshold")]


class res2tac_pair(ctypes.Structure):
    _fields_ = [("left", ctypes.c_void_p), ("right", ctypes.c_void_p), ("in_pitch", ctypes.c_int64),
                ("disp", ctypes.c_void_p), ("out_pitch", ctypes.c_int64),
                ("width", ctypes.c_int32), ("height", ctypes.c_int32),
                ("max_disp", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class res2tac_tuning(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int32) for n in ("agg_dpl", "agg_warps", "wta_chunk", "shear_dpl",
                                               "row_mode", "shear_cpl", "cost_mode",
                                               "row_cost")]


class res2tac_batch_tuning(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int32) for n in ("max_disp", "large", "row_dpl", "shear_dpl",
                                               "shear_cpl", "wta_px")]

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_}


class Res2tacError(RuntimeError):
    def __init__(self, code: int, message: str):
        super().__init__(f"res2tac error {code}: {message}")
        self.code = code


_lib = None


def library_path() -> str:
    return _build.LIB


def load(path: str | None = None):
    """Loads libres2tac.so (or the library at path); raises if it has not been built (no
    fallback exists)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    path = path or _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(
            "libres2tac.so is not built: run `python -c 'import __graft_entry__ as g; g.build()'` "
            "(needs nvcc); the SGM path has no CPU fallback")
    lib = ctypes.CDLL(path)
    P, I32, I64, S = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t
    PP = ctypes.POINTER(res2tac_params)
    sig = {
        "res2tac_create": (ctypes.c_int, [PP, ctypes.POINTER(ctypes.c_void_p)]),
        "res2tac_compute": (ctypes.c_int, [P, P, P, I64, P, I64, P]),
        "res2tac_compute_host": (ctypes.c_int, [P, P, P, I64, P, I64, P]),
        "res2tac_compute_batch": (ctypes.c_int, [P, ctypes.POINTER(res2tac_pair), I32, P]),
        "res2tac_debug_outputs": (ctypes.c_int, [P, P, P, P, P, P, P]),
        "res2tac_workspace_bytes": (S, [PP]),
        "res2tac_batch_workspace_bytes": (S, [PP, ctypes.POINTER(res2tac_pair), I32]),
        "res2tac_get_tuning": (ctypes.c_int, [P, ctypes.POINTER(res2tac_tuning)]),
        "res2tac_set_tuning": (ctypes.c_int, [P, ctypes.POINTER(res2tac_tuning)]),
        "res2tac_autotune": (ctypes.c_int, [P, P, P, I64, P, I64, P,
                                            ctypes.POINTER(res2tac_tuning)]),
        "res2tac_last_launch_count": (ctypes.c_int, [P]),
        "res2tac_destroy": (None, [P]),
        "res2tac_strerror": (ctypes.c_char_p, [ctypes.c_int]),
        "res2tac_last_error": (ctypes.c_char_p, []),
        "res2tac_set_profiling": (ctypes.c_int, [P, ctypes.c_int]),
        "res2tac_stage_times": (ctypes.c_int, [P, ctypes.POINTER(ctypes.c_float), ctypes.c_int]),
        "res2tac_probe_int_peak": (ctypes.c_int, [ctypes.c_int, P,
                                                  ctypes.POINTER(ctypes.c_double)]),
        "res2tac_probe_red_peak": (ctypes.c_int, [I64, I32, P, ctypes.POINTER(ctypes.c_double)]),
        "res2tac_batch_reserve": (ctypes.c_int, [P, S, I32]),
        "res2tac_compute_static": (ctypes.c_int, [PP, P, P, I64, P, I64, P]),
        "res2tac_compute_subpixel": (ctypes.c_int, [P, P, P, I64, P, I64, P]),
        "res2tac_debug_subpixel": (ctypes.c_int, [P, P, P]),
        "res2tac_rectify": (ctypes.c_int, [P, I64, I32, I32, P, P, I64, P, I64, I32, I32, P]),
        "res2tac_set_rectification": (ctypes.c_int, [P, P, P, P, P, I64, I32, I32, P]),
        "res2tac_compute_raw": (ctypes.c_int, [P, P, P, I64, P, I64, P]),
        "res2tac_set_batch_tuning": (ctypes.c_int, [P, ctypes.POINTER(res2tac_batch_tuning), I32]),
        "res2tac_probe_popc_rate": (ctypes.c_int, [ctypes.c_int, P,
                                                   ctypes.POINTER(ctypes.c_double)]),
        "res2tac_bounds_status": (ctypes.c_int, [P, ctypes.POINTER(I32), ctypes.POINTER(I32),
                                                 ctypes.POINTER(I64)]),
        "res2tac_get_batch_tuning": (ctypes.c_int, [P, ctypes.POINTER(res2tac_batch_tuning)]),
        "res2tac_autotune_batch": (ctypes.c_int, [P, ctypes.POINTER(res2tac_pair), I32, P,
                                                  ctypes.POINTER(res2tac_batch_tuning), I32,
                                                  ctypes.POINTER(I32),
                                                  ctypes.POINTER(ctypes.c_float),
                                                  ctypes.POINTER(ctypes.c_float)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def use_check_library(on: bool = True):
    """Switches every function of this module to the debug build with range checks
    (libres2tac_check.so, built on first use) or, with on=False, back to libres2tac.so."""
    global _lib
    _lib = None
    return load(_build.build(check=True) if on else None)


def res2tac_bounds_status(h: int) -> tuple:
    """(checked, site, byte offset) of the context's range-check record."""
    c, s, o = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int64()
    _check(load().res2tac_bounds_status(h, ctypes.byref(c), ctypes.byref(s), ctypes.byref(o)))
    return c.value, s.value, o.value


def _check(rc: int):
    if rc != RES2TAC_OK:
        lib = load()
        raise Res2tacError(rc, lib.res2tac_last_error().decode(errors="replace"))


def make_params(width, height, max_disp, census_w=9, census_h=7, p1=10, p2=120, num_paths=8,
                flags=RES2TAC_LR_CHECK | RES2TAC_MEDIAN, lr_threshold=1) -> res2tac_params:
    return res2tac_params(width, height, max_disp, census_w, census_h, p1, p2, num_paths, flags,
                          lr_threshold)


def params_from_dict(d: dict) -> res2tac_params:
    return make_params(d["width"], d["height"], d["max_disp"], d["census_w"], d["census_h"],
                       d["p1"], d["p2"], d["num_paths"], d["flags"], d.get("lr_threshold", 1))


# --------------------------------------------------------------------------- same-name wrappers
def res2tac_create(params: res2tac_params) -> int:
    h = ctypes.c_void_p()
    _check(load().res2tac_create(ctypes.byref(params), ctypes.byref(h)))
    return h.value


def res2tac_compute(h: int, left: int, right: int, in_pitch: int, disp: int, out_pitch: int,
                    stream: int = 0) -> None:
    _check(load().res2tac_compute(h, left, right, in_pitch, disp, out_pitch, stream))


def res2tac_compute_host(h: int, left: int, right: int, in_pitch: int, disp: int, out_pitch: int,
                         stream: int = 0) -> None:
    _check(load().res2tac_compute_host(h, left, right, in_pitch, disp, out_pitch, stream))


def res2tac_compute_subpixel(h: int, left: int, right: int, in_pitch: int, disp: int,
                             out_pitch: int, stream: int = 0) -> None:
    """Pipeline with sub-pixel refinement; disp is a device float map (+inf = invalid)."""
    _check(load().res2tac_compute_subpixel(h, left, right, in_pitch, disp, out_pitch, stream))


def res2tac_rectify(raw: int, raw_pitch: int, raw_w: int, raw_h: int, mapx: int, mapy: int,
                    map_pitch: int, out: int, out_pitch: int, width: int, height: int,
                    stream: int = 0) -> None:
    _check(load().res2tac_rectify(raw, raw_pitch, raw_w, raw_h, mapx, mapy, map_pitch, out,
                                  out_pitch, width, height, stream))


def res2tac_set_rectification(h: int, mapx_l: int, mapy_l: int, mapx_r: int, mapy_r: int,
                              map_pitch: int, raw_w: int, raw_h: int, stream: int = 0) -> None:
    _check(load().res2tac_set_rectification(h, mapx_l, mapy_l, mapx_r, mapy_r, map_pitch, raw_w,
                                            raw_h, stream))


def res2tac_compute_raw(h: int, raw_left: int, raw_right: int, raw_pitch: int, disp: int,
                        out_pitch: int, stream: int = 0) -> None:
    _check(load().res2tac_compute_raw(h, raw_left, raw_right, raw_pitch, disp, out_pitch, stream))


def res2tac_debug_subpixel(h: int, dl_sub: int, stream: int = 0) -> None:
    _check(load().res2tac_debug_subpixel(h, dl_sub, stream))


def res2tac_compute_static(params: res2tac_params, left: int, right: int, in_pitch: int,
                           disp: int, out_pitch: int, stream: int = 0) -> None:
    """No-allocation variant of res2tac_compute: no context; scratch is the library's fixed
    device array (RES2TAC_STATIC_SCRATCH_BYTES), shared by every call."""
    _check(load().res2tac_compute_static(ctypes.byref(params), left, right, in_pitch, disp,
                                         out_pitch, stream))


def res2tac_compute_batch(h: int, pairs, stream: int = 0) -> None:
    arr = (res2tac_pair * len(pairs))(*pairs)
    _check(load().res2tac_compute_batch(h, arr, len(pairs), stream))


def res2tac_debug_outputs(h: int, cost=0, agg=0, dl=0, dr=0, mask=0, stream: int = 0) -> None:
    _check(load().res2tac_debug_outputs(h, cost or None, agg or None, dl or None, dr or None,
                                        mask or None, stream))


def res2tac_workspace_bytes(params: res2tac_params) -> int:
    return int(load().res2tac_workspace_bytes(ctypes.byref(params)))


def res2tac_batch_workspace_bytes(params: res2tac_params, pairs) -> int:
    arr = (res2tac_pair * len(pairs))(*pairs)
    return int(load().res2tac_batch_workspace_bytes(ctypes.byref(params), arr, len(pairs)))


def res2tac_batch_reserve(h: int, scratch_bytes: int, max_pairs: int) -> None:
    _check(load().res2tac_batch_reserve(h, scratch_bytes, max_pairs))


def res2tac_get_tuning(h: int) -> res2tac_tuning:
    t = res2tac_tuning()
    _check(load().res2tac_get_tuning(h, ctypes.byref(t)))
    return t


def res2tac_set_tuning(h: int, t: res2tac_tuning) -> None:
    _check(load().res2tac_set_tuning(h, ctypes.byref(t)))


def res2tac_autotune(h: int, left: int, right: int, in_pitch: int, disp: int, out_pitch: int,
                     stream: int = 0) -> res2tac_tuning:
    t = res2tac_tuning()
    _check(load().res2tac_autotune(h, left, right, in_pitch, disp, out_pitch, stream,
                                   ctypes.byref(t)))
    return t


def res2tac_last_launch_count(h: int) -> int:
    return int(load().res2tac_last_launch_count(h))


def res2tac_set_profiling(h: int, enable: bool) -> None:
    _check(load().res2tac_set_profiling(h, 1 if enable else 0))


def res2tac_stage_times(h: int) -> dict:
    ms = (ctypes.c_float * len(STAGES))()
    _check(load().res2tac_stage_times(h, ms, len(STAGES)))
    return dict(zip(STAGES, [float(v) for v in ms]))


def res2tac_set_batch_tuning(h: int, entries) -> None:
    arr = (res2tac_batch_tuning * len(entries))(*entries)
    _check(load().res2tac_set_batch_tuning(h, arr, len(entries)))


def res2tac_get_batch_tuning(h: int, max_disp: int, large: int) -> res2tac_batch_tuning:
    t = res2tac_batch_tuning(max_disp, large, 0, 0, 0, 0)
    _check(load().res2tac_get_batch_tuning(h, ctypes.byref(t)))
    return t


def res2tac_autotune_batch(h: int, pairs, stream: int = 0):
    """Returns (table entries of the tuned buckets, batch ms with the defaults, ms tuned)."""
    arr = (res2tac_pair * len(pairs))(*pairs)
    cap = 34
    table = (res2tac_batch_tuning * cap)()
    count = ctypes.c_int32()
    m0, m1 = ctypes.c_float(), ctypes.c_float()
    _check(load().res2tac_autotune_batch(h, arr, len(pairs), stream, table, cap,
                                         ctypes.byref(count), ctypes.byref(m0), ctypes.byref(m1)))
    return [table[i] for i in range(count.value)], m0.value, m1.value


def res2tac_probe_red_peak(nbytes: int, passes: int = 16, stream: int = 0) -> float:
    v = ctypes.c_double()
    _check(load().res2tac_probe_red_peak(nbytes, passes, stream, ctypes.byref(v)))
    return v.value


def res2tac_probe_int_peak(iters: int = 20000, stream: int = 0) -> float:
    v = ctypes.c_double()
    _check(load().res2tac_probe_int_peak(iters, stream, ctypes.byref(v)))
    return v.value


def res2tac_probe_popc_rate(iters: int = 20000, stream: int = 0) -> float:
    v = ctypes.c_double()
    _check(load().res2tac_probe_popc_rate(iters, stream, ctypes.byref(v)))
    return v.value


def res2tac_destroy(h: int) -> None:
    if h:
        load().res2tac_destroy(h)


def res2tac_strerror(code: int) -> str:
    return load().res2tac_strerror(code).decode()


def res2tac_last_error() -> str:
    return load().res2tac_last_error().decode(errors="replace")


# ------------------------------------------------------------------ torch convenience (plumbing)
class Stereo:
    """One context bound to torch CUDA tensors: torch supplies device memory and the stream only;
    all computation happens in the library's kernels."""

    def __init__(self, params):
        self.params = params if isinstance(params, res2tac_params) else params_from_dict(params)
        self.handle = res2tac_create(self.params)

    def close(self):
        if self.handle:
            res2tac_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def _stream():
        import torch
        return torch.cuda.current_stream().cuda_stream

    def compute(self, left, right, out=None):
        """left, right: uint8 CUDA tensors [H, W] (rows may be padded); returns uint16 [H, W]
        stored in an int16 tensor (torch has no uint16 arithmetic on older versions)."""
        import torch
        H, W = self.params.height, self.params.width
        assert left.is_cuda and left.dtype == torch.uint8 and tuple(left.shape) == (H, W)
        assert right.stride() == left.stride() and left.stride(1) == 1
        if out is None:
            out = torch.empty((H, W), dtype=torch.int16, device=left.device)
        res2tac_compute(self.handle, left.data_ptr(), right.data_ptr(), left.stride(0),
                        out.data_ptr(), out.stride(0) * 2, self._stream())
        return out

    def compute_subpixel(self, left, right, out=None):
        """As compute, with sub-pixel refinement: returns a float32 [H, W] map, +inf where the
        left-right check rejected the pixel."""
        import torch
        H, W = self.params.height, self.params.width
        assert left.is_cuda and left.dtype == torch.uint8 and tuple(left.shape) == (H, W)
        assert right.stride() == left.stride() and left.stride(1) == 1
        if out is None:
            out = torch.empty((H, W), dtype=torch.float32, device=left.device)
        res2tac_compute_subpixel(self.handle, left.data_ptr(), right.data_ptr(), left.stride(0),
                                 out.data_ptr(), out.stride(0) * 4, self._stream())
        return out

    def debug_subpixel(self):
        """Sub-pixel D^L (before the check and the median) of the last compute_subpixel."""
        import torch
        H, W = self.params.height, self.params.width
        o = torch.empty((H, W), dtype=torch.float32, device="cuda")
        res2tac_debug_subpixel(self.handle, o.data_ptr(), self._stream())
        return o

    def debug_outputs(self):
        import torch
        H, W, D = self.params.height, self.params.width, self.params.max_disp
        dev = torch.device("cuda")
        o = {
            "cost": torch.empty((H, W, D), dtype=torch.uint8, device=dev),
            "agg": torch.empty((H, W, D), dtype=torch.int16, device=dev),
            "dl": torch.empty((H, W), dtype=torch.int16, device=dev),
            "dr": torch.empty((H, W), dtype=torch.int16, device=dev),
            "mask": torch.empty((H, W), dtype=torch.uint8, device=dev),
        }
        res2tac_debug_outputs(self.handle, o["cost"].data_ptr(), o["agg"].data_ptr(),
                              o["dl"].data_ptr(), o["dr"].data_ptr(), o["mask"].data_ptr(),
                              self._stream())
        return o


def u16(t) -> "numpy.ndarray":
    """int16 torch tensor holding uint16 values -> numpy uint16 array."""
    return t.cpu().numpy().view("uint16")
