"""Seeded synthetic stereo pairs shaped like the paper's workloads.

The paper measures on KITTI 2015 (1242x375) and Middlebury 2014 Q pairs (Sec. 3.1); neither
dataset is used here. These generators stand in for them: rectified 8-bit grayscale pairs with a
known integer disparity field, so both the CUDA library and the CPU oracle read identical bytes.
This module holds only the input recipes (noise, blur, warps); none of the stereo method's
arithmetic. numpy only, deterministic for a given seed.

Scene kinds:
  "rects"   320x240-style: blurred uniform noise, d = 0 background plus 6 fronto-parallel
            rectangles with d in 5..50, right = warp + N(0, 2).
  "road"    KITTI-like: ground plane whose disparity rises linearly to 110 at the bottom row,
            20 slanted planes (rectangles / ellipses) with d = a + b x + c y, 4-octave value-noise
            texture, right = rounded warp + N(0, 3).
  "nadir"   aerial: d = 40 + 60 * diamond-square heightmap (roughness 0.6) + 30 boxes of +10..40,
            band-limited texture with 10 % of the area in constant patches dithered by +-1.
Disparities of "road" and "nadir" are scaled by D / 128 so the field fits the searched range.
"""
from __future__ import annotations

import numpy as np

FLAG_LR_CHECK = 1
FLAG_MEDIAN = 2

BATCH_WIDTHS = (320, 640, 1024, 1242, 1920)
BATCH_HEIGHTS = (240, 375, 512, 768, 1080)
BATCH_DISPS = (64, 128, 256)


def _gauss_kernel(sigma: float) -> np.ndarray:
    r = int(np.ceil(3 * sigma))
    t = np.arange(-r, r + 1, dtype=np.float64)
    k = np.exp(-0.5 * (t / sigma) ** 2)
    return k / k.sum()


def _blur(a: np.ndarray, sigma: float) -> np.ndarray:
    k = _gauss_kernel(sigma)
    r = len(k) // 2
    p = np.pad(a, ((0, 0), (r, r)), mode="reflect")
    a = sum(k[i] * p[:, i:i + a.shape[1]] for i in range(len(k)))
    p = np.pad(a, ((r, r), (0, 0)), mode="reflect")
    return sum(k[i] * p[i:i + a.shape[0], :] for i in range(len(k)))


def _to_u8(a: np.ndarray) -> np.ndarray:
    lo, hi = float(a.min()), float(a.max())
    if hi <= lo:
        return np.zeros(a.shape, np.uint8)
    return np.clip(np.rint((a - lo) / (hi - lo) * 255.0), 0, 255).astype(np.uint8)


def _bilinear_grid(rng, H: int, W: int, cell: float) -> np.ndarray:
    gh, gw = int(np.ceil(H / cell)) + 2, int(np.ceil(W / cell)) + 2
    g = rng.random((gh, gw))
    ys = np.arange(H) / cell
    xs = np.arange(W) / cell
    y0, x0 = np.floor(ys).astype(int), np.floor(xs).astype(int)
    fy, fx = (ys - y0)[:, None], (xs - x0)[None, :]
    a = g[y0][:, x0]
    b = g[y0][:, x0 + 1]
    c = g[y0 + 1][:, x0]
    d = g[y0 + 1][:, x0 + 1]
    return (a * (1 - fx) + b * fx) * (1 - fy) + (c * (1 - fx) + d * fx) * fy


def value_noise(rng, H: int, W: int, octaves: int = 4, base_cell: float = 32.0) -> np.ndarray:
    out = np.zeros((H, W))
    amp, cell = 1.0, base_cell
    for _ in range(octaves):
        out += amp * _bilinear_grid(rng, H, W, max(cell, 1.0))
        amp *= 0.5
        cell /= 2.0
    return out


def diamond_square(rng, H: int, W: int, roughness: float = 0.6) -> np.ndarray:
    n = 1
    while (1 << n) + 1 < max(H, W):
        n += 1
    size = (1 << n) + 1
    h = np.zeros((size, size))
    h[0, 0], h[0, -1], h[-1, 0], h[-1, -1] = rng.random(4)
    step, scale = size - 1, 1.0
    while step > 1:
        half = step // 2
        corners = h[0::step, 0::step]  # (n+1, n+1)
        # diamond step: centres of squares
        avg = (corners[:-1, :-1] + corners[:-1, 1:] + corners[1:, :-1] + corners[1:, 1:]) / 4.0
        h[half::step, half::step] = avg + (rng.random(avg.shape) - 0.5) * scale
        cent = h[half::step, half::step]  # (n, n)
        nanrow = np.full((1, cent.shape[1]), np.nan)
        nancol = np.full((cent.shape[0], 1), np.nan)
        # square step, horizontal edge midpoints (y = k*step, x = half + k*step)
        up = np.vstack([nanrow, cent])
        down = np.vstack([cent, nanrow])
        nb = np.stack([corners[:, :-1], corners[:, 1:], up, down])
        mid = np.nanmean(nb, axis=0)
        h[0::step, half::step] = mid + (rng.random(mid.shape) - 0.5) * scale
        # square step, vertical edge midpoints (y = half + k*step, x = k*step)
        lft = np.hstack([nancol, cent])
        rgt = np.hstack([cent, nancol])
        nb = np.stack([corners[:-1, :], corners[1:, :], lft, rgt])
        mid = np.nanmean(nb, axis=0)
        h[half::step, 0::step] = mid + (rng.random(mid.shape) - 0.5) * scale
        step = half
        scale *= roughness
    h = h[:H, :W]
    return (h - h.min()) / max(h.max() - h.min(), 1e-12)


def band_noise(rng, H: int, W: int, f_lo: float = 0.02, f_hi: float = 0.25) -> np.ndarray:
    spec = np.fft.rfft2(rng.standard_normal((H, W)))
    fy = np.fft.fftfreq(H)[:, None]
    fx = np.fft.rfftfreq(W)[None, :]
    f = np.sqrt(fx * fx + fy * fy)
    spec[(f < f_lo) | (f > f_hi)] = 0
    return np.fft.irfft2(spec, s=(H, W))


def forward_warp(rng, left: np.ndarray, disp: np.ndarray) -> np.ndarray:
    """Right image R(x - d, y) = L(x, y), nearer surfaces (larger d) written last; holes get
    fresh uniform noise."""
    H, W = left.shape
    right = np.full(H * W, -1, np.int32)
    ys, xs = np.mgrid[0:H, 0:W]
    d = disp.astype(np.int64).ravel()
    xr = xs.ravel() - d
    ok = xr >= 0
    tgt = (ys.ravel() * W + xr)[ok]
    src = left.ravel()[ok]
    dk = d[ok]
    order = np.lexsort((dk, tgt))  # by target, then by disparity ascending
    tgt_s = tgt[order]
    last = np.ones(tgt_s.shape, bool)
    last[:-1] = tgt_s[1:] != tgt_s[:-1]  # the largest d per target wins (z-order)
    right[tgt_s[last]] = src[order][last]
    right = right.reshape(H, W)
    holes = right < 0
    right[holes] = rng.integers(0, 256, int(holes.sum()))
    return right.astype(np.uint8)


def _add_noise(rng, img: np.ndarray, sigma: float) -> np.ndarray:
    noisy = img.astype(np.float64) + rng.normal(0.0, sigma, img.shape)
    return np.clip(np.rint(noisy), 0, 255).astype(np.uint8)


def scene_rects(seed: int, W: int = 320, H: int = 240, D: int = 64):
    rng = np.random.default_rng(seed)
    left = _to_u8(_blur(rng.random((H, W)), 1.5))
    disp = np.zeros((H, W), np.int32)
    for _ in range(6):
        w, h = int(rng.integers(W // 10, W // 3)), int(rng.integers(H // 10, H // 3))
        x0, y0 = int(rng.integers(0, W - w)), int(rng.integers(0, H - h))
        dv = int(rng.integers(5, 51))
        disp[y0:y0 + h, x0:x0 + w] = np.maximum(disp[y0:y0 + h, x0:x0 + w], min(dv, D - 1))
    right = _add_noise(rng, forward_warp(rng, left, disp), 2.0)
    return left, right, disp


def scene_road(seed: int, W: int = 1242, H: int = 375, D: int = 128):
    rng = np.random.default_rng(seed)
    s = D / 128.0
    left = _to_u8(value_noise(rng, H, W, octaves=4, base_cell=24.0))
    dfield = np.repeat((110.0 * np.arange(H) / max(H - 1, 1))[:, None], W, axis=1)
    for _ in range(20):
        cx, cy = rng.uniform(0, W), rng.uniform(0, H)
        rw, rh = rng.uniform(W / 30, W / 6), rng.uniform(H / 20, H / 4)
        a = rng.uniform(2, 120)
        b, c = rng.uniform(-0.2, 0.2, 2)
        box = rng.random() < 0.5
        x0, x1 = max(int(np.floor(cx - rw)), 0), min(int(np.ceil(cx + rw)) + 1, W)
        y0, y1 = max(int(np.floor(cy - rh)), 0), min(int(np.ceil(cy + rh)) + 1, H)
        yy, xx = np.mgrid[y0:y1, x0:x1].astype(np.float64)
        if box:
            inside = (np.abs(xx - cx) <= rw) & (np.abs(yy - cy) <= rh)
        else:
            inside = ((xx - cx) / rw) ** 2 + ((yy - cy) / rh) ** 2 <= 1.0
        plane = a + b * (xx - cx) + c * (yy - cy)
        sub = dfield[y0:y1, x0:x1]
        dfield[y0:y1, x0:x1] = np.where(inside, np.maximum(sub, plane), sub)
    disp = np.clip(np.rint(dfield * s), 0, D - 1).astype(np.int32)
    right = _add_noise(rng, forward_warp(rng, left, disp), 3.0)
    return left, right, disp


def scene_nadir(seed: int, W: int = 1024, H: int = 768, D: int = 128):
    rng = np.random.default_rng(seed)
    s = D / 128.0
    dfield = 40.0 + 60.0 * diamond_square(rng, H, W, 0.6)
    for _ in range(30):
        w, h = int(rng.integers(W // 40 + 1, W // 8 + 2)), int(rng.integers(H // 40 + 1, H // 8 + 2))
        x0, y0 = int(rng.integers(0, max(W - w, 1))), int(rng.integers(0, max(H - h, 1)))
        dfield[y0:y0 + h, x0:x0 + w] += rng.uniform(10, 40)
    disp = np.clip(np.rint(dfield * s), 0, D - 1).astype(np.int32)
    tex = _to_u8(band_noise(rng, H, W)).astype(np.int32)
    covered, target = 0, 0.10 * W * H
    while covered < target:
        w, h = int(rng.integers(8, max(W // 10, 9))), int(rng.integers(8, max(H // 10, 9)))
        x0, y0 = int(rng.integers(0, max(W - w, 1))), int(rng.integers(0, max(H - h, 1)))
        c = int(rng.integers(2, 254))
        tex[y0:y0 + h, x0:x0 + w] = c + rng.integers(-1, 2, (min(h, H - y0), min(w, W - x0)))
        covered += w * h
    left = np.clip(tex, 0, 255).astype(np.uint8)
    right = _add_noise(rng, forward_warp(rng, left, disp), 1.0)
    return left, right, disp


def params(W, H, D, census_w, census_h, P1, P2, num_paths, flags, lr_threshold=1) -> dict:
    return dict(width=W, height=H, max_disp=D, census_w=census_w, census_h=census_h, p1=P1,
                p2=P2, num_paths=num_paths, flags=flags, lr_threshold=lr_threshold)


# The three single-pair workloads: 320x240 D=64 5x5 4 paths WTA only; 1242x375 D=128 9x7
# 8 paths with LR check + median; 1024x768 D=128 9x7 8 paths, P1=8 P2=96, LR check + median.
SINGLE = {
    "320x240_d64_ct5x5_r4": dict(kind="rects", prm=params(320, 240, 64, 5, 5, 10, 120, 4, 0)),
    "1242x375_d128_ct9x7_r8": dict(kind="road", prm=params(1242, 375, 128, 9, 7, 10, 120, 8,
                                                         FLAG_LR_CHECK | FLAG_MEDIAN)),
    "1024x768_d128_ct9x7_r8": dict(kind="nadir", prm=params(1024, 768, 128, 9, 7, 8, 96, 8,
                                                          FLAG_LR_CHECK | FLAG_MEDIAN)),
}

_KINDS = {"rects": scene_rects, "road": scene_road, "nadir": scene_nadir}


def make_scene(kind: str, seed: int, W: int, H: int, D: int):
    return _KINDS[kind](seed, W, H, D)


def single_pair(name: str, seed: int = 0):
    """(left, right, gt_disparity, params) of one named single-pair workload."""
    w = SINGLE[name]
    p = w["prm"]
    left, right, gt = make_scene(w["kind"], seed, p["width"], p["height"], p["max_disp"])
    return left, right, gt, dict(p)


def batch_specs(seed: int = 0, n: int = 64, big_fraction: float = 0.0):
    """Sizes of a batch of uneven pairs: W, H, D drawn uniformly from the listed sets, scene kind
    "road" or "nadir" by coin flip; with big_fraction > 0 that share are 3840x2160, D = 256."""
    rng = np.random.default_rng(seed)
    specs = []
    for i in range(n):
        if big_fraction > 0 and rng.random() < big_fraction:
            W, H, D = 3840, 2160, 256
        else:
            W = int(rng.choice(BATCH_WIDTHS))
            H = int(rng.choice(BATCH_HEIGHTS))
            D = int(rng.choice(BATCH_DISPS))
        kind = "road" if rng.random() < 0.5 else "nadir"
        specs.append(dict(kind=kind, seed=seed * 100003 + i,
                          prm=params(W, H, D, 9, 7, 10, 120, 8, FLAG_LR_CHECK | FLAG_MEDIAN)))
    return specs


def batch_pairs(seed: int = 0, n: int = 64, big_fraction: float = 0.0):
    out = []
    for s in batch_specs(seed, n, big_fraction):
        p = s["prm"]
        left, right, gt = make_scene(s["kind"], s["seed"], p["width"], p["height"], p["max_disp"])
        out.append((left, right, gt, dict(p)))
    return out


def rectification_maps(seed: int, W: int, H: int, raw_w: int | None = None,
                       raw_h: int | None = None, strength: float = 1.0):
    """Seeded float32 maps (mapx, mapy) [H, W] of a calibration-like rectification: for each
    rectified pixel the source coordinate in a raw_w x raw_h image under a small in-plane rotation
    (up to 1 degree), a sub-pixel shift and radial lens distortion (|k1| <= 0.08 at the image
    corners). These are inputs, as a calibration routine would deliver them; no matching here."""
    raw_w = raw_w or W
    raw_h = raw_h or H
    rng = np.random.default_rng(seed)
    f = 0.9 * max(W, H)
    theta = np.deg2rad(rng.uniform(-1.0, 1.0)) * strength
    k1 = rng.uniform(-0.08, 0.08) * strength
    tx, ty = rng.uniform(-1.5, 1.5, size=2) * strength
    v, u = np.mgrid[0:H, 0:W].astype(np.float64)
    xn, yn = (u - (W - 1) / 2) / f, (v - (H - 1) / 2) / f
    c, s = np.cos(theta), np.sin(theta)
    xr, yr = c * xn - s * yn, s * xn + c * yn
    corner2 = max(((W - 1) / 2 / f) ** 2 + ((H - 1) / 2 / f) ** 2, 1e-12)
    r2 = (xr * xr + yr * yr) / corner2
    xd, yd = xr * (1 + k1 * r2), yr * (1 + k1 * r2)
    mapx = f * xd + (raw_w - 1) / 2 + tx
    mapy = f * yd + (raw_h - 1) / 2 + ty
    return mapx.astype(np.float32), mapy.astype(np.float32)
