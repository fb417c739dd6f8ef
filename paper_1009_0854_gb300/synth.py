"""Seeded synthetic inputs shaped like the paper's workloads.

The paper measures on RGB16Million (a 4096x4096 image holding every 24-bit
colour once) and on 100 photographs; neither is available, so these
generators stand in for them.  This module holds no colour-space arithmetic:
it only produces uint8 RGB bytes (and float inputs for the gradient
workload), so the same bytes feed the CUDA library and the oracle.

All generators use numpy's PCG64 with an explicit seed.
"""
import math

import numpy as np

SPACES = ("cielab", "hsi", "sct")


def rgb_cube():
    """All 2^24 uint8 triplets in lexicographic order, R outermost, shape
    (4096, 4096, 3): the content of RGB16Million in a fixed order."""
    v = np.arange(1 << 24, dtype=np.uint32)
    out = np.empty((1 << 24, 3), dtype=np.uint8)
    out[:, 0] = (v >> 16) & 255
    out[:, 1] = (v >> 8) & 255
    out[:, 2] = v & 255
    return out.reshape(4096, 4096, 3)


def gradient_noise_image(height=512, width=512, seed=0):
    """Upper half: smooth 2D gradients across all three channels
    (R along x, G along y, B along x+y); lower half: i.i.d. uniform 0..255."""
    rng = np.random.default_rng(seed)
    img = np.empty((height, width, 3), dtype=np.uint8)
    hu = height // 2
    y, x = np.mgrid[0:hu, 0:width].astype(np.float64)
    wx = max(width - 1, 1)
    hy = max(hu - 1, 1)
    img[:hu, :, 0] = np.rint(x * 255.0 / wx)
    img[:hu, :, 1] = np.rint(y * 255.0 / hy)
    img[:hu, :, 2] = np.rint((x + y) * 255.0 / (wx + hy))
    img[hu:] = rng.integers(0, 256, size=(height - hu, width, 3), dtype=np.uint8)
    return img


def _content(rng, h, w, kind):
    """One image: 0 = smooth gradients, 1 = piecewise-constant rectangles,
    2 = gradients plus Gaussian noise (sigma 12) clipped to 0..255."""
    if kind == 1:
        img = np.empty((h, w, 3), dtype=np.uint8)
        img[:] = rng.integers(0, 256, size=3, dtype=np.uint8)
        for _ in range(int(rng.integers(4, 24))):
            y0, y1 = np.sort(rng.integers(0, h + 1, size=2))
            x0, x1 = np.sort(rng.integers(0, w + 1, size=2))
            img[y0:y1, x0:x1] = rng.integers(0, 256, size=3, dtype=np.uint8)
        return img
    c0 = rng.uniform(0, 255, size=3)
    cx = rng.uniform(-255, 255, size=3)
    cy = rng.uniform(-255, 255, size=3)
    y = np.linspace(0.0, 1.0, h, dtype=np.float32)[:, None, None]
    x = np.linspace(0.0, 1.0, w, dtype=np.float32)[None, :, None]
    img = c0[None, None, :] + cx[None, None, :] * x + cy[None, None, :] * y
    img = 255.0 * np.abs(((img / 255.0) + 1.0) % 2.0 - 1.0)   # fold into [0, 255]
    if kind == 2:
        img = img + rng.normal(0.0, 12.0, size=img.shape)
    return np.clip(np.rint(img), 0, 255).astype(np.uint8)


def batch_specs(count=256, seed=0, lo=64, hi=4096):
    """(height, width, kind, space) for the uneven batch: sides drawn
    log-uniform in [lo, hi], content kind uniform over the three kinds,
    target space uniform over CIELAB / HSI / SCT."""
    rng = np.random.default_rng(seed)
    specs = []
    for _ in range(count):
        h = int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))
        w = int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))
        specs.append((h, w, int(rng.integers(0, 3)), SPACES[int(rng.integers(0, 3))]))
    return specs


def batch_images(count=256, seed=0, lo=64, hi=4096):
    """Images of ``batch_specs``; image i is generated from seed (seed, i)."""
    out = []
    for i, (h, w, kind, space) in enumerate(batch_specs(count, seed, lo, hi)):
        rng = np.random.default_rng([seed, i])
        out.append((_content(rng, h, w, kind), space))
    return out


def serve_trace(rate=2000.0, duration=60.0, seed=0, lo_mpx=0.1, hi_mpx=24.0,
                mix=(0.5, 0.25, 0.25)):
    """Poisson arrivals: list of (arrival_s, height, width, kind, space) with
    sizes log-uniform in [lo_mpx, hi_mpx] Mpixel at aspect 4:3."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    while True:
        t += rng.exponential(1.0 / rate)
        if t >= duration:
            break
        mpx = math.exp(rng.uniform(math.log(lo_mpx), math.log(hi_mpx)))
        h = max(1, int(round(math.sqrt(mpx * 1e6 * 3.0 / 4.0))))
        w = max(1, int(round(mpx * 1e6 / h)))
        u = rng.uniform()
        space = SPACES[0] if u < mix[0] else (SPACES[1] if u < mix[0] + mix[1] else SPACES[2])
        out.append((t, h, w, int(rng.integers(0, 3)), space))
    return out


def request_image(h, w, kind, seed):
    return _content(np.random.default_rng(seed), h, w, kind)


def linear_rgb_batch(n=64, h=512, w=512, seed=0, knee=0.008856, frac=0.05):
    """FP32 linear RGB in [0,1], shape (n, 3, h, w); a fraction ``frac`` of the
    pixels get three equal channels, half of them exactly 0 and half within
    1e-4 of the linear-segment knee.  Returns (x, target_rgb)."""
    rng = np.random.default_rng(seed)
    x = rng.uniform(0.0, 1.0, size=(n, 3, h, w)).astype(np.float32)
    npx = n * h * w
    sel = rng.choice(npx, size=int(frac * npx), replace=False)
    half = len(sel) // 2
    flat = x.transpose(0, 2, 3, 1).reshape(npx, 3)
    flat[sel[:half]] = 0.0
    v = (knee + rng.uniform(-1e-4, 1e-4, size=len(sel) - half)).astype(np.float32)
    flat[sel[half:]] = v[:, None]
    x = flat.reshape(n, h, w, 3).transpose(0, 3, 1, 2).copy()
    target = np.random.default_rng(seed + 1).uniform(0.0, 1.0, size=(n, 3, h, w)).astype(np.float32)
    return x, target
