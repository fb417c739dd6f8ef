"""Comparison helpers for the GPU-vs-oracle parity tests.

Tolerances (stated per transform; the kernels compute in FP32, the oracle in
FP64, both evaluate the same approximant):
  CIELAB  |delta| <= 2e-4 per component (L*, a*, b*)
  CIELUV  |delta| <= 2e-4 per component (L*, u*, v*), as CIELAB
  HSI     hue: circular |delta| <= 1e-3 degree = 1.745e-5 rad;
          S and I: |delta| <= 1e-6
  SCT     |delta| <= 1e-5 * max(1, |ref|) per component (relative for L,
          1e-5 rad for the angles)
  LUT     selection ids identical; values |delta| <= 2e-4
FP16 outputs add half a unit in the last place of the FP16 value.
"""
import math

import numpy as np
import torch

LAB_TOL = 2e-4
HUE_TOL = math.radians(1e-3)
SI_TOL = 1e-6
SCT_REL = 1e-5


def to_np(t):
    return t.detach().float().cpu().numpy().astype(np.float64)


def _half_ulp(ref, dtype):
    if dtype != torch.float16:
        return 0.0
    r = np.abs(ref).astype(np.float16).astype(np.float64)
    return 0.5 * np.spacing(r.astype(np.float16)).astype(np.float64) + 1e-12


def check_space(space, gpu_planes, ref_planes, dtype=torch.float32, what=""):
    """Assert GPU planes (3, ...) match oracle planes (list of 3 arrays)."""
    g = [to_np(gpu_planes[c]).ravel() for c in range(3)]
    r = [np.asarray(ref_planes[c], dtype=np.float64).ravel() for c in range(3)]
    if space in ("cielab", "cieluv"):
        for c in range(3):
            err = np.abs(g[c] - r[c]) - _half_ulp(r[c], dtype)
            k = int(np.argmax(err))
            assert err[k] <= LAB_TOL, "%s Lab[%d] |d| %.3g at %d (gpu %r ref %r)" % (what, c, err[k] + 0, k, g[c][k], r[c][k])
    elif space == "hsi":
        d = np.abs(g[0] - r[0])
        d = np.minimum(d, 2 * math.pi - d) - _half_ulp(r[0], dtype)
        k = int(np.argmax(d))
        assert d[k] <= HUE_TOL, "%s hue |d| %.3g rad at %d (gpu %r ref %r)" % (what, d[k], k, g[0][k], r[0][k])
        for c in (1, 2):
            err = np.abs(g[c] - r[c]) - _half_ulp(r[c], dtype)
            k = int(np.argmax(err))
            assert err[k] <= SI_TOL, "%s HSI[%d] |d| %.3g at %d" % (what, c, err[k], k)
    elif space == "sct":
        for c in range(3):
            err = np.abs(g[c] - r[c]) - _half_ulp(r[c], dtype)
            lim = SCT_REL * np.maximum(1.0, np.abs(r[c]))
            k = int(np.argmax(err - lim))
            assert err[k] <= lim[k], "%s SCT[%d] |d| %.3g at %d (gpu %r ref %r)" % (what, c, err[k], k, g[c][k], r[c][k])
    else:
        raise ValueError(space)


def max_errors(space, gpu_planes, ref_planes):
    g = [to_np(gpu_planes[c]).ravel() for c in range(3)]
    r = [np.asarray(ref_planes[c], dtype=np.float64).ravel() for c in range(3)]
    out = []
    for c in range(3):
        d = np.abs(g[c] - r[c])
        if space == "hsi" and c == 0:
            d = np.minimum(d, 2 * math.pi - d)
        out.append(float(d.max()) if d.size else 0.0)
    return out


def oracle_planes(space, rgb_np, exact=False, cfg=None):
    """Oracle output for a configuration (dict of degree fields)."""
    import oracle as O
    cfg = cfg or {}
    if space == "cielab":
        return O.cielab(rgb_np, exact=exact, n=cfg.get("lab_n", 4), m=cfg.get("lab_m", 4))
    if space == "cieluv":
        return O.cieluv(rgb_np, exact=exact, n=cfg.get("lab_n", 4), m=cfg.get("lab_m", 4))
    if space == "hsi":
        return O.hsi(rgb_np, mode="exact" if exact else "approx", n=cfg.get("hsi_n", 5),
                     printed=cfg.get("hsi_coeffs", 0) == 1)
    return O.sct(rgb_np, exact=exact, n=cfg.get("sct_n", 5), m=cfg.get("sct_m", 5), r=cfg.get("sct_r", 5))
