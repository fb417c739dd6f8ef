"""FP64 CPU oracle for MACT (Celebi, Kingravi & Celiker, "Fast Color Space
Transformations Using Minimax Approximations").

TEST INFRASTRUCTURE.  Only tests/, ``__graft_entry__.smoke()`` and bench.py's
cpu_baseline / reference legs may import this package.  It shares no code
with the CUDA library: the per-pixel formulas live in ``mact_oracle.c``
(plain double precision, written from the paper's equations), the paper's
coefficient tables in ``tables.py`` and the Remez exchange in ``remez.py``.

Functions take uint8 interleaved RGB as a numpy array of shape (..., 3) and
return float64 planes.  Parity status of every function is pinned by the
``-m "not gpu"`` tests (closed forms, the paper's printed numbers, brute
force over all 2^24 colours, Remez recomputation), with these exceptions,
each stated again where it applies:
  - ``cube_eps_hsi``: the HSI average error is parity unpinned (both
    coefficient sets land 1-3% from the printed averages);
  - ``cube_eps_hsi_lut``: the angular HSI LUT's maximum error is parity
    unpinned (its average is pinned within 0.5%);
  - ``cube_eps_lut`` with the pyramidal method: the averages are pinned only
    within 0.07% (parity partial); its maxima are exact.
"""
import ctypes
import os

import numpy as np

from . import remez, tables
from .build import build as _build_lib

_lib = None


class RGBDef(ctypes.Structure):
    _fields_ = [("threshold", ctypes.c_double), ("slope", ctypes.c_double),
                ("offset", ctypes.c_double), ("exponent", ctypes.c_double),
                ("m", ctypes.c_double * 9), ("white", ctypes.c_double * 3)]


class SCTCoeffs(ctypes.Structure):
    _fields_ = [("p", ctypes.POINTER(ctypes.c_double)), ("n", ctypes.c_int),
                ("q", ctypes.POINTER(ctypes.c_double)), ("m", ctypes.c_int),
                ("f", ctypes.POINTER(ctypes.c_double)), ("rf", ctypes.c_int),
                ("g", ctypes.POINTER(ctypes.c_double)), ("rg", ctypes.c_int)]


TRILINEAR, PRISM, PYRAMID, TETRA = 0, 1, 2, 3
LUT_METHODS = {"trilinear": TRILINEAR, "prism": PRISM, "pyramid": PYRAMID, "tetra": TETRA}

_D = ctypes.POINTER(ctypes.c_double)
_F = ctypes.POINTER(ctypes.c_float)
_U8 = ctypes.POINTER(ctypes.c_uint8)
_I32 = ctypes.POINTER(ctypes.c_int32)


def lib():
    global _lib
    if _lib is None:
        path = _build_lib()
        L = ctypes.CDLL(path)
        L.orc_gamma_inverse.restype = ctypes.c_double
        L.orc_gamma_inverse.argtypes = [ctypes.POINTER(RGBDef), ctypes.c_double]
        L.orc_rgb_to_t.argtypes = [ctypes.POINTER(RGBDef)] + [ctypes.c_double] * 3 + [_D]
        L.orc_cielab_pixel.argtypes = [ctypes.POINTER(RGBDef), ctypes.c_int, _D, ctypes.c_int, _D,
                                       ctypes.c_int] + [ctypes.c_double] * 3 + [_D]
        L.orc_cielab.argtypes = [ctypes.POINTER(RGBDef), ctypes.c_int, _D, ctypes.c_int, _D,
                                 ctypes.c_int, _U8, ctypes.c_int64, _D, _D, _D, ctypes.c_int]
        L.orc_cieluv_pixel.argtypes = L.orc_cielab_pixel.argtypes
        L.orc_cieluv.argtypes = L.orc_cielab.argtypes
        L.orc_hsi.argtypes = [ctypes.c_int, _D, ctypes.c_int, _U8, ctypes.c_int64, _D, _D, _D,
                              ctypes.c_int]
        L.orc_sct.argtypes = [ctypes.POINTER(SCTCoeffs), _U8, ctypes.c_int64, _D, _D, _D,
                              ctypes.c_int]
        L.orc_sct_inverse.argtypes = [_D, _D]
        L.orc_delta_e.restype = ctypes.c_double
        L.orc_delta_e.argtypes = [_D, _D]
        L.orc_d_hsi.restype = ctypes.c_double
        L.orc_d_hsi.argtypes = [_D, _D]
        L.orc_lut_build.argtypes = [ctypes.POINTER(RGBDef), ctypes.c_int, _F]
        L.orc_lut_interp.argtypes = [ctypes.c_int, _F, ctypes.c_int, _U8, ctypes.c_int64,
                                     _D, _D, _D, _I32, ctypes.c_int]
        L.orc_cube_cbrt_probs.argtypes = [ctypes.POINTER(RGBDef), _D]
        L.orc_cube_sct_probs.argtypes = [_D]
        L.orc_cube_eps_cielab.argtypes = [ctypes.POINTER(RGBDef), _D, ctypes.c_int, _D,
                                          ctypes.c_int, _D]
        L.orc_cube_eps_hsi.argtypes = [_D, ctypes.c_int, _D]
        L.orc_cube_eps_sct.argtypes = [ctypes.POINTER(RGBDef), ctypes.POINTER(SCTCoeffs), _D]
        L.orc_cube_eps_lut.argtypes = [ctypes.POINTER(RGBDef), ctypes.c_int, _F, ctypes.c_int, _D]
        L.orc_lut_build_hsi.argtypes = [ctypes.c_int, _F]
        L.orc_lut_interp_hsi_pixel.restype = ctypes.c_double
        L.orc_lut_interp_hsi_pixel.argtypes = [_F, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _D]
        L.orc_lut_interp_hsi.argtypes = [_F, ctypes.c_int, _U8, ctypes.c_int64, _D, _D, _D, _D, ctypes.c_int]
        L.orc_cube_eps_hsi_lut.argtypes = [_F, ctypes.c_int, _D]
        L.orc_lab_linear.argtypes = [ctypes.POINTER(RGBDef), ctypes.c_int, _D, ctypes.c_int, _D, ctypes.c_int,
                                     _D, ctypes.c_int64, ctypes.c_int64, _D]
        L.orc_lab_loss_grad.argtypes = [ctypes.POINTER(RGBDef), ctypes.c_int, _D, ctypes.c_int, _D, ctypes.c_int,
                                        _D, _D, ctypes.c_int64, ctypes.c_int64, _D]
        L.orc_lab_loss_grad.restype = ctypes.c_double
        L.orc_max_threads.restype = ctypes.c_int
        _lib = L
    return _lib


def max_threads():
    return lib().orc_max_threads()


# ------------------------------------------------------------------ inputs

def bt709_d65(matrix=None, white=None, gamma=None):
    """The paper's RGB definition (Eq. equ_rgb_lin, equ_rgb_xyz, D65)."""
    g = dict(tables.BT709_GAMMA, **(gamma or {}))
    d = RGBDef()
    d.threshold, d.slope, d.offset, d.exponent = g["threshold"], g["slope"], g["offset"], g["exponent"]
    for i, v in enumerate(matrix or tables.BT709_MATRIX):
        d.m[i] = v
    for i, v in enumerate(white or tables.D65_WHITE):
        d.white[i] = v
    return d


def _darr(v):
    a = (ctypes.c_double * max(1, len(v)))()
    for i, x in enumerate(v):
        a[i] = float(x)
    return a


def _rgb(rgb):
    rgb = np.ascontiguousarray(rgb, dtype=np.uint8)
    if rgb.shape[-1] != 3:
        raise ValueError("rgb must have a trailing dimension of 3")
    return rgb, rgb.size // 3


def _planes(npix, shape):
    return [np.empty(npix, dtype=np.float64) for _ in range(3)], shape


def _ptr(a, t):
    return a.ctypes.data_as(t)


def cbrt_coeffs(n, m):
    """(p, q) for the cube root: a rational from Table tab_cbrt_rat when m > 0,
    a polynomial from Table tab_cbrt_poly when m == 0 (q = None)."""
    if m == 0:
        return tables.CBRT_POLY[n][1], None
    _, p, q = tables.CBRT_RAT[(n, m)]
    return p, q


_CBRT_FITS = {}


def cbrt_minimax(n, m):
    """(p, q, E) of the minimax rational p_n/q_m of t^(1/3) on [0.008856, 1]
    (the interval of Figure fig_cbrt), from the oracle's own Remez exchange,
    q(0) = 1: for the degrees Table tab_cbrt_rat does not print (and the
    converged form of those it does)."""
    if (n, m) not in _CBRT_FITS:
        p, q, E, xs, es = remez.remez_rational(np.cbrt, n, m, 0.008856, 1.0)
        _CBRT_FITS[(n, m)] = (list(p), list(q), E, xs, es)
    p, q, E, _, _ = _CBRT_FITS[(n, m)]
    return p, q, E


def cbrt_minimax_extrema(n, m):
    """The reference points and signed errors of cbrt_minimax(n, m)."""
    cbrt_minimax(n, m)
    return _CBRT_FITS[(n, m)][3], _CBRT_FITS[(n, m)][4]


def hsi_coeffs(n, printed=False):
    """Coefficients replacing arctan(sqrt(3) x): the oracle's own Remez fit on
    [0, 1] (default) or Table tab_arctan as printed (n=2 sign read as minus)."""
    if printed:
        return tables.HSI_ARCTAN[n][1]
    return remez.hsi_arctan_unit(n)[0]


# ------------------------------------------------------------- transforms

def cielab(rgb, exact=False, n=4, m=4, p=None, q=None, rgbdef=None, nthreads=0):
    """RGB -> CIELAB (Eq. equ_rgb_lin, equ_rgb_xyz, equ_xyz_lab).  With
    exact=False the cube root is replaced by p/q (default: Table tab_cbrt_rat
    (4,4)); m == 0 selects the polynomial of Table tab_cbrt_poly."""
    rgb, npix = _rgb(rgb)
    if p is None:
        p, q = cbrt_coeffs(n, m)
    d = rgbdef or bt709_d65()
    pa, qa = _darr(p), _darr(q or [1.0])
    (L, A, B), _ = _planes(npix, rgb.shape[:-1])
    lib().orc_cielab(ctypes.byref(d), 0 if exact else 1, pa, len(p) - 1, qa,
                     (len(q) - 1) if q is not None else -1,
                     _ptr(rgb, _U8), npix, _ptr(L, _D), _ptr(A, _D), _ptr(B, _D), nthreads)
    return [x.reshape(rgb.shape[:-1]) for x in (L, A, B)]


def cieluv(rgb, exact=False, n=4, m=4, p=None, q=None, rgbdef=None, nthreads=0):
    """RGB -> CIE 1976 L*u*v* (the CIELUV variant the Conclusions name): L* as
    in CIELAB (the cube root exact or replaced by p/q, default Table
    tab_cbrt_rat (4,4)), u* = 13 L* (u' - u'n), v* = 13 L* (v' - v'n)."""
    rgb, npix = _rgb(rgb)
    if p is None:
        p, q = cbrt_coeffs(n, m)
    d = rgbdef or bt709_d65()
    pa, qa = _darr(p), _darr(q or [1.0])
    (L, U, V), _ = _planes(npix, rgb.shape[:-1])
    lib().orc_cieluv(ctypes.byref(d), 0 if exact else 1, pa, len(p) - 1, qa,
                     (len(q) - 1) if q is not None else -1,
                     _ptr(rgb, _U8), npix, _ptr(L, _D), _ptr(U, _D), _ptr(V, _D), nthreads)
    return [x.reshape(rgb.shape[:-1]) for x in (L, U, V)]


def hsi(rgb, mode="approx", n=5, printed=False, coeffs=None, nthreads=0):
    """RGB -> HSI.  mode "exact" (Kender, Eq. equ_rgb_kender), "approx"
    (Kender with P_n), "arccos" (Eq. equ_rgb_hsi).  H radians, S, I in [0,1]."""
    rgb, npix = _rgb(rgb)
    c = coeffs if coeffs is not None else hsi_coeffs(n, printed)
    md = {"exact": 0, "approx": 1, "arccos": 2}[mode]
    (H, S, I), _ = _planes(npix, rgb.shape[:-1])
    lib().orc_hsi(md, _darr(c), len(c) - 1, _ptr(rgb, _U8), npix,
                  _ptr(H, _D), _ptr(S, _D), _ptr(I, _D), nthreads)
    return [x.reshape(rgb.shape[:-1]) for x in (H, S, I)]


def _sct_coeffs(n, m, r):
    keep = [_darr(tables.SCT_ARCSIN[n][1]), _darr(tables.SCT_ARCCOS[m][1]),
            _darr(tables.SCT_F[r][1]), _darr(tables.SCT_G[r][1])]
    co = SCTCoeffs(keep[0], n, keep[1], m, keep[2], r, keep[3], r)
    co._keep = keep
    return co


def sct(rgb, exact=False, n=5, m=5, r=5, nthreads=0):
    """RGB -> SCT (Eq. equ_rgb_sct, equ_sct_b), L in code units, angles in
    radians; approximants from Tables tab_arcsin, tab_arccos, tab_f, tab_g."""
    rgb, npix = _rgb(rgb)
    co = None if exact else _sct_coeffs(n, m, r)
    (L, A, B), _ = _planes(npix, rgb.shape[:-1])
    lib().orc_sct(ctypes.byref(co) if co is not None else None, _ptr(rgb, _U8), npix,
                  _ptr(L, _D), _ptr(A, _D), _ptr(B, _D), nthreads)
    return [x.reshape(rgb.shape[:-1]) for x in (L, A, B)]


def sct_inverse(L, A, B):
    """Eq. equ_sct_rgb for one pixel."""
    s = _darr([L, A, B])
    out = (ctypes.c_double * 3)()
    lib().orc_sct_inverse(s, out)
    return list(out)


def delta_e(x, y):
    return lib().orc_delta_e(_darr(x), _darr(y))


def d_hsi(x, y):
    return lib().orc_d_hsi(_darr(x), _darr(y))


def gamma_inverse(kp, rgbdef=None):
    d = rgbdef or bt709_d65()
    return lib().orc_gamma_inverse(ctypes.byref(d), float(kp))


# -------------------------------------------------------------------- LUTs

def lut_build(N, rgbdef=None):
    """N^3 x 3 FP32 LUT of the exact CIELAB at nodes k' = i/(N-1), R outermost."""
    d = rgbdef or bt709_d65()
    lut = np.empty((N, N, N, 3), dtype=np.float32)
    lib().orc_lut_build(ctypes.byref(d), N, _ptr(lut, _F))
    return lut


def lut_build_hsi(N):
    """N^3 x 3 FP32 LUT of the exact HSI (H, S, I) at nodes k' = i/(N-1),
    R outermost; H = 0 at gray nodes (S = 0)."""
    lut = np.empty((N, N, N, 3), dtype=np.float32)
    lib().orc_lut_build_hsi(N, _ptr(lut, _F))
    return lut


def lut_interp_hsi(lut, rgb, nthreads=0):
    """Trilinear interpolation of an HSI LUT with angular hue mixing
    (Eq. equ_angular along B, then G, then R; gray nodes carry no hue).
    Returns ([H, S, I], cond), cond the smallest mix modulus per pixel."""
    rgb, npix = _rgb(rgb)
    lut = np.ascontiguousarray(lut, dtype=np.float32)
    (H, S, I), _ = _planes(npix, rgb.shape[:-1])
    cond = np.empty(npix, dtype=np.float64)
    lib().orc_lut_interp_hsi(_ptr(lut, _F), lut.shape[0], _ptr(rgb, _U8), npix, _ptr(H, _D), _ptr(S, _D),
                             _ptr(I, _D), _ptr(cond, _D), nthreads)
    sh = rgb.shape[:-1]
    return [x.reshape(sh) for x in (H, S, I)], cond.reshape(sh)


def cube_eps_hsi_lut(lut):
    """(eps^T_avg, eps^T_max) in D_HSI of the angular HSI LUT over all 2^24 colours."""
    lut = np.ascontiguousarray(lut, dtype=np.float32)
    out = (ctypes.c_double * 2)()
    lib().orc_cube_eps_hsi_lut(_ptr(lut, _F), lut.shape[0], out)
    return list(out)


def lut_interp(method, lut, rgb, nthreads=0):
    """FP64 interpolation of an FP32 LUT.  Returns (planes, selection ids);
    a selection id is (lower-corner node index) * 8 + simplex id."""
    rgb, npix = _rgb(rgb)
    lut = np.ascontiguousarray(lut, dtype=np.float32)
    N = lut.shape[0]
    md = LUT_METHODS[method] if isinstance(method, str) else int(method)
    (o0, o1, o2), _ = _planes(npix, rgb.shape[:-1])
    sel = np.empty(npix, dtype=np.int32)
    lib().orc_lut_interp(md, _ptr(lut, _F), N, _ptr(rgb, _U8), npix,
                         _ptr(o0, _D), _ptr(o1, _D), _ptr(o2, _D), _ptr(sel, _I32), nthreads)
    sh = rgb.shape[:-1]
    return [x.reshape(sh) for x in (o0, o1, o2)], sel.reshape(sh)


# ------------------------------------------------- statistics over the cube

def cube_cbrt_probs(rgbdef=None):
    d = rgbdef or bt709_d65()
    out = (ctypes.c_double * 3)()
    lib().orc_cube_cbrt_probs(ctypes.byref(d), out)
    return list(out)


def cube_sct_probs():
    out = (ctypes.c_double * 2)()
    lib().orc_cube_sct_probs(out)
    return list(out)


def cube_eps_cielab(n=4, m=4, p=None, q=None, rgbdef=None):
    """(eps^T_avg, eps^T_max) in Delta E*ab over all 2^24 colours."""
    if p is None:
        p, q = cbrt_coeffs(n, m)
    d = rgbdef or bt709_d65()
    out = (ctypes.c_double * 2)()
    lib().orc_cube_eps_cielab(ctypes.byref(d), _darr(p), len(p) - 1, _darr(q or [1.0]),
                              (len(q) - 1) if q is not None else -1, out)
    return list(out)


def cube_eps_cieluv(n=4, m=4, p=None, q=None, rgbdef=None):
    """(eps_avg, eps_max) in Delta E*uv of MACT CIELUV over all 2^24 colours."""
    if p is None:
        p, q = cbrt_coeffs(n, m)
    d = rgbdef or bt709_d65()
    out = (ctypes.c_double * 2)()
    lib().orc_cube_eps_cieluv(ctypes.byref(d), _darr(p), len(p) - 1, _darr(q or [1.0]),
                              (len(q) - 1) if q is not None else -1, out)
    return list(out)


def cube_eps_hsi(n=5, printed=False, coeffs=None):
    """(eps^T_avg, eps^T_max) in D_HSI over all 2^24 colours.  The maximum is
    pinned by the paper's Table tab_hsi; the average is parity unpinned (it
    matches the printed values only to about 3%)."""
    c = coeffs if coeffs is not None else hsi_coeffs(n, printed)
    out = (ctypes.c_double * 2)()
    lib().orc_cube_eps_hsi(_darr(c), len(c) - 1, out)
    return list(out)


def cube_eps_sct(n=5, m=5, r=5, rgbdef=None):
    d = rgbdef or bt709_d65()
    co = _sct_coeffs(n, m, r)
    out = (ctypes.c_double * 2)()
    lib().orc_cube_eps_sct(ctypes.byref(d), ctypes.byref(co), out)
    return list(out)


def cube_eps_lut(method, lut, rgbdef=None):
    d = rgbdef or bt709_d65()
    lut = np.ascontiguousarray(lut, dtype=np.float32)
    md = LUT_METHODS[method] if isinstance(method, str) else int(method)
    out = (ctypes.c_double * 2)()
    lib().orc_cube_eps_lut(ctypes.byref(d), md, _ptr(lut, _F), lut.shape[0], out)
    return list(out)


# --------------------------------------------- differentiable RGB -> CIELAB

def _lab_args(exact, n, m, p=None, q=None):
    if p is None:
        p, q = cbrt_coeffs(n, m)
    return (0 if exact else 1), _darr(p), len(p) - 1, _darr(q or [1.0]), ((len(q) - 1) if q is not None else -1)


def lab_linear(x, exact=False, n=4, m=4, rgbdef=None, p=None, q=None):
    """CIELAB of LINEAR RGB x, shape (N, 3, ...) -> same shape (FP64).  p, q:
    explicit cube-root coefficients (default: Table tab_cbrt_rat (n, m))."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    nb, hw = x.shape[0], x[0, 0].size
    out = np.empty_like(x)
    d = rgbdef or bt709_d65()
    mode, pa, pn, qa, qm = _lab_args(exact, n, m, p, q)
    lib().orc_lab_linear(ctypes.byref(d), mode, pa, pn, qa, qm, _ptr(x, _D), nb, hw, _ptr(out, _D))
    return out


def lab_loss_grad(x, target, exact=False, n=4, m=4, rgbdef=None, grad=True, p=None, q=None):
    """(mean Delta E*ab of lab_linear(x) vs target, analytic dLoss/dx)."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    t = np.ascontiguousarray(target, dtype=np.float64)
    nb, hw = x.shape[0], x[0, 0].size
    g = np.empty_like(x) if grad else None
    d = rgbdef or bt709_d65()
    mode, pa, pn, qa, qm = _lab_args(exact, n, m, p, q)
    loss = lib().orc_lab_loss_grad(ctypes.byref(d), mode, pa, pn, qa, qm, _ptr(x, _D), _ptr(t, _D), nb, hw,
                                   _ptr(g, _D) if grad else None)
    return loss, g
