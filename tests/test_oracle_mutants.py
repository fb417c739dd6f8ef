"""Planted mistakes in the oracle, on the CPU: the pins must catch each one.

Each mutant is a copy of ``oracle/mact_oracle.c`` with one plausible slip
(a sign, a dropped term, a wrong index, a transposed operand, a swapped
branch), compiled with the oracle's own gcc flags and loaded in place of the
oracle's library.  A battery of pins that do not come from the oracle itself
-- textbook colorimetry, closed forms, the paper's printed numbers
(``tests/golden/``), interpolation identities and finite differences -- runs
against it and must fail.  The unmutated oracle must pass the whole battery.
"""
import concurrent.futures as cf
import math
import os

import numpy as np
import pytest

import oracle as O
from oracle import build as oracle_build
from conftest import read_golden

# (id, text in mact_oracle.c (must occur exactly once), replacement)
MUTANTS = [
    # CIELAB (Eq. equ_rgb_lin, equ_rgb_xyz, equ_xyz_lab)
    ("lab_a_sign", "lab[1] = 500.0 * (fx - fy);", "lab[1] = 500.0 * (fy - fx);"),
    ("lab_b_index", "lab[2] = 200.0 * (fy - fz);", "lab[2] = 200.0 * (fy - fx);"),
    ("matrix_transposed",
     "double xyz = d->m[3 * c + 0] * k[0] + d->m[3 * c + 1] * k[1] + d->m[3 * c + 2] * k[2];",
     "double xyz = d->m[c] * k[0] + d->m[3 + c] * k[1] + d->m[6 + c] * k[2];"),
    ("white_not_divided", "t[c] = xyz / d->white[c];", "t[c] = xyz;"),
    ("linear_segment_offset_dropped",
     "    if (t > 0.008856) return cbrt(t);\n    return 7.787 * t + 16.0 / 116.0;",
     "    if (t > 0.008856) return cbrt(t);\n    return 7.787 * t;"),
    ("knee_comparison_flipped", "if (t > 0.008856) return cbrt(t);", "if (t < 0.008856) return cbrt(t);"),
    ("gamma_toe_multiplies", "if (kp < d->threshold) return kp / d->slope;",
     "if (kp < d->threshold) return kp * d->slope;"),
    ("rational_denominator_dropped", "double den = (m >= 0) ? orc_poly(q, m, t) : 1.0;", "double den = 1.0;"),
    # HSI (Eq. equ_rgb_kender, Table tab_arctan)
    ("hsi_s_factor_dropped", "hsi[1] = sum > 0.0 ? 1.0 - 3.0 * mn / sum : 0.0;",
     "hsi[1] = sum > 0.0 ? 1.0 - mn / sum : 0.0;"),
    ("hsi_i_not_averaged", "hsi[2] = (sum / 255.0) / 3.0;", "hsi[2] = sum / 255.0;"),
    ("hue_case2_sign", "return ORC_PI + orc_atan_sqrt3((b - g) / (b - r + g - r), c, n);",
     "return ORC_PI + orc_atan_sqrt3((g - b) / (b - r + g - r), c, n);"),
    ("arctan_odd_symmetry_lost", "if (x < 0.0) return -orc_poly(c, n, -x);",
     "if (x < 0.0) return orc_poly(c, n, -x);"),
    # SCT (Eq. equ_rgb_sct, equ_sct_b, equ_arccos_cheap, arctan_split)
    ("sct_length_index", "double L = sqrt(r * r + g * g + b * b);", "double L = sqrt(r * r + g * g + b * g);"),
    ("sct_arcsin_argument", "double y = sqrt(1.0 - x);", "double y = sqrt(x);"),
    ("sct_f_g_split_flipped", "} else if (g < r) {", "} else if (g > r) {"),
    ("sct_inverse_sin_cos", "rgb[2] = s[0] * cos(s[1]);", "rgb[2] = s[0] * sin(s[1]);"),
    # error measures (Eq. equ_cielab_dist, equ_hsi_dist)
    ("delta_e_term_repeated", "return sqrt(dl * dl + da * da + db * db);", "return sqrt(dl * dl + da * da + da * da);"),
    ("d_hsi_cosine_sign", "double v = x[1] * x[1] + y[1] * y[1] - 2.0 * x[1] * y[1] * cos(th) + di * di;",
     "double v = x[1] * x[1] + y[1] * y[1] + 2.0 * x[1] * y[1] * cos(th) + di * di;"),
    # LUTs (Section "Comparison with 3D Lookup Table Interpolation Methods")
    ("lut_build_axes_transposed", "lut[((int64_t)(i * N + j) * N + k) * 3 + c] = (float)lab[c];",
     "lut[((int64_t)(k * N + j) * N + i) * 3 + c] = (float)lab[c];"),
    ("lut_remainder_modulus", "*rem = s % 255;", "*rem = s % 256;"),
    ("trilinear_weight_axes", "+ c100 * fr * (1 - fg) * (1 - fb) + c101 * fr * (1 - fg) * fb",
     "+ c100 * fb * (1 - fg) * (1 - fr) + c101 * fr * (1 - fg) * fb"),
    ("prism_wrong_vertex",
     "v = c000 + (c010 - c000) * fg + (c011 - c010) * fb + (c100 - c000) * fr",
     "v = c000 + (c010 - c000) * fg + (c011 - c010) * fb + (c010 - c000) * fr"),
    ("pyramid_wrong_vertex", "v = c000 + (c111 - c110) * fb + (c100 - c000) * fr + (c010 - c000) * fg",
     "v = c000 + (c111 - c011) * fb + (c100 - c000) * fr + (c010 - c000) * fg"),
    ("tetra_wrong_vertex", "v = c000 + (c100 - c000) * fr + (c110 - c100) * fg + (c111 - c110) * fb;",
     "v = c000 + (c100 - c000) * fr + (c110 - c100) * fg + (c111 - c101) * fb;"),
    ("angular_mix_operand", "double x = (1.0 - a) * cos(h0) + a * cos(h1);",
     "double x = (1.0 - a) * cos(h0) + a * cos(h0);"),
    # backward (derivative of Eq. equ_xyz_lab through Eq. equ_rgb_xyz)
    ("dpoly_factor_dropped", "s += i * a[i] * xp;", "s += a[i] * xp;"),
    ("grad_a_sign", "double gf[3] = {500.0 * ga, 116.0 * gL - 500.0 * ga + 200.0 * gb, -200.0 * gb};",
     "double gf[3] = {500.0 * ga, 116.0 * gL + 500.0 * ga + 200.0 * gb, -200.0 * gb};"),
    ("grad_white_dropped", "for (int c = 0; c < 3; ++c) gt[c] = gf[c] * df[c] / d->white[c];",
     "for (int c = 0; c < 3; ++c) gt[c] = gf[c] * df[c];"),
    ("grad_matrix_not_transposed",
     "grad[b * 3 * hw + j * hw + i] = d->m[j] * gt[0] + d->m[3 + j] * gt[1] + d->m[6 + j] * gt[2];",
     "grad[b * 3 * hw + j * hw + i] = d->m[3 * j] * gt[0] + d->m[3 * j + 1] * gt[1] + d->m[3 * j + 2] * gt[2];"),
    ("grad_linear_slope", "        *df = 7.787;\n", "        *df = 7.787 * t;\n"),
    # shared pieces and the cube statistics
    ("poly_power_shift", "        s += a[i] * xp;\n        xp *= x;", "        xp *= x;\n        s += a[i] * xp;"),
    ("gamma_exponent_inverted", "return pow((kp + d->offset) / (1.0 + d->offset), d->exponent);",
     "return pow((kp + d->offset) / (1.0 + d->offset), 1.0 / d->exponent);"),
    ("hue_case1_base", "if (r > b && g > b) return ORC_PI / 3.0 + orc_atan_sqrt3(",
     "if (r > b && g > b) return ORC_PI / 6.0 + orc_atan_sqrt3("),
    ("hue_case3_base", "if (b > g) return 5.0 * ORC_PI / 3.0 + orc_atan_sqrt3(",
     "if (b > g) return 4.0 * ORC_PI / 3.0 + orc_atan_sqrt3("),
    ("hue_arccos_reflection", "if (b > g) h = 2.0 * ORC_PI - h;", "if (b < g) h = 2.0 * ORC_PI - h;"),
    ("sct_branch_threshold", "} else if (x >= 0.5) {", "} else if (x >= 0.6) {"),
    ("sct_r_zero_angle", "B = ORC_PI / 2.0;                         /* R = 0, G > 0 */",
     "B = 0.0;                                  /* R = 0, G > 0 */"),
    ("hsi_lut_weight_axis", "(((c >> 1) & 1) ? f[1] : 1.0 - f[1])", "(((c >> 1) & 1) ? f[2] : 1.0 - f[1])"),
    ("eps_cielab_compares_itself",
     "orc_cielab_pixel(d, 0, NULL, 0, NULL, 0, r, g, b, e);\n                orc_cielab_pixel(d, 1, p, n, q, m, r, g, b, a);",
     "orc_cielab_pixel(d, 1, p, n, q, m, r, g, b, e);\n                orc_cielab_pixel(d, 1, p, n, q, m, r, g, b, a);"),
    ("eps_sct_inverse_channels", "orc_cielab_pixel(d, 0, NULL, 0, NULL, 0, back[0], back[1], back[2], a);",
     "orc_cielab_pixel(d, 0, NULL, 0, NULL, 0, back[0], back[2], back[1], a);"),
    ("cbrt_probs_channel", "c2 += t[2] > 0.008856;", "c2 += t[1] > 0.008856;"),
    # CIELUV (CIE 1976 L*u*v*, the variant the Conclusions name)
    ("luv_denominator_weight", "const double den = X + 15.0 * Y + 3.0 * Z;", "const double den = X + 5.0 * Y + 3.0 * Z;"),
    ("luv_u_numerator", "luv[1] = 13.0 * L * (4.0 * X / den - un);", "luv[1] = 13.0 * L * (4.0 * Y / den - un);"),
    ("luv_v_white_term", "luv[2] = 13.0 * L * (9.0 * Y / den - vn);", "luv[2] = 13.0 * L * (9.0 * Y / den - un);"),
    ("luv_lightness_channel", "const double fy = mode ? orc_f_approx(t[1], p, n, q, m) : orc_f_exact(t[1]);",
     "const double fy = mode ? orc_f_approx(t[0], p, n, q, m) : orc_f_exact(t[0]);"),
    ("luv_white_u_numerator", "const double un = 4.0 * Xn / dn, vn = 9.0 * Yn / dn;",
     "const double un = 4.0 * Yn / dn, vn = 9.0 * Yn / dn;"),
]

TWO_PI = 2.0 * math.pi


def _px(*rows):
    return np.array(rows, dtype=np.uint8).reshape(-1, 3)


def _circ(a, b):
    d = np.abs(np.asarray(a, dtype=np.float64) - np.asarray(b, dtype=np.float64)) % TWO_PI
    return np.minimum(d, TWO_PI - d)


# ---------------------------------------------------------------- the pins

def pin_primaries_lab():
    """Textbook CIELAB of the BT.709 primaries, secondaries, white and black."""
    for row in read_golden("primaries_lab.txt"):
        got = [float(x[0]) for x in O.cielab(_px([int(v) for v in row[:3]]), exact=True)]
        assert max(abs(a - float(b)) for a, b in zip(got, row[3:])) < 0.02, row


def pin_grays():
    """Grays: a* = b* = 0 in both CIELAB forms (each matrix row sums to its
    white component), L* increasing; HSI S = 0, H = 0, I = v/255; SCT
    L = v sqrt(3), angle A = arccos(1/sqrt(3)), angle B = pi/4."""
    v = np.arange(256, dtype=np.uint8)
    grays = np.stack([v, v, v], axis=1)
    for exact in (True, False):
        L, A, B = O.cielab(grays, exact=exact)
        assert np.abs(A).max() < 1e-9 and np.abs(B).max() < 1e-9 and np.all(np.diff(L) > 0)
    H, S, I = O.hsi(grays, mode="exact")
    assert np.all(H == 0.0) and np.all(S == 0.0) and np.abs(I - v / 255.0).max() < 1e-15
    for exact, tol in ((True, 1e-13), (False, 1e-4)):
        L, A, B = O.sct(grays[1:], exact=exact)
        assert np.abs(L - v[1:] * math.sqrt(3.0)).max() < 1e-11
        assert np.abs(A - math.acos(1.0 / math.sqrt(3.0))).max() < tol
        assert np.abs(B - math.pi / 4).max() < tol


def pin_hsi_primaries():
    """Hues of red, green, blue, yellow, cyan, magenta: 0, 120, 240, 60, 180,
    300 degrees; S = 1 (min = 0); I = (R + G + B)/765.  The approximant
    deviates by its own maximum error at |x| = 1 (1.9e-4 rad for n = 5)."""
    rgb = _px([255, 0, 0], [0, 255, 0], [0, 0, 255], [255, 255, 0], [0, 255, 255], [255, 0, 255])
    hue = np.radians([0, 120, 240, 60, 180, 300])
    for mode, tol in (("exact", 1e-12), ("arccos", 1e-12), ("approx", 3e-4)):
        H, S, I = O.hsi(rgb, mode=mode)
        assert _circ(H, hue).max() <= tol, mode
        assert np.abs(S - 1.0).max() < 1e-15
        assert np.abs(I - rgb.sum(axis=1) / 765.0).max() < 1e-15


def pin_sct_primaries():
    """Red: angle A = pi/2, angle B = 0; green: A = B = pi/2; blue: A = 0;
    L = 255 for each."""
    rgb = _px([255, 0, 0], [0, 255, 0], [0, 0, 255])
    for exact, tol in ((True, 1e-12), (False, 1e-4)):
        L, A, B = O.sct(rgb, exact=exact)
        assert np.abs(L - 255.0).max() < 1e-12
        assert abs(A[0] - math.pi / 2) <= tol and abs(B[0]) <= tol
        assert abs(A[1] - math.pi / 2) <= tol and abs(B[1] - math.pi / 2) <= tol
        assert abs(A[2]) <= tol


def pin_sct_round_trip():
    """Eq. equ_sct_rgb inverts the exact SCT (spherical coordinates)."""
    rgb = np.random.default_rng(5).integers(0, 256, (300, 3)).astype(np.uint8)
    L, A, B = O.sct(rgb, exact=True)
    back = np.array([O.sct_inverse(L[k], A[k], B[k]) for k in range(len(rgb))])
    assert np.abs(back - rgb).max() < 1e-9


def pin_distances():
    """Delta E*ab on Pythagorean quadruples; D_HSI by the law of cosines in
    the (S, H) plane plus the intensity difference."""
    assert abs(O.delta_e([0, 0, 0], [3, 4, 12]) - 13.0) < 1e-12
    assert abs(O.delta_e([1, 2, 3], [3, 5, 9]) - 7.0) < 1e-12
    assert abs(O.d_hsi([0.0, 1.0, 0.5], [math.pi / 3, 1.0, 0.5]) - 1.0) < 1e-12      # equilateral
    assert abs(O.d_hsi([0.3, 0.3, 0.2], [0.3 + math.pi, 0.4, 0.2]) - 0.7) < 1e-12   # opposite hues
    assert abs(O.d_hsi([1.0, 0.5, 0.1], [1.0, 0.5, 0.4]) - 0.3) < 1e-12             # intensity only


def pin_lut_linear_reproduction():
    """All four interpolators reproduce a LUT whose nodes are a linear
    function of the node indices, at every code (they are exact for linear
    functions; the code v sits at v (N - 1)/255 node units)."""
    N = 6
    i, j, k = np.meshgrid(np.arange(N), np.arange(N), np.arange(N), indexing="ij")
    coef = [(3.0, -2.0, 5.0), (-1.0, 4.0, 2.0), (7.0, 1.0, -3.0)]
    lut = np.stack([a * i + b * j + c * k for a, b, c in coef], axis=-1).astype(np.float32)
    rgb = np.random.default_rng(9).integers(0, 256, (4000, 3)).astype(np.uint8)
    rgb = np.concatenate([rgb, _px([255, 255, 255], [0, 0, 0], [255, 0, 51])])
    x = rgb.astype(np.float64) * (N - 1) / 255.0
    for method in ("trilinear", "prism", "pyramid", "tetra"):
        planes, _ = O.lut_interp(method, lut, rgb)
        for c, (a, b, cc) in enumerate(coef):
            assert np.abs(planes[c] - (a * x[:, 0] + b * x[:, 1] + cc * x[:, 2])).max() < 1e-9, method


def _node_codes(N=18):
    codes = np.arange(N) * (255 // (N - 1))
    r, g, b = np.meshgrid(codes, codes, codes, indexing="ij")
    return np.stack([r, g, b], axis=-1).reshape(-1, 3).astype(np.uint8)


def pin_lut_nodes():
    """With N = 18 the nodes sit on the codes 0, 15, ..., 255: every method
    returns the node's stored value, the exact CIELAB of the node colour
    rounded to FP32."""
    rgb = _node_codes()
    ref = O.cielab(rgb, exact=True)
    lut = O.lut_build(18)
    for method in ("trilinear", "prism", "pyramid", "tetra"):
        planes, _ = O.lut_interp(method, lut, rgb)
        for c in range(3):
            assert np.abs(planes[c] - ref[c]).max() < 1e-4, method


def pin_hsi_lut_nodes():
    """The angular HSI LUT returns the exact HSI at its nodes."""
    rgb = _node_codes()
    (H, S, I), _ = O.lut_interp_hsi(O.lut_build_hsi(18), rgb)
    eh, es, ei = O.hsi(rgb, mode="exact")
    assert _circ(H, eh).max() <= 1e-6 and np.abs(S - es).max() <= 1e-7 and np.abs(I - ei).max() <= 1e-7


def pin_gradient_finite_differences():
    """The analytic gradient of the mean Delta E*ab loss against central
    differences, for the exact and the (4,4) cube root, with points on the
    linear segment below the knee and above it."""
    rng = np.random.default_rng(3)
    x = rng.uniform(0.05, 0.95, size=(1, 3, 2, 4))
    x[0, :, 0, 0] = [0.002, 0.003, 0.001]
    x[0, :, 1, 3] = [0.0025, 0.0025, 0.0025]
    tgt = rng.uniform(-20.0, 60.0, size=x.shape)
    h = 1e-7
    for exact in (True, False):
        _, g = O.lab_loss_grad(x, tgt, exact=exact)
        fd = np.empty_like(x)
        for idx in np.ndindex(*x.shape):
            xp, xm = x.copy(), x.copy()
            xp[idx] += h
            xm[idx] -= h
            fd[idx] = (O.lab_loss_grad(xp, tgt, exact=exact, grad=False)[0] -
                       O.lab_loss_grad(xm, tgt, exact=exact, grad=False)[0]) / (2 * h)
        assert np.abs(g - fd).max() <= 1e-6 * max(1.0, np.abs(fd).max()), exact


def pin_probabilities():
    """Eq. equ_cbrt_prob and equ_sct_arcsin_arccos_prob, printed to 6 decimals."""
    g = {k: float(v) for k, v in read_golden("probabilities.txt")}
    px, py, pz = O.cube_cbrt_probs()
    assert (round(px, 6), round(py, 6), round(pz, 6)) == (
        g["P_X_over_X0_gt_knee"], g["P_Y_over_Y0_gt_knee"], g["P_Z_over_Z0_gt_knee"])
    pa, _ = O.cube_sct_probs()
    assert round(pa, 6) == g["P_arcsin"]


def pin_printed_cube_errors():
    """Table tab_cielab (4,4), Table tab_hsi n = 5 (maximum), Table tab_sct
    (5,5,5) and Table tab_lut trilinear 17^3, over every 24-bit colour."""
    row = [r for r in read_golden("tab_cielab.txt") if r[:2] == ["4", "4"]][0]
    a, b = O.cube_eps_cielab(4, 4)
    assert a == pytest.approx(float(row[2]), rel=1e-3) and b == pytest.approx(float(row[3]), rel=1e-3)
    row = [r for r in read_golden("tab_hsi.txt") if r[0] == "5"][0]
    assert abs(O.cube_eps_hsi(5)[1] - float(row[2])) <= 5e-7
    row = [r for r in read_golden("tab_sct.txt") if r[:3] == ["5", "5", "5"]][0]
    a, b = O.cube_eps_sct(5, 5, 5)
    assert abs(a - float(row[3])) <= 2e-6 and b == pytest.approx(float(row[4]), rel=1e-2)
    row = [r for r in read_golden("tab_lut.txt") if r[:2] == ["trilinear", "17"]][0]
    a, b = O.cube_eps_lut("trilinear", O.lut_build(17))
    assert abs(a - float(row[2])) <= 1e-6 and abs(b - float(row[3])) <= 2e-6


def pin_cieluv():
    """CIELUV: L* equals CIELAB's L*; grays have u* = v* = 0; the primaries'
    u', v' recovered from u*, v* and L* equal the CIE 1976 UCS values of the
    ITU-R BT.709 chromaticities (tests/golden/bt709_chromaticities.txt)."""
    rgb = np.random.default_rng(4).integers(0, 256, (3000, 3)).astype(np.uint8)
    for exact in (True, False):
        assert np.array_equal(O.cieluv(rgb, exact=exact)[0], O.cielab(rgb, exact=exact)[0])
    v = np.arange(256, dtype=np.uint8)
    _, U, V = O.cieluv(np.stack([v, v, v], axis=1), exact=True)
    assert np.abs(U).max() < 1e-9 and np.abs(V).max() < 1e-9
    rows = {r[0]: r[1:] for r in read_golden("bt709_chromaticities.txt")}

    def uv(x, y):
        d = -2.0 * x + 12.0 * y + 3.0
        return 4.0 * x / d, 9.0 * y / d
    un, vn = uv(float(rows["white"][3]), float(rows["white"][4]))
    for name in ("red", "green", "blue"):
        r, g, b, x, y = rows[name]
        L, U, V = O.cieluv(_px([int(r), int(g), int(b)]), exact=True)
        ur, vr = uv(float(x), float(y))
        assert abs(U[0] / (13.0 * L[0]) + un - ur) < 2e-5 and abs(V[0] / (13.0 * L[0]) + vn - vr) < 2e-5, name


PINS = [pin_primaries_lab, pin_grays, pin_cieluv, pin_hsi_primaries, pin_sct_primaries, pin_sct_round_trip, pin_distances,
        pin_lut_linear_reproduction, pin_lut_nodes, pin_hsi_lut_nodes, pin_gradient_finite_differences,
        pin_probabilities, pin_printed_cube_errors]


def first_failure():
    """Name of the first pin that fails, or None."""
    for pin in PINS:
        try:
            pin()
        except (AssertionError, FloatingPointError, ValueError):
            return pin.__name__
    return None


class _Using:
    """Load another build of the oracle's source in place of its library."""

    def __init__(self, path):
        self.path = path

    def __enter__(self):
        self.saved = (O._lib, O._build_lib)
        O._lib = None
        O._build_lib = lambda: self.path
        return self

    def __exit__(self, *exc):
        O._lib, O._build_lib = self.saved
        return False


@pytest.fixture(scope="module")
def mutant_libs(tmp_path_factory):
    src = open(oracle_build.SRC).read()
    d = tmp_path_factory.mktemp("oracle_mutants")
    jobs = {}
    for mid, find, repl in MUTANTS:
        assert src.count(find) == 1, mid
        c = d / (mid + ".c")
        c.write_text(src.replace(find, repl))
        jobs[mid] = (str(c), str(d / ("lib_%s.so" % mid)))
    with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 2)) as ex:
        list(ex.map(lambda a: oracle_build.compile_lib(*a), jobs.values()))
    return {mid: out for mid, (_, out) in jobs.items()}


def test_unmutated_oracle_passes_every_pin():
    """The control: the committed oracle passes the whole battery."""
    with _Using(oracle_build.build()):
        for pin in PINS:
            pin()


@pytest.mark.parametrize("mid", [m[0] for m in MUTANTS])
def test_planted_mistake_is_caught(mutant_libs, mid):
    with np.errstate(all="ignore"), _Using(mutant_libs[mid]):
        caught = first_failure()
    assert caught is not None, "no pin catches the planted mistake %s" % mid


# ------------------------------------------- mistakes in the Python side

def _cbrt44(mp, p=None, q=None):
    eps, p0, q0 = O.tables.CBRT_RAT[(4, 4)]
    rat = dict(O.tables.CBRT_RAT)
    rat[(4, 4)] = (eps, p if p is not None else p0, q if q is not None else q0)
    mp.setattr(O.tables, "CBRT_RAT", rat)


def _sct(mp, name, n, fn):
    tab = dict(getattr(O.tables, name))
    eps, c = tab[n]
    tab[n] = (eps, fn(list(c)))
    mp.setattr(O.tables, name, tab)


def _hsi_wrong_interval(mp):
    mp.setattr(O.remez, "_HSI01", {})
    mp.setattr(O.remez, "hsi_arctan_unit", lambda n: (
        list(map(float, O.remez.remez_poly(lambda x: np.arctan(np.sqrt(3.0) * x), n, 0.0, 254.0 / 256.0)[0])), 0.0))


PY_MUTANTS = [
    # the paper's tables, transcribed in oracle/tables.py
    ("table_cbrt44_digits_transposed",
     lambda mp: _cbrt44(mp, q=[4.022100e-04, 5.414536e-02, 8.221562e-01, 1.800167, 3.513617e-01])),
    ("table_cbrt44_numerator_denominator_swapped",
     lambda mp: _cbrt44(mp, p=O.tables.CBRT_RAT[(4, 4)][2], q=O.tables.CBRT_RAT[(4, 4)][1])),
    ("table_sct_f_a1_sign", lambda mp: _sct(mp, "SCT_F", 5, lambda c: c[:1] + [-c[1]] + c[2:])),
    ("table_sct_arcsin_reversed", lambda mp: _sct(mp, "SCT_ARCSIN", 5, lambda c: c[::-1])),
    ("table_sct_g_a2_scaled", lambda mp: _sct(mp, "SCT_G", 5, lambda c: c[:2] + [c[2] * 10.0] + c[3:])),
    # the RGB definition (Eq. equ_rgb_lin, equ_rgb_xyz, the D65 white)
    ("gamma_exponent_not_inverted", lambda mp: mp.setattr(O.tables, "BT709_GAMMA",
                                                          dict(O.tables.BT709_GAMMA, exponent=0.45))),
    ("white_point_digit", lambda mp: mp.setattr(O.tables, "D65_WHITE", [0.950456, 1.0, 1.088058])),
    ("matrix_rows_swapped", lambda mp: mp.setattr(O.tables, "BT709_MATRIX",
                                                  O.tables.BT709_MATRIX[6:] + O.tables.BT709_MATRIX[3:6] +
                                                  O.tables.BT709_MATRIX[:3])),
    # the HSI set: a fit on the printed rows' interval instead of [0, 1]
    ("hsi_fit_on_printed_interval", _hsi_wrong_interval),
]


@pytest.mark.parametrize("mid", [m[0] for m in PY_MUTANTS])
def test_planted_python_mistake_is_caught(monkeypatch, mid):
    patch = dict(PY_MUTANTS)[mid]
    with monkeypatch.context() as mp:
        patch(mp)
        with np.errstate(all="ignore"):
            caught = first_failure()
    assert caught is not None, "no pin catches the planted mistake %s" % mid
