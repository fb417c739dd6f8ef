"""Closed forms, textbook values and invariants that pin the oracle's
per-pixel transforms independently of its own formulas."""
import math

import numpy as np
import pytest

import oracle as O
from oracle import tables
from conftest import read_golden

LAB_ROWS = [(n, m) for (n, m) in tables.CBRT_RAT]


def _px(*rgb):
    return np.array([rgb], dtype=np.uint8)


def test_primaries_match_textbook_lab():
    """CIELAB of the BT.709 primaries/secondaries under D65 agrees with the
    standard tabulated values (two decimals; the paper's 6-digit matrix and
    white move them by at most 0.012)."""
    for row in read_golden("primaries_lab.txt"):
        r, g, b = (int(v) for v in row[:3])
        ref = [float(v) for v in row[3:]]
        L, A, B = O.cielab(_px(r, g, b), exact=True)
        assert abs(L[0] - ref[0]) < 0.02 and abs(A[0] - ref[1]) < 0.02 and abs(B[0] - ref[2]) < 0.02


def test_white_and_grays_exact():
    """White gives t = (1,1,1) -> L* = 100, a* = b* = 0; every gray has
    t_X = t_Y = t_Z because each matrix row sums to its white component, so
    a* = b* = 0."""
    v = np.arange(256, dtype=np.uint8)
    grays = np.stack([v, v, v], axis=1)
    L, A, B = O.cielab(grays, exact=True)
    assert abs(L[255] - 100.0) < 1e-9
    assert np.abs(A).max() < 1e-9 and np.abs(B).max() < 1e-9
    assert np.all(np.diff(L) > 0)


@pytest.mark.parametrize("nm", LAB_ROWS)
def test_grays_mact(nm):
    """The gray invariant holds for the approximant too: f is applied to three
    equal arguments."""
    v = np.arange(256, dtype=np.uint8)
    _, A, B = O.cielab(np.stack([v, v, v], axis=1), n=nm[0], m=nm[1])
    assert np.abs(A).max() < 1e-9 and np.abs(B).max() < 1e-9


def test_mact_lightness_error_bounded_by_table_eps():
    """For grays only L* differs from the exact transform, by 116 |p/q - cbrt|,
    which Table tab_cbrt_rat bounds by 116 eps^A_max on [0.008856, 1]."""
    v = np.arange(256, dtype=np.uint8)
    g = np.stack([v, v, v], axis=1)
    Le, _, _ = O.cielab(g, exact=True)
    for (n, m), (eps, _, _) in tables.CBRT_RAT.items():
        La, _, _ = O.cielab(g, n=n, m=m)
        assert np.abs(La - Le).max() <= 116 * eps * 1.002


def test_gamma_inverse_bt709():
    """Eq. equ_rgb_lin: 0 -> 0, 1 -> 1, linear below 0.081 with slope 1/4.5,
    and the two branches meet at the threshold to within 0.4% (BT.709 has a
    small jump there: 0.018 vs 0.017945)."""
    assert O.gamma_inverse(0.0) == 0.0
    assert abs(O.gamma_inverse(1.0) - 1.0) < 1e-15
    assert abs(O.gamma_inverse(0.05) - 0.05 / 4.5) < 1e-15
    lo = 0.081 / 4.5
    hi = O.gamma_inverse(0.081)
    assert 2e-3 < abs(hi - lo) / lo < 4e-3
    # BT.709 mid-gray: ((0.5 + 0.099) / 1.099) ** (1 / 0.45)
    assert O.gamma_inverse(0.5) == pytest.approx(math.exp(math.log(0.599 / 1.099) / 0.45), rel=1e-14)


def test_linear_segment_below_knee():
    """t <= 0.008856 uses 7.787 t + 16/116 in both paths, so codes whose three
    t values are below the knee give identical exact and MACT results."""
    rgb = np.array([[1, 2, 3], [5, 5, 5], [0, 0, 9], [3, 0, 0]], dtype=np.uint8)
    e = O.cielab(rgb, exact=True)
    a = O.cielab(rgb)
    for x, y in zip(e, a):
        assert np.array_equal(x, y)
    # black: f = 16/116 -> L* = 0
    L, A, B = O.cielab(_px(0, 0, 0), exact=True)
    assert L[0] == pytest.approx(0.0, abs=1e-12)


def test_hsi_primaries_exact():
    """Hue of the primaries and secondaries (radians), S and I closed forms."""
    pi = math.pi
    cases = {(255, 0, 0): 0.0, (255, 255, 0): pi / 3, (0, 255, 0): 2 * pi / 3,
             (0, 255, 255): pi, (0, 0, 255): 4 * pi / 3, (255, 0, 255): 5 * pi / 3}
    for rgb, h in cases.items():
        H, S, I = O.hsi(_px(*rgb), mode="exact")
        assert H[0] == pytest.approx(h, abs=1e-12)
        assert S[0] == pytest.approx(1.0, abs=1e-15)
        assert I[0] == pytest.approx(sum(rgb) / 765.0, abs=1e-15)
    v = np.arange(256, dtype=np.uint8)
    H, S, I = O.hsi(np.stack([v, v, v], axis=1), mode="approx")
    assert np.all(H == 0.0) and np.all(S == 0.0)
    assert np.allclose(I, v / 255.0, atol=1e-15)


def test_hsi_mact_primaries():
    """MACT hue: red takes the "R > B -> 0" branch exactly; green and blue sit
    at |x| = 1, where the [0, 1] fit's error is its full eps^A."""
    for n in (2, 3, 4, 5):
        c, E = O.remez.hsi_arctan_unit(n)
        H, _, _ = O.hsi(np.array([[255, 0, 0], [0, 255, 0], [0, 0, 255]], dtype=np.uint8), n=n)
        assert H[0] == 0.0
        assert abs(H[1] - 2 * math.pi / 3) == pytest.approx(E, rel=1e-6)
        assert abs(H[2] - 4 * math.pi / 3) == pytest.approx(E, rel=1e-6)


def test_hsi_approx_hue_error_bounded():
    """|H_mact - H_exact| <= eps^A of the fit, on random colours."""
    rng = np.random.default_rng(7)
    rgb = rng.integers(0, 256, size=(200000, 3), dtype=np.uint8)
    He, _, _ = O.hsi(rgb, mode="exact")
    for n in (2, 3, 4, 5):
        _, E = O.remez.hsi_arctan_unit(n)
        Ha, _, _ = O.hsi(rgb, n=n)
        d = np.abs(He - Ha)
        d = np.minimum(d, 2 * math.pi - d)
        assert d.max() <= E * (1 + 1e-9)


def test_d_hsi():
    """Eq. equ_hsi_dist: identical pixels -> 0; hue difference wraps at pi;
    opposite hues at equal S, I give 2 s."""
    assert O.d_hsi([1.0, 0.5, 0.3], [1.0, 0.5, 0.3]) == 0.0
    assert O.d_hsi([0.1, 0.5, 0.3], [2 * math.pi - 0.1, 0.5, 0.3]) == pytest.approx(
        O.d_hsi([0.1, 0.5, 0.3], [0.3, 0.5, 0.3]), rel=1e-12)
    assert O.d_hsi([0.0, 0.7, 0.2], [math.pi, 0.7, 0.2]) == pytest.approx(1.4, rel=1e-12)
    assert O.d_hsi([0.0, 0.0, 0.2], [1.0, 0.0, 0.5]) == pytest.approx(0.3, rel=1e-12)


def test_delta_e():
    assert O.delta_e([50, 10, -10], [53, 14, -10]) == pytest.approx(5.0)


def test_sct_closed_forms_exact_and_mact():
    """Eq. equ_rgb_sct: gray v -> L = v sqrt(3), A = arccos(1/sqrt(3)),
    B = pi/4; blue -> A = 0; red -> A = pi/2, B = 0; green -> B = pi/2;
    black -> all 0.  MACT angles agree to within the fits' eps^A."""
    s3 = math.sqrt(3.0)
    for exact in (True, False):
        tolA = 0.0 if exact else max(tables.SCT_ARCSIN[5][0], tables.SCT_ARCCOS[5][0]) * 1.5
        tolB = 0.0 if exact else max(tables.SCT_F[5][0], tables.SCT_G[5][0]) * 1.5
        L, A, B = O.sct(np.array([[100, 100, 100]], dtype=np.uint8), exact=exact)
        assert L[0] == pytest.approx(100 * s3, rel=1e-15)
        assert abs(A[0] - math.acos(1 / s3)) <= tolA + 1e-15
        assert abs(B[0] - math.pi / 4) <= tolB + 1e-15
        L, A, B = O.sct(np.array([[0, 0, 255], [255, 0, 0], [0, 255, 0], [0, 0, 0]], dtype=np.uint8),
                        exact=exact)
        assert abs(A[0]) <= tolA + 1e-15 and B[0] == 0.0
        assert abs(A[1] - math.pi / 2) <= tolA + 1e-15 and abs(B[1]) <= tolB + 1e-15
        assert B[2] == pytest.approx(math.pi / 2, abs=1e-15)
        assert L[3] == 0.0 and A[3] == 0.0 and B[3] == 0.0


def test_sct_inverse_roundtrip():
    """Eq. equ_sct_rgb inverts Eq. equ_rgb_sct."""
    rng = np.random.default_rng(3)
    rgb = rng.integers(0, 256, size=(20000, 3), dtype=np.uint8)
    L, A, B = O.sct(rgb, exact=True)
    for i in range(0, 20000, 97):
        back = O.sct_inverse(L[i], A[i], B[i])
        assert np.allclose(back, rgb[i].astype(float), atol=1e-9)


def test_sct_mact_angle_error_bounded():
    """|A_mact - A_exact| and |B_mact - B_exact| stay within the printed
    eps^A of the fits used (plus their 7-digit rounding)."""
    rng = np.random.default_rng(5)
    rgb = rng.integers(0, 256, size=(300000, 3), dtype=np.uint8)
    _, Ae, Be = O.sct(rgb, exact=True)
    for n, m, r in [(4, 4, 4), (5, 5, 5)]:
        _, Aa, Ba = O.sct(rgb, n=n, m=m, r=r)
        epsA = max(tables.SCT_ARCSIN[n][0], tables.SCT_ARCCOS[m][0])
        epsB = max(tables.SCT_F[r][0], tables.SCT_G[r][0])
        assert np.abs(Aa - Ae).max() <= 1.5 * epsA
        assert np.abs(Ba - Be).max() <= 1.05 * epsB
