"""Pins of the oracle's CIELUV (the variant the paper's Conclusions name;
CIE 1976 L*u*v*, defined by the CIE rather than printed in the paper),
independent of its own formulas:

- L* is CIELAB's L* (already pinned against textbook values and the printed
  error tables), in both the exact and the MACT form;
- white gives (100, 0, 0) and every gray has u* = v* = 0;
- the BT.709 primaries' chromaticities u', v', recovered from the oracle's
  u*, v* and L*, equal those computed from the ITU-R BT.709 xy values through
  the CIE 1976 UCS relation (tests/golden/bt709_chromaticities.txt);
- the MACT L* error is bounded by 116 times the printed approximant error."""
import numpy as np

import oracle as O
from oracle import tables
from conftest import read_golden


def _uv_from_xy(x, y):
    d = -2.0 * x + 12.0 * y + 3.0
    return 4.0 * x / d, 9.0 * y / d


def test_white_black_and_grays():
    v = np.arange(256, dtype=np.uint8)
    grays = np.stack([v, v, v], axis=1)
    for exact in (True, False):
        L, U, V = O.cieluv(grays, exact=exact)
        assert np.abs(U).max() < 1e-9 and np.abs(V).max() < 1e-9
        assert L[0] == 0.0 and U[0] == 0.0 and V[0] == 0.0
        assert np.all(np.diff(L) > 0)
    L, U, V = O.cieluv(grays[255:], exact=True)
    assert abs(L[0] - 100.0) < 1e-9


def test_lightness_is_cielab_lightness():
    rgb = np.random.default_rng(5).integers(0, 256, size=(20000, 3), dtype=np.uint8)
    for exact in (True, False):
        assert np.array_equal(O.cieluv(rgb, exact=exact)[0], O.cielab(rgb, exact=exact)[0])


def test_primary_chromaticities_match_bt709():
    """u' = u*/(13 L*) + u'n and v' = v*/(13 L*) + v'n of each primary agree
    with the BT.709 xy values to the rounding of the paper's 6-digit matrix
    and white (a few 1e-6)."""
    rows = {r[0]: r[1:] for r in read_golden("bt709_chromaticities.txt")}
    un, vn = _uv_from_xy(float(rows["white"][3]), float(rows["white"][4]))
    for name in ("red", "green", "blue"):
        r, g, b, x, y = rows[name]
        L, U, V = O.cieluv(np.array([[int(r), int(g), int(b)]], dtype=np.uint8), exact=True)
        u_ref, v_ref = _uv_from_xy(float(x), float(y))
        assert abs(U[0] / (13.0 * L[0]) + un - u_ref) < 2e-5, name
        assert abs(V[0] / (13.0 * L[0]) + vn - v_ref) < 2e-5, name


def test_mact_lightness_error_within_printed_bound():
    """|L*_MACT - L*_exact| = 116 |p/q(t) - t^(1/3)| <= 116 eps^A_max of
    Table tab_cbrt_rat (4,4) (printed to 7 digits: 0.5% slack)."""
    eps = tables.CBRT_RAT[(4, 4)][0]
    rgb = np.random.default_rng(6).integers(0, 256, size=(200000, 3), dtype=np.uint8)
    la = O.cieluv(rgb)[0]
    le = O.cieluv(rgb, exact=True)[0]
    assert np.abs(la - le).max() <= 116.0 * eps * 1.005
