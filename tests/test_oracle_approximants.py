"""The printed approximant tables against minimax theory: each row's maximum
error on its interval equals the printed eps^A_max, its error alternates in
sign n+2 (polynomial) or n+m+2 (rational) times, and an independent Remez
exchange recomputes the converged rows (Section "Overview of Minimax
Approximation Theory" and Tables tab_cbrt_poly ... tab_g)."""
import numpy as np
import pytest

from oracle import remez, tables as T

SQ3 = np.sqrt(3.0)

POLY_TABLES = [
    ("tab_cbrt_poly", T.CBRT_POLY, np.cbrt, T.CBRT_POLY_INTERVAL),
    ("tab_arctan", T.HSI_ARCTAN, lambda x: np.arctan(SQ3 * x), T.HSI_PRINTED_INTERVAL),
    ("tab_arcsin", T.SCT_ARCSIN, lambda y: 2.0 * np.arcsin(y / np.sqrt(2.0)), T.SCT_ARCSIN_INTERVAL),
    ("tab_arccos", T.SCT_ARCCOS, np.arccos, T.SCT_ARCCOS_INTERVAL),
    ("tab_f", T.SCT_F, np.arctan, T.SCT_F_INTERVAL),
    ("tab_g", T.SCT_G, lambda w: np.pi / 2 - np.arctan(w), T.SCT_G_INTERVAL),
]
POLY_ROWS = [(name, n, f, iv, tab[n]) for name, tab, f, iv in POLY_TABLES for n in tab]


def _tol(eps, coeffs, xmax):
    return max(remez.decimal_rounding_bound(coeffs, xmax), 2e-3 * eps)


@pytest.mark.parametrize("row", POLY_ROWS, ids=lambda r: "%s_n%d" % (r[0], r[1]))
def test_printed_polynomial_max_error_and_alternation(row):
    """max |f - P| on the interval equals eps^A_max to within the effect of
    rounding the coefficients to the printed 7 digits, and the error has
    n+2 alternating extrema."""
    name, n, f, (a, b), (eps, c) = row
    err = lambda x: f(x) - remez.poly_eval(c, x)
    emax, xs, es = remez.max_error(err, a, b)
    assert abs(emax - eps) <= _tol(eps, c, b)
    big = np.abs(es) >= 0.5 * eps
    assert big.sum() >= n + 2


@pytest.mark.parametrize("row", sorted(T.CBRT_RAT), ids=lambda r: "n%d_m%d" % r)
def test_printed_rational_max_error_and_alternation(row):
    """Table tab_cbrt_rat: max |cbrt - p/q| on [0.008856, 1] equals the
    printed eps^A_max to 0.2%, and the error alternates n+m+2 times.  (The
    rows with n+m >= 6 are not equal-ripple: their ripple decays away from the
    left end, i.e. the paper's exchange stopped before convergence; the
    printed eps is the left-end error.)"""
    n, m = row
    eps, p, q = T.CBRT_RAT[row]
    a, b = T.CBRT_RAT_INTERVAL
    err = lambda x: np.cbrt(x) - remez.poly_eval(p, x) / remez.poly_eval(q, x)
    emax, xs, es = remez.max_error(err, a, b)
    assert emax == pytest.approx(eps, rel=2e-3)
    assert len(xs) == n + m + 2
    assert np.all(np.sign(es[1:]) == -np.sign(es[:-1]))
    assert abs(es[0]) == pytest.approx(eps, rel=1e-3)


EQUAL_RIPPLE_POLY = [r for r in POLY_ROWS if not (r[0] == "tab_arccos" and r[1] == 5)]


@pytest.mark.parametrize("row", EQUAL_RIPPLE_POLY, ids=lambda r: "%s_n%d" % (r[0], r[1]))
def test_remez_recomputes_printed_polynomials(row):
    """An independent Remez exchange on the same interval reproduces each
    printed polynomial row to 5 significant digits (the cube-root n=2 row to
    3: the paper's own fit stopped 0.15% above the true minimax error), and
    the true minimax error never exceeds the printed one by more than the
    printed rounding."""
    name, n, f, (a, b), (eps, c) = row
    cc, E, xs, es = remez.remez_poly(f, n, a, b)
    scale = np.maximum(np.abs(c), 1e-2)
    rel = 2e-3 if (name == "tab_cbrt_poly" and n == 2) else 1e-4
    assert np.max(np.abs(cc - np.array(c)) / scale) <= rel
    assert E <= eps * (1 + 1e-4)
    assert np.max(np.abs(es)) - np.min(np.abs(es)) <= 1e-8 * E


def test_arccos_m5_dominated_by_printed_rounding():
    """Table tab_arccos m=5: the printed a0 = 1.570798 carries a rounding
    error (up to 5e-7) comparable to eps^A = 1.19e-6, so the printed row is
    not equal-ripple; the Remez fit is, and matches eps^A to 0.2%."""
    eps, c = T.SCT_ARCCOS[5]
    cc, E, xs, es = remez.remez_poly(np.arccos, 5, *T.SCT_ARCCOS_INTERVAL)
    assert E == pytest.approx(eps, rel=2e-3)
    assert np.max(np.abs(cc - np.array(c))) <= 1e-4


@pytest.mark.parametrize("row", [(2, 2), (2, 3)], ids=lambda r: "n%d_m%d" % r)
def test_remez_recomputes_converged_rationals(row):
    """For the low-degree rationals the paper's fit is close to equal ripple
    (extrema within 0.6% of each other); an independent rational Remez
    converges to the same function: coefficients (normalised to q0 = 1) agree
    to 3e-3 and the minimax error is at most the printed one."""
    eps, p, q = T.CBRT_RAT[row]
    pp, qq, E, xs, es = remez.remez_rational(np.cbrt, row[0], row[1], *T.CBRT_RAT_INTERVAL)
    pn, qn = np.array(p) / q[0], np.array(q) / q[0]
    assert np.max(np.abs(pp - pn) / np.abs(pn)) < 3e-3
    assert np.max(np.abs(qq - qn) / np.abs(qn)) < 3e-3
    assert E <= eps
    assert E == pytest.approx(eps, rel=5e-3)
    assert np.max(np.abs(es)) - np.min(np.abs(es)) <= 1e-6 * E


def test_remez_rational_is_optimal_for_every_printed_degree():
    """For (4,4) the true minimax rational has an error well below the printed
    eps (the printed row is an unconverged fit); the exchange still ends
    equal-ripple with n+m+2 alternations."""
    eps, p, q = T.CBRT_RAT[(4, 4)]
    pp, qq, E, xs, es = remez.remez_rational(np.cbrt, 4, 4, *T.CBRT_RAT_INTERVAL)
    assert E < eps
    assert len(xs) == 10
    assert np.max(np.abs(es)) - np.min(np.abs(es)) <= 1e-6 * E


def test_hsi_unit_interval_fit():
    """The oracle's default HSI set: minimax for arctan(sqrt(3) x) on [0, 1],
    equal ripple with n+2 alternations, and the error at x = 1 is its full
    minimax error (the hue of pure green/blue)."""
    for n in (2, 3, 4, 5):
        c, E = remez.hsi_arctan_unit(n)
        err = lambda x: np.arctan(SQ3 * x) - remez.poly_eval(c, x)
        emax, xs, es = remez.max_error(err, 0.0, 1.0)
        assert len(xs) == n + 2
        assert emax == pytest.approx(E, rel=1e-8)
        assert abs(err(np.array([1.0]))[0]) == pytest.approx(E, rel=1e-8)


def test_hsi_printed_n2_sign():
    """Table tab_arctan prints a2 = +7.497879e-01 for n = 2; with that sign
    the error at x = 1 is about 1.5 rad, so the oracle reads it as minus."""
    bad = T.HSI_ARCTAN_PRINTED_N2_AS_PRINTED
    good = T.HSI_ARCTAN[2][1]
    x = np.array([1.0])
    assert abs(np.arctan(SQ3 * x) - remez.poly_eval(bad, x))[0] > 1.0
    cc, E, _, _ = remez.remez_poly(lambda x: np.arctan(SQ3 * x), 2, *T.HSI_PRINTED_INTERVAL)
    assert cc[2] == pytest.approx(good[2], rel=1e-4)


# ---- cube-root rationals beyond the printed degrees ----------------------

import oracle as O  # noqa: E402


@pytest.mark.parametrize("n,m", [(4, 4), (5, 5), (6, 6), (5, 6)])
def test_fitted_cube_root_rational_is_minimax(n, m):
    """The oracle's Remez fit of t^(1/3) on [0.008856, 1] (the interval of
    Figure fig_cbrt): by Chebyshev's alternation theorem the minimax rational
    has n+m+2 error extrema of alternating sign and equal modulus; a dense
    log-spaced grid, independent of the exchange's own, finds nothing above
    that level, and the denominator has no zero on the interval."""
    p, q, E = O.cbrt_minimax(n, m)
    xs, es = O.cbrt_minimax_extrema(n, m)
    es = np.asarray(es)
    assert len(xs) == n + m + 2
    assert np.all(np.sign(es[1:]) == -np.sign(es[:-1]))
    assert np.max(np.abs(es)) - np.min(np.abs(es)) <= 1e-4 * E
    t = np.geomspace(0.008856, 1.0, 400001)
    den = np.polyval(np.asarray(q)[::-1], t)
    assert np.all(den > 0)
    err = np.cbrt(t) - np.polyval(np.asarray(p)[::-1], t) / den
    assert np.max(np.abs(err)) <= E * (1 + 1e-4)


def test_fitted_errors_fall_with_degree_and_beat_the_printed_row():
    """Each added degree lowers the minimax error, and the converged (4,4)
    lies below the printed (4,4) row's error (an unconverged fit)."""
    eps44_printed = T.CBRT_RAT[(4, 4)][0]
    E = {d: O.cbrt_minimax(*d)[2] for d in [(4, 4), (5, 5), (6, 6)]}
    assert E[(6, 6)] < E[(5, 5)] < E[(4, 4)] < eps44_printed


def test_fitted_six_six_cube_error_below_1e4():
    """Over every 24-bit colour the (6,6) fit's CIELAB error (Delta E*ab in
    FP64 against the exact transform) stays below 1e-4: the approximant
    matches the exact transform to the level of FP32 rounding."""
    p, q, _ = O.cbrt_minimax(6, 6)
    avg, mx = O.cube_eps_cielab(p=p, q=q)
    assert mx < 1e-4 and avg < mx
    p4, q4, _ = O.cbrt_minimax(4, 4)
    assert O.cube_eps_cielab(p=p4, q=q4)[1] > 10 * mx
