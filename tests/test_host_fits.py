"""The library's host-side minimax fits (``mact_fit_cbrt_rational``,
``mact_fit_hsi_arctan``), checked on the CPU: no GPU and no handle needed.

The library's Remez exchange (C++) and the oracle's (numpy) are separate
implementations of the same best-approximation problems, whose solutions
are unique; they must agree.  Beyond that, each library fit is pinned by the
alternation theorem (n + m + 2 or n + 2 sign-alternating extrema of equal
size, found by the oracle's extremum search) and, for arctan, by the
maxima the paper prints in Table tab_hsi."""
import ctypes

import numpy as np
import pytest

import oracle as O
from conftest import read_golden
from oracle import remez
from paper_1009_0854_gb300 import mact

CBRT_LO = 0.008856


def _rat(p, q, x):
    return np.polyval(np.asarray(p)[::-1], x) / np.polyval(np.asarray(q)[::-1], x)


@pytest.mark.parametrize("n,m", [(1, 1), (2, 2), (3, 3), (4, 4), (3, 5), (5, 3), (2, 6), (5, 5), (6, 6)])
def test_cbrt_rational_fit_matches_oracle(n, m):
    p, q, e = mact.mact_fit_cbrt_rational(n, m)
    po, qo, eo = O.cbrt_minimax(n, m)
    assert q[0] == 1.0 and len(p) == n + 1 and len(q) == m + 1
    x = np.exp(np.linspace(np.log(CBRT_LO), 0.0, 20001))
    assert abs(e - eo) <= 1e-5 * eo
    assert np.abs(_rat(p, q, x) - _rat(po, qo, x)).max() <= 1e-4 * eo
    assert np.all(np.polyval(np.asarray(q)[::-1], x) > 0.0)        # no pole on the interval


@pytest.mark.parametrize("n,m", [(2, 2), (4, 4), (6, 6)])
def test_cbrt_rational_fit_equioscillates(n, m):
    """Alternation theorem: n + m + 2 alternating extrema, all of size E."""
    p, q, e = mact.mact_fit_cbrt_rational(n, m)
    xs, es = remez.alternating_extrema(lambda t: np.cbrt(t) - _rat(p, q, t), CBRT_LO, 1.0)
    big = np.abs(es) >= 0.999 * e
    assert big.sum() >= n + m + 2
    assert np.abs(es).max() <= e * (1.0 + 1e-6)


@pytest.mark.parametrize("row", read_golden("tab_hsi.txt"), ids=lambda r: "n%s" % r[0])
def test_hsi_arctan_fit_matches_oracle_and_paper(row):
    """Degrees 2..5: the library's fit equals the oracle's; its levelled error
    is the maximum Table tab_hsi prints (to the printed 6 decimals), and it
    equioscillates at n + 2 points."""
    n = int(row[0])
    c, e = mact.mact_fit_hsi_arctan(n)
    co = O.hsi_coeffs(n)
    x = np.linspace(0.0, 1.0, 20001)
    f = lambda t: np.arctan(np.sqrt(3.0) * t)
    assert np.abs(np.polyval(c[::-1], x) - np.polyval(np.asarray(co)[::-1], x)).max() <= 1e-6 * e
    assert abs(e - float(row[2])) <= 5e-7
    xs, es = remez.alternating_extrema(lambda t: f(t) - np.polyval(c[::-1], t), 0.0, 1.0)
    assert (np.abs(es) >= 0.999 * e).sum() >= n + 2


def test_fit_argument_checks():
    L = mact.lib()
    buf = (ctypes.c_double * 7)()
    for n, m in [(0, 2), (2, 0), (7, 2), (2, 7)]:
        assert L.mact_fit_cbrt_rational(n, m, buf, buf, None) == mact.MACT_E_INVAL
    assert L.mact_fit_cbrt_rational(2, 2, None, buf, None) == mact.MACT_E_INVAL
    assert L.mact_fit_cbrt_rational(2, 2, buf, None, None) == mact.MACT_E_INVAL
    for n in (1, 6):
        assert L.mact_fit_hsi_arctan(n, buf, None) == mact.MACT_E_INVAL
    assert L.mact_fit_hsi_arctan(3, None, None) == mact.MACT_E_INVAL
    assert L.mact_fit_hsi_arctan(3, buf, None) == mact.MACT_OK      # max_err may be NULL
