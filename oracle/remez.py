"""Remez exchange for minimax polynomials and rationals, plus an
equioscillation checker.

Test infrastructure (part of the oracle).  The paper computes every
approximant with the Remez exchange algorithm (Section "Overview of Minimax
Approximation Theory", citing Fraser 1965 for the implementation); it prints
the results but not the program.  This module restates the method from its
definition so that tests can (a) confirm that a printed table row is the
minimax fit it claims to be and (b) produce the HSI arctan(sqrt(3) x) fit on
[0, 1], which the oracle uses as its default HSI set.

Method (Chebyshev alternation theorem): p* is the minimax polynomial of degree
n for f on [a, b] iff the error f - p* reaches its maximum modulus at n+2
points with alternating signs.  The exchange algorithm repeatedly
  1. solves f(x_j) - p(x_j) = (-1)^j E on a reference x_0 < ... < x_{n+1};
  2. locates the extrema of the resulting error and takes them as the next
     reference;
until the extrema have equal modulus.  For a rational p/q (q(0) normalised to
1) the reference system p(x_j) - (f(x_j) - (-1)^j E) q(x_j) = 0 is nonlinear
in E; it is solved by fixed-point iteration on E, each step a linear solve.
Error extrema are located on a dense grid and refined by golden-section search.
"""
import math

import numpy as np


def _vander(x, n):
    return np.vander(np.asarray(x, dtype=np.float64), n + 1, increasing=True)


def poly_eval(c, x):
    """a0 + a1 x + ... (plain sum of powers)."""
    x = np.asarray(x, dtype=np.float64)
    return _vander(x.ravel(), len(c) - 1).dot(np.asarray(c, dtype=np.float64)).reshape(x.shape)


def dense_grid(a, b, npts=200001):
    """Uniform grid, plus a geometric cluster near each end so that endpoint
    singularities (cube root at 0) are resolved."""
    u = np.linspace(a, b, npts)
    span = b - a
    g = span * np.logspace(-12, -1, 2000)
    pts = np.concatenate([u, a + g, b - g])
    pts = pts[(pts >= a) & (pts <= b)]
    return np.unique(pts)


def _golden_max(h, lo, hi, iters=80):
    """Maximise h on [lo, hi] by golden-section search."""
    invphi = (math.sqrt(5.0) - 1.0) / 2.0
    c = hi - invphi * (hi - lo)
    d = lo + invphi * (hi - lo)
    hc, hd = h(c), h(d)
    for _ in range(iters):
        if hc > hd:
            hi, d, hd = d, c, hc
            c = hi - invphi * (hi - lo)
            hc = h(c)
        else:
            lo, c, hc = c, d, hd
            d = lo + invphi * (hi - lo)
            hd = h(d)
    x = 0.5 * (lo + hi)
    return x


def alternating_extrema(err, a, b, grid=None, refine=True):
    """Local extrema of the error function err on [a, b], one per run of
    constant sign, each refined by golden-section search.  Returns arrays
    (x, e) in increasing x; consecutive entries alternate in sign."""
    x = dense_grid(a, b) if grid is None else grid
    e = err(x)
    s = np.sign(e)
    s[s == 0] = 1
    xs, es = [], []
    start = 0
    n = len(x)
    for i in range(1, n + 1):
        if i == n or s[i] != s[start]:
            seg = slice(start, i)
            k = start + int(np.argmax(np.abs(e[seg])))
            xk = x[k]
            if refine and 0 < k < n - 1:
                sign = s[k]
                xk = _golden_max(lambda t: sign * float(err(np.array([t]))[0]), x[k - 1], x[k + 1])
                if sign * float(err(np.array([xk]))[0]) < sign * e[k]:
                    xk = x[k]
            xs.append(xk)
            es.append(float(err(np.array([xk]))[0]))
            start = i
    return np.array(xs), np.array(es)


def _pick_reference(xs, es, npts):
    """Choose npts consecutive alternating extrema that contain the largest."""
    xs, es = list(xs), list(es)
    while len(xs) > npts:
        kmax = int(np.argmax(np.abs(es)))
        # drop the smaller end, never the global maximum
        if (abs(es[0]) <= abs(es[-1]) and kmax != 0) or kmax == len(xs) - 1:
            xs.pop(0); es.pop(0)
        else:
            xs.pop(); es.pop()
    return np.array(xs), np.array(es)


def remez_poly(f, n, a, b, tol=1e-12, maxiter=60):
    """Minimax polynomial of degree n for f on [a, b].
    Returns (coefficients ascending, E, extrema x, extrema e)."""
    k = np.arange(n + 2)
    ref = 0.5 * (a + b) - 0.5 * (b - a) * np.cos(np.pi * k / (n + 1))
    grid = dense_grid(a, b)
    c = None
    for _ in range(maxiter):
        A = np.hstack([_vander(ref, n), ((-1.0) ** k)[:, None]])
        sol = np.linalg.solve(A, f(ref))
        c, E = sol[:-1], sol[-1]
        err = lambda x, c=c: f(x) - poly_eval(c, x)
        xs, es = alternating_extrema(err, a, b, grid)
        if len(xs) < n + 2:
            break
        xs, es = _pick_reference(xs, es, n + 2)
        emax, emin = np.max(np.abs(es)), np.min(np.abs(es))
        ref = xs
        if emax - emin <= tol * emax:
            break
    return c, float(emax), xs, es


def remez_rational(f, n, m, a, b, init=None, tol=1e-10, maxiter=80, inner=60):
    """Minimax rational p_n/q_m for f on [a, b], normalised to q(0) = 1.
    init: optional (p, q) starting guess (any normalisation).
    Returns (p, q, E, extrema x, extrema e)."""
    N = n + m + 2
    k = np.arange(N)
    sgn = (-1.0) ** k
    ref = 0.5 * (a + b) - 0.5 * (b - a) * np.cos(np.pi * k / (N - 1))
    grid = dense_grid(a, b)
    if init is not None:
        p0 = np.asarray(init[0], dtype=np.float64)
        q0 = np.asarray(init[1], dtype=np.float64)
        p0, q0 = p0 / q0[0], q0 / q0[0]
        E = 0.0
    else:
        q0 = np.zeros(m + 1)
        q0[0] = 1.0
        E = 0.0
    q = q0.copy()
    p = None
    for _ in range(maxiter):
        fr = f(ref)
        for _ in range(inner):
            qo = poly_eval(q, ref)
            # unknowns: p_0..p_n, q_1..q_m, E
            A = np.zeros((N, N))
            A[:, : n + 1] = _vander(ref, n)
            Vq = _vander(ref, m)
            A[:, n + 1: n + 1 + m] = -(fr[:, None]) * Vq[:, 1:]
            A[:, -1] = sgn * qo
            rhs = fr.copy()
            sol = np.linalg.solve(A, rhs)
            p = sol[: n + 1]
            qn = np.concatenate([[1.0], sol[n + 1: n + 1 + m]])
            En = sol[-1]
            done = abs(En - E) <= 1e-15 + 1e-13 * abs(En) and np.allclose(qn, q, rtol=1e-13, atol=1e-15)
            q, E = qn, En
            if done:
                break
        err = lambda x, p=p, q=q: f(x) - poly_eval(p, x) / poly_eval(q, x)
        xs, es = alternating_extrema(err, a, b, grid)
        if len(xs) < N:
            break
        xs, es = _pick_reference(xs, es, N)
        emax, emin = np.max(np.abs(es)), np.min(np.abs(es))
        ref = xs
        if emax - emin <= tol * emax:
            break
    return p, q, float(emax), xs, es


def max_error(err, a, b):
    """max |err| on [a, b] over the dense grid with refined extrema."""
    xs, es = alternating_extrema(err, a, b)
    return float(np.max(np.abs(es))), xs, es


def decimal_rounding_bound(coeffs, xmax):
    """First-order bound on the change of a polynomial's value when each
    coefficient is rounded to the 7 significant digits the paper prints:
    sum_i (half a unit in the last printed digit of a_i) * xmax^i."""
    tot = 0.0
    for i, a in enumerate(coeffs):
        if a == 0.0:
            continue
        e = math.floor(math.log10(abs(a)))
        half_ulp = 0.5 * 10.0 ** (e - 6)
        tot += half_ulp * xmax ** i
    return tot


# -- the oracle's HSI default set ------------------------------------------

_HSI01 = {}


def hsi_arctan_unit(n):
    """Minimax polynomial of degree n for arctan(sqrt(3) x) on [0, 1]
    (the domain Kender's formula needs, since |x| = 1 occurs)."""
    if n not in _HSI01:
        c, E, _, _ = remez_poly(lambda x: np.arctan(np.sqrt(3.0) * x), n, 0.0, 1.0)
        _HSI01[n] = (list(map(float, c)), E)
    return _HSI01[n]
