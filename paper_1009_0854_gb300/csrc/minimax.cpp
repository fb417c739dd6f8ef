// minimax.cpp -- Remez exchange in double precision, run at mact_create:
//  - the polynomial fit of arctan(sqrt(3) x) on [0, 1] for the HSI transform
//    (Section "Approximation of the Inverse Tangent Function": the paper's
//    fits come from the Remez exchange algorithm; Kender's formula needs the
//    whole of |x| <= 1);
//  - rational fits p_n/q_m of t^(1/3) on [0.008856, 1] (the interval of
//    Figure fig_cbrt) for degrees the cube-root table does not print.
//
// Chebyshev alternation: the degree-n minimax polynomial makes the error
// reach its maximum modulus n+2 times with alternating signs (n+m+2 times
// for a non-degenerate rational p_n/q_m).  Each exchange levels the error on
// the current reference, then moves the reference to the extrema of the
// error, located on a grid and refined by golden-section search, until the
// extrema are level.
#include <cmath>
#include <vector>

namespace mact {

namespace {

double eval(const std::vector<double> &c, double x)
{
    double s = 0.0;
    for (int i = (int)c.size() - 1; i >= 0; --i) s = s * x + c[i];
    return s;
}

// Gaussian elimination with partial pivoting; a is n x n row-major.
bool solve(std::vector<double> a, std::vector<double> b, std::vector<double> &x)
{
    const int n = (int)b.size();
    for (int k = 0; k < n; ++k) {
        int p = k;
        for (int i = k + 1; i < n; ++i)
            if (std::fabs(a[i * n + k]) > std::fabs(a[p * n + k])) p = i;
        if (a[p * n + k] == 0.0) return false;
        if (p != k) {
            for (int j = 0; j < n; ++j) std::swap(a[k * n + j], a[p * n + j]);
            std::swap(b[k], b[p]);
        }
        for (int i = k + 1; i < n; ++i) {
            double m = a[i * n + k] / a[k * n + k];
            for (int j = k; j < n; ++j) a[i * n + j] -= m * a[k * n + j];
            b[i] -= m * b[k];
        }
    }
    x.assign(n, 0.0);
    for (int i = n - 1; i >= 0; --i) {
        double s = b[i];
        for (int j = i + 1; j < n; ++j) s -= a[i * n + j] * x[j];
        x[i] = s / a[i * n + i];
    }
    return true;
}

}  // namespace

// One extremum of err per run of constant sign on the grid gx (ge receives
// err on the grid), refined by golden-section search between the grid
// neighbours; then N consecutive extrema that contain the largest.  False
// if there are fewer than N sign runs.
template <class E>
bool reference_from_extrema(E err, const std::vector<double> &gx, std::vector<double> &ge, int N,
                            std::vector<double> &ex, std::vector<double> &ee)
{
    const int G = (int)gx.size() - 1;
    for (int i = 0; i <= G; ++i) ge[i] = err(gx[i]);
    ex.clear();
    ee.clear();
    int start = 0;
    for (int i = 1; i <= G + 1; ++i) {
        if (i == G + 1 || (ge[i] >= 0) != (ge[start] >= 0)) {
            int k = start;
            for (int j = start; j < i; ++j)
                if (std::fabs(ge[j]) > std::fabs(ge[k])) k = j;
            double xk = gx[k];
            if (k > 0 && k < G) {
                const double sg = ge[k] >= 0 ? 1.0 : -1.0;
                double lo = gx[k - 1], hi = gx[k + 1];
                const double ip = 0.6180339887498949;
                double c = hi - ip * (hi - lo), d = lo + ip * (hi - lo);
                double fc = sg * err(c), fd = sg * err(d);
                for (int s = 0; s < 60; ++s) {
                    if (fc > fd) { hi = d; d = c; fd = fc; c = hi - ip * (hi - lo); fc = sg * err(c); }
                    else { lo = c; c = d; fc = fd; d = lo + ip * (hi - lo); fd = sg * err(d); }
                }
                double xm = 0.5 * (lo + hi);
                if (sg * err(xm) > sg * ge[k]) xk = xm;
            }
            ex.push_back(xk);
            ee.push_back(err(xk));
            start = i;
        }
    }
    if ((int)ex.size() < N) return false;
    while ((int)ex.size() > N) {   // keep N consecutive extrema containing the largest
        int km = 0;
        for (int i = 1; i < (int)ee.size(); ++i)
            if (std::fabs(ee[i]) > std::fabs(ee[km])) km = i;
        bool drop_front = (std::fabs(ee.front()) <= std::fabs(ee.back()) && km != 0) ||
                          km == (int)ee.size() - 1;
        if (drop_front) { ex.erase(ex.begin()); ee.erase(ee.begin()); }
        else { ex.pop_back(); ee.pop_back(); }
    }
    return true;
}

// Degree-n minimax polynomial of f on [a, b]; coefficients ascending.
// Returns false if the exchange fails to produce n+2 alternating extrema.
template <class F>
bool remez_poly(F f, int n, double a, double b, std::vector<double> &coef, double *err_out)
{
    const int N = n + 2;
    std::vector<double> ref(N);
    for (int j = 0; j < N; ++j) ref[j] = 0.5 * (a + b) - 0.5 * (b - a) * std::cos(M_PI * j / (N - 1));
    const int G = 20000;
    std::vector<double> gx(G + 1), ge(G + 1);
    for (int i = 0; i <= G; ++i) gx[i] = a + (b - a) * i / G;
    double E = 0.0;
    for (int it = 0; it < 50; ++it) {
        std::vector<double> A(N * N), rhs(N), sol;
        for (int j = 0; j < N; ++j) {
            double p = 1.0;
            for (int i = 0; i <= n; ++i) { A[j * N + i] = p; p *= ref[j]; }
            A[j * N + n + 1] = (j % 2 == 0) ? 1.0 : -1.0;
            rhs[j] = f(ref[j]);
        }
        if (!solve(A, rhs, sol)) return false;
        coef.assign(sol.begin(), sol.begin() + n + 1);
        auto err = [&](double x) { return f(x) - eval(coef, x); };
        std::vector<double> ex, ee;
        if (!reference_from_extrema(err, gx, ge, N, ex, ee)) return false;
        double emax = 0.0, emin = 1e300;
        for (double e : ee) { emax = std::fmax(emax, std::fabs(e)); emin = std::fmin(emin, std::fabs(e)); }
        ref = ex;
        E = emax;
        if (emax - emin <= 1e-12 * emax) break;
    }
    if (err_out) *err_out = E;
    return true;
}

// Minimax rational p_n/q_m of f on [a, b] (0 < a), normalised to q(0) = 1;
// p and q ascending.  On each reference x_j the levelled error
// f - p/q = (-1)^j E is the nonlinear system p(x_j) - f_j q(x_j) + (-1)^j E q(x_j) = 0
// in p, q_1..q_m and E.  The E q term takes the previous denominator, and
// the linear system is re-solved until q stops changing (the columns are
// equilibrated before elimination, since monomials on [a, 1] span many
// orders of magnitude).  The grid is log-spaced, dense where t^(1/3) bends
// most.  False if the exchange does not level the error to 1e-3 relative,
// or if q changes sign on [a, b].
template <class F>
bool remez_rational(F f, int n, int m, double a, double b, std::vector<double> &p, std::vector<double> &q,
                    double *err_out)
{
    const int N = n + m + 2;
    std::vector<double> ref(N);
    for (int j = 0; j < N; ++j) ref[j] = 0.5 * (a + b) - 0.5 * (b - a) * std::cos(M_PI * j / (N - 1));
    const int G = 40000;
    std::vector<double> gx(G + 1), ge(G + 1);
    for (int i = 0; i <= G; ++i) gx[i] = a * std::pow(b / a, (double)i / G);
    gx[G] = b;
    q.assign(m + 1, 0.0);
    q[0] = 1.0;
    p.assign(n + 1, 0.0);
    double E = 0.0, ripple = 1.0;
    for (int it = 0; it < 80; ++it) {
        std::vector<double> fr(N), q0(N);
        for (int j = 0; j < N; ++j) fr[j] = f(ref[j]);
        for (int inner = 0; inner < 60; ++inner) {
            for (int j = 0; j < N; ++j) q0[j] = eval(q, ref[j]);
            // unknowns p_0..p_n, q_1..q_m, E
            std::vector<double> A(N * N, 0.0), rhs(N), sol;
            for (int j = 0; j < N; ++j) {
                double xp = 1.0;
                for (int i = 0; i <= n; ++i) { A[j * N + i] = xp; xp *= ref[j]; }
                xp = ref[j];
                for (int k = 1; k <= m; ++k) { A[j * N + n + k] = -fr[j] * xp; xp *= ref[j]; }
                A[j * N + N - 1] = ((j % 2 == 0) ? 1.0 : -1.0) * q0[j];
                rhs[j] = fr[j];
            }
            std::vector<double> scale(N, 0.0);
            for (int c = 0; c < N; ++c) {
                for (int j = 0; j < N; ++j) scale[c] = std::fmax(scale[c], std::fabs(A[j * N + c]));
                if (scale[c] == 0.0) return false;
                for (int j = 0; j < N; ++j) A[j * N + c] /= scale[c];
            }
            if (!solve(A, rhs, sol)) return false;
            for (int c = 0; c < N; ++c) sol[c] /= scale[c];
            p.assign(sol.begin(), sol.begin() + n + 1);
            double dq = 0.0;
            for (int k = 1; k <= m; ++k) {
                dq = std::fmax(dq, std::fabs(sol[n + k] - q[k]) / (1.0 + std::fabs(sol[n + k])));
                q[k] = sol[n + k];
            }
            const double En = sol[N - 1];
            const bool done = std::fabs(En - E) <= 1e-15 + 1e-13 * std::fabs(En) && dq <= 1e-13;
            E = En;
            if (done) break;
        }
        auto err = [&](double x) { return f(x) - eval(p, x) / eval(q, x); };
        std::vector<double> ex, ee;
        if (!reference_from_extrema(err, gx, ge, N, ex, ee)) return false;
        double emax = 0.0, emin = 1e300;
        for (double e : ee) { emax = std::fmax(emax, std::fabs(e)); emin = std::fmin(emin, std::fabs(e)); }
        ref = ex;
        E = emax;
        ripple = (emax - emin) / emax;
        if (ripple <= 1e-9) break;
    }
    for (int i = 0; i <= G; ++i)
        if (!(eval(q, gx[i]) > 0.0)) return false;
    if (!(ripple <= 1e-3)) return false;
    if (err_out) *err_out = E;
    return true;
}

// arctan(sqrt(3) x) on [0, 1], degree n (2..5).
bool hsi_unit_interval_fit(int n, double *coef6, double *err)
{
    std::vector<double> c;
    const double s3 = std::sqrt(3.0);
    if (!remez_poly([s3](double x) { return std::atan(s3 * x); }, n, 0.0, 1.0, c, err)) return false;
    for (int i = 0; i < 6; ++i) coef6[i] = i <= n ? c[i] : 0.0;
    return true;
}

// t^(1/3) on [0.008856, 1] as p_n/q_m (n, m in 1..6), q(0) = 1; p7 and q7
// receive the ascending coefficients, zero-padded to 7 entries.
bool cbrt_rational_fit(int n, int m, double *p7, double *q7, double *err)
{
    if (n < 1 || n > 6 || m < 1 || m > 6) return false;
    std::vector<double> p, q;
    if (!remez_rational([](double t) { return std::cbrt(t); }, n, m, 0.008856, 1.0, p, q, err)) return false;
    for (int i = 0; i < 7; ++i) {
        p7[i] = i <= n ? p[i] : 0.0;
        q7[i] = i <= m ? q[i] : 0.0;
    }
    return true;
}

}  // namespace mact
