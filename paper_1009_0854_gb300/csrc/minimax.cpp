// minimax.cpp -- polynomial Remez exchange in double precision, used at
// mact_create to fit arctan(sqrt(3) x) on [0, 1] for the HSI transform
// (Section "Approximation of the Inverse Tangent Function": the paper's
// fits come from the Remez exchange algorithm; Kender's formula needs the
// whole of |x| <= 1).
//
// Chebyshev alternation: the degree-n minimax polynomial makes the error
// reach its maximum modulus n+2 times with alternating signs.  Each exchange
// solves p(x_j) + (-1)^j E = f(x_j) on the current reference, then moves
// the reference to the extrema of the error, located on a uniform grid and
// refined by golden-section search, until the extrema are level.
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
        for (int i = 0; i <= G; ++i) ge[i] = err(gx[i]);
        // one extremum per run of constant sign
        std::vector<double> ex, ee;
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
        double emax = 0.0, emin = 1e300;
        for (double e : ee) { emax = std::fmax(emax, std::fabs(e)); emin = std::fmin(emin, std::fabs(e)); }
        ref = ex;
        E = emax;
        if (emax - emin <= 1e-12 * emax) break;
    }
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

}  // namespace mact
