"""Coefficient tables of the MACT approximants, as printed in the paper.

Test infrastructure: this module belongs to the FP64 oracle. Only tests/,
``__graft_entry__.smoke()`` and bench.py's cpu_baseline leg may import it.

Every table lists coefficients in ascending powers (a0 + a1 x + ... ) exactly
as the paper prints them, together with the stated approximation error
epsilon^A_max and the interval on which the paper says the approximant is used.

Readings of the paper that these tables encode:
  * Table "Minimax polynomials for the inverse tangent function" (HSI), row
    n=2 prints a2 = +7.497879e-01.  With that sign the error at x=1 is about
    1.49, so the sign is a transcription slip: the value here is -7.497879e-01
    (a polynomial Remez fit reproduces -7.49788e-01).  The printed sign is kept
    in ``HSI_ARCTAN_PRINTED_N2_AS_PRINTED`` for the test that documents it.
  * The HSI rows are the minimax fits on [0, 254/256] rather than on [0, 1];
    the oracle's default HSI set is its own Remez fit on [0, 1]
    (see ``oracle.remez``) and these printed rows are the alternative set.
"""

# Section "Approximation of the Cube-Root Function", Table tab_cbrt_poly:
# minimax polynomials p_n(t) ~ t^(1/3); degree -> (eps^A_max, coefficients).
CBRT_POLY = {
    2: (1.271154e-01, [1.268979e-01, 2.393873, -1.647669]),
    3: (9.787829e-02, [9.787826e-02, 4.057495, -7.388864, 4.331370]),
    4: (8.111150e-02, [8.111133e-02, 5.926004, -2.017165e+01, 2.833070e+01,
                       -1.324728e+01]),
    5: (7.002956e-02, [7.002910e-02, 7.961214, -4.329352e+01, 1.063182e+02,
                       -1.135685e+02, 4.358268e+01]),
}

# Section "Approximation of the Cube-Root Function", Table tab_cbrt_rat:
# minimax rationals p_n(t)/q_m(t) ~ t^(1/3) on [0.008856, 1];
# (n, m) -> (eps^A_max, numerator coefficients, denominator coefficients).
CBRT_RAT = {
    (2, 2): (2.060996e-03,
             [6.309655e-03, 5.785782e-01, 1.591005],
             [4.482646e-02, 1.175862, 9.596879e-01]),
    (2, 3): (7.210231e-04,
             [2.500705e-03, 3.447113e-01, 1.942708],
             [1.978701e-02, 8.542797e-01, 1.664540, -2.503267e-01]),
    (3, 2): (5.931593e-04,
             [1.776519e-03, 2.632323e-01, 1.751297, 3.836709e-01],
             [1.432256e-02, 6.779998e-01, 1.706260]),
    (2, 4): (3.107735e-04,
             [1.317899e-03, 2.390113e-01, 2.099395],
             [1.124254e-02, 6.726679e-01, 2.184656, -7.511150e-01,
              2.229717e-01]),
    (3, 3): (1.858694e-04,
             [4.370889e-04, 9.526952e-02, 1.252009, 1.302733],
             [3.912364e-03, 2.954084e-01, 1.717143, 6.343408e-01]),
    (4, 2): (2.334688e-04,
             [7.589302e-04, 1.519784e-01, 1.663584, 8.368075e-01,
              -1.657269e-01],
             [6.644723e-03, 4.506424e-01, 2.030622]),
    (3, 4): (8.539863e-05,
             [1.683667e-04, 4.667675e-02, 9.106812e-01, 1.810577],
             [1.610864e-03, 1.617974e-01, 1.494070, 1.218468, -1.079451e-01]),
    (4, 3): (8.052920e-05,
             [1.349673e-04, 3.832079e-02, 7.870174e-01, 1.799062,
              2.071170e-01],
             [1.299250e-03, 1.345420e-01, 1.330358, 1.365369]),
    (4, 4): (3.856930e-05,
             [3.927283e-05, 1.392318e-02, 4.114739e-01, 1.734853,
              8.679223e-01],
             [4.022100e-04, 5.414536e-02, 8.221526e-01, 1.800167,
              3.513617e-01]),
}

# Section "Approximation of the Inverse Tangent Function" (HSI), Table
# tab_arctan: polynomials P_n(x) ~ arctan(sqrt(3) x); n -> (eps^A_max, coeffs).
HSI_ARCTAN = {
    2: (6.907910e-03, [5.959793e-03, 1.782975, -7.497879e-01]),
    3: (3.654156e-03, [-3.654076e-03, 1.884080, -9.805583e-01, 1.430580e-01]),
    4: (1.286371e-03, [-1.286369e-03, 1.796716, -4.958969e-01, -6.927404e-01,
                       4.421541e-01]),
    5: (1.801311e-04, [-1.801283e-04, 1.739333, -2.039848e-02, -2.065512,
                       2.052837, -6.591729e-01]),
}
HSI_ARCTAN_PRINTED_N2_AS_PRINTED = [5.959793e-03, 1.782975, 7.497879e-01]

# Section "Approximation of the Inverse Cosine Function", Table tab_arcsin:
# polynomials P_n(y) ~ 2 arcsin(y / sqrt(2)) on y in [0, 1/sqrt(2)].
SCT_ARCSIN = {
    4: (2.097814e-05, [2.097797e-05, 1.412840, 1.429881e-02, 6.704361e-02,
                       6.909677e-02]),
    5: (2.370540e-06, [-2.370048e-06, 1.414434, -3.300037e-03, 1.354670e-01,
                       -3.994259e-02, 6.099502e-02]),
}

# Same section, Table tab_arccos: polynomials Q_m(x) ~ arccos(x) on [0, 0.5].
SCT_ARCCOS = {
    4: (1.048949e-05, [1.570786, -9.990285e-01, -1.429899e-02, -9.481335e-02,
                       -1.381942e-01]),
    5: (1.186403e-06, [1.570798, -1.000156, 3.299810e-03, -1.915780e-01,
                       7.988231e-02, -1.725177e-01]),
}

# Section "Approximation of the Inverse Tangent Function" (SCT), Table tab_f:
# polynomials f_r(x) ~ arctan(x) on [0, 254/255].
SCT_F = {
    4: (1.036515e-04, [-1.036508e-04, 1.003740, -1.773538e-02, -3.390563e-01,
                       1.386796e-01]),
    5: (2.073939e-05, [2.073866e-05, 9.982666e-01, 2.352573e-02, -4.506862e-01,
                       2.635050e-01, -4.920822e-02]),
}

# Same section, Table tab_g: polynomials g_r(w) ~ pi/2 - arctan(w) on
# [1/255, 1], where w = R/G.
SCT_G = {
    4: (1.051643e-04, [1.570917, -1.004004, 1.885694e-02, 3.373159e-01,
                       -1.377930e-01]),
    5: (2.012104e-05, [1.570769, -9.981253e-01, -2.440212e-02, 4.528921e-01,
                       -2.659181e-01, 5.016228e-02]),
}

# Intervals on which each approximant is fitted and used.
CBRT_KNEE = 0.008856                      # Eq. equ_xyz_lab, branch point of f(t)
CBRT_RAT_INTERVAL = (0.008856, 1.0)       # Figure fig_cbrt
CBRT_POLY_INTERVAL = (0.0, 1.0)           # reading: the printed fits equioscillate on [0,1]
HSI_PRINTED_INTERVAL = (0.0, 254.0 / 256.0)
HSI_INTERVAL = (0.0, 1.0)
SCT_ARCSIN_INTERVAL = (0.0, 2.0 ** -0.5)
SCT_ARCCOS_INTERVAL = (0.0, 0.5)
SCT_F_INTERVAL = (0.0, 254.0 / 255.0)
SCT_G_INTERVAL = (1.0 / 255.0, 1.0)

# The paper's default ("highest order") degrees, Section "Calculation of the
# Computational Gain Values".
DEFAULT_LAB = (4, 4)
DEFAULT_HSI = 5
DEFAULT_SCT = (5, 5, 5)

# RGB definition: ITU-R BT.709 inverse gamma (Eq. equ_rgb_lin), BT.709
# primaries to CIEXYZ (Eq. equ_rgb_xyz) and the D65 white point.
BT709_GAMMA = dict(threshold=0.081, slope=4.5, offset=0.099, exponent=1.0 / 0.45)
BT709_MATRIX = [0.412391, 0.357584, 0.180481,
                0.212639, 0.715169, 0.072192,
                0.019331, 0.119195, 0.950532]
D65_WHITE = [0.950456, 1.0, 1.089058]
