"""Pins of the oracle's analytic gradient of the mean Delta E*ab loss of
RGB -> CIELAB on linear RGB: central finite differences of the oracle's own
forward (a different computation from the analytic chain rule), the linear
segment below the knee, and the Delta E = 0 convention."""
import numpy as np
import pytest

import oracle as O

KNEE = 0.008856


def _fd(x, t, exact, h, one_sided=0):
    g = np.zeros_like(x)
    for idx in np.ndindex(x.shape):
        xp = x.copy()
        xm = x.copy()
        if one_sided == 0:
            xp[idx] += h
            xm[idx] -= h
            den = 2 * h
        elif one_sided > 0:
            xp[idx] += h
            den = h
        else:
            xm[idx] -= h
            den = h
        g[idx] = (O.lab_loss_grad(xp, t, exact=exact, grad=False)[0] -
                  O.lab_loss_grad(xm, t, exact=exact, grad=False)[0]) / den
    return g


@pytest.mark.parametrize("exact", [False, True])
@pytest.mark.parametrize("h", [1e-6, 1e-3])
def test_gradient_matches_central_differences(exact, h):
    """Away from the knee (t > 0.05) central differences agree with the
    analytic gradient: to 1e-7 relative with h = 1e-6 and to 2e-3 with the
    h = 1e-3 step (truncation error of the second-order formula)."""
    rng = np.random.default_rng(1)
    x = rng.uniform(0.1, 1.0, size=(2, 3, 6))
    t = rng.uniform(-60, 90, size=(2, 3, 6))
    loss, g = O.lab_loss_grad(x, t, exact=exact)
    fd = _fd(x, t, exact, h)
    tol = 1e-7 if h < 1e-5 else 2e-3
    assert np.abs(fd - g).max() <= tol * np.abs(g).max()


def test_linear_segment_gradient():
    """Pixels with all three channels below the knee use f = 7.787 t + 16/116:
    the loss is smooth there and the gradient matches central differences."""
    rng = np.random.default_rng(2)
    v = rng.uniform(0.0005, 0.006, size=(1, 1, 8))
    x = np.repeat(v, 3, axis=1)
    t = rng.uniform(-5, 5, size=(1, 3, 8))
    _, g = O.lab_loss_grad(x, t, exact=False)
    fd = _fd(x, t, False, 1e-7)
    assert np.abs(fd - g).max() <= 1e-6 * np.abs(g).max()


def test_knee_one_sided_differences():
    """Gray pixels just above / below the knee: the analytic gradient equals
    the one-sided difference taken on the pixel's own side."""
    eps = 3e-5
    for side in (+1, -1):
        x = np.full((1, 3, 1), KNEE + side * eps)
        t = np.array([[[10.0], [5.0], [-3.0]]])
        for exact in (False, True):
            _, g = O.lab_loss_grad(x, t, exact=exact)
            fd = _fd(x, t, exact, 1e-6, one_sided=side)
            assert np.abs(fd - g).max() <= 1e-3 * np.abs(g).max()


def test_zero_input_and_zero_delta_e():
    """x = 0 (black) lies on the linear segment: finite gradient; where the
    target equals Lab(x) exactly the gradient is defined as 0."""
    x = np.zeros((1, 3, 2))
    x[0, :, 1] = 0.5
    lab = O.lab_linear(x)
    t = lab.copy()
    t[0, 0, 0] += 1.0
    loss, g = O.lab_loss_grad(x, t)
    assert np.all(np.isfinite(g))
    assert np.all(g[0, :, 1] == 0.0)
    assert loss == pytest.approx(0.5, rel=1e-12)


def test_lab_linear_matches_code_path():
    """Linear-RGB forward equals the 8-bit path when x is the BT.709
    linearisation of the codes."""
    codes = np.array([[10, 200, 30], [255, 255, 255], [1, 2, 3], [128, 64, 32]], dtype=np.uint8)
    x = np.array([[O.gamma_inverse(c / 255.0) for c in px] for px in codes]).T[None]
    lab = O.lab_linear(x)
    for exact in (False, True):
        L, A, B = O.cielab(codes, exact=exact)
        ll = O.lab_linear(x, exact=exact)
        assert np.allclose(ll[0], np.stack([L, A, B]), atol=1e-12)
    assert lab.shape == x.shape
