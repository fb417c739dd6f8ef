"""The C ABI library loads and exports every entry point include/mact.h
declares; argument validation that needs no GPU behaves as documented."""
import ctypes
import os
import re

import pytest

from conftest import ROOT

HEADER = os.path.join(ROOT, "include", "mact.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_ ]*?[\s\*]+(mact_[a-z_0-9]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def L():
    from paper_1009_0854_gb300 import mact
    return mact.lib()


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ["mact_create", "mact_destroy", "mact_convert", "mact_convert_batch", "mact_lut_build",
              "mact_lut_interp", "mact_strerror", "mact_last_error", "mact_config_default"]:
        assert n in names


def test_library_exports_every_declared_symbol(L):
    for n in declared_functions():
        assert hasattr(L, n), n


def test_config_default_is_the_papers(L):
    from paper_1009_0854_gb300 import mact
    cfg = mact.mact_config_default()
    assert (cfg.lab_n, cfg.lab_m, cfg.hsi_n, cfg.hsi_coeffs) == (4, 4, 5, 0)
    assert (cfg.sct_n, cfg.sct_m, cfg.sct_r, cfg.exact) == (5, 5, 5, 0)
    assert list(cfg.rgb.white) == [0.950456, 1.0, 1.089058]
    assert list(cfg.rgb.rgb_to_xyz)[:3] == [0.412391, 0.357584, 0.180481]
    assert cfg.rgb.gamma_threshold == 0.081 and cfg.rgb.gamma_slope == 4.5


@pytest.mark.parametrize("field,value", [("lab_n", 5), ("lab_m", 1), ("hsi_n", 6), ("hsi_coeffs", 2),
                                         ("sct_n", 3), ("sct_r", 6), ("exact", 2)])
def test_create_rejects_bad_config_before_touching_the_gpu(L, field, value):
    from paper_1009_0854_gb300 import mact
    cfg = mact.mact_config_default(**{field: value})
    h = ctypes.c_void_p()
    assert L.mact_create(ctypes.byref(cfg), ctypes.byref(h)) == -1
    assert h.value is None
    assert L.mact_last_error()


@pytest.mark.parametrize("fields", [
    dict(gamma_offset=-0.5),                           # negative base of the power: NaN codes
    dict(gamma_slope=0.01),                            # the linear toe climbs above 1
    dict(gamma_threshold=0.5, gamma_slope=0.6),        # the toe ends above the power segment: not monotone
    dict(gamma_exponent=1.0, gamma_offset=0.0, gamma_threshold=-1.0, gamma_slope=1.0)])
def test_create_rejects_gamma_curves_outside_the_unit_interval(L, fields):
    """Eq. equ_rgb_lin with user parameters must give finite, non-decreasing
    linear codes in [0, 1]; the check runs on the host before any CUDA call.
    The last case is the identity curve, which is accepted."""
    from paper_1009_0854_gb300 import mact
    cfg = mact.mact_config_default(**fields)
    h = ctypes.c_void_p()
    st = L.mact_create(ctypes.byref(cfg), ctypes.byref(h))
    if fields.get("gamma_exponent") == 1.0:
        assert st in (0, -3)              # valid: fails only at the device without a GPU
        if st == 0:
            L.mact_destroy(h)
    else:
        assert st == -1 and h.value is None
        assert b"gamma" in L.mact_last_error()


def test_create_rejects_white_above_reference(L):
    from paper_1009_0854_gb300 import mact
    cfg = mact.mact_config_default(white=[0.9, 1.0, 1.089058])
    h = ctypes.c_void_p()
    assert L.mact_create(ctypes.byref(cfg), ctypes.byref(h)) == -1


def test_null_arguments(L):
    from paper_1009_0854_gb300 import mact
    assert L.mact_create(None, None) == -1
    img = mact.Image()
    assert L.mact_convert(None, ctypes.byref(img), None) == -1
    assert L.mact_convert_batch(None, None, 0, None) == -1
    assert L.mact_lut_build(None, 17, None, None) == -1
    assert L.mact_destroy(None) == -1


def test_strerror(L):
    from paper_1009_0854_gb300 import mact
    assert mact.mact_strerror(0) == "ok"
    assert mact.mact_strerror(-1) == "invalid argument"
    assert mact.mact_strerror(-2).startswith("out of memory")
    assert mact.mact_strerror(-5) == "timed out"


def test_config_default_uses_the_printed_cube_root(L):
    from paper_1009_0854_gb300 import mact
    assert mact.mact_config_default().lab_coeffs == 0


@pytest.mark.parametrize("fields", [dict(lab_coeffs=2), dict(lab_coeffs=1, lab_n=7, lab_m=6),
                                    dict(lab_coeffs=1, lab_n=6, lab_m=0), dict(lab_coeffs=-1)])
def test_create_rejects_bad_fitted_rational_config(L, fields):
    from paper_1009_0854_gb300 import mact
    cfg = mact.mact_config_default(**fields)
    h = ctypes.c_void_p()
    assert L.mact_create(ctypes.byref(cfg), ctypes.byref(h)) == -1
    assert h.value is None


def test_fitted_rational_fit_runs_on_the_host(L):
    """The (6,6) Remez fit happens on the host before any CUDA call: without
    a GPU mact_create gets past it and fails only at the device (MACT_E_CUDA),
    never with MACT_E_UNSUPPORTED (a fit that did not converge)."""
    from paper_1009_0854_gb300 import mact
    for n, m in [(6, 6), (5, 6), (1, 1)]:
        cfg = mact.mact_config_default(lab_coeffs=1, lab_n=n, lab_m=m)
        h = ctypes.c_void_p()
        st = L.mact_create(ctypes.byref(cfg), ctypes.byref(h))
        assert st in (0, -3), (n, m, st)
        if st == 0:
            L.mact_destroy(h)


def test_newest_entry_points_reject_null(L):
    assert L.mact_host_memory_access(None) == -1
    assert L.mact_serve_set_mode(None, 0) == -1
    assert L.mact_lut_build_hsi(None, 17, None, None) == -1


@pytest.mark.parametrize("nb,hw", [(1, (1 << 31) + 1), ((1 << 31) + 1, 1), (1 << 16, 1 << 16), (1 << 40, 1 << 40),
                                   (-1, 4), (4, -1)])
def test_gradient_sizes_refused_before_the_handle(L, nb, hw):
    """The gradient entry points admit at most 2^31 pixels (their kernels use
    32-bit grid-stride indices, which must not wrap); oversized or negative
    calls are refused on the host before anything else, products included."""
    calls = [lambda: L.mact_lab_forward(None, None, nb, hw, None, None),
             lambda: L.mact_lab_backward(None, None, None, nb, hw, None, None),
             lambda: L.mact_lab_delta_e_loss(None, None, None, nb, hw, None, None, None)]
    for call in calls:
        assert call() == -1
        msg = L.mact_last_error()
        assert b"2^31" in msg or b"negative" in msg, msg


def test_gradient_size_limit_is_inclusive(L):
    """Exactly 2^31 pixels passes the size check (then fails on the NULL handle)."""
    assert L.mact_lab_forward(None, None, 2, 1 << 30, None, None) == -1
    assert b"NULL handle" in L.mact_last_error()


@pytest.mark.parametrize("fields", [
    dict(gamma_threshold=0.04045, gamma_slope=12.92, gamma_offset=0.055, gamma_exponent=2.4),   # sRGB
    dict(gamma_threshold=0.0, gamma_slope=1.0, gamma_offset=0.0, gamma_exponent=2.2),          # pure power
    dict(gamma_threshold=2.0, gamma_slope=1.0, gamma_offset=0.0, gamma_exponent=1.0)])         # linear codes
def test_create_accepts_common_gamma_curves(L, fields):
    """Valid curves pass the host checks; without a GPU the call then fails
    only at the device (MACT_E_CUDA)."""
    from paper_1009_0854_gb300 import mact
    cfg = mact.mact_config_default(**fields)
    h = ctypes.c_void_p()
    st = L.mact_create(ctypes.byref(cfg), ctypes.byref(h))
    assert st in (0, -3), L.mact_last_error()
    if st == 0:
        L.mact_destroy(h)
