"""Pins of the oracle's 3D-LUT packing, extraction and the four
interpolators (Section "Comparison with 3D Lookup Table Interpolation
Methods"), independent of the per-method formulas."""
import itertools

import numpy as np
import pytest

import oracle as O

METHODS = ["trilinear", "prism", "pyramid", "tetra"]


def _lut_of(fn, N):
    """LUT whose node (i, j, k) holds fn(i, j, k)/(N-1) scaled, 3 channels."""
    g = np.arange(N) / (N - 1)
    R, G, B = np.meshgrid(g, g, g, indexing="ij")
    return np.stack(fn(R, G, B), axis=-1).astype(np.float32)


def _all_codes_sample(rng, n=50000):
    return rng.integers(0, 256, size=(n, 3), dtype=np.uint8)


def test_lut_build_nodes_are_exact_cielab():
    """Packing: node (i,j,k) is the exact CIELAB of codes 255 (i,j,k)/(N-1)."""
    N = 6   # 255/5 = 51: every node is an integer code
    lut = O.lut_build(N)
    codes = np.array(list(itertools.product(range(0, 256, 51), repeat=3)), dtype=np.uint8)
    L, A, B = O.cielab(codes, exact=True)
    ref = np.stack([L, A, B], axis=1).astype(np.float32).reshape(N, N, N, 3)
    assert np.array_equal(lut, ref)


@pytest.mark.parametrize("method", METHODS)
@pytest.mark.parametrize("N", [4, 6, 16, 18])
def test_interp_reproduces_nodes(method, N):
    """At a lattice point every method returns the node value."""
    rng = np.random.default_rng(N)
    lut = rng.normal(size=(N, N, N, 3)).astype(np.float32)
    step = 255 // (N - 1)
    codes = np.array(list(itertools.product(range(0, 256, step), repeat=3)), dtype=np.uint8)
    out, _ = O.lut_interp(method, lut, codes)
    idx = codes.astype(int) // step
    ref = lut[idx[:, 0], idx[:, 1], idx[:, 2]].astype(np.float64)
    assert np.allclose(np.stack(out, axis=1), ref, atol=1e-12, rtol=0)


@pytest.mark.parametrize("method", METHODS)
@pytest.mark.parametrize("N", [2, 9, 17, 33])
def test_interp_exact_for_affine_functions(method, N):
    """Every method is exact for an affine function of (R, G, B): a dropped
    term, a wrong sign or a swapped corner breaks this."""
    lut = _lut_of(lambda r, g, b: (3 * r - 2 * g + 0.5 * b + 1, -r + 4 * g + 2 * b, 0.25 * r + g - 3 * b), N)
    rng = np.random.default_rng(11)
    codes = _all_codes_sample(rng)
    out, _ = O.lut_interp(method, lut, codes)
    x = codes.astype(np.float64) / 255.0
    ref = [3 * x[:, 0] - 2 * x[:, 1] + 0.5 * x[:, 2] + 1, -x[:, 0] + 4 * x[:, 1] + 2 * x[:, 2],
           0.25 * x[:, 0] + x[:, 1] - 3 * x[:, 2]]
    for o, r in zip(out, ref):
        assert np.abs(o - r).max() < 2e-6  # FP32 node rounding only


def test_trilinear_exact_for_multilinear_functions():
    """Trilinear interpolation reproduces r*g*b (multilinear) exactly."""
    N = 5
    lut = _lut_of(lambda r, g, b: (r * g * b, r * g, g * b), N)
    rng = np.random.default_rng(12)
    codes = _all_codes_sample(rng)
    out, _ = O.lut_interp("trilinear", lut, codes)
    x = codes.astype(np.float64) / 255.0
    assert np.abs(out[0] - x[:, 0] * x[:, 1] * x[:, 2]).max() < 1e-6


def _locate(v, N):
    s = v * (N - 1)
    i, r = s // 255, s % 255
    if i == N - 1:
        i, r = N - 2, 255
    return i, r


@pytest.mark.parametrize("N", [9, 17, 33])
def test_extraction_cell_ids(N):
    """Selection id = lower-corner node index * 8 + simplex; the cell must
    contain the code: node(i)/(N-1) <= v/255 <= node(i+1)/(N-1)."""
    rng = np.random.default_rng(N)
    lut = np.zeros((N, N, N, 3), dtype=np.float32)
    codes = np.concatenate([_all_codes_sample(rng, 20000),
                            np.array([[0, 0, 0], [255, 255, 255], [255, 0, 128]], dtype=np.uint8)])
    _, sel = O.lut_interp("tetra", lut, codes)
    base = sel // 8
    ib, ig, ir = base % N, (base // N) % N, base // (N * N)
    for k, (i, v) in enumerate(zip(np.stack([ir, ig, ib], axis=1), codes)):
        for a in range(3):
            assert i[a] <= N - 2
            assert i[a] * 255 <= int(v[a]) * (N - 1) <= (i[a] + 1) * 255


def _vertices(method, sid):
    """Cube corners (x=R, y=G, z=B) of the simplex/prism/pyramid picked."""
    if method == "tetra":
        paths = {0: "RGB", 1: "RBG", 2: "BRG", 3: "GRB", 4: "GBR", 5: "BGR"}
        p = [0, 0, 0]
        out = [tuple(p)]
        for ch in paths[sid]:
            p["RGB".index(ch)] = 1
            out.append(tuple(p))
        return out
    raise ValueError(method)


def test_tetra_is_barycentric_on_selected_simplex():
    """Brute force: tetrahedral interpolation equals the barycentric
    interpolation on the 4 corners of the chosen tetrahedron (weights solved
    by least squares), and those weights are non-negative, i.e. the simplex
    contains the point."""
    N = 3
    rng = np.random.default_rng(21)
    lut = rng.normal(size=(N, N, N, 3)).astype(np.float32)
    codes = _all_codes_sample(rng, 3000)
    out, sel = O.lut_interp("tetra", lut, codes)
    for k in range(len(codes)):
        cell = [_locate(int(v), N) for v in codes[k]]
        f = np.array([r / 255.0 for _, r in cell])
        verts = _vertices("tetra", int(sel[k] % 8))
        M = np.vstack([np.array(verts, dtype=float).T, np.ones(4)])
        w = np.linalg.solve(M, np.append(f, 1.0))
        assert w.min() > -1e-12
        vals = np.array([lut[cell[0][0] + a, cell[1][0] + b, cell[2][0] + c] for a, b, c in verts],
                        dtype=np.float64)
        assert np.allclose(w @ vals, [o[k] for o in out], atol=1e-12)


def test_prism_is_triangle_times_segment():
    """Brute force: prism interpolation = barycentric interpolation on the
    G-B triangle that contains (fG, fB), then linear along R."""
    N = 3
    rng = np.random.default_rng(22)
    lut = rng.normal(size=(N, N, N, 3)).astype(np.float64).astype(np.float32)
    codes = _all_codes_sample(rng, 3000)
    out, sel = O.lut_interp("prism", lut, codes)
    for k in range(len(codes)):
        cell = [_locate(int(v), N) for v in codes[k]]
        fr, fg, fb = (r / 255.0 for _, r in cell)
        tri = [(0, 0), (1, 0), (1, 1)] if fg >= fb else [(0, 0), (0, 1), (1, 1)]
        assert int(sel[k] % 8) == (0 if fg >= fb else 1)
        M = np.vstack([np.array(tri, dtype=float).T, np.ones(3)])
        w = np.linalg.solve(M, np.array([fg, fb, 1.0]))
        assert w.min() > -1e-12

        def face(x):
            return sum(wi * lut[cell[0][0] + x, cell[1][0] + a, cell[2][0] + b].astype(np.float64)
                       for wi, (a, b) in zip(w, tri))
        ref = (1 - fr) * face(0) + fr * face(1)
        assert np.allclose(ref, [o[k] for o in out], atol=1e-12)


def test_pyramid_apex_and_base():
    """Pyramidal interpolation: on the base face (smallest fraction 0) it is
    bilinear on that face; along the segment to the apex c111 it is linear."""
    N = 2
    rng = np.random.default_rng(23)
    lut = rng.normal(size=(2, 2, 2, 3)).astype(np.float32)
    c = lut.astype(np.float64)
    # codes with B = 0: base B=0 face, bilinear in (R, G)
    for r, g in [(10, 200), (128, 64), (255, 3)]:
        out, sel = O.lut_interp("pyramid", lut, np.array([[r, g, 0]], dtype=np.uint8))
        fr, fg = r / 255.0, g / 255.0
        ref = ((1 - fr) * (1 - fg) * c[0, 0, 0] + fr * (1 - fg) * c[1, 0, 0]
               + (1 - fr) * fg * c[0, 1, 0] + fr * fg * c[1, 1, 0])
        assert sel[0] % 8 == 0
        assert np.allclose([o[0] for o in out], ref, atol=1e-12)
    # the apex edges from base corners c110, c100, c010 to c111 are linear
    # (the cross-term form is not linear on the c000-c111 diagonal)
    for t in (0, 51, 102, 204, 255):
        f = t / 255.0
        for code, corner in [((255, 255, t), c[1, 1, 0]), ((255, t, t), c[1, 0, 0]),
                             ((t, 255, t), c[0, 1, 0])]:
            out, _ = O.lut_interp("pyramid", lut, np.array([code], dtype=np.uint8))
            assert np.allclose([o[0] for o in out], (1 - f) * corner + f * c[1, 1, 1], atol=1e-12)


def test_code_255_uses_last_cell():
    """v = 255 maps to cell N-2 with fraction 1 (not a cell N-1)."""
    for N in (9, 17, 33):
        lut = np.zeros((N, N, N, 3), dtype=np.float32)
        _, sel = O.lut_interp("trilinear", lut, np.array([[255, 255, 255]], dtype=np.uint8))
        assert sel[0] // 8 == ((N - 2) * N + (N - 2)) * N + (N - 2)
