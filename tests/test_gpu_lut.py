"""GPU parity of the LUT packing and the four interpolators against the
oracle: selection (cell and simplex) bit-identical, values within 2e-4."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1009_0854_gb300 import mact
from parity import LAB_TOL, to_np

pytestmark = pytest.mark.gpu

METHODS = ["trilinear", "prism", "pyramid", "tetra"]


@pytest.fixture(scope="module")
def h():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return mact.mact_create()


_LUT = {}


def oracle_lut(N):
    if N not in _LUT:
        _LUT[N] = O.lut_build(N)
    return _LUT[N]


@pytest.mark.parametrize("N", [2, 9, 17, 33, 64])
def test_lut_build_matches_oracle(h, N):
    """Packing on the GPU (FP64 then rounded) equals the oracle's FP32 LUT to
    one FP32 ulp (plus 1e-12 where the value is 0 up to cancellation)."""
    g = mact.mact_lut_build(h, N).cpu().numpy()
    ref = oracle_lut(N) if N != 64 else O.lut_build(64)
    d = np.abs(g.astype(np.float64) - ref.astype(np.float64))
    assert np.all(d <= np.spacing(np.abs(ref)).astype(np.float64) + 1e-12)


@pytest.mark.parametrize("method", METHODS)
@pytest.mark.parametrize("N", [9, 17, 33])
def test_interp_full_cube(h, cube_rgb, method, N):
    """Every 24-bit colour, the oracle-built LUT fed to both sides."""
    lut = oracle_lut(N)
    rgb = cube_rgb.reshape(-1, 3)
    out, sel = mact.mact_lut_interp(h, method, torch.from_numpy(lut).cuda(),
                                    torch.from_numpy(rgb).cuda(), sel=True)
    torch.cuda.synchronize()
    ref, rsel = O.lut_interp(method, lut, rgb)
    assert np.array_equal(sel.cpu().numpy(), rsel)
    for c in range(3):
        d = np.abs(to_np(out[c]) - ref[c])
        assert d.max() <= LAB_TOL, (method, N, c, d.max())


@pytest.mark.parametrize("method", METHODS)
@pytest.mark.parametrize("N", [2, 5, 18, 40, 64])
def test_interp_other_sizes_and_ragged(h, method, N):
    rng = np.random.default_rng(N)
    lut = rng.normal(scale=50.0, size=(N, N, N, 3)).astype(np.float32)
    for npix in (1, 7, 2047, 4099):
        rgb = rng.integers(0, 256, size=(npix, 3), dtype=np.uint8)
        rgb[0] = (255, 255, 255)
        out, sel = mact.mact_lut_interp(h, method, torch.from_numpy(lut).cuda(), torch.from_numpy(rgb).cuda(),
                                        sel=True)
        torch.cuda.synchronize()
        ref, rsel = O.lut_interp(method, lut, rgb)
        assert np.array_equal(sel.cpu().numpy(), rsel)
        for c in range(3):
            assert np.abs(to_np(out[c]) - ref[c]).max() <= LAB_TOL


def test_interp_without_selection_output(h, cube_rgb):
    lut = oracle_lut(17)
    rgb = torch.from_numpy(cube_rgb.reshape(-1, 3)[:100000].copy()).cuda()
    a = mact.mact_lut_interp(h, "tetra", torch.from_numpy(lut).cuda(), rgb)
    b, _ = mact.mact_lut_interp(h, "tetra", torch.from_numpy(lut).cuda(), rgb, sel=True)
    torch.cuda.synchronize()
    assert torch.equal(a, b)


@pytest.mark.parametrize("N", [9, 17, 33])
def test_cache_layout_records(h, N):
    """Caching layout: record of cell (i,j,k) = [c000, c_xyz - c000 ...] in
    slot order x*4 + y*2 + z, computed in FP32 exactly as numpy does."""
    lut = oracle_lut(N)
    cache = mact.mact_lut_cache_build(h, torch.from_numpy(lut).cuda()).cpu().numpy()
    m = N - 1
    rec = cache.reshape(m, m, m, 8, 4)
    assert np.array_equal(rec[..., 0, :3], lut[:m, :m, :m])
    for slot in range(1, 8):
        x, y, z = slot >> 2, (slot >> 1) & 1, slot & 1
        d = lut[x:x + m, y:y + m, z:z + m] - lut[:m, :m, :m]
        assert np.array_equal(rec[..., slot, :3], d)


@pytest.mark.parametrize("method", METHODS)
@pytest.mark.parametrize("N", [9, 17, 33])
def test_cached_interp_full_cube(h, cube_rgb, method, N):
    """The caching form selects the same cells and simplices (bit-identical
    ids) and gives the same values within 2e-4."""
    lut = oracle_lut(N)
    rgb = cube_rgb.reshape(-1, 3)
    cache = mact.mact_lut_cache_build(h, torch.from_numpy(lut).cuda())
    out, sel = mact.mact_lut_interp_cached(h, method, cache, N, torch.from_numpy(rgb).cuda(), sel=True)
    torch.cuda.synchronize()
    ref, rsel = O.lut_interp(method, lut, rgb)
    assert np.array_equal(sel.cpu().numpy(), rsel)
    for c in range(3):
        assert np.abs(to_np(out[c]) - ref[c]).max() <= LAB_TOL


def test_cached_interp_ragged(h):
    rng = np.random.default_rng(77)
    lut = rng.normal(scale=40.0, size=(5, 5, 5, 3)).astype(np.float32)
    cache = mact.mact_lut_cache_build(h, torch.from_numpy(lut).cuda())
    for npix in (1, 3, 4097):
        rgb = rng.integers(0, 256, size=(npix, 3), dtype=np.uint8)
        out, sel = mact.mact_lut_interp_cached(h, "pyramid", cache, 5, torch.from_numpy(rgb).cuda(), sel=True)
        ref, rsel = O.lut_interp("pyramid", lut, rgb)
        assert np.array_equal(sel.cpu().numpy(), rsel)
        for c in range(3):
            assert np.abs(to_np(out[c]) - ref[c]).max() <= LAB_TOL


@pytest.mark.parametrize("method", METHODS)
@pytest.mark.parametrize("N", [5, 17, 33, 40])
def test_packed_lut_equals_unpacked(h, method, N):
    """mact_lut_pack + mact_lut_interp_packed: the packed nodes are the LUT's
    values padded with 0, the edge records pair each node with the next
    along B and along R, and interpolation from them gives the same
    selections and the same bits as mact_lut_interp, and the oracle's values,
    on all 2^24 colours for 17^3 and 33^3 and on a ragged random sample
    otherwise."""
    rng = np.random.default_rng(100 + N)
    lut = oracle_lut(N) if N in (17, 33) else rng.normal(scale=50.0, size=(N, N, N, 3)).astype(np.float32)
    lt = torch.from_numpy(lut).cuda()
    lut4 = mact.mact_lut_pack(h, lt)
    torch.cuda.synchronize()
    p = lut4.cpu().numpy()
    m = N ** 3
    nodes = p[:4 * m].reshape(N, N, N, 4)
    assert np.array_equal(nodes[..., :3], lut) and np.all(nodes[..., 3] == 0.0)
    # B-edge records: (x_i, y_i, x_{i+1}, y_{i+1}) and (z_i, z_{i+1}); the last
    # node of a B row repeats itself
    nb = np.concatenate([lut[:, :, 1:], lut[:, :, -1:]], axis=2)     # next along B
    nr = np.concatenate([lut[1:], lut[-1:]], axis=0)                 # next along R
    for xoff, zoff, nxt in ((4 * m, 12 * m, nb), (8 * m, 14 * m, nr)):
        xy = p[xoff:xoff + 4 * m].reshape(N, N, N, 4)
        z = p[zoff:zoff + 2 * m].reshape(N, N, N, 2)
        assert np.array_equal(xy[..., 0:2], lut[..., 0:2]) and np.array_equal(xy[..., 2:4], nxt[..., 0:2])
        assert np.array_equal(z[..., 0], lut[..., 2]) and np.array_equal(z[..., 1], nxt[..., 2])
    assert np.array_equal(p[16 * m:18 * m].reshape(N, N, N, 2), lut[..., 0:2])
    assert np.array_equal(p[18 * m:19 * m].reshape(N, N, N), lut[..., 2])
    if N in (17, 33):
        rgb = torch.from_numpy(np.ascontiguousarray(
            np.stack(np.meshgrid(np.arange(256), np.arange(256), np.arange(256), indexing="ij"), -1)
            .reshape(-1, 3).astype(np.uint8))).cuda()
    else:
        rgb = torch.from_numpy(rng.integers(0, 256, size=(5003, 3), dtype=np.uint8)).cuda()
    a, sa = mact.mact_lut_interp_packed(h, method, lut4, N, rgb, sel=True)
    b, sb = mact.mact_lut_interp(h, method, lt, rgb, sel=True)
    torch.cuda.synchronize()
    assert torch.equal(sa, sb) and torch.equal(a, b)
    ref, rsel = O.lut_interp(method, lut, rgb.cpu().numpy())
    assert np.array_equal(sa.cpu().numpy(), rsel)
    for c in range(3):
        assert np.abs(to_np(a[c]) - ref[c]).max() <= LAB_TOL
