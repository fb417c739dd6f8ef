"""Thin ctypes binding of libmact.so (include/mact.h).

Argument marshalling only: every step of every transform runs in the CUDA
kernels of libmact.so.  PyTorch supplies device memory (tensors) and streams;
the functions below take torch tensors, pass their device pointers and sizes
through the C ABI, and raise ``MactError`` on any non-zero status.  There is
no CPU fallback: if the library cannot be loaded, every call raises.

Names mirror the C entry points (``mact_create``, ``mact_convert``, ...).
"""
import ctypes
import os

import torch

from . import _build

SPACES = {"cielab": 0, "hsi": 1, "sct": 2, "cieluv": 3}
DTYPES = {torch.float32: 0, torch.float16: 1}
METHODS = {"trilinear": 0, "prism": 1, "pyramid": 2, "tetra": 3}

MACT_OK = 0
MACT_E_INVAL = -1
MACT_E_NOMEM = -2
MACT_E_CUDA = -3
MACT_E_UNSUPPORTED = -4
MACT_E_TIMEOUT = -5
MACT_E_BUSY = -6


class MactError(RuntimeError):
    def __init__(self, status, where, detail=""):
        self.status = status
        super().__init__("%s failed: status %d (%s)%s" % (
            where, status, _lib_strerror(status), (": " + detail) if detail else ""))


class RGBDef(ctypes.Structure):
    _fields_ = [("gamma_threshold", ctypes.c_double), ("gamma_slope", ctypes.c_double),
                ("gamma_offset", ctypes.c_double), ("gamma_exponent", ctypes.c_double),
                ("rgb_to_xyz", ctypes.c_double * 9), ("white", ctypes.c_double * 3)]


class Config(ctypes.Structure):
    _fields_ = [("rgb", RGBDef), ("exact", ctypes.c_int32), ("lab_n", ctypes.c_int32),
                ("lab_m", ctypes.c_int32), ("hsi_n", ctypes.c_int32), ("hsi_coeffs", ctypes.c_int32),
                ("sct_n", ctypes.c_int32), ("sct_m", ctypes.c_int32), ("sct_r", ctypes.c_int32),
                ("lab_coeffs", ctypes.c_int32)]


class Image(ctypes.Structure):
    _fields_ = [("rgb", ctypes.c_void_p), ("width", ctypes.c_int64), ("height", ctypes.c_int64),
                ("pitch_bytes", ctypes.c_int64), ("space", ctypes.c_int32), ("dtype", ctypes.c_int32),
                ("out", ctypes.c_void_p * 3), ("out_pitch_elems", ctypes.c_int64)]


class TuneEntry(ctypes.Structure):
    _fields_ = [("threads", ctypes.c_int32), ("px_per_thread", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32),
                ("ms", ctypes.c_float)]


class ServeStats(ctypes.Structure):
    _fields_ = [("completed", ctypes.c_int64), ("failed", ctypes.c_int64), ("batches", ctypes.c_int64),
                ("queued", ctypes.c_int64), ("in_flight", ctypes.c_int64), ("pixels", ctypes.c_int64),
                ("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double), ("max_ms", ctypes.c_double),
                ("gpix_per_s", ctypes.c_double),
                ("queue_p50_ms", ctypes.c_double), ("h2d_p50_ms", ctypes.c_double),
                ("compute_p50_ms", ctypes.c_double), ("d2h_p50_ms", ctypes.c_double),
                ("queue_p99_ms", ctypes.c_double), ("h2d_p99_ms", ctypes.c_double),
                ("compute_p99_ms", ctypes.c_double), ("d2h_p99_ms", ctypes.c_double),
                ("d2h_busy_ms", ctypes.c_double), ("d2h_copy_gbs", ctypes.c_double),
                ("inflight_bytes_max", ctypes.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None
_VP = ctypes.c_void_p


def lib_path():
    return _build.LIB


def lib():
    """Load libmact.so (building it first if it is absent)."""
    global _lib
    if _lib is None:
        path = _build.LIB
        if not os.path.exists(path):
            _build.build()
        L = ctypes.CDLL(path)
        L.mact_config_default.argtypes = [ctypes.POINTER(Config)]
        L.mact_config_default.restype = None
        L.mact_create.argtypes = [ctypes.POINTER(Config), ctypes.POINTER(_VP)]
        L.mact_destroy.argtypes = [_VP]
        L.mact_convert.argtypes = [_VP, ctypes.POINTER(Image), _VP]
        L.mact_convert_batch.argtypes = [_VP, ctypes.POINTER(Image), ctypes.c_int32, _VP]
        L.mact_convert_batch_static.argtypes = [_VP, ctypes.POINTER(Image), ctypes.c_int32, _VP]
        L.mact_lut_build.argtypes = [_VP, ctypes.c_int32, _VP, _VP]
        L.mact_lut_interp.argtypes = [_VP, ctypes.c_int32, _VP, ctypes.c_int32, _VP, ctypes.c_int64,
                                      ctypes.POINTER(_VP * 3), _VP, _VP]
        L.mact_lut_pack.argtypes = [_VP, _VP, ctypes.c_int32, _VP, _VP]
        L.mact_lut_interp_packed.argtypes = L.mact_lut_interp.argtypes
        L.mact_serve_create.argtypes = [_VP, ctypes.c_size_t, ctypes.c_int32, ctypes.POINTER(_VP)]
        L.mact_serve_submit.argtypes = [_VP, ctypes.POINTER(Image), ctypes.POINTER(ctypes.c_uint64)]
        L.mact_serve_poll.argtypes = [_VP, ctypes.c_uint64, ctypes.POINTER(ctypes.c_int32),
                                      ctypes.POINTER(ctypes.c_double)]
        L.mact_serve_wait.argtypes = [_VP, ctypes.c_uint64, ctypes.c_double, ctypes.POINTER(ctypes.c_double)]
        L.mact_serve_cancel.argtypes = [_VP, ctypes.c_uint64]
        L.mact_serve_release.argtypes = [_VP, ctypes.c_uint64]
        L.mact_serve_stats.argtypes = [_VP, ctypes.POINTER(ServeStats)]
        L.mact_serve_destroy.argtypes = [_VP, ctypes.c_double]
        L.mact_serve_set_mode.argtypes = [_VP, ctypes.c_int32]
        L.mact_serve_set_mode.restype = ctypes.c_int
        for name in ("mact_serve_create", "mact_serve_submit", "mact_serve_poll", "mact_serve_wait",
                     "mact_serve_cancel", "mact_serve_release", "mact_serve_stats", "mact_serve_destroy"):
            getattr(L, name).restype = ctypes.c_int
        L.mact_batch_plan_create.argtypes = [_VP, ctypes.POINTER(Image), ctypes.c_int32, ctypes.POINTER(_VP)]
        L.mact_batch_plan_launch.argtypes = [_VP, _VP]
        L.mact_batch_plan_graph_launch.argtypes = [_VP, _VP]
        L.mact_batch_plan_destroy.argtypes = [_VP]
        L.mact_autotune_batch.argtypes = [_VP, ctypes.POINTER(Image), ctypes.c_int32, ctypes.c_int32,
                                          ctypes.POINTER(TuneEntry), ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)]
        L.mact_set_batch_shape.argtypes = [_VP, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32]
        L.mact_get_batch_shape.argtypes = [_VP] + [ctypes.POINTER(ctypes.c_int32)] * 3
        for name in ("mact_batch_plan_create", "mact_batch_plan_launch", "mact_batch_plan_graph_launch",
                     "mact_batch_plan_destroy", "mact_autotune_batch", "mact_set_batch_shape",
                     "mact_get_batch_shape"):
            getattr(L, name).restype = ctypes.c_int
        L.mact_lut_cache_build.argtypes = [_VP, _VP, ctypes.c_int32, _VP, _VP]
        L.mact_lut_interp_cached.argtypes = [_VP, ctypes.c_int32, _VP, ctypes.c_int32, _VP, ctypes.c_int64,
                                             ctypes.POINTER(_VP * 3), _VP, _VP]
        L.mact_lut_cache_build.restype = ctypes.c_int
        L.mact_lut_interp_cached.restype = ctypes.c_int
        L.mact_cube_error.argtypes = [_VP, ctypes.c_int32, ctypes.POINTER(ctypes.c_double),
                                      ctypes.POINTER(ctypes.c_double)]
        L.mact_cube_error_lut.argtypes = [_VP, ctypes.c_int32, _VP, ctypes.c_int32, ctypes.POINTER(ctypes.c_double),
                                          ctypes.POINTER(ctypes.c_double)]
        L.mact_cube_error.restype = ctypes.c_int
        L.mact_cube_error_lut.restype = ctypes.c_int
        L.mact_lab_forward.argtypes = [_VP, _VP, ctypes.c_int64, ctypes.c_int64, _VP, _VP]
        L.mact_lab_backward.argtypes = [_VP, _VP, _VP, ctypes.c_int64, ctypes.c_int64, _VP, _VP]
        L.mact_lab_delta_e_loss.argtypes = [_VP, _VP, _VP, ctypes.c_int64, ctypes.c_int64, _VP, _VP, _VP]
        for name in ("mact_lab_forward", "mact_lab_backward", "mact_lab_delta_e_loss"):
            getattr(L, name).restype = ctypes.c_int
        L.mact_strerror.argtypes = [ctypes.c_int]
        L.mact_strerror.restype = ctypes.c_char_p
        L.mact_last_error.argtypes = []
        L.mact_last_error.restype = ctypes.c_char_p
        L.mact_lut_build_hsi.argtypes = [_VP, ctypes.c_int32, _VP, _VP]
        L.mact_lut_build_hsi.restype = ctypes.c_int
        L.mact_lut_interp_hsi.argtypes = [_VP, _VP, ctypes.c_int32, _VP, ctypes.c_int64, ctypes.POINTER(_VP), _VP]
        L.mact_lut_interp_hsi.restype = ctypes.c_int
        L.mact_fit_cbrt_rational.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(ctypes.c_double),
                                             ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
        L.mact_fit_cbrt_rational.restype = ctypes.c_int
        L.mact_fit_hsi_arctan.argtypes = [ctypes.c_int32, ctypes.POINTER(ctypes.c_double),
                                          ctypes.POINTER(ctypes.c_double)]
        L.mact_fit_hsi_arctan.restype = ctypes.c_int
        L.mact_host_memory_access.argtypes = [_VP]
        L.mact_host_memory_access.restype = ctypes.c_int32
        for name in ("mact_create", "mact_destroy", "mact_convert", "mact_convert_batch", "mact_convert_batch_static",
                     "mact_lut_build", "mact_lut_interp"):
            getattr(L, name).restype = ctypes.c_int
        _lib = L
    return _lib


def _lib_strerror(st):
    try:
        return lib().mact_strerror(st).decode()
    except Exception:  # noqa: BLE001 - message formatting only
        return "?"


def _check(st, where):
    if st != MACT_OK:
        raise MactError(st, where, lib().mact_last_error().decode())


def _need(t, name, shape, dtype=torch.float32):
    """Refuse a caller-supplied tensor whose size, type or layout differs from
    what the kernel will read or write (the C ABI cannot see buffer sizes)."""
    if not isinstance(t, torch.Tensor):
        raise TypeError("%s must be a torch.Tensor" % name)
    if t.dtype != dtype or tuple(t.shape) != tuple(shape) or not t.is_contiguous():
        raise ValueError("%s must be a contiguous %s tensor of shape %s (got %s %s%s)" % (
            name, dtype, tuple(shape), t.dtype, tuple(t.shape), "" if t.is_contiguous() else ", strided"))
    return t


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return _VP(stream.cuda_stream)


def mact_config_default(**overrides):
    """The paper's defaults (BT.709, D65, CIELAB (4,4), HSI n=5 on [0,1],
    SCT (5,5,5)); keyword overrides set top-level fields (exact, lab_n, ...)."""
    cfg = Config()
    lib().mact_config_default(ctypes.byref(cfg))
    for k, v in overrides.items():
        if k in ("matrix", "rgb_to_xyz"):
            for i, x in enumerate(v):
                cfg.rgb.rgb_to_xyz[i] = x
        elif k == "white":
            for i, x in enumerate(v):
                cfg.rgb.white[i] = x
        elif k.startswith("gamma_"):
            setattr(cfg.rgb, k, v)
        else:
            setattr(cfg, k, int(v))
    return cfg


class Handle:
    """Owns a mact_handle; destroyed with the object."""

    def __init__(self, ptr, cfg):
        self.ptr = ptr
        self.cfg = cfg

    def close(self):
        if self.ptr:
            lib().mact_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001 - interpreter shutdown
            pass


def mact_create(cfg=None, **overrides):
    if cfg is None:
        cfg = mact_config_default(**overrides)
    h = _VP()
    _check(lib().mact_create(ctypes.byref(cfg), ctypes.byref(h)), "mact_create")
    return Handle(h, cfg)


def _image(rgb, space, out):
    if rgb.dtype != torch.uint8 or rgb.dim() != 3 or rgb.shape[2] != 3:
        raise ValueError("rgb must be a (H, W, 3) uint8 tensor")
    if rgb.stride(2) != 1 or rgb.stride(1) != 3:
        raise ValueError("rgb pixels must be interleaved and rows dense (stride (pitch, 3, 1))")
    if out.dim() != 3 or out.shape[0] != 3 or out.shape[1:] != rgb.shape[:2]:
        raise ValueError("out must have shape (3, H, W)")
    if out.dtype not in DTYPES:
        raise ValueError("out must be float32 or float16")
    if out.stride(2) != 1:
        raise ValueError("out rows must be dense")
    H, W = rgb.shape[0], rgb.shape[1]
    img = Image()
    img.rgb = rgb.data_ptr()
    img.width = W
    img.height = H
    img.pitch_bytes = rgb.stride(0)
    img.space = SPACES[space] if isinstance(space, str) else int(space)
    img.dtype = DTYPES[out.dtype]
    for c in range(3):
        img.out[c] = out[c].data_ptr()
    img.out_pitch_elems = out.stride(1)
    return img


def mact_convert(h, rgb, space="cielab", dtype=torch.float32, out=None, stream=None):
    """Convert one (H, W, 3) uint8 CUDA image; returns a (3, H, W) tensor."""
    if out is None:
        out = torch.empty((3, rgb.shape[0], rgb.shape[1]), dtype=dtype, device=rgb.device,
                          pin_memory=rgb.device.type == "cpu")
    img = _image(rgb, space, out)
    _check(lib().mact_convert(h.ptr, ctypes.byref(img), _stream(stream)), "mact_convert")
    return out


def mact_convert_batch(h, images, dtype=torch.float32, outs=None, stream=None):
    """images: list of (rgb (H, W, 3) uint8 CUDA tensor, space); one launch.
    Returns the list of (3, H, W) outputs."""
    n = len(images)
    if outs is None:
        outs = [torch.empty((3, r.shape[0], r.shape[1]), dtype=dtype, device=r.device,
                         pin_memory=r.device.type == "cpu") for r, _ in images]
    if len(outs) != n:
        raise ValueError("outs must hold one output per image")
    arr = (Image * max(n, 1))()
    for i, ((rgb, space), out) in enumerate(zip(images, outs)):
        arr[i] = _image(rgb, space, out)
    _check(lib().mact_convert_batch(h.ptr, arr, n, _stream(stream)), "mact_convert_batch")
    return outs


def mact_convert_batch_static(h, images, dtype=torch.float32, outs=None, stream=None):
    """As mact_convert_batch, through the entry point that allocates nothing
    in the library (its work list lives in a fixed device array; at most 1024
    images).  Output tensors are still created here unless outs is given."""
    n = len(images)
    if outs is None:
        outs = [torch.empty((3, r.shape[0], r.shape[1]), dtype=dtype, device=r.device,
                         pin_memory=r.device.type == "cpu") for r, _ in images]
    if len(outs) != n:
        raise ValueError("outs must hold one output per image")
    arr = (Image * max(n, 1))()
    for i, ((rgb, space), out) in enumerate(zip(images, outs)):
        arr[i] = _image(rgb, space, out)
    _check(lib().mact_convert_batch_static(h.ptr, arr, n, _stream(stream)), "mact_convert_batch_static")
    return outs


def mact_lut_build(h, n, out=None, device="cuda", stream=None):
    """n^3 x 3 FP32 LUT of the exact CIELAB at the lattice nodes."""
    if out is None:
        out = torch.empty((n, n, n, 3), dtype=torch.float32, device=device)
    _need(out, "out", (n, n, n, 3))
    _check(lib().mact_lut_build(h.ptr, n, _VP(out.data_ptr()), _stream(stream)), "mact_lut_build")
    return out


def mact_lut_interp(h, method, lut, rgb, out=None, sel=False, stream=None):
    """Interpolate the (npix, 3) or (H, W, 3) uint8 pixels of rgb in an
    (n, n, n, 3) FP32 LUT.  Returns (3, npix) planes and, if sel, the int32
    selection ids ((lower-corner node)*8 + simplex)."""
    if lut.dtype != torch.float32 or not lut.is_contiguous() or lut.dim() != 4 or lut.shape[3] != 3:
        raise ValueError("lut must be a contiguous (n, n, n, 3) float32 tensor")
    if rgb.dtype != torch.uint8 or not rgb.is_contiguous() or rgb.shape[-1] != 3:
        raise ValueError("rgb must be a contiguous (..., 3) uint8 tensor")
    n = lut.shape[0]
    if lut.shape[1] != n or lut.shape[2] != n:
        raise ValueError("lut must be a cube (n, n, n, 3)")
    npix = rgb.numel() // 3
    if out is None:
        out = torch.empty((3, npix), dtype=torch.float32, device=rgb.device,
                          pin_memory=rgb.device.type == "cpu")
    _need(out, "out", (3, npix))
    ptrs = (_VP * 3)(*(out[c].data_ptr() for c in range(3)))
    s = (torch.empty(npix, dtype=torch.int32, device=rgb.device, pin_memory=rgb.device.type == "cpu")
         if sel else None)
    m = METHODS[method] if isinstance(method, str) else int(method)
    _check(lib().mact_lut_interp(h.ptr, m, _VP(lut.data_ptr()), n, _VP(rgb.data_ptr()), npix,
                                 ctypes.byref(ptrs), _VP(s.data_ptr() if s is not None else 0),
                                 _stream(stream)), "mact_lut_interp")
    return (out, s) if sel else out


LUT_PACKED_FLOATS = 19   # floats per node of the packed layout (mact_lut_pack)


def mact_lut_pack(h, lut, out=None, stream=None):
    """The (n, n, n, 3) FP32 LUT in the packed layout the interpolation
    kernels read (a flat FP32 tensor of 19 n^3 values: the nodes padded to
    16 bytes, the B-edge and R-edge xy and z records, and the nodes' dense xy
    and z planes), for repeated
    interpolation with mact_lut_interp_packed."""
    if lut.dtype != torch.float32 or not lut.is_contiguous() or lut.dim() != 4 or lut.shape[3] != 3:
        raise ValueError("lut must be a contiguous (n, n, n, 3) float32 tensor")
    n = lut.shape[0]
    if lut.shape[1] != n or lut.shape[2] != n:
        raise ValueError("lut must be a cube (n, n, n, 3)")
    size = LUT_PACKED_FLOATS * n ** 3
    if out is None:
        out = torch.empty(size, dtype=torch.float32, device=lut.device)
    _need(out, "out", (size,))
    _check(lib().mact_lut_pack(h.ptr, _VP(lut.data_ptr()), n, _VP(out.data_ptr()), _stream(stream)), "mact_lut_pack")
    return out


def mact_lut_interp_packed(h, method, packed, n, rgb, out=None, sel=False, stream=None):
    """mact_lut_interp on a LUT of size n packed by mact_lut_pack."""
    _need(packed, "packed", (LUT_PACKED_FLOATS * n ** 3,))
    if rgb.dtype != torch.uint8 or not rgb.is_contiguous() or rgb.shape[-1] != 3:
        raise ValueError("rgb must be a contiguous (..., 3) uint8 tensor")
    npix = rgb.numel() // 3
    if out is None:
        out = torch.empty((3, npix), dtype=torch.float32, device=rgb.device,
                          pin_memory=rgb.device.type == "cpu")
    _need(out, "out", (3, npix))
    ptrs = (_VP * 3)(*(out[c].data_ptr() for c in range(3)))
    s = (torch.empty(npix, dtype=torch.int32, device=rgb.device, pin_memory=rgb.device.type == "cpu")
         if sel else None)
    m = METHODS[method] if isinstance(method, str) else int(method)
    _check(lib().mact_lut_interp_packed(h.ptr, m, _VP(packed.data_ptr()), n, _VP(rgb.data_ptr()), npix,
                                        ctypes.byref(ptrs), _VP(s.data_ptr() if s is not None else 0),
                                        _stream(stream)), "mact_lut_interp_packed")
    return (out, s) if sel else out


# ------------------------------------------------ error over the RGB cube

def mact_cube_error(h, space):
    """(eps_avg, eps_max) of the handle's transform over all 2^24 colours."""
    a, m = ctypes.c_double(), ctypes.c_double()
    sp = SPACES[space] if isinstance(space, str) else int(space)
    _check(lib().mact_cube_error(h.ptr, sp, ctypes.byref(a), ctypes.byref(m)), "mact_cube_error")
    return a.value, m.value


def mact_cube_error_lut(h, method, lut):
    """(eps_avg, eps_max) of LUT interpolation over all 2^24 colours."""
    n = lut.shape[0] if isinstance(lut, torch.Tensor) and lut.dim() == 4 else 0
    _need(lut, "lut", (n, n, n, 3))
    a, m = ctypes.c_double(), ctypes.c_double()
    md = METHODS[method] if isinstance(method, str) else int(method)
    _check(lib().mact_cube_error_lut(h.ptr, md, _VP(lut.data_ptr()), lut.shape[0], ctypes.byref(a),
                                     ctypes.byref(m)), "mact_cube_error_lut")
    return a.value, m.value


# ------------------------------------------------ batched plans, autotuner

def _image_array(images, outs):
    if len(outs) != len(images):
        raise ValueError("outs must hold one output per image")
    arr = (Image * max(len(images), 1))()
    for i, ((rgb, space), out) in enumerate(zip(images, outs)):
        arr[i] = _image(rgb, space, out)
    return arr


def _default_outs(images, dtype):
    return [torch.empty((3, r.shape[0], r.shape[1]), dtype=dtype, device=r.device,
                         pin_memory=r.device.type == "cpu") for r, _ in images]


class BatchPlan:
    """A fixed image list with its device work list (mact_batch_plan_t)."""

    def __init__(self, ptr, keep):
        self.ptr = ptr
        self._keep = keep

    def launch(self, stream=None):
        _check(lib().mact_batch_plan_launch(self.ptr, _stream(stream)), "mact_batch_plan_launch")

    def graph_launch(self, stream=None):
        _check(lib().mact_batch_plan_graph_launch(self.ptr, _stream(stream)), "mact_batch_plan_graph_launch")

    def close(self):
        if self.ptr:
            lib().mact_batch_plan_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001 - interpreter shutdown
            pass


def mact_batch_plan_create(h, images, dtype=torch.float32, outs=None):
    """Plan for a list of (rgb, space); returns (plan, outs)."""
    outs = _default_outs(images, dtype) if outs is None else outs
    arr = _image_array(images, outs)
    p = _VP()
    _check(lib().mact_batch_plan_create(h.ptr, arr, len(images), ctypes.byref(p)), "mact_batch_plan_create")
    return BatchPlan(p, (h, images, outs)), outs


def mact_autotune_batch(h, images, dtype=torch.float32, outs=None, reps=5):
    """Time every batch launch shape on these images; the fastest becomes the
    handle's shape.  Returns (table of dicts, chosen (threads, px/thread, ctas/SM))."""
    outs = _default_outs(images, dtype) if outs is None else outs
    arr = _image_array(images, outs)
    table = (TuneEntry * 32)()
    n = ctypes.c_int32()
    _check(lib().mact_autotune_batch(h.ptr, arr, len(images), int(reps), table, 32, ctypes.byref(n)),
           "mact_autotune_batch")
    rows = [{k: getattr(table[i], k) for k, _ in TuneEntry._fields_} for i in range(n.value)]
    return rows, mact_get_batch_shape(h)


def mact_set_batch_shape(h, threads, px_per_thread, ctas_per_sm=0):
    _check(lib().mact_set_batch_shape(h.ptr, threads, px_per_thread, ctas_per_sm), "mact_set_batch_shape")


def mact_get_batch_shape(h):
    v = [ctypes.c_int32() for _ in range(3)]
    _check(lib().mact_get_batch_shape(h.ptr, *[ctypes.byref(x) for x in v]), "mact_get_batch_shape")
    return tuple(x.value for x in v)


# ------------------------------------------------ differentiable CIELAB

def _planar(x):
    if x.dtype != torch.float32 or not x.is_contiguous() or x.dim() < 2 or x.shape[1] != 3:
        raise ValueError("expected a contiguous float32 tensor of shape (N, 3, ...)")
    nb = x.shape[0]
    return nb, (x.numel() // (3 * nb)) if nb else 0


def mact_lab_forward(h, x, out=None, stream=None):
    """CIELAB of linear RGB x (N, 3, ...) -> same shape."""
    nb, hw = _planar(x)
    out = torch.empty_like(x) if out is None else _need(out, "out", x.shape)
    _check(lib().mact_lab_forward(h.ptr, _VP(x.data_ptr()), nb, hw, _VP(out.data_ptr()), _stream(stream)),
           "mact_lab_forward")
    return out


def mact_lab_backward(h, x, grad_lab, out=None, stream=None):
    """Vector-Jacobian product J(x)^T grad_lab."""
    nb, hw = _planar(x)
    if not isinstance(grad_lab, torch.Tensor):
        raise TypeError("grad_lab must be a torch.Tensor")
    grad_lab = _need(grad_lab.contiguous(), "grad_lab", x.shape)
    out = torch.empty_like(x) if out is None else _need(out, "out", x.shape)
    _check(lib().mact_lab_backward(h.ptr, _VP(x.data_ptr()), _VP(grad_lab.data_ptr()), nb, hw,
                                   _VP(out.data_ptr()), _stream(stream)), "mact_lab_backward")
    return out


def mact_lab_delta_e_loss(h, x, target_lab, grad=True, loss=None, grad_out=None, stream=None):
    """(mean Delta E*ab of Lab(x) vs target_lab as a 0-d tensor, dLoss/dx or None)."""
    nb, hw = _planar(x)
    _need(target_lab, "target_lab", x.shape)
    loss = torch.empty((), dtype=torch.float32, device=x.device) if loss is None else _need(loss, "loss", ())
    g = (torch.empty_like(x) if grad_out is None else _need(grad_out, "grad_out", x.shape)) if grad else None
    _check(lib().mact_lab_delta_e_loss(h.ptr, _VP(x.data_ptr()), _VP(target_lab.data_ptr()), nb, hw,
                                       _VP(loss.data_ptr()), _VP(g.data_ptr() if g is not None else 0),
                                       _stream(stream)), "mact_lab_delta_e_loss")
    return loss, g


# ------------------------------------------------------------- served form

class Server:
    """Owns a mact_server_t (continuous-batching conversion server)."""

    def __init__(self, ptr, handle):
        self.ptr = ptr
        self.handle = handle      # keep the handle alive as long as the server
        self._keep = {}           # ticket -> tensors referenced by the request

    def close(self, timeout_ms=60000.0):
        if self.ptr:
            st = lib().mact_serve_destroy(self.ptr, timeout_ms)
            self.ptr = None
            self._keep.clear()
            return st
        return MACT_OK

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001 - interpreter shutdown
            pass


def mact_serve_create(h, mem_budget_bytes, max_slots=64):
    p = _VP()
    _check(lib().mact_serve_create(h.ptr, int(mem_budget_bytes), int(max_slots), ctypes.byref(p)),
           "mact_serve_create")
    return Server(p, h)


SERVE_MODES = {"direct": 0, "staged": 1}


def mact_serve_set_mode(srv, mode):
    """'direct' (host buffers the kernel can address are used in place) or
    'staged' (every host buffer is copied through the device arena)."""
    m = SERVE_MODES[mode] if isinstance(mode, str) else int(mode)
    _check(lib().mact_serve_set_mode(srv.ptr, m), "mact_serve_set_mode")


def mact_serve_submit(srv, rgb, space="cielab", out=None, dtype=torch.float32):
    """Queue one (H, W, 3) uint8 image; rgb and out may be host (pinned or
    pageable) or CUDA tensors.  Returns (ticket, out)."""
    if out is None:
        out = torch.empty((3, rgb.shape[0], rgb.shape[1]), dtype=dtype, device=rgb.device,
                          pin_memory=(rgb.device.type == "cpu"))
    img = _image(rgb, space, out)
    t = ctypes.c_uint64()
    _check(lib().mact_serve_submit(srv.ptr, ctypes.byref(img), ctypes.byref(t)), "mact_serve_submit")
    srv._keep[t.value] = (rgb, out)
    return t.value, out


def mact_serve_poll(srv, ticket):
    """(done, latency_ms); raises MactError for a failed request."""
    d = ctypes.c_int32()
    lat = ctypes.c_double()
    _check(lib().mact_serve_poll(srv.ptr, ticket, ctypes.byref(d), ctypes.byref(lat)), "mact_serve_poll")
    return bool(d.value), lat.value


def mact_serve_wait(srv, ticket, timeout_ms=60000.0):
    lat = ctypes.c_double()
    _check(lib().mact_serve_wait(srv.ptr, ticket, float(timeout_ms), ctypes.byref(lat)), "mact_serve_wait")
    return lat.value


def mact_serve_cancel(srv, ticket):
    _check(lib().mact_serve_cancel(srv.ptr, ticket), "mact_serve_cancel")


def mact_serve_release(srv, ticket):
    _check(lib().mact_serve_release(srv.ptr, ticket), "mact_serve_release")
    srv._keep.pop(ticket, None)


def mact_serve_stats(srv):
    st = ServeStats()
    _check(lib().mact_serve_stats(srv.ptr, ctypes.byref(st)), "mact_serve_stats")
    return st.as_dict()


def mact_serve_destroy(srv, timeout_ms=60000.0):
    return srv.close(timeout_ms)


def mact_lut_cache_build(h, lut, out=None, stream=None):
    """Caching layout of an (n, n, n, 3) FP32 LUT: ((n-1)^3, 8, 4) float32."""
    n = lut.shape[0] if isinstance(lut, torch.Tensor) and lut.dim() == 4 else 0
    _need(lut, "lut", (n, n, n, 3))
    if out is None:
        out = torch.empty(((n - 1) ** 3, 8, 4), dtype=torch.float32, device=lut.device)
    _need(out, "out", ((n - 1) ** 3, 8, 4))
    _check(lib().mact_lut_cache_build(h.ptr, _VP(lut.data_ptr()), n, _VP(out.data_ptr()), _stream(stream)),
           "mact_lut_cache_build")
    return out


def mact_lut_interp_cached(h, method, cache, n, rgb, out=None, sel=False, stream=None):
    """As mact_lut_interp, from the caching layout of an n^3 LUT."""
    if rgb.dtype != torch.uint8 or not rgb.is_contiguous() or rgb.shape[-1] != 3:
        raise ValueError("rgb must be a contiguous (..., 3) uint8 tensor")
    _need(cache, "cache", ((n - 1) ** 3, 8, 4))
    npix = rgb.numel() // 3
    if out is None:
        out = torch.empty((3, npix), dtype=torch.float32, device=rgb.device,
                          pin_memory=rgb.device.type == "cpu")
    _need(out, "out", (3, npix))
    ptrs = (_VP * 3)(*(out[c].data_ptr() for c in range(3)))
    s = (torch.empty(npix, dtype=torch.int32, device=rgb.device, pin_memory=rgb.device.type == "cpu")
         if sel else None)
    m = METHODS[method] if isinstance(method, str) else int(method)
    _check(lib().mact_lut_interp_cached(h.ptr, m, _VP(cache.data_ptr()), n, _VP(rgb.data_ptr()), npix,
                                        ctypes.byref(ptrs), _VP(s.data_ptr() if s is not None else 0),
                                        _stream(stream)), "mact_lut_interp_cached")
    return (out, s) if sel else out


def mact_lut_build_hsi(h, n, out=None, device="cuda", stream=None):
    """(n, n, n, 4) FP32 HSI LUT: (cos H, sin H, S, I) of the exact HSI at the
    nodes (gray nodes: (0, 0, 0, I))."""
    if out is None:
        out = torch.empty((n, n, n, 4), dtype=torch.float32, device=device)
    _need(out, "out", (n, n, n, 4))
    _check(lib().mact_lut_build_hsi(h.ptr, n, _VP(out.data_ptr()), _stream(stream)), "mact_lut_build_hsi")
    return out


def mact_lut_interp_hsi(h, lut4, rgb, out=None, stream=None):
    """Trilinear HSI interpolation with angular hue mixing of the (npix, 3)
    or (H, W, 3) uint8 pixels of rgb.  Returns (3, npix) planes H, S, I."""
    if lut4.dtype != torch.float32 or not lut4.is_contiguous() or lut4.dim() != 4 or lut4.shape[3] != 4:
        raise ValueError("lut4 must be a contiguous (n, n, n, 4) float32 tensor")
    if rgb.dtype != torch.uint8 or not rgb.is_contiguous() or rgb.shape[-1] != 3:
        raise ValueError("rgb must be a contiguous (..., 3) uint8 tensor")
    n = lut4.shape[0]
    if lut4.shape[1] != n or lut4.shape[2] != n:
        raise ValueError("lut4 must be a cube (n, n, n, 4)")
    npix = rgb.numel() // 3
    if out is None:
        out = torch.empty((3, npix), dtype=torch.float32, device=rgb.device,
                          pin_memory=rgb.device.type == "cpu")
    _need(out, "out", (3, npix))
    ptrs = (_VP * 3)(*(out[c].data_ptr() for c in range(3)))
    _check(lib().mact_lut_interp_hsi(h.ptr, _VP(lut4.data_ptr()), lut4.shape[0], _VP(rgb.data_ptr()), npix, ptrs,
                                     _stream(stream)), "mact_lut_interp_hsi")
    return out


def mact_host_memory_access(h):
    """1 if the kernels of h may be given any host memory (the device walks
    the host page tables), 0 if only device and pinned/registered host memory
    (other host pointers are then rejected before launch)."""
    r = lib().mact_host_memory_access(h.ptr)
    if r < 0:
        _check(r, "mact_host_memory_access")
    return r


def mact_fit_cbrt_rational(n, m):
    """The library's host-side minimax rational of t^(1/3) on [0.008856, 1]:
    (p, q, max_err), ascending coefficients with q[0] = 1."""
    p, q, e = (ctypes.c_double * 7)(), (ctypes.c_double * 7)(), ctypes.c_double()
    _check(lib().mact_fit_cbrt_rational(int(n), int(m), p, q, ctypes.byref(e)), "mact_fit_cbrt_rational")
    return list(p)[: n + 1], list(q)[: m + 1], e.value


def mact_fit_hsi_arctan(n):
    """The library's host-side minimax polynomial of arctan(sqrt(3) x) on
    [0, 1]: (c, max_err), ascending coefficients."""
    c, e = (ctypes.c_double * 6)(), ctypes.c_double()
    _check(lib().mact_fit_hsi_arctan(int(n), c, ctypes.byref(e)), "mact_fit_hsi_arctan")
    return list(c)[: n + 1], e.value


def mact_strerror(status):
    return lib().mact_strerror(status).decode()


def mact_last_error():
    return lib().mact_last_error().decode()
