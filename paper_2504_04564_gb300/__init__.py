"""Python binding of libvdbc (include/vdbc.h): argument marshalling only.

Every step of encoding and rendering runs in the library's CUDA kernels.  The
binding converts torch tensors (device memory, via ``data_ptr()``), numpy
arrays (host memory) and plain Python values into the C structs, and turns a
non-OK status into ``VdbcError``.  There is no fallback: if ``libvdbc.so`` is
missing the import of :func:`lib` raises.

Functions keep the C names: ``vdbc_encode``, ``vdbc_render``,
``vdbc_render_dense``, ``vdbc_volume_create``, ``vdbc_grid_decode`` ...
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

# VDBC_CHECKED=1 in the environment selects the bounds-checked build,
# VDBC_SANITIZE=1 the build whose host code runs under ASan/UBSan
CHECKED = os.environ.get("VDBC_CHECKED", "") == "1"
SANITIZE = not CHECKED and os.environ.get("VDBC_SANITIZE", "") == "1"
LIB_PATH = _build.LIB_CHECKED if CHECKED else (_build.LIB_ASAN if SANITIZE else _build.LIB)

OK, ERR_INVALID_ARG, ERR_OOM, ERR_CUDA, ERR_FORMAT, ERR_TIMEOUT, ERR_DEVICE_FLAG, ERR_UNSUPPORTED = range(8)
F1, F2, F3 = 1, 2, 3
FP32, FP16, FP8, LEARNED = 0, 1, 2, 3
CAM_ORTHO, CAM_PINHOLE = 0, 1
MODE_EA, MODE_PT, MODE_ISO = 0, 1, 2
FILTER_TEXTURE, FILTER_LINEAR = 0, 1

STATUS_NAMES = {0: "OK", 1: "INVALID_ARG", 2: "OOM", 3: "CUDA", 4: "FORMAT", 5: "TIMEOUT",
                6: "DEVICE_FLAG", 7: "UNSUPPORTED"}


class VdbcError(RuntimeError):
    def __init__(self, status, message):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), message))
        self.status = status


class Dense(ctypes.Structure):
    _fields_ = [("dims", ctypes.c_int32 * 3), ("on_device", ctypes.c_int32), ("data", ctypes.c_void_p)]


class EncodeParams(ctypes.Structure):
    _fields_ = [("ratio", ctypes.c_double), ("metric", ctypes.c_int32), ("payload", ctypes.c_int32),
                ("macrocell", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class GridInfo(ctypes.Structure):
    _fields_ = [("dims", ctypes.c_int32 * 3), ("payload", ctypes.c_int32), ("macrocell", ctypes.c_int32),
                ("metric", ctypes.c_int32), ("background_bits", ctypes.c_uint32), ("reserved", ctypes.c_int32),
                ("ratio", ctypes.c_double), ("n_bricks", ctypes.c_int64), ("n_nonempty", ctypes.c_int64),
                ("budget", ctypes.c_int64), ("n_active", ctypes.c_int64), ("n_upper", ctypes.c_int64),
                ("n_lower", ctypes.c_int64), ("n_leaves", ctypes.c_int64), ("n_tiles", ctypes.c_int64),
                ("n_neural", ctypes.c_int64), ("payload_bytes", ctypes.c_uint64), ("node_bytes", ctypes.c_uint64),
                ("total_bytes", ctypes.c_uint64)]

    def as_dict(self):
        d = {}
        for name, _ in self._fields_:
            v = getattr(self, name)
            d[name] = list(v) if name == "dims" else v
        return d


class Camera(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("width", ctypes.c_int32), ("height", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("eye", ctypes.c_double * 3), ("look", ctypes.c_double * 3),
                ("up", ctypes.c_double * 3), ("fovy_or_height", ctypes.c_double)]


class Medium(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("tf_n", ctypes.c_int32), ("tf_rgba", ctypes.c_void_p),
                ("step", ctypes.c_float), ("density_scale", ctypes.c_float), ("albedo", ctypes.c_float),
                ("g", ctypes.c_float), ("max_bounces", ctypes.c_int32), ("iso", ctypes.c_float),
                ("sun_dir", ctypes.c_float * 3), ("sun_rad", ctypes.c_float * 3), ("env_rad", ctypes.c_float * 3)]


class Job(ctypes.Structure):
    _fields_ = [("grid", ctypes.c_void_p), ("camera", Camera), ("medium", Medium), ("spp", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("seed", ctypes.c_uint64), ("rgba_out", ctypes.c_void_p)]


class Tuning(ctypes.Structure):
    _fields_ = [("threads", ctypes.c_int32), ("chunk", ctypes.c_int32), ("coarse", ctypes.c_int32),
                ("depth", ctypes.c_int32), ("frame_ms", ctypes.c_float)]


class RenderStats(ctypes.Structure):
    _fields_ = [("lookups", ctypes.c_uint64), ("paths", ctypes.c_uint64), ("error_flags", ctypes.c_uint64),
                ("events", ctypes.c_uint64 * 8), ("kernel_ms", ctypes.c_float), ("reserved", ctypes.c_int32)]


class LearnState(ctypes.Structure):
    _fields_ = [("params", ctypes.c_void_p), ("params_m", ctypes.c_void_p), ("params_v", ctypes.c_void_p),
                ("latents", ctypes.c_void_p), ("latents_m", ctypes.c_void_p), ("latents_v", ctypes.c_void_p),
                ("step", ctypes.c_int64)]


class LearnParams(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_int32), ("samples_per_leaf", ctypes.c_int32), ("lr", ctypes.c_float),
                ("lr_latent", ctypes.c_float), ("max_error", ctypes.c_float), ("reserved", ctypes.c_int32),
                ("max_bytes", ctypes.c_uint64), ("seed", ctypes.c_uint64), ("init_params", ctypes.c_void_p),
                ("init_latents", ctypes.c_void_p), ("force", ctypes.c_void_p),
                ("resume", ctypes.POINTER(LearnState)), ("save", ctypes.POINTER(LearnState))]


MLP_PARAMS = 1729   # 19 -> 32 -> 32 -> 1: W1, b1, W2, b2, w3, b3

_lib = None

# name -> (restype, argtypes); the exported surface of include/vdbc.h
_vp = ctypes.c_void_p
class ErrorStats(ctypes.Structure):
    _fields_ = [("mse", ctypes.c_double), ("rmse", ctypes.c_double), ("mean_abs", ctypes.c_double),
                ("max_abs", ctypes.c_double), ("psnr", ctypes.c_double), ("n", ctypes.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


SIGNATURES = {
    "vdbc_encode": (ctypes.c_int, [ctypes.POINTER(Dense), ctypes.POINTER(EncodeParams), _vp, ctypes.POINTER(_vp)]),
    "vdbc_grid_get_info": (ctypes.c_int, [_vp, ctypes.POINTER(GridInfo)]),
    "vdbc_grid_decode": (ctypes.c_int, [_vp, _vp, ctypes.c_int32, _vp]),
    "vdbc_grid_active_bricks": (ctypes.c_int, [_vp, _vp]),
    "vdbc_grid_macrocells": (ctypes.c_int, [_vp, _vp, _vp]),
    "vdbc_grid_save": (ctypes.c_int, [_vp, ctypes.c_char_p]),
    "vdbc_grid_load": (ctypes.c_int, [ctypes.c_char_p, _vp, ctypes.POINTER(_vp)]),
    "vdbc_grid_free": (None, [_vp]),
    "vdbc_render": (ctypes.c_int, [_vp, ctypes.POINTER(Camera), ctypes.POINTER(Medium), ctypes.c_int32,
                                   ctypes.c_uint64, _vp, ctypes.c_int32, _vp]),
    "vdbc_render_stats_get": (ctypes.c_int, [_vp, _vp, ctypes.POINTER(RenderStats)]),
    "vdbc_volume_create": (ctypes.c_int, [ctypes.POINTER(Dense), ctypes.c_int32, ctypes.c_int32, _vp,
                                          ctypes.POINTER(_vp)]),
    "vdbc_volume_free": (None, [_vp]),
    "vdbc_render_dense": (ctypes.c_int, [_vp, ctypes.POINTER(Camera), ctypes.POINTER(Medium), ctypes.c_int32,
                                         ctypes.c_uint64, _vp, ctypes.c_int32, _vp]),
    "vdbc_volume_render_stats_get": (ctypes.c_int, [_vp, _vp, ctypes.POINTER(RenderStats)]),
    "vdbc_philox": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int32]),
    "vdbc_compare": (ctypes.c_int, [_vp, _vp, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, _vp,
                                    ctypes.POINTER(ErrorStats)]),
    "vdbc_select_bricks_noalloc": (ctypes.c_int, [ctypes.POINTER(Dense), ctypes.POINTER(EncodeParams), _vp, _vp,
                                                  _vp, _vp]),
    "vdbc_batch_create": (ctypes.c_int, [ctypes.POINTER(Job), ctypes.c_int32, ctypes.c_int32, _vp,
                                         ctypes.POINTER(_vp)]),
    "vdbc_batch_render_frames": (ctypes.c_int, [_vp, ctypes.c_int32, _vp]),
    "vdbc_batch_reset": (ctypes.c_int, [_vp, _vp]),
    "vdbc_batch_state_size": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_int64)]),
    "vdbc_batch_get_state": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_int32), _vp, _vp]),
    "vdbc_batch_set_state": (ctypes.c_int, [_vp, ctypes.c_int32, _vp, _vp]),
    "vdbc_batch_get_tuning": (ctypes.c_int, [_vp, ctypes.POINTER(Tuning)]),
    "vdbc_batch_stats_get": (ctypes.c_int, [_vp, _vp, ctypes.POINTER(RenderStats)]),
    "vdbc_batch_free": (None, [_vp]),
    "vdbc_learn": (ctypes.c_int, [_vp, ctypes.POINTER(LearnParams), _vp, ctypes.POINTER(_vp), _vp]),
    "vdbc_learn_loss_grad": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int64, _vp, _vp, _vp, _vp]),
    "vdbc_learn_get_params": (ctypes.c_int, [_vp, _vp]),
    "vdbc_kernel_launches": (ctypes.c_uint64, []),
    "vdbc_last_error": (ctypes.c_char_p, []),
    "vdbc_version": (ctypes.c_char_p, []),
}


def lib():
    """The loaded libvdbc.so.  Raises if it has not been built (no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("%s is not built; run __graft_entry__.build() "
                              "or python -m paper_2504_04564_gb300.build%s"
                              % (LIB_PATH, " --checked" if CHECKED else (" --sanitize" if SANITIZE else "")))
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(status):
    if status != OK:
        msg = lib().vdbc_last_error()
        raise VdbcError(status, msg.decode() if msg else "")


# ---------------------------------------------------------------- marshalling helpers
def _is_torch(x):
    return type(x).__module__.startswith("torch")


def _ptr(x):
    """(address, on_device) of a torch tensor or a numpy array."""
    if _is_torch(x):
        return x.data_ptr(), int(x.is_cuda)
    if isinstance(x, np.ndarray):
        return x.ctypes.data, 0
    raise TypeError("expected a torch tensor or a numpy array, got %r" % type(x))


def _stream(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except ImportError:
            pass
        return 0
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def make_dense(vol) -> Dense:
    """Descriptor of an x-fastest (nz, ny, nx) float32 volume (torch or numpy)."""
    if _is_torch(vol):
        assert vol.dtype.__str__() == "torch.float32" and vol.is_contiguous()
    else:
        assert vol.dtype == np.float32 and vol.flags["C_CONTIGUOUS"]
    nz, ny, nx = vol.shape
    d = Dense()
    d.dims[0], d.dims[1], d.dims[2] = nx, ny, nz
    p, on_dev = _ptr(vol)
    d.data = p
    d.on_device = on_dev
    return d


def make_camera(kind, width, height, eye, look, up, fovy_or_height) -> Camera:
    c = Camera()
    c.kind, c.width, c.height = int(kind), int(width), int(height)
    for a in range(3):
        c.eye[a], c.look[a], c.up[a] = float(eye[a]), float(look[a]), float(up[a])
    c.fovy_or_height = float(fovy_or_height)
    return c


def make_medium(mode, tf=None, step=0.5, density_scale=1.0, albedo=0.9, g=0.0, max_bounces=1,
                sun_dir=(0, 0, 1), sun_rad=(0, 0, 0), env_rad=(0, 0, 0), iso=0.5) -> Medium:
    m = Medium()
    m.mode = int(mode)
    m._tf = None
    if tf is not None:
        m._tf = np.ascontiguousarray(tf, dtype=np.float32).reshape(-1, 4)
        m.tf_n = m._tf.shape[0]
        m.tf_rgba = m._tf.ctypes.data
    m.step, m.density_scale, m.albedo, m.g = float(step), float(density_scale), float(albedo), float(g)
    m.max_bounces = int(max_bounces)
    m.iso = float(iso)
    for a in range(3):
        m.sun_dir[a], m.sun_rad[a], m.env_rad[a] = float(sun_dir[a]), float(sun_rad[a]), float(env_rad[a])
    return m


# ---------------------------------------------------------------- the C entry points
class Grid:
    """Owning wrapper of a vdbc_grid*; frees it on close()/garbage collection."""

    def __init__(self, handle):
        self.handle = handle

    @property
    def info(self) -> GridInfo:
        return vdbc_grid_get_info(self)

    def close(self):
        if self.handle:
            lib().vdbc_grid_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Volume:
    """Owning wrapper of a vdbc_volume* (the plain dense form)."""

    def __init__(self, handle):
        self.handle = handle

    def close(self):
        if self.handle:
            lib().vdbc_volume_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def vdbc_encode(vol, ratio, metric=F2, payload=FP32, macrocell=8, stream=None) -> Grid:
    d = make_dense(vol)
    p = EncodeParams(float(ratio), int(metric), int(payload), int(macrocell), 0)
    h = ctypes.c_void_p()
    _check(lib().vdbc_encode(ctypes.byref(d), ctypes.byref(p), _stream(stream), ctypes.byref(h)))
    return Grid(h.value)


def vdbc_grid_get_info(grid: Grid) -> GridInfo:
    info = GridInfo()
    _check(lib().vdbc_grid_get_info(grid.handle, ctypes.byref(info)))
    return info


def vdbc_grid_decode(grid: Grid, out, stream=None):
    p, on_dev = _ptr(out)
    _check(lib().vdbc_grid_decode(grid.handle, p, on_dev, _stream(stream)))
    return out


def vdbc_grid_active_bricks(grid: Grid) -> np.ndarray:
    out = np.zeros(grid.info.n_bricks, dtype=np.uint8)
    _check(lib().vdbc_grid_active_bricks(grid.handle, out.ctypes.data))
    return out


def vdbc_grid_macrocells(grid: Grid):
    i = grid.info
    mc = i.macrocell
    n = int(np.prod([(d + mc - 1) // mc for d in i.dims]))
    mn = np.zeros(n, dtype=np.float32)
    mx = np.zeros(n, dtype=np.float32)
    _check(lib().vdbc_grid_macrocells(grid.handle, mn.ctypes.data, mx.ctypes.data))
    return mn, mx


def vdbc_grid_save(grid: Grid, path: str) -> None:
    _check(lib().vdbc_grid_save(grid.handle, path.encode()))


def vdbc_grid_load(path: str, stream=None) -> Grid:
    h = ctypes.c_void_p()
    _check(lib().vdbc_grid_load(path.encode(), _stream(stream), ctypes.byref(h)))
    return Grid(h.value)


def vdbc_render(grid: Grid, camera: Camera, medium: Medium, spp, seed, out, stream=None):
    p, on_dev = _ptr(out)
    _check(lib().vdbc_render(grid.handle, ctypes.byref(camera), ctypes.byref(medium), int(spp),
                             ctypes.c_uint64(int(seed)), p, on_dev, _stream(stream)))
    return out


def vdbc_render_stats_get(grid: Grid, stream=None) -> RenderStats:
    s = RenderStats()
    _check(lib().vdbc_render_stats_get(grid.handle, _stream(stream), ctypes.byref(s)))
    return s


def vdbc_volume_create(vol, filter=FILTER_TEXTURE, macrocell=8, stream=None) -> Volume:
    d = make_dense(vol)
    h = ctypes.c_void_p()
    _check(lib().vdbc_volume_create(ctypes.byref(d), int(filter), int(macrocell), _stream(stream),
                                    ctypes.byref(h)))
    return Volume(h.value)


def vdbc_render_dense(volume: Volume, camera: Camera, medium: Medium, spp, seed, out, stream=None):
    p, on_dev = _ptr(out)
    _check(lib().vdbc_render_dense(volume.handle, ctypes.byref(camera), ctypes.byref(medium), int(spp),
                                   ctypes.c_uint64(int(seed)), p, on_dev, _stream(stream)))
    return out


def vdbc_volume_render_stats_get(volume: Volume, stream=None) -> RenderStats:
    s = RenderStats()
    _check(lib().vdbc_volume_render_stats_get(volume.handle, _stream(stream), ctypes.byref(s)))
    return s


class Batch:
    """Owning wrapper of a vdbc_batch*; keeps its grids and outputs alive."""

    def __init__(self, handle, keep):
        self.handle = handle
        self._keep = keep

    def close(self):
        if self.handle:
            lib().vdbc_batch_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def make_job(grid: Grid, camera: Camera, medium: Medium, spp, seed, out) -> Job:
    j = Job()
    j.grid = grid.handle
    j.camera = camera
    j.medium = medium
    j.spp = int(spp)
    j.seed = int(seed)
    j.rgba_out = _ptr(out)[0]
    return j


def vdbc_batch_create(jobs, autotune=True, stream=None, keep=()) -> Batch:
    """jobs: a list of Job structs (see make_job); `keep` holds Python objects
    (grids, output tensors) that must outlive the batch."""
    arr = (Job * len(jobs))(*jobs)
    h = ctypes.c_void_p()
    _check(lib().vdbc_batch_create(arr, len(jobs), int(bool(autotune)), _stream(stream), ctypes.byref(h)))
    return Batch(h.value, (list(keep), jobs))


def vdbc_batch_render_frames(batch: Batch, frames=1, stream=None):
    _check(lib().vdbc_batch_render_frames(batch.handle, int(frames), _stream(stream)))


def vdbc_batch_reset(batch: Batch, stream=None):
    _check(lib().vdbc_batch_reset(batch.handle, _stream(stream)))


def vdbc_batch_get_state(batch: Batch, stream=None):
    """(frame, per-pixel sums as a float32 numpy array of vdbc_batch_state_size floats)."""
    n = ctypes.c_int64(0)
    _check(lib().vdbc_batch_state_size(batch.handle, ctypes.byref(n)))
    sums = np.zeros(n.value, dtype=np.float32)
    frame = ctypes.c_int32(0)
    _check(lib().vdbc_batch_get_state(batch.handle, ctypes.byref(frame), sums.ctypes.data, _stream(stream)))
    return int(frame.value), sums


def vdbc_batch_set_state(batch: Batch, frame: int, sums, stream=None):
    n = ctypes.c_int64(0)
    _check(lib().vdbc_batch_state_size(batch.handle, ctypes.byref(n)))
    a = np.ascontiguousarray(sums, dtype=np.float32)
    if a.size != n.value:
        raise ValueError("state of %d floats for a batch of %d" % (a.size, n.value))
    _check(lib().vdbc_batch_set_state(batch.handle, int(frame), a.ctypes.data, _stream(stream)))


def vdbc_batch_get_tuning(batch: Batch) -> Tuning:
    t = Tuning()
    _check(lib().vdbc_batch_get_tuning(batch.handle, ctypes.byref(t)))
    return t


def vdbc_batch_stats_get(batch: Batch, stream=None) -> RenderStats:
    st = RenderStats()
    _check(lib().vdbc_batch_stats_get(batch.handle, _stream(stream), ctypes.byref(st)))
    return st


def vdbc_compare(a, b, stride=1, channels=1, stream=None) -> ErrorStats:
    """FP64 error of device array `a` against `b` (same shape): elements of
    `stride` floats, the first `channels` of each compared (an RGBA image:
    stride=4, channels=3)."""
    if not (a.is_cuda and b.is_cuda) or a.numel() != b.numel() or a.numel() % stride:
        raise ValueError("vdbc_compare: two CUDA arrays of the same size, a multiple of the stride")
    if not (a.is_contiguous() and b.is_contiguous()) or str(a.dtype) != "torch.float32" or str(b.dtype) != "torch.float32":
        raise ValueError("vdbc_compare: contiguous float32 arrays")
    out = ErrorStats()
    _check(lib().vdbc_compare(a.data_ptr(), b.data_ptr(), a.numel() // stride, int(stride), int(channels),
                              _stream(stream), ctypes.byref(out)))
    return out


def vdbc_select_bricks_noalloc(vol, ratio, background_bits_out, active_out, counts_out, metric=F2, payload=FP32,
                               stream=None):
    """Brick selection of vdbc_encode without allocating (device tensors in
    and out; see include/vdbc.h for who needs it and its limits).  The
    outputs must be CUDA tensors: one uint32 (or int32) word, one uint8 per
    32^3 brick and three int64."""
    dims = [int(x) for x in vol.shape[::-1]]
    nb = 1
    for n in dims:
        nb *= (n + 31) // 32
    for name, t, dtypes, need in (("background_bits_out", background_bits_out, ("torch.uint32", "torch.int32"), 1),
                                  ("active_out", active_out, ("torch.uint8",), nb),
                                  ("counts_out", counts_out, ("torch.int64",), 3)):
        if not (hasattr(t, "is_cuda") and t.is_cuda):
            raise TypeError("%s must be a CUDA tensor" % name)
        if str(t.dtype) not in dtypes:
            raise TypeError("%s must have dtype %s, not %s" % (name, " or ".join(dtypes), t.dtype))
        if not t.is_contiguous() or t.numel() < need:
            raise ValueError("%s must be contiguous with at least %d elements (has %d)" % (name, need, t.numel()))
    d = make_dense(vol)
    p = EncodeParams(float(ratio), int(metric), int(payload), 8, 0)
    _check(lib().vdbc_select_bricks_noalloc(ctypes.byref(d), ctypes.byref(p), _ptr(background_bits_out)[0],
                                            _ptr(active_out)[0], _ptr(counts_out)[0], _stream(stream)))


class LearnCheckpoint:
    """The arrays of a vdbc_learn_state (device tensors the caller owns) and
    its step count.  ``LearnCheckpoint.zeros(grid, torch, device)`` sizes them
    for `grid`'s leaf positions."""
    FIELDS = ("params", "params_m", "params_v", "latents", "latents_m", "latents_v")

    def __init__(self, arrays, step=0):
        self.arrays = dict(arrays)
        self.step = int(step)

    @classmethod
    def zeros(cls, grid, torch, device):
        npos = 1
        for d in grid.info.dims:
            npos *= (int(d) + 7) // 8
        n = dict(params=MLP_PARAMS, params_m=MLP_PARAMS, params_v=MLP_PARAMS, latents=npos * 16,
                 latents_m=npos * 16, latents_v=npos * 16)
        return cls({k: torch.zeros(n[k], dtype=torch.float32, device=device) for k in cls.FIELDS})

    def struct(self) -> LearnState:
        return LearnState(*[_ptr(self.arrays[k])[0] for k in self.FIELDS], self.step)


def vdbc_learn(grid: Grid, steps=200, samples_per_leaf=64, lr=1e-3, lr_latent=1e-2, max_error=0.0, max_bytes=0,
               seed=0, init_params=None, init_latents=None, force=None, resume=None, save=None, stream=None):
    """Learned grid from `grid` (see include/vdbc.h).  init_params (1729),
    init_latents (per leaf position x 16) and force (per leaf position,
    uint8) are device tensors or None; resume / save are LearnCheckpoint or
    None (save.step is updated).  Returns (Grid, per-step losses)."""
    p = LearnParams(int(steps), int(samples_per_leaf), float(lr), float(lr_latent), float(max_error), 0,
                    int(max_bytes), int(seed), _ptr(init_params)[0] if init_params is not None else None,
                    _ptr(init_latents)[0] if init_latents is not None else None,
                    _ptr(force)[0] if force is not None else None)
    rs = resume.struct() if resume is not None else None
    sv = save.struct() if save is not None else None
    if rs is not None:
        p.resume = ctypes.pointer(rs)
    if sv is not None:
        p.save = ctypes.pointer(sv)
    out = _vp()
    losses = np.zeros(max(int(steps), 1), dtype=np.float64)
    _check(lib().vdbc_learn(grid.handle, ctypes.byref(p), _stream(stream), ctypes.byref(out), losses.ctypes.data))
    if sv is not None:
        save.step = int(sv.step)
    return Grid(out.value), losses[:int(steps)]


def vdbc_learn_loss_grad(params, inputs, targets, grad_params, grad_inputs=None, stream=None) -> float:
    """Loss and gradients of the training kernels on explicit samples (device tensors)."""
    n = int(targets.numel())
    loss = ctypes.c_double(0.0)
    _check(lib().vdbc_learn_loss_grad(_ptr(params)[0], _ptr(inputs)[0], _ptr(targets)[0], n, ctypes.byref(loss),
                                      _ptr(grad_params)[0],
                                      _ptr(grad_inputs)[0] if grad_inputs is not None else None, _stream(stream)))
    return loss.value


def vdbc_learn_get_params(grid: Grid) -> np.ndarray:
    out = np.zeros(MLP_PARAMS, dtype=np.float32)
    _check(lib().vdbc_learn_get_params(grid.handle, out.ctypes.data))
    return out


def vdbc_philox(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(-1, 4)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros_like(c)
    _check(lib().vdbc_philox(c.ctypes.data, k.ctypes.data, out.ctypes.data, c.shape[0]))
    return out


def vdbc_kernel_launches() -> int:
    return int(lib().vdbc_kernel_launches())


def vdbc_last_error() -> str:
    return lib().vdbc_last_error().decode()


def vdbc_version() -> str:
    return lib().vdbc_version().decode()
