"""CPU oracle -- TEST INFRASTRUCTURE ONLY.

A plain, slow, FP64 restatement in C of what arXiv 2504.04564 computes (see
``oracle.h`` for the list).  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py`` (its ``cpu_baseline`` leg and ``--impl reference``) may import
this package.  The product path (``paper_2504_04564_gb300``) never does: it
shares no code, header, table or helper with this directory.

This module compiles ``liboracle.so`` with gcc (``build()``) and wraps its
functions with numpy-friendly signatures.  With ORACLE_SANITIZE=1 in the
environment it builds and loads ``liboracle_asan.so`` instead, instrumented
by AddressSanitizer and UndefinedBehaviorSanitizer (the process must then
start with libasan preloaded).
"""
from __future__ import annotations

import contextlib
import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
SANITIZE = os.environ.get("ORACLE_SANITIZE", "") == "1"
LIB = os.path.join(_BUILD, "liboracle_asan.so" if SANITIZE else "liboracle.so")
SOURCES = ["philox.c", "encode.c", "render.c", "mlp.c"]
SANITIZE_FLAGS = ["-g", "-fno-omit-frame-pointer", "-fsanitize=address,undefined", "-fno-sanitize-recover=all"]

F1, F2, F3 = 1, 2, 3
FP32, FP16, FP8 = 0, 1, 2
CAM_ORTHO, CAM_PINHOLE = 0, 1
MODE_EA, MODE_PT, MODE_ISO = 0, 1, 2

c_i64p = ctypes.POINTER(ctypes.c_int64)


def compile_library(src_dir: str, out: str, sanitize: bool = False) -> str:
    """Compile the oracle's C sources found in `src_dir` into the shared
    library `out` (the flags every build of the oracle uses)."""
    srcs = [os.path.join(src_dir, s) for s in SOURCES if os.path.exists(os.path.join(src_dir, s))]
    cmd = ["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared"] + (SANITIZE_FLAGS if sanitize else []) + srcs + ["-o", out, "-lm"]
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
    if r.returncode != 0:
        raise RuntimeError("oracle build failed:\n" + r.stdout.decode())
    return r.stdout.decode()


def build(verbose: bool = False) -> None:
    os.makedirs(_BUILD, exist_ok=True)
    srcs = [os.path.join(_HERE, s) for s in SOURCES if os.path.exists(os.path.join(_HERE, s))]
    deps = srcs + [os.path.join(_HERE, "oracle.h")]
    if os.path.exists(LIB) and all(os.path.getmtime(d) <= os.path.getmtime(LIB) for d in deps):
        return
    log = compile_library(_HERE, LIB, SANITIZE)
    if verbose and log:
        print(log)


class Camera(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("width", ctypes.c_int32), ("height", ctypes.c_int32),
                ("eye", ctypes.c_double * 3), ("look", ctypes.c_double * 3),
                ("up", ctypes.c_double * 3), ("fovy_or_height", ctypes.c_double)]


class Medium(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("tf_n", ctypes.c_int32),
                ("tf_rgba", ctypes.POINTER(ctypes.c_float)), ("step", ctypes.c_double),
                ("density_scale", ctypes.c_double), ("albedo", ctypes.c_double),
                ("g", ctypes.c_double), ("max_bounces", ctypes.c_int32),
                ("macrocell", ctypes.c_int32), ("sun_dir", ctypes.c_double * 3),
                ("sun_rad", ctypes.c_double * 3), ("env_rad", ctypes.c_double * 3), ("iso", ctypes.c_double)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = _bind(ctypes.CDLL(LIB))
    return _lib


@contextlib.contextmanager
def library(path: str):
    """Bind every wrapper of this module to another build of the oracle's
    sources for the duration of the block (the pin tests load a copy with a
    deliberately planted mistake this way, to show that a pin catches it)."""
    global _lib
    saved = _lib
    _lib = _bind(ctypes.CDLL(path))
    try:
        yield _lib
    finally:
        _lib = saved


def _bind(L):
    vp = ctypes.c_void_p
    L.or_philox4x32_10.argtypes = [vp, vp, vp]
    L.or_u01.argtypes = [ctypes.c_uint32]
    L.or_u01.restype = ctypes.c_double
    L.or_background_bits.argtypes = [vp, ctypes.c_int64]
    L.or_background_bits.restype = ctypes.c_uint32
    L.or_brick_grid.argtypes = [vp, vp]
    L.or_brick_ranges.argtypes = [vp, vp, vp, vp]
    L.or_brick_scores.argtypes = [vp, vp, ctypes.c_int64, ctypes.c_uint32, ctypes.c_int, vp, vp]
    L.or_brick_budget.argtypes = [ctypes.c_int64, ctypes.c_double, ctypes.c_int]
    L.or_brick_budget.restype = ctypes.c_int64
    L.or_select.argtypes = [vp, vp, ctypes.c_int64, ctypes.c_int64, vp]
    L.or_select.restype = ctypes.c_int64
    L.or_decode_dense.argtypes = [vp, vp, vp, ctypes.c_uint32, ctypes.c_int, vp]
    L.or_round_fp16.argtypes = [ctypes.c_float]
    L.or_round_fp16.restype = ctypes.c_float
    L.or_round_e4m3.argtypes = [ctypes.c_float]
    L.or_round_e4m3.restype = ctypes.c_float
    L.or_quantize_leaf.argtypes = [vp, ctypes.c_int, vp, vp, vp]
    L.or_tree_build.argtypes = [vp, vp, vp, ctypes.c_uint32, ctypes.c_int]
    L.or_tree_build.restype = vp
    L.or_tree_value.argtypes = [vp, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64]
    L.or_tree_value.restype = ctypes.c_float
    L.or_tree_counts.argtypes = [vp, vp]
    L.or_tree_free.argtypes = [vp]
    L.or_trilinear.argtypes = [vp, vp, vp]
    L.or_trilinear.restype = ctypes.c_double
    L.or_macrocell_minmax.argtypes = [vp, vp, ctypes.c_int32, vp, vp]
    L.or_clip_box.argtypes = [vp, vp, vp, vp, vp]
    L.or_clip_box.restype = ctypes.c_int
    L.or_dda_cells.argtypes = [vp, ctypes.c_int32, vp, vp, ctypes.c_double, ctypes.c_double,
                               vp, vp, vp, ctypes.c_int64]
    L.or_dda_cells.restype = ctypes.c_int64
    L.or_hg_eval.argtypes = [ctypes.c_double, ctypes.c_double]
    L.or_hg_eval.restype = ctypes.c_double
    L.or_hg_sample_mu.argtypes = [ctypes.c_double, ctypes.c_double]
    L.or_hg_sample_mu.restype = ctypes.c_double
    L.or_onb.argtypes = [vp, vp, vp]
    L.or_scatter_dir.argtypes = [vp, ctypes.c_double, ctypes.c_double, vp]
    L.or_camera_ray.argtypes = [ctypes.POINTER(Camera), vp, ctypes.c_int64, ctypes.c_int64,
                                ctypes.c_double, ctypes.c_double, vp, vp]
    L.or_ratio_transmittance.argtypes = [vp, vp, vp, ctypes.POINTER(Medium), vp, vp,
                                         ctypes.c_uint32, ctypes.c_uint32, vp, vp]
    L.or_ratio_transmittance.restype = ctypes.c_double
    L.or_render_pixels.argtypes = [vp, vp, vp, ctypes.POINTER(Camera), ctypes.POINTER(Medium),
                                   ctypes.c_int32, ctypes.c_uint64, vp, ctypes.c_int64, vp]
    if hasattr(L, "or_mlp_forward"):
        _bind_mlp(L)
    return L


def _bind_mlp(L):
    vp = ctypes.c_void_p
    L.or_mlp_num_params.restype = ctypes.c_int
    L.or_mlp_forward.argtypes = [vp, vp, ctypes.c_int64, vp]
    L.or_mlp_loss_grad.argtypes = [vp, vp, vp, ctypes.c_int64, vp, vp]
    L.or_mlp_loss_grad.restype = ctypes.c_double
    L.or_adam_step.argtypes = [vp, vp, vp, vp, ctypes.c_int64, ctypes.c_int64, ctypes.c_double,
                               ctypes.c_double, ctypes.c_double, ctypes.c_double]
    L.or_round_bf16.argtypes = [ctypes.c_float]
    L.or_round_bf16.restype = ctypes.c_float
    L.or_mlp_forward_bf16.argtypes = [vp, vp, ctypes.c_int64, vp]
    L.or_learned_leaf.argtypes = [vp, vp, vp, vp]
    L.or_mlp_loss_grad_bf16.argtypes = [vp, vp, vp, ctypes.c_int64, vp, vp]
    L.or_mlp_loss_grad_bf16.restype = ctypes.c_double
    L.or_tree_leaf.argtypes = [vp, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, vp]
    L.or_tree_leaf.restype = ctypes.c_int


def _p(a):
    return ctypes.c_void_p(a.ctypes.data)


def _dims(vol):
    nz, ny, nx = vol.shape
    return np.array([nx, ny, nz], dtype=np.int64)


# ---------------------------------------------------------------- RNG
def philox(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().or_philox4x32_10(_p(c), _p(k), _p(out))
    return out


# ---------------------------------------------------------------- encoder
def background_bits(vol: np.ndarray) -> int:
    v = np.ascontiguousarray(vol, dtype=np.float32)
    return int(lib().or_background_bits(_p(v), v.size))


def brick_grid(dims):
    d = np.asarray(dims, dtype=np.int64)
    nb = np.zeros(3, dtype=np.int64)
    lib().or_brick_grid(_p(d), _p(nb))
    return nb


def brick_ranges(vol: np.ndarray):
    v = np.ascontiguousarray(vol, dtype=np.float32)
    d = _dims(v)
    nb = brick_grid(d)
    n = int(np.prod(nb))
    lo = np.zeros(n, dtype=np.uint32)
    hi = np.zeros(n, dtype=np.uint32)
    lib().or_brick_ranges(_p(v), _p(d), _p(lo), _p(hi))
    return lo, hi


def brick_scores(lo, hi, b_bits: int, metric: int = F2):
    n = lo.size
    f = np.zeros(n, dtype=np.float64)
    e = np.zeros(n, dtype=np.uint8)
    lib().or_brick_scores(_p(lo), _p(hi), n, b_bits, metric, _p(f), _p(e))
    return f, e


def brick_budget(nbricks: int, ratio: float, payload: int = FP32) -> int:
    return int(lib().or_brick_budget(nbricks, float(ratio), payload))


def select(f, empty, n_budget: int):
    a = np.zeros(f.size, dtype=np.uint8)
    take = lib().or_select(_p(f), _p(empty), f.size, int(n_budget), _p(a))
    return a, int(take)


def encode(vol: np.ndarray, ratio: float, metric: int = F2, payload: int = FP32) -> dict:
    """Algorithm 1 end to end: B, ranges, scores, budget, selection."""
    v = np.ascontiguousarray(vol, dtype=np.float32)
    b = background_bits(v)
    lo, hi = brick_ranges(v)
    f, empty = brick_scores(lo, hi, b, metric)
    n = brick_budget(lo.size, ratio, payload)
    active, take = select(f, empty, n)
    return dict(background_bits=b, lo=lo, hi=hi, f=f, empty=empty, budget=n, active=active,
                n_active=take, payload=payload, dims=_dims(v))


def decode_dense(vol: np.ndarray, active, b_bits: int, payload: int = FP32) -> np.ndarray:
    v = np.ascontiguousarray(vol, dtype=np.float32)
    out = np.empty_like(v)
    a = np.ascontiguousarray(active, dtype=np.uint8)
    lib().or_decode_dense(_p(v), _p(_dims(v)), _p(a), b_bits, payload, _p(out))
    return out


def round_fp16(x: float) -> float:
    return float(lib().or_round_fp16(x))


def round_e4m3(x: float) -> float:
    return float(lib().or_round_e4m3(x))


def quantize_leaf(leaf, payload):
    a = np.ascontiguousarray(leaf, dtype=np.float32).reshape(512)
    out = np.zeros(512, dtype=np.float32)
    s = ctypes.c_float()
    o = ctypes.c_float()
    lib().or_quantize_leaf(_p(a), payload, _p(out), ctypes.byref(s), ctypes.byref(o))
    return out, s.value, o.value


class Tree:
    """The oracle's 4-level tree; value(i,j,k) descends root -> upper -> lower -> leaf."""

    def __init__(self, vol, active, b_bits, payload=FP32):
        self._v = np.ascontiguousarray(vol, dtype=np.float32)
        a = np.ascontiguousarray(active, dtype=np.uint8)
        self.h = lib().or_tree_build(_p(self._v), _p(_dims(self._v)), _p(a), b_bits, payload)

    def value(self, i, j, k) -> float:
        return float(lib().or_tree_value(self.h, i, j, k))

    def leaf(self, li, lj, lk):
        """The 512 values of the leaf node at leaf position (li, lj, lk), or None for a tile."""
        out = np.zeros(512, dtype=np.float32)
        return out if lib().or_tree_leaf(self.h, li, lj, lk, _p(out)) else None

    def counts(self) -> dict:
        out = np.zeros(6, dtype=np.int64)
        lib().or_tree_counts(self.h, _p(out))
        return dict(root=int(out[0]), upper=int(out[1]), lower=int(out[2]), leaves=int(out[3]),
                    lower_tiles=int(out[4]), upper_tiles=int(out[5]))

    def close(self):
        if self.h:
            lib().or_tree_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------- renderer
def make_camera(kind, width, height, eye, look, up, fovy_or_height) -> Camera:
    c = Camera()
    c.kind, c.width, c.height = int(kind), int(width), int(height)
    for a in range(3):
        c.eye[a], c.look[a], c.up[a] = float(eye[a]), float(look[a]), float(up[a])
    c.fovy_or_height = float(fovy_or_height)
    return c


def make_medium(mode, tf=None, step=0.5, density_scale=1.0, albedo=0.9, g=0.0, max_bounces=1,
                macrocell=8, sun_dir=(0, 0, 1), sun_rad=(0, 0, 0), env_rad=(0, 0, 0), iso=0.5):
    m = Medium()
    m.mode = int(mode)
    keep = None
    if tf is not None:
        keep = np.ascontiguousarray(tf, dtype=np.float32).reshape(-1, 4)
        m.tf_n = keep.shape[0]
        m.tf_rgba = keep.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
    m.step, m.density_scale, m.albedo, m.g = float(step), float(density_scale), float(albedo), float(g)
    m.max_bounces, m.macrocell = int(max_bounces), int(macrocell)
    m.iso = float(iso)
    for a in range(3):
        m.sun_dir[a], m.sun_rad[a], m.env_rad[a] = float(sun_dir[a]), float(sun_rad[a]), float(env_rad[a])
    m._keep = keep
    return m


def trilinear(d: np.ndarray, p) -> float:
    pp = np.ascontiguousarray(p, dtype=np.float64)
    return float(lib().or_trilinear(_p(d), _p(_dims(d)), _p(pp)))


def macrocell_minmax(d: np.ndarray, cell: int = 8):
    dims = _dims(d)
    nc = (dims + cell - 1) // cell
    mn = np.zeros(int(np.prod(nc)), dtype=np.float32)
    mx = np.zeros_like(mn)
    lib().or_macrocell_minmax(_p(d), _p(dims), cell, _p(mn), _p(mx))
    return mn, mx


def dda_cells(dims, cell, o, d, tmin, tmax, cap=100000):
    dd = np.asarray(dims, dtype=np.int64)
    oo = np.ascontiguousarray(o, dtype=np.float64)
    di = np.ascontiguousarray(d, dtype=np.float64)
    cells = np.zeros(cap, dtype=np.int64)
    t0 = np.zeros(cap)
    t1 = np.zeros(cap)
    n = lib().or_dda_cells(_p(dd), cell, _p(oo), _p(di), tmin, tmax, _p(cells), _p(t0), _p(t1), cap)
    return cells[:n], t0[:n], t1[:n]


def clip_box(dims, o, d):
    dd = np.asarray(dims, dtype=np.int64)
    oo = np.ascontiguousarray(o, dtype=np.float64)
    di = np.ascontiguousarray(d, dtype=np.float64)
    tin = ctypes.c_double()
    tout = ctypes.c_double()
    hit = lib().or_clip_box(_p(dd), _p(oo), _p(di), ctypes.byref(tin), ctypes.byref(tout))
    return bool(hit), tin.value, tout.value


def scatter_dir(dirn, mu: float, phi: float) -> np.ndarray:
    """The direction after scattering from `dirn` at polar cosine mu and azimuth phi (radians)."""
    d = np.ascontiguousarray(dirn, dtype=np.float64)
    out = np.zeros(3)
    lib().or_scatter_dir(_p(d), float(mu), float(phi), _p(out))
    return out


def camera_ray(cam: Camera, dims, px, py, jx=0.5, jy=0.5):
    dd = np.asarray(dims, dtype=np.int64)
    o = np.zeros(3)
    d = np.zeros(3)
    lib().or_camera_ray(ctypes.byref(cam), _p(dd), px, py, jx, jy, _p(o), _p(d))
    return o, d


def ratio_transmittance(d, cell_max, medium, o, dirn, pixel, sample, seed):
    dims = _dims(d)
    oo = np.ascontiguousarray(o, dtype=np.float64)
    di = np.ascontiguousarray(dirn, dtype=np.float64)
    call = np.zeros(1, dtype=np.uint32)
    key = np.array([seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF], dtype=np.uint32)
    return float(lib().or_ratio_transmittance(_p(d), _p(dims), _p(cell_max), ctypes.byref(medium),
                                              _p(oo), _p(di), pixel, sample, _p(call), _p(key)))


def render_pixels(d: np.ndarray, cell_max, cam: Camera, medium: Medium, spp: int, seed: int,
                  pixels, threads: int = 1) -> np.ndarray:
    """RGBA (FP64) of the listed pixel ids (py * width + px); rows split over threads."""
    d = np.ascontiguousarray(d, dtype=np.float32)
    dims = _dims(d)
    cm = np.ascontiguousarray(cell_max if cell_max is not None else np.zeros(1), dtype=np.float32)
    pix = np.ascontiguousarray(pixels, dtype=np.int64)
    out = np.zeros((pix.size, 4), dtype=np.float64)
    L = lib()
    if threads <= 1 or pix.size < 2:
        L.or_render_pixels(_p(d), _p(dims), _p(cm), ctypes.byref(cam), ctypes.byref(medium), spp,
                           ctypes.c_uint64(seed), _p(pix), pix.size, _p(out))
        return out
    chunks = np.array_split(np.arange(pix.size), threads * 8)
    lock = threading.Lock()
    queue = list(chunks)

    def worker():
        while True:
            with lock:
                if not queue:
                    return
                c = queue.pop()
            if c.size == 0:
                continue
            sub = np.ascontiguousarray(pix[c])
            o = np.zeros((c.size, 4))
            L.or_render_pixels(_p(d), _p(dims), _p(cm), ctypes.byref(cam), ctypes.byref(medium),
                               spp, ctypes.c_uint64(seed), _p(sub), sub.size, _p(o))
            out[c] = o

    ts = [threading.Thread(target=worker) for _ in range(threads)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    return out


def render_image(d, cell_max, cam, medium, spp, seed, threads=1):
    pix = np.arange(cam.width * cam.height, dtype=np.int64)
    return render_pixels(d, cell_max, cam, medium, spp, seed, pix, threads).reshape(
        cam.height, cam.width, 4)


# ---------------------------------------------------------------- errors
def mse(a, b) -> float:
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.mean((a - b) ** 2))


def psnr(a, b) -> float:
    """PSNR with peak 1 (the convention that reproduces the paper's MSE/PSNR table)."""
    m = mse(a, b)
    return float("inf") if m == 0 else 10.0 * np.log10(1.0 / m)


# ---------------------------------------------------------------- learned leaf decoder
MLP_IN, MLP_HID, MLP_LATENT = 19, 32, 16


def mlp_num_params() -> int:
    return int(lib().or_mlp_num_params())


def mlp_forward(params, inputs) -> np.ndarray:
    p = np.ascontiguousarray(params, dtype=np.float64)
    x = np.ascontiguousarray(inputs, dtype=np.float64).reshape(-1, MLP_IN)
    out = np.zeros(x.shape[0])
    lib().or_mlp_forward(_p(p), _p(x), x.shape[0], _p(out))
    return out


def mlp_forward_bf16(params, inputs) -> np.ndarray:
    """The forward pass at the tensor-core path's precision (bf16 operands and activations)."""
    p = np.ascontiguousarray(params, dtype=np.float64)
    x = np.ascontiguousarray(inputs, dtype=np.float64).reshape(-1, MLP_IN)
    out = np.zeros(x.shape[0])
    lib().or_mlp_forward_bf16(_p(p), _p(x), x.shape[0], _p(out))
    return out


def round_bf16(x: float) -> float:
    return float(lib().or_round_bf16(x))


def mlp_loss_grad(params, inputs, targets):
    p = np.ascontiguousarray(params, dtype=np.float64)
    x = np.ascontiguousarray(inputs, dtype=np.float64).reshape(-1, MLP_IN)
    t = np.ascontiguousarray(targets, dtype=np.float64)
    gp = np.zeros_like(p)
    gx = np.zeros_like(x)
    loss = lib().or_mlp_loss_grad(_p(p), _p(x), _p(t), x.shape[0], _p(gp), _p(gx))
    return float(loss), gp, gx


def mlp_loss_grad_bf16(params, inputs, targets):
    """Loss and gradients at the tensor cores' precision (see or_mlp_loss_grad_bf16)."""
    p = np.ascontiguousarray(params, dtype=np.float64)
    x = np.ascontiguousarray(inputs, dtype=np.float64).reshape(-1, MLP_IN)
    t = np.ascontiguousarray(targets, dtype=np.float64)
    gp = np.zeros_like(p)
    gx = np.zeros_like(x)
    loss = lib().or_mlp_loss_grad_bf16(_p(p), _p(x), _p(t), x.shape[0], _p(gp), _p(gx))
    return float(loss), gp, gx


def adam_step(params, grads, m, v, step, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """In place on float64 arrays params, m, v."""
    g = np.ascontiguousarray(grads, dtype=np.float64)
    lib().or_adam_step(_p(params), _p(g), _p(m), _p(v), params.size, step, lr, beta1, beta2, eps)


def leaf_inputs(latent, n=None):
    """The 512 network inputs of one leaf (x fastest): (i, j, k) / 7 and the latent."""
    z = np.asarray(latent, dtype=np.float64).reshape(MLP_LATENT)
    idx = np.arange(512)
    uvw = np.stack([(idx & 7) / 7.0, ((idx >> 3) & 7) / 7.0, (idx >> 6) / 7.0], axis=1)
    return np.concatenate([uvw, np.broadcast_to(z, (512, MLP_LATENT))], axis=1)


def learned_leaf(params, latent, src):
    """Decoded values of a neural leaf whose source values are `src` (512)."""
    p = np.ascontiguousarray(params, dtype=np.float64)
    z = np.ascontiguousarray(latent, dtype=np.float32).reshape(MLP_LATENT)
    v = np.ascontiguousarray(src, dtype=np.float32).reshape(512)
    out = np.zeros(512, dtype=np.float32)
    lib().or_learned_leaf(_p(p), _p(z), _p(v), _p(out))
    return out


def learned_decode(vol, active, b_bits, params, latents, force):
    """Dense decode of the learned grid built from the FP32 grid of
    (vol, active, b_bits): the leaf at position p = (lk*nly + lj)*nlx + li is
    neural when force[p] == 1 (latent latents[p]), raw FP16 when force[p] == 2;
    tiles and the background as in the FP32 grid.  Returns (dense, kinds)
    with kinds[p] = 0 tile, 1 neural, 2 raw."""
    v = np.ascontiguousarray(vol, dtype=np.float32)
    nz, ny, nx = v.shape
    nl = ((nx + 7) // 8, (ny + 7) // 8, (nz + 7) // 8)
    out = decode_dense(v, active, b_bits, FP32)
    tree = Tree(v, active, b_bits, FP32)
    kinds = np.zeros(nl[0] * nl[1] * nl[2], dtype=np.uint8)
    lat = np.asarray(latents, dtype=np.float32).reshape(-1, MLP_LATENT)
    for lk in range(nl[2]):
        for lj in range(nl[1]):
            for li in range(nl[0]):
                pidx = (lk * nl[1] + lj) * nl[0] + li
                src = tree.leaf(li, lj, lk)
                if src is None:
                    continue
                if force[pidx] == 2:
                    dec, _, _ = quantize_leaf(src, FP16)
                    kinds[pidx] = 2
                elif force[pidx] == 1:
                    dec = learned_leaf(params, lat[pidx], src)
                    kinds[pidx] = 1
                else:
                    raise ValueError("learned_decode needs force 1 or 2 at every leaf")
                blk = dec.reshape(8, 8, 8)
                z0, y0, x0 = lk * 8, lj * 8, li * 8
                ez, ey, ex = min(8, nz - z0), min(8, ny - y0), min(8, nx - x0)
                out[z0:z0 + ez, y0:y0 + ey, x0:x0 + ex] = blk[:ez, :ey, :ex]
    tree.close()
    return out, kinds
