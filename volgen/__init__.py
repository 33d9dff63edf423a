"""Seeded synthetic volumes shaped like the paper's workloads (inputs only).

The generator holds none of the method's arithmetic.  One C source
(``volgen.h``) is compiled for the host (gcc) and for the device (nvcc with
``--fmad=false``); both produce the same bytes, so the oracle and the CUDA path
read identical inputs.  Random parameters (blob centres, sizes, amplitudes)
are drawn here with numpy's PCG64 from the seed.

Workloads (x-fastest float32 volumes):

* ``blobs``       8 Gaussian blobs (sigma 4-12 voxels at 64^3, amplitude
                  0.5-1) plus 0.35 x 4-octave value-noise fBm (period 16 at
                  64^3), clamped to [0,1], a bias subtracted so that ~70 % of
                  the voxels fall below 0.01, those set to exactly 0;
* ``turbulence``  6-octave fBm x spherical falloff, ~50 % exactly 0;
* ``cloud``       Worley-modulated 8-octave fBm with an anvil height
                  profile, ~60 % exactly 0 (the WDAS-shaped cloud);
* ``noise``       dense noise in (0,1] (the paper's lossless worst case).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
HOST_LIB = os.path.join(_BUILD, "libvolgen_host.so")
DEV_LIB = os.path.join(_BUILD, "libvolgen_dev.so")

KINDS = {"blobs": 0, "turbulence": 1, "cloud": 2, "noise": 3}
MAX_BLOBS = 16


class VgParams(ctypes.Structure):
    _fields_ = [
        ("kind", ctypes.c_int32),
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
        ("seed", ctypes.c_uint32),
        ("octaves", ctypes.c_int32),
        ("period", ctypes.c_float),
        ("noise_amp", ctypes.c_float),
        ("bias", ctypes.c_float),
        ("zero_below", ctypes.c_float),
        ("worley_period", ctypes.c_float),
        ("nblobs", ctypes.c_int32),
        ("blob_c", (ctypes.c_float * 3) * MAX_BLOBS),
        ("blob_s", ctypes.c_float * MAX_BLOBS),
        ("blob_a", ctypes.c_float * MAX_BLOBS),
    ]


def build(verbose: bool = False) -> None:
    """Compile the host library (gcc) and, when nvcc is present, the device one."""
    os.makedirs(_BUILD, exist_ok=True)
    src_h = os.path.join(_HERE, "volgen.h")
    jobs = []
    host_src = os.path.join(_HERE, "volgen_host.c")
    if _stale(HOST_LIB, [host_src, src_h]):
        jobs.append(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
                     "-shared", host_src, "-o", HOST_LIB, "-lm"])
    dev_src = os.path.join(_HERE, "volgen_dev.cu")
    if _have_nvcc() and _stale(DEV_LIB, [dev_src, src_h]):
        jobs.append(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "--fmad=false",
                     "-prec-div=true", "-prec-sqrt=true", "-shared", "-Xcompiler", "-fPIC",
                     "-Xcompiler", "-ffp-contract=off", dev_src, "-o", DEV_LIB])
    procs = [subprocess.Popen(j, stdout=subprocess.PIPE, stderr=subprocess.STDOUT) for j in jobs]
    for j, p in zip(jobs, procs):
        out, _ = p.communicate()
        if p.returncode != 0:
            raise RuntimeError("volgen build failed: %s\n%s" % (" ".join(j), out.decode()))
        if verbose and out:
            print(out.decode())


def _have_nvcc() -> bool:
    from shutil import which
    return which("nvcc") is not None


def _stale(target: str, sources) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(s) > t for s in sources)


_host = None
_dev = None


def _host_lib():
    global _host
    if _host is None:
        if not os.path.exists(HOST_LIB):
            build()
        _host = ctypes.CDLL(HOST_LIB)
        _host.vg_fill_host.argtypes = [ctypes.POINTER(VgParams), ctypes.c_int32, ctypes.c_int32,
                                       ctypes.c_void_p]
        _host.vg_fill_host.restype = None
        assert _host.vg_params_size() == ctypes.sizeof(VgParams)
    return _host


def _dev_lib():
    global _dev
    if _dev is None:
        if not os.path.exists(DEV_LIB):
            build()
        _dev = ctypes.CDLL(DEV_LIB)
        _dev.vg_fill_device.argtypes = [ctypes.POINTER(VgParams), ctypes.c_void_p, ctypes.c_void_p]
        _dev.vg_fill_device.restype = ctypes.c_int
        assert _dev.vg_params_size_device() == ctypes.sizeof(VgParams)
    return _dev


def make_params(kind: str, dims, seed: int = 0) -> VgParams:
    """Parameters of a workload; dims = (nx, ny, nz)."""
    nx, ny, nz = (int(d) for d in dims)
    p = VgParams()
    p.kind = KINDS[kind]
    p.nx, p.ny, p.nz = nx, ny, nz
    p.seed = int(seed) & 0xFFFFFFFF
    p.zero_below = 0.01
    rng = np.random.default_rng(int(seed))
    m = float(min(nx, ny, nz))
    if kind == "blobs":
        s = m / 64.0
        p.octaves, p.period, p.noise_amp = 4, 16.0 * s, 0.35
        p.bias = 0.245
        p.nblobs = 8
        for b in range(8):
            for a, n in enumerate((nx, ny, nz)):
                p.blob_c[b][a] = float(rng.uniform(n / 8.0, 7.0 * n / 8.0))
            p.blob_s[b] = float(rng.uniform(4.0, 12.0) * s)
            p.blob_a[b] = float(rng.uniform(0.5, 1.0))
    elif kind == "turbulence":
        p.octaves, p.period = 6, m / 4.0
        p.bias = 0.0
    elif kind == "cloud":
        p.octaves, p.period = 8, m / 3.0
        p.worley_period = m / 6.0
        p.bias = 0.0
    elif kind == "noise":
        p.zero_below = -1.0
    else:
        raise ValueError(kind)
    return p


def generate_host(params: VgParams, threads: int | None = None) -> np.ndarray:
    """The volume as a (nz, ny, nx) float32 array, z slabs filled in parallel."""
    lib = _host_lib()
    out = np.empty((params.nz, params.ny, params.nx), dtype=np.float32)
    nthreads = max(1, min(threads or os.cpu_count() or 1, params.nz))
    bounds = np.linspace(0, params.nz, nthreads + 1).astype(int)
    ptr = out.ctypes.data_as(ctypes.c_void_p)

    def run(z0, z1):
        lib.vg_fill_host(ctypes.byref(params), int(z0), int(z1), ptr)

    ts = [threading.Thread(target=run, args=(bounds[i], bounds[i + 1])) for i in range(nthreads)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    return out


def generate_device(params: VgParams, out_ptr: int, stream: int = 0) -> None:
    """Fill a device buffer of nx*ny*nz float32 (x fastest) on `stream`."""
    rc = _dev_lib().vg_fill_device(ctypes.byref(params), ctypes.c_void_p(out_ptr),
                                   ctypes.c_void_p(stream))
    if rc != 0:
        raise RuntimeError("vg_fill_device failed with cudaError %d" % rc)


def generate_torch(params: VgParams, device="cuda"):
    """Convenience: a torch tensor (nz, ny, nx) on `device` filled by the device generator."""
    import torch
    t = torch.empty((params.nz, params.ny, params.nx), dtype=torch.float32, device=device)
    generate_device(params, t.data_ptr(), torch.cuda.current_stream(t.device).cuda_stream)
    return t
