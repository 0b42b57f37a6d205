"""ctypes wrapper of the GPU input generators (synth.cu); torch tensors in,
torch tensors out.  Input generation only."""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

from . import _ZipfRI, gaussian_mixture_params

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "synth.cu")
LIB = os.path.join(HERE, "_lib", "libsynth.so")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + ".tmp"
        subprocess.check_call([NVCC, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17",
                               "-Xcompiler", "-fPIC", "-shared", SRC, "-o", tmp])
        os.replace(tmp, LIB)
    return LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB):
                raise ImportError("libsynth.so not built; call synth.gpu.build()")
            L = ctypes.CDLL(LIB)
            vp, u64, i32, d = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int, ctypes.c_double
            L.synth_iota_u64.argtypes = [vp, u64, u64, vp]
            L.synth_iota_u32.argtypes = [vp, u64, u64, vp]
            L.synth_uniform_mod.argtypes = [vp, u64, u64, u64, u64, vp]
            L.synth_uniform_exact.argtypes = [vp, u64, u64, u64, u64, u64, vp]
            L.synth_zipf.argtypes = [vp, u64, u64, u64, d, u64, d, d, d, i32, vp]
            L.synth_exponential.argtypes = [vp, u64, u64, u64, d, vp]
            L.synth_gaussian_mixture.argtypes = [vp, u64, u64, u64, vp, vp, vp, i32, vp]
            L.synth_rmat.argtypes = [vp, vp, u64, u64, u64, i32, d, d, d, vp]
            _lib = L
    return _lib


def _s():
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


def _chk(rc):
    if rc != 0:
        raise RuntimeError(f"synth kernel launch failed: cuda error {rc}")


def _empty(n, dtype=None, out=None):
    import torch
    return out if out is not None else torch.empty(n, dtype=dtype or torch.uint64, device="cuda")


def iota(n, start=0, dtype=None, out=None):
    import torch
    dtype = dtype or torch.uint64
    o = _empty(n, dtype, out)
    f = _load().synth_iota_u64 if dtype == torch.uint64 else _load().synth_iota_u32
    _chk(f(_p(o), n, start, _s()))
    return o


def uniform_mod(seed, n, mu, start=0, out=None):
    o = _empty(n, out=out)
    _chk(_load().synth_uniform_mod(_p(o), n, start, seed, mu, _s()))
    return o


def uniform_exact(seed, n, mu, start=0, count=None, out=None):
    count = n - start if count is None else count
    o = _empty(count, out=out)
    _chk(_load().synth_uniform_exact(_p(o), count, start, n, mu, seed, _s()))
    return o


def zipf(seed, n, s, N=10**9, start=0, out=None, ranks_only=False):
    z = _ZipfRI(s, N)
    o = _empty(n, out=out)
    _chk(_load().synth_zipf(_p(o), n, start, seed, float(s), int(N), float(z.h_x1), float(z.h_n), float(z.sq),
                            int(ranks_only), _s()))
    return o


def exponential(seed, n, lam, start=0, out=None):
    o = _empty(n, out=out)
    _chk(_load().synth_exponential(_p(o), n, start, seed, float(lam), _s()))
    return o


def gaussian_mixture(seed, n, k=8, start=0, out=None):
    import numpy as np
    means, sigmas, w = gaussian_mixture_params(seed, k)
    cw = np.ascontiguousarray(np.cumsum(w), dtype=np.float64)
    means = np.ascontiguousarray(means, dtype=np.float64)
    sigmas = np.ascontiguousarray(sigmas, dtype=np.float64)
    o = _empty(n, out=out)
    _chk(_load().synth_gaussian_mixture(_p(o), n, start, seed, cw.ctypes.data_as(ctypes.c_void_p),
                                        means.ctypes.data_as(ctypes.c_void_p),
                                        sigmas.ctypes.data_as(ctypes.c_void_p), k, _s()))
    return o


def rmat_edges(seed, m, scale, abcd=(0.57, 0.19, 0.19, 0.05), start=0):
    import torch
    src = torch.empty(m, dtype=torch.uint32, device="cuda")
    dst = torch.empty(m, dtype=torch.uint32, device="cuda")
    a, b, c, _ = abcd
    _chk(_load().synth_rmat(_p(src), _p(dst), m, start, seed, scale, a, b, c, _s()))
    return src, dst
