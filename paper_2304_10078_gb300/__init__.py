"""Python binding of the GB300 semisort library (libsemisort.so).

Argument marshalling only: every step of semisort / collect-reduce /
histogram runs in the CUDA kernels behind the C ABI declared in
``include/semisort.h``.  PyTorch provides device memory and streams.  There is
no CPU fallback: if the compiled library is missing, every call raises.

Key dtypes: ``torch.uint32``, ``torch.uint64``, or 128-bit keys as a
``(n, 2)`` ``torch.uint64`` tensor (lo, hi).  Value dtypes: ``torch.uint32``,
``torch.uint64``.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libsemisort.so")

SS_U32, SS_U64, SS_U128 = 0, 1, 2
OP_EQUAL, OP_LESS, OP_REDUCE, OP_HIST = 0, 1, 2, 3
FLAG_PHASE_TIMING = 0x1
FLAG_IDENTITY_HASH = 0x2
FLAG_HASH_BUCKETS = 0x4
FLAG_SWAP_OUTPUT = 0x8

STATUS = {
    0: "ok", 1: "invalid argument", 2: "unsupported type or size", 3: "workspace too small",
    4: "capacity exceeded", 5: "not enough device memory", 6: "device wait timed out",
    7: "CUDA runtime error", 8: "recursion depth limit reached",
}

STAT_NAMES = ["levels", "dist_l0", "dist_l1", "dist_l2", "dist_l3", "refined", "copied",
              "heavy_l0", "max_refine", "refine_items", "all_distinct", "l0_splitters", "l0_max_sample_range",
              "l0_max_light_bucket", "l0_light_buckets", "learn_steps"]


class SemisortError(RuntimeError):
    def __init__(self, code: int, where: str):
        super().__init__(f"{where}: {STATUS.get(code, code)} (status {code})")
        self.code = code


class Options(ctypes.Structure):
    _fields_ = [("seed", ctypes.c_uint64), ("subarray", ctypes.c_uint32), ("n_light_log2", ctypes.c_uint32),
                ("alpha", ctypes.c_uint32), ("sample_size", ctypes.c_uint32), ("splitter_mode", ctypes.c_int32),
                ("flags", ctypes.c_int32)]


_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    from . import _build
    return _build.build(force=force)


def lib():
    """The loaded C library; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise ImportError(f"libsemisort.so not built ({LIB_PATH}); call paper_2304_10078_gb300.build()")
            L = ctypes.CDLL(LIB_PATH)
            vp, u64, i32, sz = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int, ctypes.c_size_t
            L.ss_workspace_size.argtypes = [i32, i32, i32, u64, vp, ctypes.POINTER(sz)]
            L.ss_workspace_size.restype = i32
            for name in ("semisort_equal", "semisort_less"):
                f = getattr(L, name)
                f.argtypes = [i32, i32, vp, vp, vp, vp, u64, vp, sz, vp, vp]
                f.restype = i32
            L.semisort_equal_noalloc.argtypes = [i32, i32, vp, vp, vp, vp, u64, vp, vp]
            L.semisort_equal_noalloc.restype = i32
            L.ss_mlp_workspace_size.argtypes = []
            L.ss_mlp_workspace_size.restype = sz
            L.ss_mlp_loss_grad.argtypes = [vp, vp, vp, ctypes.c_uint32, vp, vp, sz, vp]
            L.ss_mlp_loss_grad.restype = i32
            L.ss_mlp_train.argtypes = [vp, vp, ctypes.c_uint32, vp, ctypes.c_uint32, ctypes.c_float, vp, vp, vp, sz,
                                       vp]
            L.ss_mlp_train.restype = i32
            L.ss_mlp_invert.argtypes = [vp, i32, u64, u64, ctypes.c_uint32, vp, vp, sz, vp]
            L.ss_mlp_invert.restype = i32
            L.ss_workspace_size_batched.argtypes = [i32, i32, i32, u64, ctypes.c_uint32, vp, ctypes.POINTER(sz)]
            L.ss_workspace_size_batched.restype = i32
            for name in ("semisort_equal_batched", "semisort_less_batched"):
                f = getattr(L, name)
                f.argtypes = [i32, i32, vp, vp, vp, vp, vp, ctypes.c_uint32, u64, vp, sz, vp, vp]
                f.restype = i32
            L.collect_reduce_batched.argtypes = [i32, vp, vp, vp, ctypes.c_uint32, u64, vp, vp, u64, vp, vp, vp, sz,
                                                 vp, vp]
            L.collect_reduce_batched.restype = i32
            L.histogram_batched.argtypes = [i32, vp, vp, ctypes.c_uint32, u64, vp, vp, u64, vp, vp, vp, sz, vp, vp]
            L.histogram_batched.restype = i32
            L.collect_reduce.argtypes = [i32, vp, vp, vp, vp, u64, vp, u64, vp, sz, vp, vp]
            L.collect_reduce.restype = i32
            L.histogram.argtypes = [i32, vp, vp, vp, u64, vp, u64, vp, sz, vp, vp]
            L.histogram.restype = i32
            L.ss_last_device_error.argtypes = [vp, vp, ctypes.POINTER(i32)]
            L.ss_last_device_error.restype = i32
            L.ss_get_stats.argtypes = [vp, vp, ctypes.POINTER(u64), i32]
            L.ss_get_stats.restype = i32
            L.ss_phase_times.argtypes = [ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_char_p), i32]
            L.ss_phase_times.restype = i32
            L.ss_status_string.argtypes = [i32]
            L.ss_status_string.restype = ctypes.c_char_p
            L.ss_kernel_launches.argtypes = []
            L.ss_kernel_launches.restype = i32
            L.ss_hash_u64.argtypes = [vp, vp, u64, u64, vp]
            L.ss_hash_u64.restype = i32
            _lib = L
    return _lib


def _torch():
    import torch
    return torch


def key_code(t) -> int:
    torch = _torch()
    if t.dim() == 2:
        if t.dtype != torch.uint64 or t.shape[1] != 2:
            raise TypeError("128-bit keys must be an (n, 2) uint64 tensor")
        return SS_U128
    if t.dtype == torch.uint32:
        return SS_U32
    if t.dtype == torch.uint64:
        return SS_U64
    raise TypeError(f"unsupported key dtype {t.dtype}")


def val_code(t) -> int:
    torch = _torch()
    if t is None or t.dtype == torch.uint64:
        return SS_U64
    if t.dtype == torch.uint32:
        return SS_U32
    raise TypeError(f"unsupported value dtype {t.dtype}")


def make_options(seed=0, subarray=0, n_light_log2=0, alpha=0, sample_size=0, splitter_mode=0, flags=0) -> Options:
    return Options(seed, subarray, n_light_log2, alpha, sample_size, splitter_mode, flags)


def _opt_ptr(opt):
    return None if opt is None else ctypes.cast(ctypes.pointer(opt), ctypes.c_void_p)


def _stream(stream):
    torch = _torch()
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _check(code: int, where: str):
    if code != 0:
        raise SemisortError(code, where)


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def workspace_size(op: int, kcode: int, vcode: int, n: int, options: Options | None = None) -> int:
    out = ctypes.c_size_t(0)
    _check(lib().ss_workspace_size(op, kcode, vcode, n, _opt_ptr(options), ctypes.byref(out)), "ss_workspace_size")
    return out.value


def alloc_workspace(op: int, keys, vals=None, options: Options | None = None, device=None):
    torch = _torch()
    nbytes = workspace_size(op, key_code(keys), val_code(vals), keys.shape[0], options)
    return torch.empty(max(nbytes, 256), dtype=torch.uint8, device=device or keys.device)


def _semisort(fn, op, keys, vals, keys_out, vals_out, workspace, options, stream):
    torch = _torch()
    n = keys.shape[0]
    if keys_out is None:
        keys_out = torch.empty_like(keys)
    if vals is not None and vals_out is None:
        vals_out = torch.empty_like(vals)
    if workspace is None:
        workspace = alloc_workspace(op, keys, vals, options)
    code = fn(key_code(keys), val_code(vals), _ptr(keys), _ptr(vals), _ptr(keys_out), _ptr(vals_out), n,
              _ptr(workspace), workspace.numel(), _opt_ptr(options), _stream(stream))
    _check(code, fn.__name__)
    return keys_out, vals_out


def semisort_equal(keys, vals=None, keys_out=None, vals_out=None, workspace=None, options=None, stream=None):
    """semisort_=: records with equal keys become contiguous, stable."""
    return _semisort(lib().semisort_equal, OP_EQUAL, keys, vals, keys_out, vals_out, workspace, options, stream)


def semisort_equal_noalloc(keys, vals, keys_out, vals_out, options=None, stream=None):
    """semisort_= on at most 2^18 records with the library's static scratch
    array (no workspace, nothing allocated); outputs are caller tensors."""
    code = lib().semisort_equal_noalloc(key_code(keys), val_code(vals), _ptr(keys), _ptr(vals), _ptr(keys_out),
                                        _ptr(vals_out), keys.shape[0], _opt_ptr(options), _stream(stream))
    _check(code, "semisort_equal_noalloc")
    return keys_out, vals_out


def semisort_less(keys, vals=None, keys_out=None, vals_out=None, workspace=None, options=None, stream=None):
    """semisort_< (range partitioned): the stable sort by key."""
    return _semisort(lib().semisort_less, OP_LESS, keys, vals, keys_out, vals_out, workspace, options, stream)


def collect_reduce(keys, vals, capacity=None, ukeys_out=None, sums_out=None, num_unique=None, workspace=None,
                   options=None, stream=None):
    """(unique keys, u64 wraparound sums) -- returns (ukeys, sums, d_num_unique)."""
    torch = _torch()
    n = keys.shape[0]
    cap = n if capacity is None else capacity
    if ukeys_out is None:
        ukeys_out = torch.empty((cap,) + tuple(keys.shape[1:]), dtype=keys.dtype, device=keys.device)
    if sums_out is None:
        sums_out = torch.empty(cap, dtype=torch.uint64, device=keys.device)
    if num_unique is None:
        num_unique = torch.zeros(1, dtype=torch.uint64, device=keys.device)
    if workspace is None:
        workspace = alloc_workspace(OP_REDUCE, keys, vals, options)
    code = lib().collect_reduce(key_code(keys), _ptr(keys), _ptr(vals), _ptr(ukeys_out), _ptr(sums_out), cap,
                                _ptr(num_unique), n, _ptr(workspace), workspace.numel(), _opt_ptr(options),
                                _stream(stream))
    _check(code, "collect_reduce")
    return ukeys_out, sums_out, num_unique


def histogram(keys, capacity=None, ukeys_out=None, counts_out=None, num_unique=None, workspace=None, options=None,
              stream=None):
    """(unique keys, u32 counts) -- returns (ukeys, counts, d_num_unique)."""
    torch = _torch()
    n = keys.shape[0]
    cap = n if capacity is None else capacity
    if ukeys_out is None:
        ukeys_out = torch.empty((cap,) + tuple(keys.shape[1:]), dtype=keys.dtype, device=keys.device)
    if counts_out is None:
        counts_out = torch.empty(cap, dtype=torch.uint32, device=keys.device)
    if num_unique is None:
        num_unique = torch.zeros(1, dtype=torch.uint64, device=keys.device)
    if workspace is None:
        workspace = alloc_workspace(OP_HIST, keys, None, options)
    code = lib().histogram(key_code(keys), _ptr(keys), _ptr(ukeys_out), _ptr(counts_out), cap, _ptr(num_unique), n,
                           _ptr(workspace), workspace.numel(), _opt_ptr(options), _stream(stream))
    _check(code, "histogram")
    return ukeys_out, counts_out, num_unique


def last_device_error(workspace, stream=None) -> int:
    code = ctypes.c_int(0)
    _check(lib().ss_last_device_error(_ptr(workspace), _stream(stream), ctypes.byref(code)), "ss_last_device_error")
    return code.value


def stats(workspace, stream=None) -> dict:
    buf = (ctypes.c_uint64 * len(STAT_NAMES))()
    m = lib().ss_get_stats(_ptr(workspace), _stream(stream), buf, len(STAT_NAMES))
    return {STAT_NAMES[i]: int(buf[i]) for i in range(m)}


def phase_times() -> list[tuple[str, float]]:
    ms = (ctypes.c_float * 64)()
    names = (ctypes.c_char_p * 64)()
    m = lib().ss_phase_times(ms, names, 64)
    return [(names[i].decode(), float(ms[i])) for i in range(m)]


def kernel_launches() -> int:
    """Kernels enqueued by the most recent library call on this thread."""
    return int(lib().ss_kernel_launches())


def hash_u64(keys, salt: int, stream=None):
    torch = _torch()
    out = torch.empty_like(keys)
    _check(lib().ss_hash_u64(_ptr(keys), _ptr(out), keys.numel(), salt & 0xFFFFFFFFFFFFFFFF, _stream(stream)),
           "ss_hash_u64")
    return out


MLP_PARAMS = 1153


def _mlp_ws(device):
    torch = _torch()
    return torch.empty(int(lib().ss_mlp_workspace_size()), dtype=torch.uint8, device=device)


def mlp_loss_grad(params, x, t, stream=None):
    """(loss, gradient) of the learned-splitter model on points (x, t); float32 device tensors."""
    torch = _torch()
    out = torch.empty(MLP_PARAMS + 1, dtype=torch.float32, device=params.device)
    ws = _mlp_ws(params.device)
    _check(lib().ss_mlp_loss_grad(_ptr(params), _ptr(x), _ptr(t), x.numel(), _ptr(out), _ptr(ws), ws.numel(),
                                  _stream(stream)), "ss_mlp_loss_grad")
    return out[MLP_PARAMS], out[:MLP_PARAMS]


def mlp_train(x, t, params0, steps, lr, stream=None):
    """Trained parameters and the loss at them (float32 device tensors)."""
    torch = _torch()
    p = torch.empty(MLP_PARAMS, dtype=torch.float32, device=params0.device)
    loss = torch.empty(1, dtype=torch.float32, device=params0.device)
    ws = _mlp_ws(params0.device)
    _check(lib().ss_mlp_train(_ptr(x), _ptr(t), x.numel(), _ptr(params0), steps, float(lr), _ptr(p), _ptr(loss),
                              _ptr(ws), ws.numel(), _stream(stream)), "ss_mlp_train")
    return p, loss


def mlp_invert(params, key_type, kmin, kmax, n_light_log2, stream=None):
    """The 2^n_light_log2 - 1 integer splitters of the model over [kmin, kmax]."""
    torch = _torch()
    nl = 1 << n_light_log2
    out = torch.empty(nl - 1, dtype=torch.uint32 if key_type == SS_U32 else torch.uint64, device=params.device)
    ws = _mlp_ws(params.device)
    _check(lib().ss_mlp_invert(_ptr(params), key_type, kmin, kmax, n_light_log2, _ptr(out), _ptr(ws), ws.numel(),
                               _stream(stream)), "ss_mlp_invert")
    return out


def workspace_size_batched(op: int, kcode: int, vcode: int, n: int, num_instances: int,
                           options: Options | None = None) -> int:
    out = ctypes.c_size_t(0)
    _check(lib().ss_workspace_size_batched(op, kcode, vcode, n, num_instances, _opt_ptr(options), ctypes.byref(out)),
           "ss_workspace_size_batched")
    return out.value


def alloc_workspace_batched(op: int, keys, offsets, vals=None, options: Options | None = None):
    torch = _torch()
    nbytes = workspace_size_batched(op, key_code(keys), val_code(vals), keys.shape[0], offsets.numel() - 1, options)
    return torch.empty(max(nbytes, 256), dtype=torch.uint8, device=keys.device)


def _semisort_batched(fn, op, keys, vals, offsets, keys_out, vals_out, workspace, options, stream):
    torch = _torch()
    if keys_out is None:
        keys_out = torch.empty_like(keys)
    if vals is not None and vals_out is None:
        vals_out = torch.empty_like(vals)
    if workspace is None:
        workspace = alloc_workspace_batched(op, keys, offsets, vals, options)
    code = fn(key_code(keys), val_code(vals), _ptr(keys), _ptr(vals), _ptr(keys_out), _ptr(vals_out), _ptr(offsets),
              offsets.numel() - 1, keys.shape[0], _ptr(workspace), workspace.numel(), _opt_ptr(options),
              _stream(stream))
    _check(code, fn.__name__)
    return keys_out, vals_out


def semisort_equal_batched(keys, vals, offsets, keys_out=None, vals_out=None, workspace=None, options=None,
                           stream=None):
    """semisort_= of every instance [offsets[i], offsets[i+1]) (offsets: uint64 device tensor)."""
    return _semisort_batched(lib().semisort_equal_batched, OP_EQUAL, keys, vals, offsets, keys_out, vals_out,
                             workspace, options, stream)


def semisort_less_batched(keys, vals, offsets, keys_out=None, vals_out=None, workspace=None, options=None,
                          stream=None):
    """semisort_< (stable sort) of every instance."""
    return _semisort_batched(lib().semisort_less_batched, OP_LESS, keys, vals, offsets, keys_out, vals_out,
                             workspace, options, stream)


def collect_reduce_batched(keys, vals, offsets, capacity=None, ukeys_out=None, sums_out=None, num_unique=None,
                           out_offsets=None, workspace=None, options=None, stream=None):
    """Per-instance (unique keys, sums): returns (ukeys, sums, num_unique[I], out_offsets[I+1])."""
    torch = _torch()
    n = keys.shape[0]
    ni = offsets.numel() - 1
    cap = n if capacity is None else capacity
    dev = keys.device
    ukeys_out = torch.empty((cap,) + tuple(keys.shape[1:]), dtype=keys.dtype, device=dev) if ukeys_out is None \
        else ukeys_out
    sums_out = torch.empty(cap, dtype=torch.uint64, device=dev) if sums_out is None else sums_out
    num_unique = torch.zeros(ni, dtype=torch.uint64, device=dev) if num_unique is None else num_unique
    out_offsets = torch.zeros(ni + 1, dtype=torch.uint64, device=dev) if out_offsets is None else out_offsets
    if workspace is None:
        workspace = alloc_workspace_batched(OP_REDUCE, keys, offsets, vals, options)
    code = lib().collect_reduce_batched(key_code(keys), _ptr(keys), _ptr(vals), _ptr(offsets), ni, n,
                                        _ptr(ukeys_out), _ptr(sums_out), cap, _ptr(num_unique), _ptr(out_offsets),
                                        _ptr(workspace), workspace.numel(), _opt_ptr(options), _stream(stream))
    _check(code, "collect_reduce_batched")
    return ukeys_out, sums_out, num_unique, out_offsets


def histogram_batched(keys, offsets, capacity=None, ukeys_out=None, counts_out=None, num_unique=None,
                      out_offsets=None, workspace=None, options=None, stream=None):
    """Per-instance (unique keys, counts): returns (ukeys, counts, num_unique[I], out_offsets[I+1])."""
    torch = _torch()
    n = keys.shape[0]
    ni = offsets.numel() - 1
    cap = n if capacity is None else capacity
    dev = keys.device
    ukeys_out = torch.empty((cap,) + tuple(keys.shape[1:]), dtype=keys.dtype, device=dev) if ukeys_out is None \
        else ukeys_out
    counts_out = torch.empty(cap, dtype=torch.uint32, device=dev) if counts_out is None else counts_out
    num_unique = torch.zeros(ni, dtype=torch.uint64, device=dev) if num_unique is None else num_unique
    out_offsets = torch.zeros(ni + 1, dtype=torch.uint64, device=dev) if out_offsets is None else out_offsets
    if workspace is None:
        workspace = alloc_workspace_batched(OP_HIST, keys, offsets, None, options)
    code = lib().histogram_batched(key_code(keys), _ptr(keys), _ptr(offsets), ni, n, _ptr(ukeys_out),
                                   _ptr(counts_out), cap, _ptr(num_unique), _ptr(out_offsets), _ptr(workspace),
                                   workspace.numel(), _opt_ptr(options), _stream(stream))
    _check(code, "histogram_batched")
    return ukeys_out, counts_out, num_unique, out_offsets

