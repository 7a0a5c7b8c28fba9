"""Thin ctypes binding of libcmg.so (include/cmg.h): the same function names,
argument marshalling only.  Every computation runs in the library's CUDA
kernels; if the library or a GPU is missing the calls raise, there is no CPU
path.

Array arguments may be NumPy arrays (passed as CMG_MEM_HOST) or CUDA torch
tensors (passed as CMG_MEM_DEVICE, read/written on the context's stream).
Outputs are NumPy arrays unless ``device=True`` (CUDA torch tensors) or an
``out`` array is given.
"""
import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libcmg.so")

CMG_OK = 0
CMG_ERR_INVALID_ARG = -1
CMG_ERR_DUPLICATE_KEY = -2
CMG_ERR_KEY_OUT_OF_RANGE = -3
CMG_ERR_MISSING_PARENT = -4
CMG_ERR_OOM = -5
CMG_ERR_CUDA = -6
CMG_ERR_NOT_CONVERGED = -7
CMG_ERR_DIVERGED = -8
CMG_ERR_TIMEOUT = -9

CMG_MEM_HOST = 0
CMG_MEM_DEVICE = 1
CMG_PREC_FP64 = 0
CMG_PREC_MIXED = 1
CMG_PREC_FFT = 2
CMG_FIELD_PHI = 0
CMG_FIELD_F = 1
CMG_OP_SWEEP, CMG_OP_RESIDUAL, CMG_OP_RESTRICT, CMG_OP_PROLONG, CMG_OP_COARSE, CMG_OP_GHOSTS = range(6)
CMG_OPR_SWEEP, CMG_OPR_RESIDUAL, CMG_OPR_RESTRICT, CMG_OPR_PROLONG, CMG_OPR_SUM_PHI, CMG_OPR_SHIFT_PHI = range(6)


class cmg_solve_params(C.Structure):
    _fields_ = [("tol", C.c_double), ("max_cycles", C.c_int), ("n_pre", C.c_int), ("n_post", C.c_int),
                ("coarse_sweeps", C.c_int), ("fixed_cycles", C.c_int), ("precision", C.c_int),
                ("inner_cycles", C.c_int), ("krylov", C.c_int)]


class cmg_solve_stats(C.Structure):
    _fields_ = [("cycles", C.c_int), ("status", C.c_int), ("rel_initial", C.c_double), ("rel_final", C.c_double),
                ("norm0", C.c_double), ("ms", C.c_double), ("cell_updates", C.c_int64),
                ("rel_history", C.c_double * 256)]


class cmg_kernel_profile(C.Structure):
    _fields_ = [("name", C.c_char * 32), ("launches", C.c_int64), ("ms", C.c_double), ("bytes", C.c_double),
                ("flops", C.c_double)]


class cmg_batch_schedule(C.Structure):
    _fields_ = [("threads", C.c_int), ("blocks_per_sm", C.c_int), ("n_pre", C.c_int), ("n_post", C.c_int),
                ("inner_cycles", C.c_int)]


class cmg_batch_stats(C.Structure):
    _fields_ = [("cycles", C.c_int), ("status", C.c_int), ("n_patches", C.c_int), ("n_converged", C.c_int),
                ("rel_max", C.c_double), ("ms", C.c_double), ("cell_updates", C.c_int64),
                ("grid_barriers", C.c_int64)]


class CmgError(RuntimeError):
    def __init__(self, code, fn, msg):
        super().__init__("%s failed (status %d): %s" % (fn, code, msg))
        self.code = code


_P = C.c_void_p
_I64 = C.c_int64
_I = C.c_int
_SIGS = {
    "cmg_version": (C.c_char_p, []),
    "cmg_last_error": (C.c_char_p, []),
    "cmg_ctx_create": (_I, [_I, _P, C.POINTER(_P)]),
    "cmg_ctx_destroy": (_I, [_P]),
    "cmg_ctx_synchronize": (_I, [_P]),
    "cmg_ctx_set_profiling": (_I, [_P, _I]),
    "cmg_ctx_get_profile": (_I, [_P, C.POINTER(cmg_kernel_profile), _I, C.POINTER(_I)]),
    "cmg_ctx_reset_profile": (_I, [_P]),
    "cmg_ctx_launch_count": (_I, [_P, C.POINTER(_I64)]),
    "cmg_morton_encode": (_I, [_P, _P, _I64, _P, _I]),
    "cmg_debug_inject_alloc_failure": (_I, [_I64]),
    "cmg_debug_neighbour_sum": (_I, [_P, _P, _I64, _I, _P, _I]),
    "cmg_morton_encode128": (_I, [_P, _P, _I64, _P, _I]),
    "cmg_morton_decode128": (_I, [_P, _P, _I64, _P, _I]),
    "cmg_level_build128": (_I, [_P, _I, _I, _I, _P, _I64, _I, _P, C.POINTER(_P)]),
    "cmg_level_key_bits": (_I, [_P, C.POINTER(_I)]),
    "cmg_level_lookup128": (_I, [_P, _P, _I64, _P, _I]),
    "cmg_level_mg_keys128": (_I, [_P, _I, _P, _I]),
    "cmg_morton_decode": (_I, [_P, _P, _I64, _P, _I]),
    "cmg_level_build": (_I, [_P, _I, _I, _I, _P, _I64, _I, _P, C.POINTER(_P)]),
    "cmg_level_destroy": (_I, [_P]),
    "cmg_level_n_octs": (_I, [_P, C.POINTER(_I64)]),
    "cmg_level_hash_capacity": (_I, [_P, C.POINTER(_I64)]),
    "cmg_level_lookup": (_I, [_P, _P, _I64, _P, _I]),
    "cmg_level_get_neighbors": (_I, [_P, _P, _I]),
    "cmg_level_get_father_cells": (_I, [_P, _P, _I]),
    "cmg_level_set_density": (_I, [_P, _P, _I, C.c_double, C.c_double]),
    "cmg_level_set_phi": (_I, [_P, _P, _I]),
    "cmg_level_get_phi": (_I, [_P, _P, _I]),
    "cmg_level_get_phi_async": (_I, [_P, _P, _I]),
    "cmg_level_get_residual": (_I, [_P, _P, _I]),
    "cmg_level_get_ghosts": (_I, [_P, _P, _I]),
    "cmg_level_solve": (_I, [_P, C.POINTER(cmg_solve_params), C.POINTER(cmg_solve_stats)]),
    "cmg_level_solve_async": (_I, [_P, C.POINTER(cmg_solve_params)]),
    "cmg_level_solve_wait": (_I, [_P, C.POINTER(cmg_solve_stats)]),
    "cmg_level_set_schedule": (_I, [_P, _I64, _I64]),
    "cmg_level_set_spin_budget": (_I, [_P, _I64]),
    "cmg_level_mg_depth": (_I, [_P, C.POINTER(_I)]),
    "cmg_level_mg_info": (_I, [_P, _I, C.POINTER(_I64), C.POINTER(_I)]),
    "cmg_level_mg_keys": (_I, [_P, _I, _P, _I]),
    "cmg_level_mg_active": (_I, [_P, _I, _P, _I]),
    "cmg_level_mg_get": (_I, [_P, _I, _I, _I, _P, _I]),
    "cmg_level_mg_set": (_I, [_P, _I, _I, _I, _P, _I]),
    "cmg_level_mg_step": (_I, [_P, _I, _I, _I, _I, C.POINTER(C.c_double)]),
    "cmg_residual_norm2_noalloc": (_I, [_P, _P, _P, _P, _I64, C.c_double, _P, _P]),
    "cmg_level_mg_step_range": (_I, [_P, _I, _I, _I, _I64, _I64, C.POINTER(C.c_double)]),
    "cmg_level_set_stencil": (_I, [_P, _I]),
    "cmg_level_mg_gather": (_I, [_P, _I, _I, _P, _I64, _P]),
    "cmg_level_mg_scatter": (_I, [_P, _I, _I, _P, _I64, _P]),
    "cmg_batch_create": (_I, [_P, _P, _I, C.POINTER(_P)]),
    "cmg_batch_destroy": (_I, [_P]),
    "cmg_batch_set_schedule": (_I, [_P, _P]),
    "cmg_batch_get_schedule": (_I, [_P, _P]),
    "cmg_batch_set_spin_budget": (_I, [_P, _I64]),
    "cmg_batch_solve": (_I, [_P, C.POINTER(cmg_solve_params), _P]),
    "cmg_batch_patch_stats": (_I, [_P, _P, _P, _P]),
    "cmg_batch_autotune": (_I, [_P, C.POINTER(cmg_solve_params), _P, C.POINTER(C.c_double)]),
    "cmg_unet_create": (_I, [_P, _I, _I, C.POINTER(_P)]),
    "cmg_unet_destroy": (_I, [_P]),
    "cmg_unet_n_params": (_I, [_P, C.POINTER(_I64)]),
    "cmg_unet_set_params": (_I, [_P, _P, _I]),
    "cmg_unet_get_params": (_I, [_P, _P, _I]),
    "cmg_unet_set_kernels": (_I, [_P, _I]),
    "cmg_unet_set_output_scale": (_I, [_P, C.c_float]),
    "cmg_unet_get_output_scale": (_I, [_P, C.POINTER(C.c_float)]),
    "cmg_unet_forward": (_I, [_P, _P, _P, _P, _I, _P, _P, _I]),
    "cmg_unet_gradients": (_I, [_P, _P, _P, _P, _P, _I, _P, C.POINTER(C.c_double), _I]),
    "cmg_unet_adam_step": (_I, [_P, C.c_float, C.c_float, C.c_float, C.c_float]),
    "cmg_unet_set_grad_clip": (_I, [_P, C.c_float]),
    "cmg_unet_grad_clip_stats": (_I, [_P, C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(_I64), C.POINTER(_I64)]),
    "cmg_dense_octs": (_I, [_P, _P, _I, _P, _I]),
}

_lib = None


def lib():
    """Load libcmg.so (built by build.py / __graft_entry__.build())."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libcmg.so is not built (%s); run __graft_entry__.build()" % LIB_PATH)
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def exported_symbols():
    return sorted(_SIGS)


def _check(rc, fn):
    if rc != CMG_OK:
        raise CmgError(rc, fn, lib().cmg_last_error().decode())
    return rc


# ------------------------------------------------------------ marshalling

def _is_torch(x):
    return type(x).__module__.startswith("torch")


def _in(x, dtype):
    """(pointer, mem, keepalive) for an input array."""
    if _is_torch(x):
        import torch
        if x.is_cuda:
            want = {np.float64: torch.float64, np.float32: torch.float32, np.uint64: torch.uint64,
                    np.uint32: torch.uint32, np.int32: torch.int32, np.uint8: torch.uint8}[dtype]
            if x.dtype != want or not x.is_contiguous():
                raise TypeError("device tensor must be contiguous %s" % want)
            return C.c_void_p(x.data_ptr()), CMG_MEM_DEVICE, x
        x = x.numpy()
    a = np.ascontiguousarray(x, dtype=dtype)
    return a.ctypes.data_as(C.c_void_p), CMG_MEM_HOST, a


def _out(shape, dtype, device=False, out=None):
    if out is not None:
        p, mem, keep = _in(out, dtype)
        if mem == CMG_MEM_HOST and keep is not out:
            raise TypeError("out must be a contiguous array of dtype %s" % np.dtype(dtype))
        return p, mem, out
    if device:
        import torch
        want = {np.float64: torch.float64, np.float32: torch.float32, np.uint64: torch.uint64,
                np.uint32: torch.uint32, np.int32: torch.int32, np.uint8: torch.uint8}[dtype]
        t = torch.empty(shape, dtype=want, device="cuda")
        return C.c_void_p(t.data_ptr()), CMG_MEM_DEVICE, t
    a = np.empty(shape, dtype=dtype)
    return a.ctypes.data_as(C.c_void_p), CMG_MEM_HOST, a


def _same_mem(m1, m2, fn):
    if m1 != m2:
        raise TypeError("%s: input and output must both be host or both be device arrays" % fn)


# ------------------------------------------------------------------ calls

def cmg_version():
    return lib().cmg_version().decode()


def cmg_last_error():
    return lib().cmg_last_error().decode()


def cmg_ctx_create(device=0, stream=None):
    """stream: a raw cudaStream_t (int), a torch.cuda.Stream, or None for the
    current torch stream (if torch is importable) else the legacy default."""
    if stream is None:
        try:
            import torch
            stream = torch.cuda.current_stream(device).cuda_stream if torch.cuda.is_available() else 0
        except ImportError:
            stream = 0
    elif not isinstance(stream, int):
        stream = stream.cuda_stream
    h = C.c_void_p()
    _check(lib().cmg_ctx_create(device, C.c_void_p(stream), C.byref(h)), "cmg_ctx_create")
    return CtxHandle(h)


class CtxHandle:
    """Owns a cmg_ctx* and tracks the levels built on it, so that destroying
    the context first destroys whatever levels are still alive (finest first)."""

    def __init__(self, h):
        self.h = h
        self.levels = []  # weak references, in build order

    @property
    def _as_parameter_(self):
        if not self.h:
            raise CmgError(CMG_ERR_INVALID_ARG, "cmg", "context already destroyed")
        return self.h

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            cmg_ctx_destroy(self)


def cmg_ctx_destroy(ctx):
    if not ctx.h:
        return
    for ref in getattr(ctx, "unets", []):
        u = ref()
        if u is not None and u.h:
            cmg_unet_destroy(u)
    for ref in reversed(ctx.levels):
        lv = ref()
        if lv is not None and lv.h:
            cmg_level_destroy(lv)
    ctx.levels = []
    h, ctx.h = ctx.h, None
    _check(lib().cmg_ctx_destroy(h), "cmg_ctx_destroy")


def cmg_ctx_synchronize(ctx):
    _check(lib().cmg_ctx_synchronize(ctx), "cmg_ctx_synchronize")


def cmg_ctx_set_profiling(ctx, enable):
    _check(lib().cmg_ctx_set_profiling(ctx, int(bool(enable))), "cmg_ctx_set_profiling")


def cmg_ctx_get_profile(ctx):
    """{family: {"launches", "ms", "bytes", "flops"}} since the last reset."""
    buf = (cmg_kernel_profile * 32)()
    n = C.c_int()
    _check(lib().cmg_ctx_get_profile(ctx, buf, 32, C.byref(n)), "cmg_ctx_get_profile")
    return {buf[i].name.decode(): {"launches": buf[i].launches, "ms": buf[i].ms, "bytes": buf[i].bytes,
                                   "flops": buf[i].flops} for i in range(n.value)}


def cmg_ctx_reset_profile(ctx):
    _check(lib().cmg_ctx_reset_profile(ctx), "cmg_ctx_reset_profile")


def cmg_ctx_launch_count(ctx):
    v = C.c_int64()
    _check(lib().cmg_ctx_launch_count(ctx, C.byref(v)), "cmg_ctx_launch_count")
    return v.value


def cmg_debug_inject_alloc_failure(after):
    """Tests: the after'th next library allocation fails with CMG_ERR_OOM."""
    _check(lib().cmg_debug_inject_alloc_failure(int(after)), "cmg_debug_inject_alloc_failure")


def cmg_debug_neighbour_sum(ctx, rows, which=0, out=None):
    """Tests: the FP64 neighbour sum of each [6] row, as the kernels form it
    (which = 0: colour passes and colour-1 residuals; 1: colour-0 residuals)."""
    p, mem, keep = _in(rows, np.float64)
    n = keep.numel() // 6 if _is_torch(keep) else keep.size // 6
    if (keep.numel() if _is_torch(keep) else keep.size) != 6 * n:
        raise ValueError("rows must hold a multiple of 6 values")
    q, mem2, res = _out((n,), np.float64, device=(mem == CMG_MEM_DEVICE), out=out)
    _same_mem(mem, mem2, "cmg_debug_neighbour_sum")
    _check(lib().cmg_debug_neighbour_sum(ctx, p, n, int(which), q, mem), "cmg_debug_neighbour_sum")
    return res


def cmg_morton_encode(ctx, ijk, out=None):
    p, mem, keep = _in(ijk, np.uint32)
    n = keep.numel() // 3 if _is_torch(keep) else keep.size // 3
    q, mem2, res = _out((n,), np.uint64, device=(mem == CMG_MEM_DEVICE), out=out)
    _same_mem(mem, mem2, "cmg_morton_encode")
    _check(lib().cmg_morton_encode(ctx, p, n, q, mem), "cmg_morton_encode")
    return res


def cmg_morton_decode(ctx, keys, out=None):
    p, mem, keep = _in(keys, np.uint64)
    n = keep.numel() if _is_torch(keep) else keep.size
    q, mem2, res = _out((n, 3), np.uint32, device=(mem == CMG_MEM_DEVICE), out=out)
    _same_mem(mem, mem2, "cmg_morton_decode")
    _check(lib().cmg_morton_decode(ctx, p, n, q, mem), "cmg_morton_decode")
    return res


def cmg_morton_encode128(ctx, ijk, out=None):
    """128-bit keys (B = 42) of [n, 3] uint64 coordinates: [n, 2] uint64
    (low word, high word)."""
    p, mem, keep = _in(ijk, np.uint64)
    n = keep.numel() // 3 if _is_torch(keep) else keep.size // 3
    q, mem2, res = _out((n, 2), np.uint64, device=(mem == CMG_MEM_DEVICE), out=out)
    _same_mem(mem, mem2, "cmg_morton_encode128")
    _check(lib().cmg_morton_encode128(ctx, p, n, q, mem), "cmg_morton_encode128")
    return res


def cmg_morton_decode128(ctx, keys, out=None):
    p, mem, keep = _in(keys, np.uint64)
    n = keep.numel() // 2 if _is_torch(keep) else keep.size // 2
    q, mem2, res = _out((n, 3), np.uint64, device=(mem == CMG_MEM_DEVICE), out=out)
    _same_mem(mem, mem2, "cmg_morton_decode128")
    _check(lib().cmg_morton_decode128(ctx, p, n, q, mem), "cmg_morton_decode128")
    return res


class LevelHandle:
    """Owns a cmg_level* (destroyed with the object) and keeps its parent alive."""

    def __init__(self, h, parent, ctx):
        import weakref
        self.h = h
        self.parent = parent
        self.ctx = ctx
        ctx.levels.append(weakref.ref(self))

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            h, self.h = self.h, None
            _lib.cmg_level_destroy(h)

    @property
    def _as_parameter_(self):
        return self.h


def cmg_level_build(ctx, level, keys, parent=None, nx=1, periodic_mask=7):
    p, mem, keep = _in(keys, np.uint64)
    n = keep.numel() if _is_torch(keep) else keep.size
    h = C.c_void_p()
    _check(lib().cmg_level_build(ctx, level, nx, periodic_mask, p, n, mem,
                                 parent.h if parent is not None else None, C.byref(h)), "cmg_level_build")
    return LevelHandle(h, parent, ctx)


def cmg_level_build128(ctx, level, keys, parent=None, nx=1, periodic_mask=7):
    """A level with 128-bit keys ([n, 2] uint64), levels up to 43."""
    p, mem, keep = _in(keys, np.uint64)
    n = keep.numel() // 2 if _is_torch(keep) else keep.size // 2
    h = C.c_void_p()
    _check(lib().cmg_level_build128(ctx, level, nx, periodic_mask, p, n, mem,
                                    parent.h if parent is not None else None, C.byref(h)), "cmg_level_build128")
    return LevelHandle(h, parent, ctx)


def cmg_level_key_bits(lvl):
    v = C.c_int()
    _check(lib().cmg_level_key_bits(lvl.h, C.byref(v)), "cmg_level_key_bits")
    return v.value


def cmg_level_destroy(lvl):
    if lvl.h:
        for ref in getattr(lvl, "batches", []):
            b = ref()
            if b is not None and b.h:
                cmg_batch_destroy(b)
        _check(lib().cmg_level_destroy(lvl.h), "cmg_level_destroy")
        lvl.h = None


class BatchHandle:
    """Owns a cmg_batch* and keeps its level alive; destroyed before it."""

    def __init__(self, h, lvl, n_patches):
        import weakref
        self.h = h
        self.lvl = lvl
        self.n_patches = n_patches
        if not hasattr(lvl, "batches"):
            lvl.batches = []
        lvl.batches.append(weakref.ref(self))

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            h, self.h = self.h, None
            _lib.cmg_batch_destroy(h)


def cmg_batch_create(lvl, offsets):
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    h = C.c_void_p()
    _check(lib().cmg_batch_create(lvl.h, off.ctypes.data_as(C.c_void_p), len(off) - 1, C.byref(h)),
           "cmg_batch_create")
    return BatchHandle(h, lvl, len(off) - 1)


def cmg_batch_destroy(b):
    if b.h:
        h, b.h = b.h, None
        _check(lib().cmg_batch_destroy(h), "cmg_batch_destroy")


def cmg_batch_set_schedule(b, threads=256, blocks_per_sm=2, n_pre=2, n_post=2, inner_cycles=1):
    s = cmg_batch_schedule(threads, blocks_per_sm, n_pre, n_post, inner_cycles)
    _check(lib().cmg_batch_set_schedule(b.h, C.byref(s)), "cmg_batch_set_schedule")


def cmg_batch_get_schedule(b):
    s = cmg_batch_schedule()
    _check(lib().cmg_batch_get_schedule(b.h, C.byref(s)), "cmg_batch_get_schedule")
    return {f: getattr(s, f) for f, _ in s._fields_}


def cmg_batch_set_spin_budget(b, cycles):
    _check(lib().cmg_batch_set_spin_budget(b.h, int(cycles)), "cmg_batch_set_spin_budget")


def cmg_batch_solve(b, params=None, raise_on_error=True, **kw):
    prm = params if params is not None else solve_params(**kw)
    st = cmg_batch_stats()
    rc = lib().cmg_batch_solve(b.h, C.byref(prm), C.byref(st))
    if raise_on_error:
        _check(rc, "cmg_batch_solve")
    return rc, {f: getattr(st, f) for f, _ in st._fields_}


def cmg_batch_patch_stats(b):
    n = b.n_patches
    rel = np.empty(n)
    conv = np.empty(n, dtype=np.int32)
    n0 = np.empty(n)
    _check(lib().cmg_batch_patch_stats(b.h, rel.ctypes.data_as(C.c_void_p), conv.ctypes.data_as(C.c_void_p),
                                       n0.ctypes.data_as(C.c_void_p)), "cmg_batch_patch_stats")
    return rel, conv, n0


def cmg_batch_autotune(b, params=None, **kw):
    prm = params if params is not None else solve_params(**kw)
    s = cmg_batch_schedule()
    ms = C.c_double()
    _check(lib().cmg_batch_autotune(b.h, C.byref(prm), C.byref(s), C.byref(ms)), "cmg_batch_autotune")
    return {f: getattr(s, f) for f, _ in s._fields_}, ms.value


def cmg_level_n_octs(lvl):
    v = C.c_int64()
    _check(lib().cmg_level_n_octs(lvl.h, C.byref(v)), "cmg_level_n_octs")
    return v.value


def cmg_level_hash_capacity(lvl):
    v = C.c_int64()
    _check(lib().cmg_level_hash_capacity(lvl.h, C.byref(v)), "cmg_level_hash_capacity")
    return v.value


def cmg_level_lookup(lvl, q, out=None):
    p, mem, keep = _in(q, np.uint64)
    n = keep.numel() if _is_torch(keep) else keep.size
    o, mem2, res = _out((n,), np.int32, device=(mem == CMG_MEM_DEVICE), out=out)
    _same_mem(mem, mem2, "cmg_level_lookup")
    _check(lib().cmg_level_lookup(lvl.h, p, n, o, mem), "cmg_level_lookup")
    return res


def cmg_level_lookup128(lvl, q, out=None):
    p, mem, keep = _in(q, np.uint64)
    n = keep.numel() // 2 if _is_torch(keep) else keep.size // 2
    o, mem2, res = _out((n,), np.int32, device=(mem == CMG_MEM_DEVICE), out=out)
    _same_mem(mem, mem2, "cmg_level_lookup128")
    _check(lib().cmg_level_lookup128(lvl.h, p, n, o, mem), "cmg_level_lookup128")
    return res


def _get(fn, lvl, shape, dtype, device, out):
    o, mem, res = _out(shape, dtype, device=device, out=out)
    _check(getattr(lib(), fn)(lvl.h, o, mem), fn)
    return res


def cmg_level_get_neighbors(lvl, device=False, out=None):
    return _get("cmg_level_get_neighbors", lvl, (cmg_level_n_octs(lvl), 7), np.int32, device, out)


def cmg_level_get_father_cells(lvl, device=False, out=None):
    return _get("cmg_level_get_father_cells", lvl, (cmg_level_n_octs(lvl), 6, 2), np.int32, device, out)


def cmg_level_get_phi(lvl, device=False, out=None):
    return _get("cmg_level_get_phi", lvl, (cmg_level_n_octs(lvl), 8), np.float64, device, out)


def cmg_level_get_phi_async(lvl, device=False, out=None):
    """Queued read-back of phi: the returned array (or `out`, which must stay
    alive) holds phi once cmg_ctx_synchronize(ctx) returns."""
    return _get("cmg_level_get_phi_async", lvl, (cmg_level_n_octs(lvl), 8), np.float64, device, out)


def cmg_level_get_residual(lvl, device=False, out=None):
    return _get("cmg_level_get_residual", lvl, (cmg_level_n_octs(lvl), 8), np.float64, device, out)


def cmg_level_get_ghosts(lvl, device=False, out=None):
    return _get("cmg_level_get_ghosts", lvl, (cmg_level_n_octs(lvl), 6, 4), np.float64, device, out)


def cmg_level_set_density(lvl, rho, rho_bar, four_pi_g=1.0):
    p, mem, keep = _in(rho, np.float64)
    _check(lib().cmg_level_set_density(lvl.h, p, mem, float(rho_bar), float(four_pi_g)), "cmg_level_set_density")


def cmg_level_set_phi(lvl, phi):
    p, mem, keep = _in(phi, np.float64)
    _check(lib().cmg_level_set_phi(lvl.h, p, mem), "cmg_level_set_phi")


def solve_params(tol=1e-10, max_cycles=100, n_pre=2, n_post=2, coarse_sweeps=4, fixed_cycles=0,
                 precision=CMG_PREC_FP64, inner_cycles=2, krylov=0):
    return cmg_solve_params(tol, max_cycles, n_pre, n_post, coarse_sweeps, fixed_cycles, precision, inner_cycles,
                            krylov)


def _stats(st):
    return {"cycles": st.cycles, "status": st.status, "rel_initial": st.rel_initial, "rel_final": st.rel_final,
            "norm0": st.norm0, "ms": st.ms, "cell_updates": st.cell_updates,
            "rel_history": list(st.rel_history[:st.cycles])}


def cmg_level_solve(lvl, params=None, raise_on_error=True, **kw):
    """Returns (status, stats dict)."""
    prm = params if params is not None else solve_params(**kw)
    st = cmg_solve_stats()
    rc = lib().cmg_level_solve(lvl.h, C.byref(prm), C.byref(st))
    if raise_on_error:
        _check(rc, "cmg_level_solve")
    return rc, _stats(st)


def cmg_level_solve_async(lvl, params=None, **kw):
    """Queue a solve without waiting; cmg_level_solve_wait reports it."""
    prm = params if params is not None else solve_params(**kw)
    _check(lib().cmg_level_solve_async(lvl.h, C.byref(prm)), "cmg_level_solve_async")


def cmg_level_solve_wait(lvl, raise_on_error=True):
    """Returns (status, stats dict) of the level's queued solve."""
    st = cmg_solve_stats()
    rc = lib().cmg_level_solve_wait(lvl.h, C.byref(st))
    if raise_on_error:
        _check(rc, "cmg_level_solve_wait")
    return rc, _stats(st)


def cmg_level_set_schedule(lvl, tail_octs_fp64=-1, tail_octs_fp32=-1):
    _check(lib().cmg_level_set_schedule(lvl.h, int(tail_octs_fp64), int(tail_octs_fp32)), "cmg_level_set_schedule")


def cmg_level_set_stencil(lvl, staged):
    """Colour passes of lexicographic full periodic levels: 0 = neighbour-table
    kernel, 1 = shared-memory brick kernel for FP32 passes (default), 2 =
    brick kernel for FP32 and FP64 passes (same bits in every mode)."""
    _check(lib().cmg_level_set_stencil(lvl.h, int(staged)), "cmg_level_set_stencil")


def cmg_level_set_spin_budget(lvl, cycles):
    _check(lib().cmg_level_set_spin_budget(lvl.h, int(cycles)), "cmg_level_set_spin_budget")


def cmg_level_mg_depth(lvl):
    v = C.c_int()
    _check(lib().cmg_level_mg_depth(lvl.h, C.byref(v)), "cmg_level_mg_depth")
    return v.value


def cmg_level_mg_info(lvl, m):
    n = C.c_int64()
    lev = C.c_int()
    _check(lib().cmg_level_mg_info(lvl.h, m, C.byref(n), C.byref(lev)), "cmg_level_mg_info")
    return n.value, lev.value


def cmg_level_mg_keys(lvl, m, device=False):
    n, _ = cmg_level_mg_info(lvl, m)
    o, mem, res = _out((n,), np.uint64, device=device)
    _check(lib().cmg_level_mg_keys(lvl.h, m, o, mem), "cmg_level_mg_keys")
    return res


def cmg_level_mg_keys128(lvl, m, device=False):
    n, _ = cmg_level_mg_info(lvl, m)
    o, mem, res = _out((n, 2), np.uint64, device=device)
    _check(lib().cmg_level_mg_keys128(lvl.h, m, o, mem), "cmg_level_mg_keys128")
    return res


def cmg_level_mg_active(lvl, m, device=False):
    n, _ = cmg_level_mg_info(lvl, m)
    o, mem, res = _out((n, 8), np.uint8, device=device)
    _check(lib().cmg_level_mg_active(lvl.h, m, o, mem), "cmg_level_mg_active")
    return res


def cmg_level_mg_get(lvl, m, field, precision=CMG_PREC_FP64, device=False):
    n, _ = cmg_level_mg_info(lvl, m)
    dt = np.float64 if precision == CMG_PREC_FP64 else np.float32
    o, mem, res = _out((n, 8), dt, device=device)
    _check(lib().cmg_level_mg_get(lvl.h, m, field, precision, o, mem), "cmg_level_mg_get")
    return res


def cmg_level_mg_set(lvl, m, field, arr, precision=CMG_PREC_FP64):
    dt = np.float64 if precision == CMG_PREC_FP64 else np.float32
    p, mem, keep = _in(arr, dt)
    _check(lib().cmg_level_mg_set(lvl.h, m, field, precision, p, mem), "cmg_level_mg_set")


def cmg_level_mg_step(lvl, m, op, precision=CMG_PREC_FP64, n=1):
    v = C.c_double(0.0)
    _check(lib().cmg_level_mg_step(lvl.h, m, op, precision, n, C.byref(v)), "cmg_level_mg_step")
    return v.value


def cmg_level_mg_step_range(lvl, m, op, arg, lo, hi, value=0.0):
    """One V-cycle operation on the octs [lo, hi) of MG level m (sharded
    solve; FP64).  Returns the value the operation reports (norm^2 or sum),
    else the value passed in."""
    v = C.c_double(float(value))
    _check(lib().cmg_level_mg_step_range(lvl.h, m, op, arg, int(lo), int(hi), C.byref(v)),
           "cmg_level_mg_step_range")
    return v.value


def _cells_and_buf(cells, buf, fn):
    pc, mc, _ = _in(cells, np.int32)
    pb, mb, _ = _in(buf, np.float64)
    if mc != CMG_MEM_DEVICE or mb != CMG_MEM_DEVICE:
        raise TypeError("%s: cells and buf must be CUDA tensors" % fn)
    if int(np.prod(buf.shape)) < int(np.prod(cells.shape)):
        raise ValueError("%s: buf holds fewer values than cells" % fn)
    return pc, pb, int(np.prod(cells.shape))


def cmg_level_mg_gather(lvl, m, field, cells, out=None):
    """Values of the listed cells (oct * 8 + child; int32 CUDA tensor) of MG
    level m: field 0 = phi, 1 = the stored source.  Returns a float64 CUDA
    tensor."""
    import torch
    if out is None:
        out = torch.empty(int(np.prod(cells.shape)), dtype=torch.float64, device=cells.device)
    pc, pb, n = _cells_and_buf(cells, out, "cmg_level_mg_gather")
    _check(lib().cmg_level_mg_gather(lvl.h, m, field, pc, n, pb), "cmg_level_mg_gather")
    return out


def cmg_level_mg_scatter(lvl, m, field, cells, values):
    """Write values (float64 CUDA tensor) into the listed cells of MG level m."""
    pc, pb, n = _cells_and_buf(cells, values, "cmg_level_mg_scatter")
    _check(lib().cmg_level_mg_scatter(lvl.h, m, field, pc, n, pb), "cmg_level_mg_scatter")


class UnetHandle:
    """Owns a cmg_unet*; destroyed before its context."""

    def __init__(self, h, ctx, grid_dim, max_batch):
        import weakref
        self.h = h
        self.ctx = ctx
        self.D = grid_dim
        self.max_batch = max_batch
        if not hasattr(ctx, "unets"):
            ctx.unets = []
        ctx.unets.append(weakref.ref(self))

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            h, self.h = self.h, None
            _lib.cmg_unet_destroy(h)


def cmg_unet_create(ctx, grid_dim=64, max_batch=4):
    h = C.c_void_p()
    _check(lib().cmg_unet_create(ctx, grid_dim, max_batch, C.byref(h)), "cmg_unet_create")
    return UnetHandle(h, ctx, grid_dim, max_batch)


def cmg_unet_destroy(net):
    if net.h:
        h, net.h = net.h, None
        _check(lib().cmg_unet_destroy(h), "cmg_unet_destroy")


def cmg_unet_n_params(net):
    v = C.c_int64()
    _check(lib().cmg_unet_n_params(net.h, C.byref(v)), "cmg_unet_n_params")
    return v.value


def cmg_unet_set_params(net, params):
    p, mem, keep = _in(params, np.float32)
    _check(lib().cmg_unet_set_params(net.h, p, mem), "cmg_unet_set_params")


def cmg_unet_get_params(net, device=False):
    o, mem, res = _out((cmg_unet_n_params(net),), np.float32, device=device)
    _check(lib().cmg_unet_get_params(net.h, o, mem), "cmg_unet_get_params")
    return res


def _batch_of(net, x):
    n = x.numel() if _is_torch(x) else np.asarray(x).size
    return n // (net.D ** 3)


def cmg_unet_set_kernels(net, tensor_path):
    """1 = tcgen05 convolutions where the grid allows (default), 0 = mma.sync."""
    _check(lib().cmg_unet_set_kernels(net.h, int(tensor_path)), "cmg_unet_set_kernels")


def cmg_unet_set_output_scale(net, scale):
    _check(lib().cmg_unet_set_output_scale(net.h, float(scale)), "cmg_unet_set_output_scale")


def cmg_unet_get_output_scale(net):
    v = C.c_float(0.0)
    _check(lib().cmg_unet_get_output_scale(net.h, C.byref(v)), "cmg_unet_get_output_scale")
    return v.value


def cmg_unet_forward(net, rho, field, base=None, delta=False):
    """Prediction base + c rms(field) delta (c: the output scale) (and delta if asked) for a batch of
    dense [B][D][D][D] fields; base defaults to field."""
    pr, mem, k1 = _in(rho, np.float32)
    pp, mem2, k2 = _in(field, np.float32)
    _same_mem(mem, mem2, "cmg_unet_forward")
    pb, k4 = None, None
    if base is not None:
        pb, _, k4 = _in(base, np.float32)
    B = _batch_of(net, rho)
    shape = (B, net.D, net.D, net.D)
    po, _, out = _out(shape, np.float32, device=(mem == CMG_MEM_DEVICE))
    pd, dres = None, None
    if delta:
        pd, _, dres = _out(shape, np.float32, device=(mem == CMG_MEM_DEVICE))
    _check(lib().cmg_unet_forward(net.h, pr, pp, pb, B, po, pd, mem), "cmg_unet_forward")
    return (out, dres) if delta else out


def cmg_unet_gradients(net, rho, field, target, base=None, grads=True):
    """(loss, gradient or None).  Host inputs give the mean loss; device inputs
    return the loss as a device sum of squares (see include/cmg.h)."""
    pr, mem, k1 = _in(rho, np.float32)
    pp, _, k2 = _in(field, np.float32)
    pn, _, k3 = _in(target, np.float32)
    pb, k4 = None, None
    if base is not None:
        pb, _, k4 = _in(base, np.float32)
    B = _batch_of(net, rho)
    pg, res = None, None
    if grads:
        pg, _, res = _out((cmg_unet_n_params(net),), np.float32, device=(mem == CMG_MEM_DEVICE))
    loss = C.c_double(0.0)
    if mem == CMG_MEM_DEVICE:
        import torch
        lt = torch.zeros(1, dtype=torch.float64, device="cuda")
        _check(lib().cmg_unet_gradients(net.h, pr, pp, pb, pn, B, pg,
                                        C.cast(C.c_void_p(lt.data_ptr()), C.POINTER(C.c_double)), mem),
               "cmg_unet_gradients")
        return lt, res
    _check(lib().cmg_unet_gradients(net.h, pr, pp, pb, pn, B, pg, C.byref(loss), mem), "cmg_unet_gradients")
    return loss.value, res


def cmg_unet_adam_step(net, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    _check(lib().cmg_unet_adam_step(net.h, lr, beta1, beta2, eps), "cmg_unet_adam_step")


def cmg_unet_set_grad_clip(net, k):
    """Cap each Adam step's gradient norm at k x its running mean (0: off)."""
    _check(lib().cmg_unet_set_grad_clip(net.h, float(k)), "cmg_unet_set_grad_clip")


def cmg_unet_grad_clip_stats(net):
    last, mean = C.c_double(), C.c_double()
    steps, clipped = C.c_int64(), C.c_int64()
    _check(lib().cmg_unet_grad_clip_stats(net.h, C.byref(last), C.byref(mean), C.byref(steps), C.byref(clipped)),
           "cmg_unet_grad_clip_stats")
    return {"last_norm": last.value, "mean_norm": mean.value, "steps": steps.value, "clipped": clipped.value}


def cmg_dense_octs(ctx, src, grid_dim, dst, to_octs):
    """Device copy dense [D^3] <-> oct-major [n][8] of a full periodic level (x-fastest octs)."""
    ps, ms, _ = _in(src, np.float64)
    pd, md, _ = _in(dst, np.float64)
    _same_mem(ms, CMG_MEM_DEVICE, "cmg_dense_octs")
    _same_mem(md, CMG_MEM_DEVICE, "cmg_dense_octs")
    _check(lib().cmg_dense_octs(ctx, ps, grid_dim, pd, int(to_octs)), "cmg_dense_octs")


def cmg_residual_norm2_noalloc(neighbors, ghosts, phi, f, h, norm2, stream=0):
    """Residual norm^2 into the one-double CUDA tensor norm2 with no device
    allocation by the library (for callers that cannot allocate at that point:
    real-time loops, hosts that own all device memory in an arena; see
    include/cmg.h).  neighbors [n][7] int32, ghosts [n][6][4] or None, phi and
    f [n][8] float64, all CUDA tensors on the current device.  Runs on
    `stream` (raw handle or torch stream); the caller synchronises before
    reading norm2.

    The library reads 7n neighbour entries, 8n values of phi and f and 24n
    ghost values, so every size is checked here before the call (ValueError)."""
    n = int(neighbors.shape[0]) if len(getattr(neighbors, "shape", ())) else -1
    sizes = [("neighbors", neighbors, 7 * n), ("phi", phi, 8 * n), ("f", f, 8 * n)]
    if ghosts is not None:
        sizes.append(("ghosts", ghosts, 24 * n))
    if n < 0:
        raise ValueError("cmg_residual_norm2_noalloc: neighbors must be an [n][7] array")
    for name, a, want in sizes:
        got = int(np.prod(a.shape))
        if got != want:
            raise ValueError("cmg_residual_norm2_noalloc: %s holds %d values, expected %d for n = %d octs"
                             % (name, got, want, n))
    if int(np.prod(norm2.shape)) < 1:
        raise ValueError("cmg_residual_norm2_noalloc: norm2 must hold at least one value")
    if not isinstance(stream, int):
        stream = stream.cuda_stream
    pn, mn, _ = _in(neighbors, np.int32)
    pp, mp, _ = _in(phi, np.float64)
    pf, mf, _ = _in(f, np.float64)
    po, mo, _ = _in(norm2, np.float64)
    pg = None
    arrays = [neighbors, phi, f, norm2]
    if ghosts is not None:
        pg, mg, _ = _in(ghosts, np.float64)
        _same_mem(mg, CMG_MEM_DEVICE, "cmg_residual_norm2_noalloc")
        arrays.append(ghosts)
    for m in (mn, mp, mf, mo):
        _same_mem(m, CMG_MEM_DEVICE, "cmg_residual_norm2_noalloc")
    import torch
    cur = torch.cuda.current_device()
    for a in arrays:
        if a.device.index != cur:
            raise ValueError("cmg_residual_norm2_noalloc: every tensor must be on the current device (cuda:%d), "
                             "got %s" % (cur, a.device))
    rc = lib().cmg_residual_norm2_noalloc(pn, pg, pp, pf, n, float(h), po, C.c_void_p(stream))
    if rc != CMG_OK:
        raise CmgError(rc, "cmg_residual_norm2_noalloc", "invalid argument or CUDA error")
