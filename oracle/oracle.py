"""ctypes wrapper around the C oracle (liboracle.so).  Test infrastructure only.

Arrays are NumPy; the oracle owns copies of everything it is given.
"""
import ctypes as C

import numpy as np

from . import build as _build

_lib = None

OR_OK = 0
OR_ERR_INVALID_ARG = -1
OR_ERR_DUPLICATE_KEY = -2
OR_ERR_KEY_OUT_OF_RANGE = -3
OR_ERR_MISSING_PARENT = -4
OR_ERR_OOM = -5
OR_ERR_NOT_CONVERGED = -7
OR_ERR_DIVERGED = -8

_P = C.c_void_p
_I64 = C.c_int64


class OrParams(C.Structure):
    _fields_ = [("tol", C.c_double), ("max_cycles", C.c_int), ("n_pre", C.c_int), ("n_post", C.c_int),
                ("coarse_sweeps", C.c_int), ("fixed_cycles", C.c_int)]


class OrStats(C.Structure):
    _fields_ = [("cycles", C.c_int), ("rel_initial", C.c_double), ("rel_final", C.c_double),
                ("norm0", C.c_double), ("rel_history", C.c_double * 256)]


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        sig = {
            "or_set_threads": (C.c_int, [C.c_int]),
            "or_get_threads": (C.c_int, []),
            "or_morton_encode": (C.c_uint64, [C.c_uint32] * 3),
            "or_encode_many": (None, [_P, _I64, _P]),
            "or_decode_many": (None, [_P, _I64, _P]),
            "or_encode128_many": (None, [_P, _I64, _P]),
            "or_decode128_many": (None, [_P, _I64, _P]),
            "or_level_build128": (C.c_int, [C.c_int, C.c_int, C.c_int, _P, _I64, _P, C.POINTER(_P)]),
            "or_level_lookup128": (None, [_P, _P, _I64, _P]),
            "or_level_mg_keys128": (None, [_P, C.c_int, _P]),
            "or_neighbor_key": (C.c_int64, [C.c_uint64, C.c_int, C.c_uint32, C.c_int]),
            "or_hash_fn": (C.c_uint64, [C.c_uint64]),
            "or_hash_capacity_for": (C.c_int64, [_I64]),
            "or_level_build": (C.c_int, [C.c_int, C.c_int, C.c_int, _P, _I64, _P, C.POINTER(_P)]),
            "or_level_free": (None, [_P]),
            "or_level_n_octs": (_I64, [_P]),
            "or_level_hash_capacity": (_I64, [_P]),
            "or_level_hash_dump": (None, [_P, _P, _P]),
            "or_level_lookup": (None, [_P, _P, _I64, _P]),
            "or_level_neighbors": (None, [_P, _P]),
            "or_level_father_cells": (None, [_P, _P]),
            "or_level_set_density": (None, [_P, _P, C.c_double, C.c_double]),
            "or_level_set_f": (None, [_P, _P]),
            "or_level_set_phi": (None, [_P, _P]),
            "or_level_get_phi": (None, [_P, _P]),
            "or_level_get_f": (None, [_P, _P]),
            "or_level_compute_ghosts": (None, [_P]),
            "or_level_get_ghosts": (None, [_P, _P]),
            "or_level_mg_depth": (C.c_int, [_P]),
            "or_level_mg_n_octs": (_I64, [_P, C.c_int]),
            "or_level_mg_lev": (C.c_int, [_P, C.c_int]),
            "or_level_mg_keys": (None, [_P, C.c_int, _P]),
            "or_level_mg_active": (None, [_P, C.c_int, _P]),
            "or_level_mg_get": (None, [_P, C.c_int, C.c_int, _P]),
            "or_level_mg_set": (None, [_P, C.c_int, C.c_int, _P]),
            "or_rb_sweeps": (None, [_P, C.c_int, C.c_int, C.c_int]),
            "or_rb_colour_pass": (None, [_P, C.c_int, C.c_int, C.c_int]),
            "or_residual": (C.c_double, [_P, C.c_int, C.c_int]),
            "or_restrict": (None, [_P, C.c_int]),
            "or_prolong": (None, [_P, C.c_int]),
            "or_coarse_solve": (None, [_P, C.c_int]),
            "or_level_solve": (C.c_int, [_P, C.POINTER(OrParams), C.POINTER(OrStats)]),
            "or_level_solve_mixed": (C.c_int, [_P, C.POINTER(OrParams), C.c_int, C.POINTER(OrStats)]),
            "or_level_solve_pcg": (C.c_int, [_P, C.POINTER(OrParams), C.POINTER(OrStats)]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def set_threads(n):
    """Threads of the oracle's per-oct loops (results are bit-identical for
    any count); returns the count in force (1 without OpenMP)."""
    return int(lib().or_set_threads(int(n)))


def get_threads():
    return int(lib().or_get_threads())


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p)


def morton_encode(ijk):
    ijk = np.ascontiguousarray(ijk, dtype=np.uint32).reshape(-1, 3)
    out = np.empty(len(ijk), dtype=np.uint64)
    lib().or_encode_many(_ptr(ijk), len(ijk), _ptr(out))
    return out


def morton_decode(keys):
    keys = np.ascontiguousarray(keys, dtype=np.uint64).ravel()
    out = np.empty((len(keys), 3), dtype=np.uint32)
    lib().or_decode_many(_ptr(keys), len(keys), _ptr(out))
    return out


def morton_encode128(ijk):
    """128-bit keys (B = 42) of [n, 3] uint64 coordinates: [n, 2] uint64
    (bits 0..63, bits 64..127)."""
    ijk = np.ascontiguousarray(ijk, dtype=np.uint64).reshape(-1, 3)
    out = np.empty((len(ijk), 2), dtype=np.uint64)
    lib().or_encode128_many(_ptr(ijk), len(ijk), _ptr(out))
    return out


def morton_decode128(keys):
    keys = np.ascontiguousarray(keys, dtype=np.uint64).reshape(-1, 2)
    out = np.empty((len(keys), 3), dtype=np.uint64)
    lib().or_decode128_many(_ptr(keys), len(keys), _ptr(out))
    return out


def neighbor_key(m, d, n_per_dim, periodic_mask=7):
    return lib().or_neighbor_key(int(m), int(d), int(n_per_dim), int(periodic_mask))


def hash_fn(h):
    return lib().or_hash_fn(int(h))


def hash_capacity_for(n):
    return lib().or_hash_capacity_for(int(n))


def params(tol=1e-10, max_cycles=100, n_pre=2, n_post=2, coarse_sweeps=4, fixed_cycles=0):
    return OrParams(tol, max_cycles, n_pre, n_post, coarse_sweeps, fixed_cycles)


class OracleError(RuntimeError):
    def __init__(self, code, what):
        super().__init__("%s failed with oracle status %d" % (what, code))
        self.code = code


class Level:
    """One AMR level of octs (plus its multigrid hierarchy) in the oracle."""

    def __init__(self, level, keys, parent=None, nx=1, periodic_mask=7):
        """keys: [n] uint64 (64-bit keys) or [n, 2] uint64 (128-bit keys)."""
        keys = np.ascontiguousarray(keys, dtype=np.uint64)
        self.wide = keys.ndim == 2
        keys = keys.reshape(-1, 2) if self.wide else keys.ravel()
        self._keys = keys
        self.level = level
        self.parent = parent  # keep alive
        h = C.c_void_p()
        build = lib().or_level_build128 if self.wide else lib().or_level_build
        rc = build(level, nx, periodic_mask, _ptr(keys), len(keys), parent._h if parent is not None else None,
                   C.byref(h))
        if rc != OR_OK:
            raise OracleError(rc, "or_level_build128" if self.wide else "or_level_build")
        self._h = h
        self.n = len(keys)

    def __del__(self):
        if getattr(self, "_h", None):
            lib().or_level_free(self._h)
            self._h = None

    # ---- structure
    @property
    def hash_capacity(self):
        return lib().or_level_hash_capacity(self._h)

    def hash_dump(self):
        cap = self.hash_capacity
        k = np.empty(cap, dtype=np.uint64)
        v = np.empty(cap, dtype=np.int32)
        lib().or_level_hash_dump(self._h, _ptr(k), _ptr(v))
        return k, v

    def lookup(self, q):
        if self.wide:
            q = np.ascontiguousarray(q, dtype=np.uint64).reshape(-1, 2)
            out = np.empty(len(q), dtype=np.int32)
            lib().or_level_lookup128(self._h, _ptr(q), len(q), _ptr(out))
            return out
        q = np.ascontiguousarray(q, dtype=np.uint64).ravel()
        out = np.empty(len(q), dtype=np.int32)
        lib().or_level_lookup(self._h, _ptr(q), len(q), _ptr(out))
        return out

    def neighbors(self):
        out = np.empty((self.n, 7), dtype=np.int32)
        lib().or_level_neighbors(self._h, _ptr(out))
        return out

    def father_cells(self):
        out = np.empty((self.n, 6, 2), dtype=np.int32)
        lib().or_level_father_cells(self._h, _ptr(out))
        return out

    # ---- fields
    def set_density(self, rho, rho_bar, four_pi_g=1.0):
        rho = np.ascontiguousarray(rho, dtype=np.float64).reshape(self.n, 8)
        lib().or_level_set_density(self._h, _ptr(rho), float(rho_bar), float(four_pi_g))

    def set_f(self, f):
        f = np.ascontiguousarray(f, dtype=np.float64).reshape(self.n, 8)
        lib().or_level_set_f(self._h, _ptr(f))

    def set_phi(self, phi):
        phi = np.ascontiguousarray(phi, dtype=np.float64).reshape(self.n, 8)
        lib().or_level_set_phi(self._h, _ptr(phi))

    def get_phi(self):
        out = np.empty((self.n, 8))
        lib().or_level_get_phi(self._h, _ptr(out))
        return out

    def get_f(self):
        out = np.empty((self.n, 8))
        lib().or_level_get_f(self._h, _ptr(out))
        return out

    def ghosts(self):
        lib().or_level_compute_ghosts(self._h)
        out = np.empty((self.n, 6, 4))
        lib().or_level_get_ghosts(self._h, _ptr(out))
        return out

    # ---- multigrid hierarchy
    @property
    def mg_depth(self):
        return lib().or_level_mg_depth(self._h)

    def mg_n_octs(self, m):
        return lib().or_level_mg_n_octs(self._h, m)

    def mg_lev(self, m):
        return lib().or_level_mg_lev(self._h, m)

    def mg_keys(self, m):
        if self.wide:
            out = np.empty((self.mg_n_octs(m), 2), dtype=np.uint64)
            lib().or_level_mg_keys128(self._h, m, _ptr(out))
            return out
        out = np.empty(self.mg_n_octs(m), dtype=np.uint64)
        lib().or_level_mg_keys(self._h, m, _ptr(out))
        return out

    def mg_active(self, m):
        out = np.empty((self.mg_n_octs(m), 8), dtype=np.uint8)
        lib().or_level_mg_active(self._h, m, _ptr(out))
        return out

    def mg_get(self, m, field):
        out = np.empty((self.mg_n_octs(m), 8))
        lib().or_level_mg_get(self._h, m, {"phi": 0, "f": 1, "r": 2}[field], _ptr(out))
        return out

    def mg_set(self, m, field, arr):
        arr = np.ascontiguousarray(arr, dtype=np.float64).reshape(self.mg_n_octs(m), 8)
        lib().or_level_mg_set(self._h, m, {"phi": 0, "f": 1, "r": 2}[field], _ptr(arr))

    # ---- steps
    def rb_sweeps(self, m=0, n=1, use_ghost=True):
        if use_ghost:
            lib().or_level_compute_ghosts(self._h)
        lib().or_rb_sweeps(self._h, m, n, int(use_ghost))

    def residual(self, m=0, use_ghost=True):
        if use_ghost:
            lib().or_level_compute_ghosts(self._h)
        return lib().or_residual(self._h, m, int(use_ghost))

    def restrict(self, m):
        lib().or_restrict(self._h, m)

    def prolong(self, m):
        lib().or_prolong(self._h, m)

    def coarse_solve(self, coarse_sweeps=4):
        lib().or_coarse_solve(self._h, coarse_sweeps)

    def solve(self, tol=1e-10, max_cycles=100, n_pre=2, n_post=2, coarse_sweeps=4, fixed_cycles=0,
              raise_on_error=True):
        p = params(tol, max_cycles, n_pre, n_post, coarse_sweeps, fixed_cycles)
        st = OrStats()
        rc = lib().or_level_solve(self._h, C.byref(p), C.byref(st))
        if rc != OR_OK and raise_on_error:
            raise OracleError(rc, "or_level_solve")
        return rc, _stats_dict(st)

    def solve_mixed(self, tol=1e-10, max_cycles=100, n_pre=2, n_post=2, coarse_sweeps=4, fixed_cycles=0,
                    inner_cycles=1, raise_on_error=True):
        p = params(tol, max_cycles, n_pre, n_post, coarse_sweeps, fixed_cycles)
        st = OrStats()
        rc = lib().or_level_solve_mixed(self._h, C.byref(p), inner_cycles, C.byref(st))
        if rc != OR_OK and raise_on_error:
            raise OracleError(rc, "or_level_solve_mixed")
        return rc, _stats_dict(st)


def _solve_pcg(self, tol=1e-10, max_cycles=100, n_pre=2, n_post=2, coarse_sweeps=4, fixed_cycles=0,
               raise_on_error=True):
    """Multigrid-preconditioned (flexible) conjugate gradients: cycles = CG
    iterations, one V-cycle preconditioner application each."""
    p = params(tol, max_cycles, n_pre, n_post, coarse_sweeps, fixed_cycles)
    st = OrStats()
    rc = lib().or_level_solve_pcg(self._h, C.byref(p), C.byref(st))
    if rc != OR_OK and raise_on_error:
        raise OracleError(rc, "or_level_solve_pcg")
    return rc, _stats_dict(st)


Level.solve_pcg = _solve_pcg


def _stats_dict(st):
    return {"cycles": st.cycles, "rel_initial": st.rel_initial, "rel_final": st.rel_final,
            "norm0": st.norm0, "rel_history": list(st.rel_history[:st.cycles])}
