"""CPU oracle for Z[x] products -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
(reference) leg may import this package.  The product path never imports it,
and it imports nothing from the product package.

Contents:

* ``schoolbook.c`` -- the plain definition h_k = sum_{i+j=k} f_i g_j over exact
  multi-limb integers (Harvey, Sec. 3), multithreaded over k, plus the
  (Z/pZ)[x] product of Sec. 4 and the plain bivariate product in
  (Z/pZ)[x, y] of Sec. 2.  Loaded here through ctypes.
* ``pyref`` -- a pure-Python twin of the same definition for tiny sizes.
* ``ks_steps`` -- a step model that runs each Kronecker-substitution variant
  (Sec. 3.1-3.4) on Python integers in any base, exposing the intermediates
  (evaluations, products, combined halves, the digits u_i, w_i and the
  reconstruction's alpha, beta, delta, epsilon).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compiles ``schoolbook.c`` into ``liboracle.so`` (plain gcc, no GPU)."""
    src = os.path.join(_HERE, "schoolbook.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        tmp = _SO + ".tmp.%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-Wall", "-shared", "-fPIC",
                               "-pthread", "-o", tmp, src])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_SO)
        u64p = ctypes.POINTER(ctypes.c_uint64)
        i64p = ctypes.POINTER(ctypes.c_int64)
        i64 = ctypes.c_int64
        ci = ctypes.c_int
        lib.oracle_mul.argtypes = [u64p, u64p, i64, u64p, i64, ci, ci, ci, ci]
        lib.oracle_mul.restype = ci
        lib.oracle_coeffs.argtypes = [u64p, i64p, i64, u64p, i64, u64p, i64, ci, ci, ci, ci]
        lib.oracle_coeffs.restype = ci
        lib.oracle_mul_mod.argtypes = [u64p, u64p, i64, u64p, i64, ctypes.c_uint64, ci]
        lib.oracle_mul_mod.restype = ci
        lib.oracle_mul_biv_mod.argtypes = [u64p, u64p, u64p, i64, i64, ctypes.c_uint64, ci]
        lib.oracle_mul_biv_mod.restype = ci
        _lib = lib
    return _lib


def _ptr(a: np.ndarray, ctype=ctypes.c_uint64):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def default_threads() -> int:
    return os.cpu_count() or 1


def ceil_log2(n: int) -> int:
    """Smallest e with 2^e >= n (n >= 1)."""
    return (n - 1).bit_length()


def out_limbs(len_f: int, len_g: int, coeff_bits: int, is_signed: bool) -> int:
    """Limbs per output coefficient: ceil((2b + e + signed) / 64), e = ceil(log2 min(Lf, Lg)).

    Sec. 3 bounds |h_k| by min(Lf, Lg) (2^b - 1)^2 < 2^(2b+e) (unsigned); a signed
    value needs one more bit for its sign.
    """
    e = ceil_log2(min(len_f, len_g))
    return (2 * coeff_bits + e + (1 if is_signed else 0) + 63) // 64


def mul(f: np.ndarray, g: np.ndarray, coeff_bits: int, is_signed: bool,
        n_limbs_out: int | None = None, threads: int | None = None) -> np.ndarray:
    """Exact h = f g.  f, g: (L, in_limbs) uint64.  Returns (Lf+Lg-1, out_limbs) uint64."""
    f = np.ascontiguousarray(f, dtype=np.uint64)
    g = np.ascontiguousarray(g, dtype=np.uint64)
    lf, lg = f.shape[0], g.shape[0]
    ol = n_limbs_out or out_limbs(lf, lg, coeff_bits, is_signed)
    h = np.zeros((lf + lg - 1, ol), dtype=np.uint64)
    rc = _load().oracle_mul(_ptr(h), _ptr(f), lf, _ptr(g), lg, coeff_bits, int(is_signed), ol,
                            threads or default_threads())
    if rc != 0:
        raise ValueError("oracle_mul failed: %d" % rc)
    return h


def coeffs(ks, f: np.ndarray, g: np.ndarray, coeff_bits: int, is_signed: bool,
           n_limbs_out: int | None = None, threads: int | None = None) -> np.ndarray:
    """Exact h_k for the listed k only.  Returns (len(ks), out_limbs) uint64."""
    f = np.ascontiguousarray(f, dtype=np.uint64)
    g = np.ascontiguousarray(g, dtype=np.uint64)
    ks = np.ascontiguousarray(ks, dtype=np.int64)
    lf, lg = f.shape[0], g.shape[0]
    ol = n_limbs_out or out_limbs(lf, lg, coeff_bits, is_signed)
    out = np.zeros((ks.size, ol), dtype=np.uint64)
    rc = _load().oracle_coeffs(_ptr(out), _ptr(ks, ctypes.c_int64), ks.size, _ptr(f), lf,
                               _ptr(g), lg, coeff_bits, int(is_signed), ol,
                               threads or default_threads())
    if rc != 0:
        raise ValueError("oracle_coeffs failed: %d" % rc)
    return out


def mul_mod(f: np.ndarray, g: np.ndarray, p: int, threads: int | None = None) -> np.ndarray:
    """h_k = sum f_i g_j mod p for residues in [0, p).  f, g: (L,) or (L, 1) uint64."""
    f = np.ascontiguousarray(f, dtype=np.uint64).reshape(-1)
    g = np.ascontiguousarray(g, dtype=np.uint64).reshape(-1)
    h = np.zeros(f.size + g.size - 1, dtype=np.uint64)
    rc = _load().oracle_mul_mod(_ptr(h), _ptr(f), f.size, _ptr(g), g.size, p,
                                threads or default_threads())
    if rc != 0:
        raise ValueError("oracle_mul_mod failed: %d" % rc)
    return h.reshape(-1, 1)


def mul_biv_mod(f: np.ndarray, g: np.ndarray, p: int, threads: int | None = None) -> np.ndarray:
    """The plain product in (Z/pZ)[x, y] (Sec. 2): f, g are (ly, lx) uint64 arrays
    of residues, row i the coefficients of y^i; returns (2 ly - 1, 2 lx - 1)."""
    f = np.ascontiguousarray(f, dtype=np.uint64)
    g = np.ascontiguousarray(g, dtype=np.uint64)
    if f.ndim != 2 or f.shape != g.shape:
        raise ValueError("f and g must be (ly, lx) arrays of the same shape")
    ly, lx = f.shape
    h = np.zeros((2 * ly - 1, 2 * lx - 1), dtype=np.uint64)
    rc = _load().oracle_mul_biv_mod(_ptr(h), _ptr(f), _ptr(g), lx, ly, p,
                                    threads or default_threads())
    if rc != 0:
        raise ValueError("oracle_mul_biv_mod failed: %d" % rc)
    return h
