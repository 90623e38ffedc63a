"""FP64 CPU oracle for the fibre-bundle FFT-convolution CG solve.

TEST INFRASTRUCTURE ONLY.  Only tests/, ``__graft_entry__.smoke()`` and the CPU
baseline leg of bench.py may import this package.  The CUDA library and its
Python binding never import it, and it imports nothing from them.

The arithmetic lives in ``oracle.c`` (plain C, double precision, each function
citing the passage of Gjerden, arXiv:1305.3625, that it follows); this module
compiles it with gcc on first use and wraps it with ctypes.

Parity status of each function (what pins it, in tests/test_oracle_*.py):
  G                 closed form of the self term and quadrature of Eq. 1c
  G_cell            self term closed form, adaptive quadrature of Eq. 1c,
                    additivity over 3x3 and 5x5 blocks of cells, far field
  fft, fft2         naive DFT, Parseval, inverse round trip
  conv_direct       delta response, translation invariance, symmetry,
                    positivity, quadrature-built Eq. 1c operator at small L
  conv_fft          conv_direct (independent algorithm), L <= 48
  spectrum          realness (even kernel) and DC = sum of the kernel table
  cg                L = 1 closed form, dense Cholesky and LAPACK solves
  cholesky_solve    LAPACK solve (library routine) on random SPD matrices
  masked_loop       brute force with dense re-solves, L <= 6
  front             brute force over every column of small masks
"""
from __future__ import annotations

import contextlib
import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_green_lock = threading.RLock()
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)
_ucp = ctypes.POINTER(ctypes.c_ubyte)
_lp = ctypes.POINTER(ctypes.c_long)
_ip = ctypes.POINTER(ctypes.c_int)


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (plain gcc, OpenMP over rows only)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", "-fno-fast-math", "-o", tmp, _SRC, "-lquadmath", "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.orc_G.restype = ctypes.c_double
            lib.orc_G.argtypes = [ctypes.c_long, ctypes.c_long]
            lib.orc_G_cell.restype = ctypes.c_double
            lib.orc_G_cell.argtypes = [ctypes.c_long, ctypes.c_long]
            lib.orc_set_green.argtypes = [ctypes.c_int, ctypes.c_long]
            lib.orc_padded_side.argtypes = [ctypes.c_int]
            lib.orc_kernel_table.argtypes = [ctypes.c_int, _dp]
            lib.orc_conv_direct_at.restype = ctypes.c_double
            lib.orc_conv_direct_at.argtypes = [ctypes.c_int, _dp, ctypes.c_int, ctypes.c_int]
            lib.orc_conv_direct.argtypes = [ctypes.c_int, _dp, _dp]
            lib.orc_dense_operator.argtypes = [ctypes.c_int, _dp, _dp]
            lib.orc_fft.argtypes = [ctypes.c_int, _dp, _dp, ctypes.c_int]
            lib.orc_fft2.argtypes = [ctypes.c_int, _dp, _dp, ctypes.c_int]
            lib.orc_spectrum.argtypes = [ctypes.c_int, _dp, _dp]
            lib.orc_conv_fft.argtypes = [ctypes.c_int, _dp, _dp]
            lib.orc_apply_A.argtypes = [ctypes.c_int, _dp, _ucp, _dp, _dp]
            lib.orc_cg.argtypes = [ctypes.c_int, _dp, _dp, _dp, _ucp, ctypes.c_double,
                                   ctypes.c_int, _ip, _dp]
            lib.orc_cholesky_solve.argtypes = [ctypes.c_int, _dp, _dp, _dp]
            lib.orc_argmax_ratio.restype = ctypes.c_long
            lib.orc_argmax_ratio.argtypes = [ctypes.c_long, _dp, _dp, _ucp, _dp]
            lib.orc_front.argtypes = [ctypes.c_int, _ucp, _ip, _ip]
            lib.orc_masked_loop.argtypes = [ctypes.c_int, _dp, _dp, _dp, _ucp, _dp,
                                            ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                            _lp, _dp, _ip]
            _lib = lib
    return _lib


def _d(a):
    return a.ctypes.data_as(_dp)


def _f64(a, n=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if n is not None and a.size != n:
        raise ValueError(f"expected {n} values, got {a.size}")
    return a


def _mask(mask, n):
    if mask is None:
        return None, None
    m = np.ascontiguousarray(mask, dtype=np.uint8)
    if m.size != n:
        raise ValueError("mask size")
    return m, m.ctypes.data_as(_ucp)


def _check(rc, what):
    if rc < 0:
        raise RuntimeError(f"oracle {what} failed with {rc}")
    return rc


def G(dx: int, dy: int) -> float:
    """Green's function of Eq. 1c (a = 1, (1-nu^2)/E = 1), point form + exact self term."""
    return _load().orc_G(int(dx), int(dy))


GREEN_POINT, GREEN_CELL = 0, 1


def G_cell(dx: int, dy: int) -> float:
    """The cell integral of Eq. 1c itself for offset (dx, dy) (closed-form
    antiderivative at the cell corners, quad precision)."""
    return _load().orc_G_cell(int(dx), int(dy))


@contextlib.contextmanager
def use_green(kind: int, L: int = 1):
    """Make the oracle calls inside use GREEN_POINT (the default) or
    GREEN_CELL (Eq. 1c's cell integral, tabulated for offsets below L)."""
    lib = _load()
    with _green_lock:
        _check(lib.orc_set_green(int(kind), int(max(L, 1))), "set_green")
        try:
            yield
        finally:
            lib.orc_set_green(GREEN_POINT, 1)


def padded_side(L: int) -> int:
    return _check(_load().orc_padded_side(int(L)), "padded_side")


def kernel_table(L: int) -> np.ndarray:
    M = padded_side(L)
    k = np.empty(M * M)
    _check(_load().orc_kernel_table(L, _d(k)), "kernel_table")
    return k.reshape(M, M)


def conv_direct(L: int, x) -> np.ndarray:
    x = _f64(x, L * L)
    y = np.empty(L * L)
    _check(_load().orc_conv_direct(L, _d(x), _d(y)), "conv_direct")
    return y


def conv_direct_at(L: int, x, iy: int, ix: int) -> float:
    x = _f64(x, L * L)
    return _load().orc_conv_direct_at(L, _d(x), int(iy), int(ix))


def dense_operator(L: int, s=None) -> np.ndarray:
    N = L * L
    A = np.empty(N * N)
    sp = None
    if s is not None:
        s = _f64(s, N)
        sp = _d(s)
    _check(_load().orc_dense_operator(L, sp, _d(A)), "dense_operator")
    return A.reshape(N, N)


def fft(x, sign: int = -1) -> np.ndarray:
    x = np.asarray(x, dtype=np.complex128)
    re = np.ascontiguousarray(x.real.copy())
    im = np.ascontiguousarray(x.imag.copy())
    _check(_load().orc_fft(x.size, _d(re), _d(im), sign), "fft")
    return re + 1j * im


def fft2(x, sign: int = -1) -> np.ndarray:
    x = np.asarray(x, dtype=np.complex128)
    M = x.shape[0]
    assert x.shape == (M, M)
    re = np.ascontiguousarray(x.real.copy())
    im = np.ascontiguousarray(x.imag.copy())
    _check(_load().orc_fft2(M, _d(re), _d(im), sign), "fft2")
    return (re + 1j * im).reshape(M, M)


def spectrum(L: int) -> np.ndarray:
    """Complex FFT2(k)/M^2 of the circulant-embedded kernel (M x M)."""
    M = padded_side(L)
    re = np.empty(M * M)
    im = np.empty(M * M)
    _check(_load().orc_spectrum(L, _d(re), _d(im)), "spectrum")
    return (re + 1j * im).reshape(M, M)


def conv_fft(L: int, x) -> np.ndarray:
    x = _f64(x, L * L)
    y = np.empty(L * L)
    _check(_load().orc_conv_fft(L, _d(x), _d(y)), "conv_fft")
    return y


def apply_A(L: int, s, x, mask=None) -> np.ndarray:
    N = L * L
    s, x = _f64(s, N), _f64(x, N)
    m, mp = _mask(mask, N)
    q = np.empty(N)
    _check(_load().orc_apply_A(L, _d(s), mp, _d(x), _d(q)), "apply_A")
    return q


def cg(L: int, s, b, x0=None, mask=None, rtol: float = 1e-10, maxit: int = 100000):
    """Returns (x, status, iterations, recomputed relative residual)."""
    N = L * L
    s, b = _f64(s, N), _f64(b, N)
    x = np.zeros(N) if x0 is None else _f64(x0, N).copy()
    m, mp = _mask(mask, N)
    it = ctypes.c_int(0)
    rel = ctypes.c_double(0.0)
    rc = _check(_load().orc_cg(L, _d(s), _d(b), _d(x), mp, float(rtol), int(maxit),
                               ctypes.byref(it), ctypes.byref(rel)), "cg")
    return x, rc, it.value, rel.value


def cholesky_solve(A, b) -> np.ndarray:
    A = np.ascontiguousarray(A, dtype=np.float64)
    n = A.shape[0]
    b = _f64(b, n)
    x = np.empty(n)
    _check(_load().orc_cholesky_solve(n, _d(A), _d(b), _d(x)), "cholesky_solve")
    return x


def argmax_ratio(x, t, mask=None):
    x = _f64(x)
    t = _f64(t, x.size)
    m, mp = _mask(mask, x.size)
    r = ctypes.c_double(0.0)
    k = _load().orc_argmax_ratio(x.size, _d(x), _d(t), mp, ctypes.byref(r))
    return k, r.value


def masked_loop(L: int, s, b, t, steps: int, x0=None, mask=None, rtol: float = 1e-10,
                maxit: int = 100000):
    """Returns dict(x, mask, picks, ratios, iters) after ``steps`` removals."""
    N = L * L
    s, b, t = _f64(s, N), _f64(b, N), _f64(t, N)
    x = np.zeros(N) if x0 is None else _f64(x0, N).copy()
    m = np.ones(N, np.uint8) if mask is None else np.ascontiguousarray(mask, np.uint8).copy()
    picks = np.full(steps, -1, dtype=np.int64)
    ratios = np.zeros(steps)
    iters = np.zeros(steps, dtype=np.int32)
    _check(_load().orc_masked_loop(L, _d(s), _d(b), _d(t), m.ctypes.data_as(_ucp), _d(x),
                                   int(steps), float(rtol), int(maxit),
                                   picks.ctypes.data_as(_lp), _d(ratios),
                                   iters.ctypes.data_as(_ip)), "masked_loop")
    return {"x": x, "mask": m, "picks": picks, "ratios": ratios, "iters": iters}


def front(L: int, mask):
    """(first_intact, damage_end) per column of the L x L mask."""
    m = np.ascontiguousarray(mask, dtype=np.uint8)
    if m.size != L * L:
        raise ValueError("mask size")
    fi = np.empty(L, dtype=np.int32)
    de = np.empty(L, dtype=np.int32)
    _check(_load().orc_front(L, m.ctypes.data_as(_ucp), fi.ctypes.data_as(_ip), de.ctypes.data_as(_ip)),
           "front")
    return fi, de
