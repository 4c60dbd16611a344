"""FP64 CPU oracle for the 3-D DFT -- test infrastructure only.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA library
in ``paper_1506_07933_gb300``; the two meet only in the tests, on inputs drawn
from the seeded generators of ``paper_1506_07933_gb300.synth`` (which hold none
of the transform's arithmetic).

The arithmetic lives in ``oracle.c`` (plain C, FP64, long-double unit roots);
this module only marshals numpy arrays into it.  What each function computes
and which passage of AccFFT it follows is stated in ``oracle.c``:

* forward c2c, unscaled, axes N2, N1, N0 (Algorithm 1, left column);
* backward c2c, axes N0, N1, N2 (Algorithm 1, right column), times 1/N
  (Section 2, footnote 2);
* r2c = c2c of the real field with k2 = 0 .. n2/2 kept; c2r its inverse on
  Hermitian-consistent input (Section 1 feature list: R2C, C2C, C2R).

``method="naive"`` is the O(n^2) definition per axis (long-double sums);
``method="fft"`` is a recursive mixed-radix (2, 3, 5) Cooley-Tukey, the
large-size oracle and the timed CPU baseline.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_LIB32 = os.path.join(_HERE, "liboracle_f32.so")
_lib = None
_lib32 = None

METHODS = {"naive": 0, "fft": 1}


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so with gcc (OpenMP on), and the same source with
    -DORC_REAL=float into liboracle_f32.so (the FP32 CPU baseline; never a parity reference)."""
    for lib, extra in ((_LIB, []), (_LIB32, ["-DORC_REAL=float"])):
        if force or not os.path.exists(lib) or os.path.getmtime(lib) < os.path.getmtime(_SRC):
            tmp = lib + ".tmp.%d" % os.getpid()
            subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-Wall", *extra,
                                   "-o", tmp, _SRC, "-lm"])
            os.replace(tmp, lib)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        i64, dp, c_int = ctypes.c_int64, ctypes.c_void_p, ctypes.c_int
        lib.orc_dft_axis.argtypes = [dp, i64, i64, i64, c_int, c_int, c_int]
        lib.orc_c2c_3d.argtypes = [dp, dp, i64, i64, i64, c_int, c_int, c_int]
        lib.orc_r2c_3d.argtypes = [dp, dp, i64, i64, i64, c_int, c_int]
        lib.orc_dft_bins.argtypes = [dp, c_int, i64, i64, i64, dp, i64, dp, c_int]
        lib.orc_c2r_3d.argtypes = [dp, dp, i64, i64, i64, c_int, c_int]
        for f in (lib.orc_dft_axis, lib.orc_c2c_3d, lib.orc_r2c_3d, lib.orc_c2r_3d, lib.orc_dft_bins):
            f.restype = c_int
        lib.orc_max_threads.restype = c_int
        _lib = lib
    return _lib


def _load32():
    """The FP32 build: the same entry points on float data."""
    global _lib32
    if _lib32 is None:
        build()
        lib = ctypes.CDLL(_LIB32)
        i64, dp, c_int = ctypes.c_int64, ctypes.c_void_p, ctypes.c_int
        lib.orc_r2c_3d.argtypes = [dp, dp, i64, i64, i64, c_int, c_int]
        lib.orc_c2r_3d.argtypes = [dp, dp, i64, i64, i64, c_int, c_int]
        lib.orc_r2c_3d.restype = lib.orc_c2r_3d.restype = c_int
        _lib32 = lib
    return _lib32


def r2c_f32(x, nthreads=None) -> np.ndarray:
    """r2c by the FP32 build of the same source (recursive mixed-radix engine): the CPU baseline
    of FP32 transforms.  float32 [n0, n1, n2] -> complex64 [n0, n1, n2//2 + 1]."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    n0, n1, n2 = x.shape
    out = np.empty((n0, n1, n2 // 2 + 1), dtype=np.complex64)
    _check(_load32().orc_r2c_3d(x.ctypes.data, out.ctypes.data, n0, n1, n2, METHODS["fft"], _threads(nthreads)))
    return out


def c2r_f32(X, n2: int, nthreads=None) -> np.ndarray:
    """c2r by the FP32 build (x 1/N): complex64 [n0, n1, n2//2 + 1] -> float32 [n0, n1, n2]."""
    X = np.ascontiguousarray(X, dtype=np.complex64)
    n0, n1, nh = X.shape
    if nh != n2 // 2 + 1:
        raise ValueError("half-spectrum width must be n2//2 + 1")
    out = np.empty((n0, n1, n2), dtype=np.float32)
    _check(_load32().orc_c2r_3d(X.ctypes.data, out.ctypes.data, n0, n1, n2, METHODS["fft"], _threads(nthreads)))
    return out


def max_threads() -> int:
    return int(_load().orc_max_threads())


def _threads(nthreads):
    return max_threads() if nthreads is None else int(nthreads)


def _check(status: int):
    if status != 0:
        raise RuntimeError("oracle error %d" % status)


def _c128(x):
    return np.ascontiguousarray(x, dtype=np.complex128)


def c2c(x, direction: int = -1, method: str = "fft", nthreads=None) -> np.ndarray:
    """3-D c2c of a complex [n0, n1, n2] array; direction -1 forward, +1 backward (x 1/N)."""
    x = _c128(x)
    if x.ndim != 3:
        raise ValueError("expected a 3-D array")
    out = np.empty_like(x)
    n0, n1, n2 = x.shape
    _check(_load().orc_c2c_3d(x.ctypes.data, out.ctypes.data, n0, n1, n2, int(direction),
                              METHODS[method], _threads(nthreads)))
    return out


def r2c(x, method: str = "fft", nthreads=None) -> np.ndarray:
    """3-D r2c of a real [n0, n1, n2] array -> complex [n0, n1, n2//2 + 1]."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    if x.ndim != 3:
        raise ValueError("expected a 3-D array")
    n0, n1, n2 = x.shape
    out = np.empty((n0, n1, n2 // 2 + 1), dtype=np.complex128)
    _check(_load().orc_r2c_3d(x.ctypes.data, out.ctypes.data, n0, n1, n2,
                              METHODS[method], _threads(nthreads)))
    return out


def c2r(X, n2: int, method: str = "fft", nthreads=None) -> np.ndarray:
    """3-D c2r of a half spectrum [n0, n1, n2//2 + 1] -> real [n0, n1, n2] (x 1/N)."""
    X = _c128(X)
    n0, n1, nh = X.shape
    if nh != n2 // 2 + 1:
        raise ValueError("half-spectrum width must be n2//2 + 1")
    out = np.empty((n0, n1, n2), dtype=np.float64)
    _check(_load().orc_c2r_3d(X.ctypes.data, out.ctypes.data, n0, n1, n2,
                              METHODS[method], _threads(nthreads)))
    return out


def dft_axis(x, axis: int, sign: int = -1, method: str = "fft", nthreads=None) -> np.ndarray:
    """Unscaled 1-D DFT of every line of a complex N-d array along ``axis``."""
    x = _c128(x).copy()
    shape = x.shape
    axis = axis % x.ndim
    outer = int(np.prod(shape[:axis], dtype=np.int64))
    inner = int(np.prod(shape[axis + 1:], dtype=np.int64))
    _check(_load().orc_dft_axis(x.ctypes.data, outer, shape[axis], inner, int(sign),
                                METHODS[method], _threads(nthreads)))
    return x


def dft_bins(x, ks, nthreads=None) -> np.ndarray:
    """Forward 3-D DFT bins X[k] for the (k0, k1, k2) rows of ``ks``, by the definition.

    ``x`` is a real or complex [n0, n1, n2] array; costs O(N) per bin.
    """
    is_real = not np.iscomplexobj(x)
    x = np.ascontiguousarray(x, dtype=np.float64 if is_real else np.complex128)
    ks = np.ascontiguousarray(np.asarray(ks, dtype=np.int64).reshape(-1, 3))
    n0, n1, n2 = x.shape
    out = np.empty(len(ks), dtype=np.complex128)
    _check(_load().orc_dft_bins(x.ctypes.data, int(is_real), n0, n1, n2, ks.ctypes.data, len(ks),
                                out.ctypes.data, _threads(nthreads)))
    return out


def wavenumbers(n: int) -> np.ndarray:
    """Integer wavenumbers of the periodic grid x_j = 2 pi j / n on [0, 2 pi): m for m <= n/2,
    else m - n (the Nyquist bin's sign does not matter for |k|^2)."""
    m = np.arange(n)
    return np.where(2 * m > n, m - n, m)


def poisson(f, method: str = "fft", nthreads=None) -> np.ndarray:
    """u with -Lap u = f on [0, 2 pi)^3, zero mean: u_hat = f_hat / |k|^2, u_hat(0) = 0.

    Spectral operator on the r2c spectrum (AccFFT Section 1 names fast spectral operators; the
    operator, grid and zero-mean convention are the readings stated for the serving workload)."""
    f = np.ascontiguousarray(f, dtype=np.float64)
    n0, n1, n2 = f.shape
    F = r2c(f, method, nthreads)
    k0 = wavenumbers(n0)[:, None, None]
    k1 = wavenumbers(n1)[None, :, None]
    k2 = np.arange(n2 // 2 + 1)[None, None, :]
    K = (k0 * k0 + k1 * k1 + k2 * k2).astype(np.float64)
    with np.errstate(divide="ignore", invalid="ignore"):
        U = np.where(K > 0, F / np.where(K > 0, K, 1.0), 0.0)
    return c2r(U, n2, method, nthreads)


def rel_l2(y, ref) -> float:
    """||y - ref||_2 / ||ref||_2 with float64 pairwise sums, in chunks of 2**24 values
    (both arrays divided by max|ref| first, so that squares neither overflow nor underflow)."""
    y = np.asarray(y).ravel()
    ref = np.asarray(ref).ravel()
    if y.shape != ref.shape:
        raise ValueError("shape mismatch %s vs %s" % (y.shape, ref.shape))
    num = den = 0.0
    step = 1 << 24
    scale = 0.0
    for i in range(0, ref.size, step):
        scale = max(scale, float(np.max(np.abs(ref[i:i + step]))) if ref[i:i + step].size else 0.0)
    scale = scale if scale > 0 and np.isfinite(scale) else 1.0
    for i in range(0, ref.size, step):
        r = ref[i:i + step].astype(np.complex128) / scale
        d = y[i:i + step].astype(np.complex128) / scale - r
        num += float(np.sum(d.real * d.real + d.imag * d.imag))
        den += float(np.sum(r.real * r.real + r.imag * r.imag))
    if den == 0:
        return float(np.sqrt(num))
    return float(np.sqrt(num / den))
