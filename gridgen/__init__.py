"""Seeded, counter-based synthetic grid inputs (no step of the method's arithmetic lives here).

Both the CPU oracle and the CUDA library are fed from these arrays.  See gridgen.c for the
generator's definition and the value distributions.
"""
import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gridgen.c")
_LIB = os.path.join(_HERE, "libgridgen.so")
_lock = threading.Lock()
_lib = None

N_IN = 43
# stream-id spacing between grids / fields, so that no two fields share a stream
STREAMS_PER_FIELD = 64


def build(force=False):
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + ".tmp%d" % os.getpid()
    subprocess.check_call(["gcc", "-std=c99", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
                           "-shared", "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB)
            P = ctypes.POINTER(ctypes.c_double)
            u64, i64, d = ctypes.c_uint64, ctypes.c_int64, ctypes.c_double
            L.gridgen_bits.argtypes = [u64, u64, u64]
            L.gridgen_bits.restype = u64
            L.gridgen_uniform.argtypes = [u64, u64, i64, i64, d, d, P]
            L.gridgen_normal.argtypes = [u64, u64, i64, i64, d, d, P]
            L.gridgen_random_grid.argtypes = [u64, u64, i64, i64, ctypes.POINTER(P)]
            L.gridgen_conformal_grid.argtypes = [i64, d, d, i64, i64, ctypes.POINTER(P)]
            L.gridgen_periodic_fields.argtypes = [u64, i64, i64, i64, i64, i64, ctypes.POINTER(P)]
            L.gridgen_periodic_fields.restype = None
            for f in (L.gridgen_uniform, L.gridgen_normal, L.gridgen_random_grid, L.gridgen_conformal_grid):
                f.restype = None
            _lib = L
    return _lib


def _ptr(a, offset=0):
    return ctypes.cast(a.ctypes.data + 8 * offset, ctypes.POINTER(ctypes.c_double))


def _chunks(n, threads):
    threads = max(1, min(threads, (n + 65535) // 65536))
    return [(n * t // threads, n * (t + 1) // threads) for t in range(threads)]


def _run(jobs):
    ths = [threading.Thread(target=j) for j in jobs]
    for t in ths:
        t.start()
    for t in ths:
        t.join()


def default_threads():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def random_grid(n, seed, stream_base=0, out=None, threads=None):
    """[43, n] float64 inputs with the random-grid recipe (g = delta + 0.1 S, S ~ U[-1,1]; dg ~ U[-0.1,0.1];
    K, beta, dbeta ~ N(0, 0.1); alpha ~ U[0.5, 1.5]).  `out` may be any C-contiguous [43, n] float64
    array (e.g. a pinned buffer viewed through numpy)."""
    if out is None:
        out = np.empty((N_IN, n), dtype=np.float64)
    assert out.shape == (N_IN, n) and out.dtype == np.float64 and out.flags["C_CONTIGUOUS"]
    L = lib()
    P = ctypes.POINTER(ctypes.c_double)

    def job(lo, hi):
        def f():
            tab = (P * N_IN)(*[_ptr(out[s], lo) for s in range(N_IN)])
            L.gridgen_random_grid(seed, stream_base, lo, hi - lo, tab)
        return f
    _run([job(lo, hi) for lo, hi in _chunks(n, threads or default_threads()) if hi > lo])
    return out


def conformal_grid(side, lo=-4.0, hi=4.0, out=None, threads=None):
    """[43, side^3] float64 inputs of the conformally flat metric psi = 1 + 0.5 exp(-r^2) on [lo, hi]^3."""
    n = side ** 3
    if out is None:
        out = np.empty((N_IN, n), dtype=np.float64)
    L = lib()
    P = ctypes.POINTER(ctypes.c_double)

    def job(a, b):
        def f():
            tab = (P * N_IN)(*[_ptr(out[s], a) for s in range(N_IN)])
            L.gridgen_conformal_grid(side, lo, hi, a, b - a, tab)
        return f
    _run([job(a, b) for a, b in _chunks(n, threads or default_threads()) if b > a])
    return out


def normal(n, seed, stream, sigma=1.0, mean=0.0, offset=0):
    out = np.empty(n, dtype=np.float64)
    lib().gridgen_normal(seed, stream, offset, n, mean, sigma, _ptr(out))
    return out


def uniform(n, seed, stream, lo=0.0, hi=1.0, offset=0):
    out = np.empty(n, dtype=np.float64)
    lib().gridgen_uniform(seed, stream, offset, n, lo, hi, _ptr(out))
    return out


def normal_fields(count, n, seed, stream_base, sigma=1.0):
    """[count, n] independent N(0, sigma) fields on streams stream_base .. stream_base+count-1."""
    out = np.empty((count, n), dtype=np.float64)
    L = lib()
    _run([(lambda s: (lambda: L.gridgen_normal(seed, stream_base + s, 0, n, 0.0, sigma, _ptr(out[s]))))(s)
          for s in range(count)])
    return out


def subgrid_sides(count, seed, lo=8, hi=48, stream=4095):
    """`count` integer sides uniform on [lo, hi] (multi-domain grid sizes N_d = side^3)."""
    L = lib()
    span = hi - lo + 1
    return [lo + int(L.gridgen_bits(seed, stream, d) % span) for d in range(count)]


def periodic_fields(shape, seed, out=None, threads=None):
    """[16, nx*ny*nz] smooth periodic fields g[6], K[6], alpha, beta[3] on the unit box (x fastest)."""
    nx, ny, nz = shape
    n = nx * ny * nz
    if out is None:
        out = np.empty((16, n), dtype=np.float64)
    L = lib()
    P = ctypes.POINTER(ctypes.c_double)

    def job(a, b):
        def f():
            tab = (P * 16)(*[_ptr(out[s], a) for s in range(16)])
            L.gridgen_periodic_fields(seed, nx, ny, nz, a, b - a, tab)
        return f
    _run([job(a, b) for a, b in _chunks(n, threads or default_threads()) if b > a])
    return out
