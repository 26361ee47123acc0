"""CPU oracle for the fused metric-evolution chain (test infrastructure only).

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import
this package.  The CUDA library never links or calls it, and the two share no code.

``dtg_oracle.c`` is a plain per-point loop nest in IEEE binary64 (compiled without floating-point
contraction) that follows, in order: the inverse metric (adjugate / determinant), the Christoffel
symbols of Eq. 6, the covariant derivative of the shift (footnote to Listing 1), and the metric
evolution equation Eq. 5 of Lewis & Pfeiffer, arXiv:1804.10120; plus the hand-derived adjoint.

Array layout: 43 input arrays (g[6], dg[18] with dg[3p+k] = d_k g_p, K[6], alpha, beta[3],
dbeta[9] with dbeta[3i+j] = d_j beta_i) and 39 output arrays (ginv[6], gamma[18] with
gamma[6i+p(j,k)] = Gamma^i_jk, dbcov[9] with dbcov[3i+j] = nabla_j beta_i, dtg[6]); packed symmetric
order p = (00, 01, 02, 11, 12, 22).
"""
import ctypes
import os
import subprocess
import threading

import numpy as np

N_IN = 43
N_OUT = 39
_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dtg_oracle.c")
_SRC_EXPR = os.path.join(_HERE, "expr_oracle.c")
_SRC_FD = os.path.join(_HERE, "fd_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force=False):
    """Compile liboracle.so with gcc (plain C99, -O2, no FP contraction)."""
    srcs = [_SRC, _SRC_EXPR, _SRC_FD]
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= max(os.path.getmtime(f) for f in srcs):
        return _LIB
    tmp = _LIB + ".tmp%d" % os.getpid()
    subprocess.check_call(["gcc", "-std=c99", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
                           "-shared", "-o", tmp] + srcs + ["-lm"])
    os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB)
            P = ctypes.POINTER(ctypes.c_double)
            L.oracle_dtg_forward.argtypes = [ctypes.POINTER(P), ctypes.POINTER(P), ctypes.c_int64]
            L.oracle_dtg_backward.argtypes = [ctypes.POINTER(P), ctypes.POINTER(P), ctypes.POINTER(P),
                                              ctypes.c_int64]
            L.oracle_metric_det.argtypes = [ctypes.POINTER(P), P, ctypes.c_int64]
            L.oracle_expr.argtypes = [ctypes.c_int, ctypes.POINTER(P), ctypes.POINTER(P), ctypes.c_int64]
            L.oracle_expr.restype = ctypes.c_int
            L.oracle_fd_inputs.argtypes = [ctypes.POINTER(P), ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                           ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                           ctypes.POINTER(P)]
            L.oracle_fd_inputs.restype = ctypes.c_int
            for f in (L.oracle_dtg_forward, L.oracle_dtg_backward, L.oracle_metric_det):
                f.restype = ctypes.c_int
            _lib = L
    return _lib


def _table(arrays, count, n, allow_none=False):
    P = ctypes.POINTER(ctypes.c_double)
    tab = (P * count)()
    assert len(arrays) == count
    for s, a in enumerate(arrays):
        if a is None:
            assert allow_none
            tab[s] = P()
            continue
        assert a.dtype == np.float64 and a.shape[-1] == n and a.flags["C_CONTIGUOUS"]
        tab[s] = a.ctypes.data_as(P)
    return tab


def _rows(a, count):
    """Accept a [count, n] array or a sequence of count 1-D arrays; return a list of 1-D arrays."""
    if isinstance(a, np.ndarray) and a.ndim == 2:
        assert a.shape[0] == count
        return [np.ascontiguousarray(a[s]) for s in range(count)]
    assert len(a) == count
    return [None if r is None else np.ascontiguousarray(r, dtype=np.float64) for r in a]


def forward(inputs):
    """inputs: [43, n] float64 (or 43 arrays).  Returns a [39, n] float64 array."""
    rows = _rows(inputs, N_IN)
    n = rows[0].shape[0]
    out = np.empty((N_OUT, n), dtype=np.float64)
    orows = [out[s] for s in range(N_OUT)]
    rc = lib().oracle_dtg_forward(_table(rows, N_IN, n), _table(orows, N_OUT, n), n)
    if rc != 0:
        raise ValueError("oracle_dtg_forward rejected its arguments")
    return out


def backward(inputs, gout):
    """inputs: [43, n]; gout: 39 arrays of n (None = that output does not enter the functional).
    Returns the [43, n] gradient of sum(gout * out) with respect to the stored inputs."""
    rows = _rows(inputs, N_IN)
    n = rows[0].shape[0]
    grows = _rows(gout, N_OUT)
    gin = np.empty((N_IN, n), dtype=np.float64)
    girows = [gin[s] for s in range(N_IN)]
    rc = lib().oracle_dtg_backward(_table(rows, N_IN, n), _table(grows, N_OUT, n, allow_none=True),
                                   _table(girows, N_IN, n), n)
    if rc != 0:
        raise ValueError("oracle_dtg_backward rejected its arguments")
    return gin


def metric_det(g):
    rows = _rows(g, 6)
    n = rows[0].shape[0]
    det = np.empty(n, dtype=np.float64)
    rc = lib().oracle_metric_det(_table(rows, 6, n), det.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), n)
    if rc != 0:
        raise ValueError("oracle_metric_det rejected its arguments")
    return det


def forward_threaded(inputs, out, threads):
    """Forward over [43, n] -> preallocated [39, n] using `threads` host threads on disjoint point
    ranges (the C loop is called unchanged on each range; ctypes releases the GIL).  Used to time the
    oracle on all host cores."""
    n = inputs.shape[1]
    P = ctypes.POINTER(ctypes.c_double)
    L = lib()
    bounds = [n * t // threads for t in range(threads + 1)]

    def work(t):
        lo, hi = bounds[t], bounds[t + 1]
        if hi <= lo:
            return
        itab = (P * N_IN)(*[ctypes.cast(inputs[s].ctypes.data + 8 * lo, P) for s in range(N_IN)])
        otab = (P * N_OUT)(*[ctypes.cast(out[s].ctypes.data + 8 * lo, P) for s in range(N_OUT)])
        rc = L.oracle_dtg_forward(itab, otab, hi - lo)
        assert rc == 0

    assert inputs.dtype == np.float64 and inputs.flags["C_CONTIGUOUS"] and out.flags["C_CONTIGUOUS"]
    ths = [threading.Thread(target=work, args=(t,)) for t in range(threads)]
    for th in ths:
        th.start()
    for th in ths:
        th.join()
    return out


# Benchmark expressions of Sec. 5.1: (number of input arrays, number of output arrays) per equation.
EXPR_ARITY = {9: (3, 3), 10: (9, 9), 11: (27, 27), 12: (6, 3), 13: (9, 3), 14: (12, 3), 15: (6, 9),
              16: (9, 27), 17: (12, 81), 18: (90, 81), 19: (99, 81), 20: (108, 81), 21: (10, 6)}


def expr(eq, inputs):
    """Evaluate benchmark expression `eq` (9..21) literally; inputs [n_in, n] -> outputs [n_out, n]."""
    n_in, n_out = EXPR_ARITY[eq]
    rows = _rows(inputs, n_in)
    n = rows[0].shape[0]
    out = np.empty((n_out, n), dtype=np.float64)
    orows = [out[s] for s in range(n_out)]
    rc = lib().oracle_expr(eq, _table(rows, n_in, n), _table(orows, n_out, n), n)
    if rc != 0:
        raise ValueError("oracle_expr rejected its arguments")
    return out


def fd_inputs(fields16, shape, spacing, order):
    """The 43-array chain input table from the 16 arrays g[6], K[6], alpha, beta[3] on a periodic grid
    of shape (nx, ny, nz) (x fastest) with spacings (hx, hy, hz): derivatives by centred differences of
    the given order (2 or 4)."""
    rows = _rows(fields16, 16)
    nx, ny, nz = shape
    n = nx * ny * nz
    assert rows[0].shape[0] == n
    out = np.empty((N_IN, n), dtype=np.float64)
    orows = [out[s] for s in range(N_IN)]
    rc = lib().oracle_fd_inputs(_table(rows, 16, n), nx, ny, nz, spacing[0], spacing[1], spacing[2], order,
                                _table(orows, N_IN, n))
    if rc != 0:
        raise ValueError("oracle_fd_inputs rejected its arguments")
    return out
