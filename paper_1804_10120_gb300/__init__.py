"""Python binding of the tl C ABI (include/tl.h): argument marshalling only.

Every step of the metric-evolution chain runs in the CUDA library ``libtl.so`` built from ``csrc/``
for sm_103a; this module only turns torch tensors into component pointer tables and calls the C
entry points of the same names.  There is no fallback: if the library is missing or the device is
not an sm_103 GPU, calls raise ``TLError``.

Array convention: a [43, n] tensor holds the inputs (g[6], dg[18], K[6], alpha, beta[3], dbeta[9])
and a [39, n] tensor the outputs (ginv[6], gamma[18], dbcov[9], dtg[6]); any sequence of 43 (39)
1-D tensors with unit stride works as well.
"""
import ctypes
import os
import threading

from . import build as _build

N_IN = 43
N_OUT = 39
TL_F64, TL_F32, TL_F64_FF = 0, 1, 2
DTYPES = {"f64": TL_F64, "f32": TL_F32, "f64_ff": TL_F64_FF}
STATUS = {0: "TL_OK", 1: "TL_ERR_INVALID_ARG", 2: "TL_ERR_ALIGNMENT", 3: "TL_ERR_UNSUPPORTED",
          4: "TL_ERR_CUDA", 5: "TL_ERR_TIMEOUT", 6: "TL_ERR_PLAN_MISMATCH"}

_lib = None
_lock = threading.Lock()


class TLError(RuntimeError):
    def __init__(self, status, message):
        super().__init__("%s: %s" % (STATUS.get(status, status), message))
        self.status = status


PtrTab43 = ctypes.c_void_p * N_IN
PtrTab39 = ctypes.c_void_p * N_OUT


def library_path():
    return _build.LIB


def lib():
    """Load libtl.so (built in-tree by build()); raises if it is absent."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.LIB
            if not os.path.exists(path):
                raise TLError(3, "libtl.so is not built (%s); call paper_1804_10120_gb300.build.build()" % path)
            L = ctypes.CDLL(path)
            vp, i64, i32, sz = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_size_t
            L.tl_dtg_forward.argtypes = [vp, vp, i64, i32, vp]
            L.tl_dtg_backward.argtypes = [vp, vp, vp, i64, i32, vp]
            L.tl_dtg_forward_backward.argtypes = [vp, vp, vp, vp, i64, i32, vp]
            L.tl_dtg_forward_host.argtypes = [vp, vp, i64, i32, vp, sz, vp]
            L.tl_dtg_host_workspace_bytes.argtypes = [i64, i32]
            L.tl_dtg_host_workspace_bytes.restype = sz
            for f in (L.tl_dtg_forward, L.tl_dtg_backward, L.tl_dtg_forward_backward, L.tl_dtg_forward_host):
                f.restype = i32
            L.tl_status_string.argtypes = [i32]
            L.tl_status_string.restype = ctypes.c_char_p
            L.tl_last_error.argtypes = []
            L.tl_last_error.restype = ctypes.c_char_p
            L.tl_version.restype = i32
            _lib = L
    return _lib


def _check(status):
    if status != 0:
        raise TLError(status, lib().tl_last_error().decode())


def _dtype_code(dtype):
    if isinstance(dtype, int):
        return dtype
    return DTYPES[dtype]


def _torch_dtype(code):
    import torch
    return torch.float32 if code == TL_F32 else torch.float64


def _rows(t, count, name, allow_none=False):
    """Tensor [count, n] or a sequence of count 1-D tensors -> list of 1-D tensors (None kept)."""
    if hasattr(t, "dim") and t.dim() == 2:
        if t.shape[0] != count:
            raise ValueError("%s must have %d rows, got %d" % (name, count, t.shape[0]))
        return [t[s] for s in range(count)]
    rows = list(t)
    if len(rows) != count:
        raise ValueError("%s must hold %d arrays, got %d" % (name, count, len(rows)))
    if not allow_none and any(r is None for r in rows):
        raise ValueError("%s may not contain None" % name)
    return rows


def _table(rows, count, n, tdtype, device_type, name):
    tab = (ctypes.c_void_p * count)()
    for s, r in enumerate(rows):
        if r is None:
            tab[s] = None
            continue
        if r.dim() != 1 or r.shape[0] != n or (n > 1 and r.stride(0) != 1):
            raise ValueError("%s[%d] must be a unit-stride 1-D tensor of length %d" % (name, s, n))
        if r.dtype != tdtype:
            raise TypeError("%s[%d] has dtype %s, expected %s" % (name, s, r.dtype, tdtype))
        if r.device.type != device_type:
            raise ValueError("%s[%d] must be on %s" % (name, s, device_type))
        tab[s] = r.data_ptr() if n > 0 else None
    return tab


def _stream_handle(stream, device):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream(device)
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def _nonnull_empty(tab, count):
    # n == 0: the C ABI still wants non-NULL table entries; any non-NULL value is fine as nothing is read.
    for s in range(count):
        if tab[s] is None:
            tab[s] = 16


def tl_dtg_forward(inputs, outputs=None, dtype="f64", stream=None):
    """Forward chain on device tensors.  Returns the [39, n] outputs (allocated if not given)."""
    import torch
    code = _dtype_code(dtype)
    td = _torch_dtype(code)
    rows = _rows(inputs, N_IN, "inputs")
    n = rows[0].shape[0]
    dev = rows[0].device
    if outputs is None:
        outputs = torch.empty((N_OUT, n), dtype=td, device=dev)
    orows = _rows(outputs, N_OUT, "outputs")
    itab = _table(rows, N_IN, n, td, "cuda", "inputs")
    otab = _table(orows, N_OUT, n, td, "cuda", "outputs")
    if n == 0:
        _nonnull_empty(itab, N_IN)
        _nonnull_empty(otab, N_OUT)
    with torch.cuda.device(dev):
        _check(lib().tl_dtg_forward(ctypes.byref(itab), ctypes.byref(otab), n, code, _stream_handle(stream, dev)))
    return outputs


def tl_dtg_backward(inputs, gout, gin=None, dtype="f64", stream=None):
    """Adjoint on device tensors: gout is [39, n] or 39 arrays (None = output not in the functional).
    Returns the [43, n] input gradients (allocated if not given)."""
    import torch
    code = _dtype_code(dtype)
    td = _torch_dtype(code)
    rows = _rows(inputs, N_IN, "inputs")
    n = rows[0].shape[0]
    dev = rows[0].device
    grows = _rows(gout, N_OUT, "gout", allow_none=True)
    if gin is None:
        gin = torch.empty((N_IN, n), dtype=td, device=dev)
    girows = _rows(gin, N_IN, "gin")
    itab = _table(rows, N_IN, n, td, "cuda", "inputs")
    gtab = _table(grows, N_OUT, n, td, "cuda", "gout")
    gitab = _table(girows, N_IN, n, td, "cuda", "gin")
    if n == 0:
        _nonnull_empty(itab, N_IN)
        _nonnull_empty(gitab, N_IN)
    with torch.cuda.device(dev):
        _check(lib().tl_dtg_backward(ctypes.byref(itab), ctypes.byref(gtab), ctypes.byref(gitab), n, code,
                                     _stream_handle(stream, dev)))
    return gin


def tl_dtg_forward_backward(inputs, gout, outputs=None, gin=None, dtype="f64", stream=None):
    """Forward and adjoint in one launch for upstream gradients known up front (gout: [39, n] or 39
    arrays, None = output not in the functional).  Returns (outputs [39, n], gin [43, n]), allocated
    where not given."""
    import torch
    code = _dtype_code(dtype)
    td = _torch_dtype(code)
    rows = _rows(inputs, N_IN, "inputs")
    n = rows[0].shape[0]
    dev = rows[0].device
    grows = _rows(gout, N_OUT, "gout", allow_none=True)
    if outputs is None:
        outputs = torch.empty((N_OUT, n), dtype=td, device=dev)
    if gin is None:
        gin = torch.empty((N_IN, n), dtype=td, device=dev)
    itab = _table(rows, N_IN, n, td, "cuda", "inputs")
    otab = _table(_rows(outputs, N_OUT, "outputs"), N_OUT, n, td, "cuda", "outputs")
    gtab = _table(grows, N_OUT, n, td, "cuda", "gout")
    gitab = _table(_rows(gin, N_IN, "gin"), N_IN, n, td, "cuda", "gin")
    if n == 0:
        _nonnull_empty(itab, N_IN)
        _nonnull_empty(otab, N_OUT)
        _nonnull_empty(gitab, N_IN)
    with torch.cuda.device(dev):
        _check(lib().tl_dtg_forward_backward(ctypes.byref(itab), ctypes.byref(otab), ctypes.byref(gtab),
                                             ctypes.byref(gitab), n, code, _stream_handle(stream, dev)))
    return outputs, gin


def tl_wait_timeouts():
    """Bounded device waits that gave up on the current device since the library was loaded (0 unless
    a staged kernel stopped early; synchronises)."""
    L = lib()
    L.tl_wait_timeouts.argtypes = [ctypes.c_void_p]
    L.tl_wait_timeouts.restype = ctypes.c_int
    c = ctypes.c_uint32()
    _check(L.tl_wait_timeouts(ctypes.byref(c)))
    return c.value


def tl_dtg_host_workspace_bytes(n, dtype="f64"):
    return int(lib().tl_dtg_host_workspace_bytes(n, _dtype_code(dtype)))


def tl_dtg_forward_host(inputs, outputs, workspace=None, dtype="f64", stream=None, device=None):
    """Forward with HOST tensors (page-locked for full speed): the library copies inputs in, runs the
    kernel and copies outputs back, all on `stream`.  `workspace` is a device uint8 tensor of at least
    tl_dtg_host_workspace_bytes(n) bytes (allocated if not given).  Returns outputs; they are valid
    after the stream is synchronised."""
    import torch
    code = _dtype_code(dtype)
    td = _torch_dtype(code)
    rows = _rows(inputs, N_IN, "inputs")
    orows = _rows(outputs, N_OUT, "outputs")
    n = rows[0].shape[0]
    dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
    need = tl_dtg_host_workspace_bytes(n, code)
    if workspace is None:
        workspace = torch.empty(max(need, 16), dtype=torch.uint8, device=dev)
    itab = _table(rows, N_IN, n, td, "cpu", "inputs")
    otab = _table(orows, N_OUT, n, td, "cpu", "outputs")
    if n == 0:
        _nonnull_empty(itab, N_IN)
        _nonnull_empty(otab, N_OUT)
    with torch.cuda.device(dev):
        _check(lib().tl_dtg_forward_host(ctypes.byref(itab), ctypes.byref(otab), n, code,
                                         ctypes.c_void_p(workspace.data_ptr()), workspace.numel(),
                                         _stream_handle(stream, dev)))
    return outputs


def _autograd():
    import torch

    class DtgFunction(torch.autograd.Function):
        """The fused chain as a differentiable op on a [43, n] float64 tensor.  Returns
        (ginv [6, n], gamma [18, n], dbcov [9, n], dtg [6, n]).  The backward runs the hand-written
        adjoint kernel, which recomputes g^ij and Gamma from the saved inputs; outputs that receive no
        gradient are passed to it as NULL and never read."""

        @staticmethod
        def forward(ctx, x, dtype="f64"):
            n = x.shape[1]
            dev = x.device
            ginv = torch.empty((6, n), dtype=x.dtype, device=dev)
            gamma = torch.empty((18, n), dtype=x.dtype, device=dev)
            dbcov = torch.empty((9, n), dtype=x.dtype, device=dev)
            dtg = torch.empty((6, n), dtype=x.dtype, device=dev)
            outs = [ginv[s] for s in range(6)] + [gamma[s] for s in range(18)] + \
                   [dbcov[s] for s in range(9)] + [dtg[s] for s in range(6)]
            tl_dtg_forward(x, outs, dtype=dtype)
            ctx.save_for_backward(x)
            ctx.dtype = dtype
            ctx.set_materialize_grads(False)
            return ginv, gamma, dbcov, dtg

        @staticmethod
        def backward(ctx, g_ginv, g_gamma, g_dbcov, g_dtg):
            (x,) = ctx.saved_tensors
            gout = []
            for g, rows in ((g_ginv, 6), (g_gamma, 18), (g_dbcov, 9), (g_dtg, 6)):
                if g is None:
                    gout += [None] * rows
                else:
                    g = g.contiguous()
                    gout += [g[s] for s in range(rows)]
            gin = tl_dtg_backward(x.contiguous(), gout, dtype=ctx.dtype)
            return gin, None

    return DtgFunction


_DtgFunction = None


def dtg(x, dtype="f64"):
    """Differentiable fused chain: returns (ginv, gamma, dbcov, dtg) for a [43, n] device tensor."""
    global _DtgFunction
    if _DtgFunction is None:
        _DtgFunction = _autograd()
    return _DtgFunction.apply(x, dtype)


def DtgFunction():
    """The torch.autograd.Function class behind dtg()."""
    global _DtgFunction
    if _DtgFunction is None:
        _DtgFunction = _autograd()
    return _DtgFunction


# ------------------------------------------------------------------------------------------- batched

def _batch_lib():
    L = lib()
    if not getattr(L, "_batch_ready", False):
        vp, i32 = ctypes.c_void_p, ctypes.c_int32
        L.tl_dtg_batched_prepare.argtypes = [vp, vp, vp, i32, ctypes.c_int, ctypes.POINTER(vp)]
        L.tl_dtg_batched.argtypes = [vp, vp]
        L.tl_dtg_batched_tune.argtypes = [vp, vp]
        L.tl_batch_plan_config.argtypes = [vp, ctypes.POINTER(i32), ctypes.POINTER(i32)]
        L.tl_batch_plan_set_config.argtypes = [vp, i32, i32]
        L.tl_batch_plan_points_per_thread.argtypes = [vp, ctypes.POINTER(i32)]
        L.tl_batch_plan_set_points_per_thread.argtypes = [vp, i32]
        L.tl_batch_plan_staging.argtypes = [vp, ctypes.POINTER(i32)]
        L.tl_batch_plan_set_staging.argtypes = [vp, i32]
        L.tl_batch_plan_check.argtypes = [vp]
        L.tl_batch_plan_destroy.argtypes = [vp]
        L.tl_batch_plan_destroy.restype = None
        for f in (L.tl_dtg_batched_prepare, L.tl_dtg_batched, L.tl_dtg_batched_tune, L.tl_batch_plan_config,
                  L.tl_batch_plan_set_config, L.tl_batch_plan_points_per_thread,
                  L.tl_batch_plan_set_points_per_thread, L.tl_batch_plan_check, L.tl_batch_plan_staging,
                  L.tl_batch_plan_set_staging):
            f.restype = ctypes.c_int
        L._batch_ready = True
    return L


class BatchPlan:
    """A batch plan over G grids (tl_dtg_batched_prepare).  The tensors must stay alive while the plan
    is used; the plan keeps references to them."""

    def __init__(self, inputs, outputs, dtype="f64"):
        import torch
        code = _dtype_code(dtype)
        td = _torch_dtype(code)
        G = len(inputs)
        if len(outputs) != G:
            raise ValueError("inputs and outputs must list the same number of grids")
        InTabs = (ctypes.c_void_p * (N_IN * max(G, 1)))()
        OutTabs = (ctypes.c_void_p * (N_OUT * max(G, 1)))()
        ns = (ctypes.c_int64 * max(G, 1))()
        dev = None
        for d in range(G):
            rows = _rows(inputs[d], N_IN, "inputs[%d]" % d)
            orows = _rows(outputs[d], N_OUT, "outputs[%d]" % d)
            n = rows[0].shape[0]
            dev = dev or rows[0].device
            it = _table(rows, N_IN, n, td, "cuda", "inputs[%d]" % d)
            ot = _table(orows, N_OUT, n, td, "cuda", "outputs[%d]" % d)
            if n == 0:
                _nonnull_empty(it, N_IN)
                _nonnull_empty(ot, N_OUT)
            for s in range(N_IN):
                InTabs[d * N_IN + s] = it[s]
            for s in range(N_OUT):
                OutTabs[d * N_OUT + s] = ot[s]
            ns[d] = n
        self.device = dev if dev is not None else torch.device("cuda", torch.cuda.current_device())
        self._keep = (list(inputs), list(outputs))
        self.G = G
        self.dtype = dtype
        h = ctypes.c_void_p()
        L = _batch_lib()
        with torch.cuda.device(self.device):
            _check(L.tl_dtg_batched_prepare(ctypes.byref(InTabs), ctypes.byref(OutTabs), ctypes.byref(ns), G, code,
                                            ctypes.byref(h)))
        self._h = h

    def launch(self, stream=None):
        import torch
        with torch.cuda.device(self.device):
            _check(_batch_lib().tl_dtg_batched(self._h, _stream_handle(stream, self.device)))

    def tune(self, stream=None):
        import torch
        with torch.cuda.device(self.device):
            _check(_batch_lib().tl_dtg_batched_tune(self._h, _stream_handle(stream, self.device)))
        return self.config

    @property
    def config(self):
        t, b = ctypes.c_int32(), ctypes.c_int32()
        _check(_batch_lib().tl_batch_plan_config(self._h, ctypes.byref(t), ctypes.byref(b)))
        return t.value, b.value

    def set_config(self, threads, blocks_per_sm, points_per_thread=None):
        _check(_batch_lib().tl_batch_plan_set_config(self._h, threads, blocks_per_sm))
        if points_per_thread is not None:
            _check(_batch_lib().tl_batch_plan_set_points_per_thread(self._h, points_per_thread))

    @property
    def points_per_thread(self):
        q = ctypes.c_int32()
        _check(_batch_lib().tl_batch_plan_points_per_thread(self._h, ctypes.byref(q)))
        return q.value

    @property
    def staging(self):
        """Staging depth: 0 (inputs loaded into registers) or 2 / 3 tiles through shared memory."""
        q = ctypes.c_int32()
        _check(_batch_lib().tl_batch_plan_staging(self._h, ctypes.byref(q)))
        return q.value

    def set_staging(self, stages):
        import torch
        with torch.cuda.device(self.device):
            _check(_batch_lib().tl_batch_plan_set_staging(self._h, stages))

    def check(self):
        import torch
        with torch.cuda.device(self.device):
            _check(_batch_lib().tl_batch_plan_check(self._h))

    def close(self):
        if getattr(self, "_h", None):
            _batch_lib().tl_batch_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def tl_dtg_batched_prepare(inputs, outputs, dtype="f64"):
    """inputs: list of G [43, n_d] device tensors; outputs: list of G [39, n_d].  Returns a BatchPlan."""
    return BatchPlan(inputs, outputs, dtype)


def tl_dtg_batched(plan, stream=None):
    plan.launch(stream)


def tl_dtg_batched_tune(plan, stream=None):
    return plan.tune(stream)


# ----------------------------------------------------------------------------- benchmark expressions

TL_EXPR_FUSED, TL_EXPR_ARRAYS = 0, 1
EXPR_MODES = {"fused": TL_EXPR_FUSED, "tensors": TL_EXPR_FUSED, "arrays": TL_EXPR_ARRAYS}


def tl_expr_arity(eq):
    L = lib()
    L.tl_expr_arity.argtypes = [ctypes.c_int32, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)]
    L.tl_expr_arity.restype = ctypes.c_int
    a, b = ctypes.c_int32(), ctypes.c_int32()
    _check(L.tl_expr_arity(eq, ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def tl_expr_eval(eq, inputs, outputs=None, mode="fused", stream=None):
    """Benchmark expression `eq` (Eqs. 9-21 of Sec. 5.1) on device float64 tensors: inputs [n_in, n] (or
    n_in arrays), outputs [n_out, n] (allocated if not given); mode "fused" (one kernel) or "arrays"
    (one launch per component and contracted index)."""
    import torch
    import torch as _t
    n_in, n_out = tl_expr_arity(eq)
    rows = _rows(inputs, n_in, "inputs")
    n = rows[0].shape[0]
    dev = rows[0].device
    if outputs is None:
        outputs = _t.empty((n_out, n), dtype=_t.float64, device=dev)
    orows = _rows(outputs, n_out, "outputs")
    itab = _table(rows, n_in, n, _t.float64, "cuda", "inputs")
    otab = _table(orows, n_out, n, _t.float64, "cuda", "outputs")
    if n == 0:
        _nonnull_empty(itab, n_in)
        _nonnull_empty(otab, n_out)
    L = lib()
    L.tl_expr_eval.argtypes = [ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int,
                               ctypes.c_void_p]
    L.tl_expr_eval.restype = ctypes.c_int
    with torch.cuda.device(dev):
        _check(L.tl_expr_eval(eq, ctypes.byref(itab), ctypes.byref(otab), n, EXPR_MODES[mode],
                              _stream_handle(stream, dev)))
    return outputs


# --------------------------------------------------------------------------------- runtime generator

class JitKernel:
    """A tensor-index program compiled by tl_jit_compile (parse, index checks, CUDA source, NVRTC).
    `inputs` / `outputs` list the component tables as (tensor name, index tuple); `source` is the
    generated CUDA."""

    def __init__(self, program):
        L = lib()
        vp = ctypes.c_void_p
        L.tl_jit_compile.argtypes = [ctypes.c_char_p, ctypes.POINTER(vp), ctypes.c_char_p, ctypes.c_size_t]
        L.tl_jit_compile.restype = ctypes.c_int
        L.tl_jit_info.argtypes = [vp, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32),
                                  ctypes.POINTER(ctypes.c_char_p), ctypes.POINTER(ctypes.c_char_p)]
        L.tl_jit_info.restype = ctypes.c_int
        L.tl_jit_launch.argtypes = [vp, vp, vp, ctypes.c_int64, vp]
        L.tl_jit_launch.restype = ctypes.c_int
        L.tl_jit_destroy.argtypes = [vp]
        L.tl_jit_destroy.restype = None
        h = vp()
        log = ctypes.create_string_buffer(4096)
        rc = L.tl_jit_compile(program.encode(), ctypes.byref(h), log, len(log))
        if rc != 0:
            raise TLError(rc, log.value.decode())
        self._h = h
        ni, no = ctypes.c_int32(), ctypes.c_int32()
        src, names = ctypes.c_char_p(), ctypes.c_char_p()
        _check(L.tl_jit_info(h, ctypes.byref(ni), ctypes.byref(no), ctypes.byref(src), ctypes.byref(names)))
        self.n_in, self.n_out = ni.value, no.value
        self.source = src.value.decode()
        self.inputs, self.outputs = [], []
        for line in names.value.decode().splitlines():
            kind, name, *idx = line.split()
            (self.inputs if kind == "in" else self.outputs).append((name, tuple(int(v) for v in idx)))
        L.tl_jit_reads.argtypes = [vp, vp]
        L.tl_jit_reads.restype = ctypes.c_int
        flags = (ctypes.c_uint8 * max(self.n_in, 1))()
        _check(L.tl_jit_reads(h, ctypes.cast(flags, vp)))
        self.reads = [bool(flags[q]) for q in range(self.n_in)]    # input entries the kernel loads

    def launch(self, inputs, outputs=None, stream=None):
        import torch
        rows = _rows(inputs, self.n_in, "inputs") if self.n_in else []
        n = rows[0].shape[0] if rows else (outputs.shape[1] if outputs is not None else 0)
        dev = rows[0].device if rows else torch.device("cuda", torch.cuda.current_device())
        if outputs is None:
            outputs = torch.empty((self.n_out, n), dtype=torch.float64, device=dev)
        orows = _rows(outputs, self.n_out, "outputs")
        itab = _table(rows, self.n_in, n, torch.float64, "cuda", "inputs") if self.n_in else (ctypes.c_void_p * 1)()
        otab = _table(orows, self.n_out, n, torch.float64, "cuda", "outputs")
        if n == 0:
            _nonnull_empty(itab, max(self.n_in, 1))
            _nonnull_empty(otab, self.n_out)
        with torch.cuda.device(dev):
            _check(lib().tl_jit_launch(self._h, ctypes.byref(itab), ctypes.byref(otab), n, _stream_handle(stream, dev)))
        return outputs

    def close(self):
        if getattr(self, "_h", None):
            lib().tl_jit_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def tl_jit_compile(program):
    return JitKernel(program)


# ------------------------------------------------------------------------------ on-grid derivatives

class _Grid3d(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int64), ("ny", ctypes.c_int64), ("nz", ctypes.c_int64), ("hx", ctypes.c_double),
                ("hy", ctypes.c_double), ("hz", ctypes.c_double), ("order", ctypes.c_int32)]


def tl_dtg_forward_fd(fields, shape, spacing, order=4, outputs=None, dtype="f64", stream=None):
    """Forward chain with d_k g_ij and d_j beta_i by centred differences (order 2 or 4) on a periodic
    grid of shape (nx, ny, nz), x fastest, spacings (hx, hy, hz).  fields: [16, n] device float64
    (g[6], K[6], alpha, beta[3]).  Returns the [39, n] outputs of tl_dtg_forward."""
    import torch
    code = _dtype_code(dtype)
    rows = _rows(fields, 16, "fields")
    n = rows[0].shape[0]
    if n != shape[0] * shape[1] * shape[2]:
        raise ValueError("fields hold %d points, shape %s has %d" % (n, shape, shape[0] * shape[1] * shape[2]))
    dev = rows[0].device
    if outputs is None:
        outputs = torch.empty((N_OUT, n), dtype=torch.float64, device=dev)
    orows = _rows(outputs, N_OUT, "outputs")
    itab = _table(rows, 16, n, torch.float64, "cuda", "fields")
    otab = _table(orows, N_OUT, n, torch.float64, "cuda", "outputs")
    g = _Grid3d(shape[0], shape[1], shape[2], spacing[0], spacing[1], spacing[2], order)
    L = lib()
    L.tl_dtg_forward_fd.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]
    L.tl_dtg_forward_fd.restype = ctypes.c_int
    with torch.cuda.device(dev):
        _check(L.tl_dtg_forward_fd(ctypes.byref(itab), ctypes.byref(otab), ctypes.byref(g), code,
                                   _stream_handle(stream, dev)))
    return outputs
