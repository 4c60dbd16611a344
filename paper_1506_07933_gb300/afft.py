"""ctypes binding of libafft.so -- argument marshalling only.

Every step of the transform runs in the CUDA library; this module checks
tensor shapes, dtypes and devices, passes raw pointers and the current CUDA
stream through the C ABI of ``include/afft.h``, and turns status codes into
exceptions.  PyTorch provides device memory and streams.  There is no CPU
fallback: if the library is missing or cannot be loaded, every call raises.

Low-level functions carry the C names (``afft_plan_create`` and so on);
``Plan`` wraps them for tensors.
"""
from __future__ import annotations

import ctypes
import os

import torch

from . import build as _build

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = _build.LIB

C2C, R2C = 0, 1
F32, F64, F32_SPLIT = 0, 1, 2
KINDS = {"c2c": C2C, "r2c": R2C}
PRECISIONS = {"f32": F32, "f64": F64, "f32_split": F32_SPLIT}

STATUS = {
    0: "AFFT_OK", 1: "AFFT_ERR_NULL", 2: "AFFT_ERR_SIZE", 3: "AFFT_ERR_R2C_ODD", 4: "AFFT_ERR_KIND",
    5: "AFFT_ERR_PRECISION", 6: "AFFT_ERR_NOMEM", 7: "AFFT_ERR_INPLACE", 8: "AFFT_ERR_CUDA",
    9: "AFFT_ERR_UNSUPPORTED", 10: "AFFT_ERR_SCRATCH", 11: "AFFT_ERR_TIMEOUT", 12: "AFFT_ERR_AXES",
}

# Every symbol include/afft.h declares.
EXPORTS = [
    "afft_plan_create", "afft_execute_forward", "afft_execute_backward",
    "afft_execute_forward_host", "afft_execute_backward_host", "afft_plan_destroy",
    "afft_plan_workspace_bytes", "afft_plan_input_bytes", "afft_plan_output_bytes",
    "afft_plan_launches", "afft_status_string", "afft_fill_uniform",
    "afft_plan_timing_begin", "afft_plan_timing_end", "afft_c2r_noalloc",
    "afft_plan_device_status", "afft_plan_set_l2_chunk", "afft_plan_l2_chunk",
    "afft_plan_create_batched", "afft_plan_tune", "afft_plan_describe", "afft_multi_create",
    "afft_multi_execute", "afft_multi_destroy", "afft_execute_poisson", "afft_plan_wait_probe",
    "afft_plan_set_blocked", "afft_plan_get_tuning", "afft_plan_set_tuning", "afft_plan_create_axes",
    "afft_plan_set_backward_scale", "afft_plan_backward_scale", "afft_copy_2d", "afft_queue_create",
    "afft_queue_execute", "afft_queue_status", "afft_queue_items", "afft_queue_destroy",
    "afft_plan_set_l2_order", "afft_plan_l2_order",
]

_lib = None


class AfftError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__("%s: %s (%s)" % (where, STATUS.get(status, status), status_string(status)))


def load(path: str = None):
    """Load libafft.so (in-tree).  Raises if it is missing: there is no fallback."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError("libafft.so not built (%s); run paper_1506_07933_gb300/build.py" % path)
    lib = ctypes.CDLL(path)
    vp, i64p, c_int, sz = ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64), ctypes.c_int, ctypes.c_size_t
    lib.afft_plan_create.argtypes = [ctypes.POINTER(vp), i64p, c_int, c_int]
    lib.afft_plan_create_batched.argtypes = [ctypes.POINTER(vp), i64p, ctypes.c_int64, c_int, c_int]
    lib.afft_plan_create_axes.argtypes = [ctypes.POINTER(vp), i64p, ctypes.c_int64, c_int, c_int, c_int]
    lib.afft_plan_set_backward_scale.argtypes = [vp, ctypes.c_double]
    lib.afft_plan_backward_scale.argtypes = [vp]
    lib.afft_plan_backward_scale.restype = ctypes.c_double
    lib.afft_copy_2d.argtypes = [vp, sz, vp, sz, sz, sz, vp]
    lib.afft_queue_create.argtypes = [ctypes.POINTER(vp), c_int, ctypes.POINTER(vp)]
    lib.afft_queue_execute.argtypes = [vp, c_int, ctypes.POINTER(vp), ctypes.POINTER(vp), vp]
    lib.afft_queue_status.argtypes = [vp]
    lib.afft_queue_items.argtypes = [vp, c_int]
    lib.afft_queue_destroy.argtypes = [vp]
    lib.afft_plan_tune.argtypes = [vp, vp]
    lib.afft_execute_poisson.argtypes = [vp, vp, vp, vp]
    lib.afft_plan_describe.argtypes = [vp, ctypes.c_char_p, sz]
    lib.afft_multi_create.argtypes = [ctypes.POINTER(vp), c_int, ctypes.POINTER(vp)]
    lib.afft_multi_execute.argtypes = [vp, c_int, ctypes.POINTER(vp), ctypes.POINTER(vp), vp]
    lib.afft_multi_destroy.argtypes = [vp]
    lib.afft_execute_forward.argtypes = [vp, vp, vp, vp]
    lib.afft_execute_backward.argtypes = [vp, vp, vp, vp]
    lib.afft_execute_forward_host.argtypes = [vp, vp, vp, vp, vp, vp]
    lib.afft_execute_backward_host.argtypes = [vp, vp, vp, vp, vp, vp]
    lib.afft_plan_destroy.argtypes = [vp]
    for f in ("afft_plan_workspace_bytes", "afft_plan_input_bytes", "afft_plan_output_bytes"):
        getattr(lib, f).argtypes = [vp]
        getattr(lib, f).restype = sz
    lib.afft_plan_launches.argtypes = [vp, c_int]
    lib.afft_status_string.argtypes = [c_int]
    lib.afft_status_string.restype = ctypes.c_char_p
    lib.afft_fill_uniform.argtypes = [vp, ctypes.c_int64, ctypes.c_uint64, c_int, vp]
    lib.afft_plan_timing_begin.argtypes = [vp, c_int]
    lib.afft_plan_timing_end.argtypes = [vp, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(c_int)]
    lib.afft_c2r_noalloc.argtypes = [i64p, c_int, vp, vp, vp]
    lib.afft_plan_device_status.argtypes = [vp]
    lib.afft_plan_wait_probe.argtypes = [vp, c_int, vp]
    lib.afft_plan_set_l2_chunk.argtypes = [vp, sz]
    lib.afft_plan_set_blocked.argtypes = [vp, c_int]
    lib.afft_plan_set_l2_order.argtypes = [vp, c_int]
    lib.afft_plan_l2_order.argtypes = [vp]
    lib.afft_plan_get_tuning.argtypes = [vp, i64p]
    lib.afft_plan_set_tuning.argtypes = [vp, i64p]
    lib.afft_plan_l2_chunk.argtypes = [vp]
    lib.afft_plan_l2_chunk.restype = sz
    for f in ("afft_plan_create", "afft_plan_create_batched", "afft_execute_forward", "afft_execute_backward",
              "afft_execute_forward_host", "afft_execute_backward_host", "afft_plan_destroy",
              "afft_plan_launches", "afft_fill_uniform", "afft_plan_timing_begin",
              "afft_plan_timing_end", "afft_c2r_noalloc", "afft_plan_device_status",
              "afft_plan_set_l2_chunk", "afft_plan_tune", "afft_plan_describe", "afft_multi_create",
              "afft_multi_execute", "afft_multi_destroy", "afft_execute_poisson", "afft_plan_wait_probe",
              "afft_plan_set_blocked", "afft_plan_get_tuning", "afft_plan_set_tuning", "afft_plan_create_axes",
              "afft_plan_set_backward_scale", "afft_copy_2d", "afft_queue_create", "afft_queue_execute",
              "afft_queue_status", "afft_queue_items", "afft_queue_destroy", "afft_plan_set_l2_order",
              "afft_plan_l2_order"):
        getattr(lib, f).restype = c_int
    _lib = lib
    return lib


def status_string(status: int) -> str:
    return load().afft_status_string(int(status)).decode()


def _check(status: int, where: str):
    if status != 0:
        raise AfftError(status, where)


def _stream_handle(stream) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream) if hasattr(stream, "cuda_stream") else int(stream)


# ------------------------------------------------------------------ C names --

def afft_plan_create(shape, kind: int, precision: int) -> ctypes.c_void_p:
    n = (ctypes.c_int64 * 3)(*[int(s) for s in shape])
    p = ctypes.c_void_p()
    _check(load().afft_plan_create(ctypes.byref(p), n, int(kind), int(precision)), "afft_plan_create")
    return p


def afft_plan_create_batched(shape, batch: int, kind: int, precision: int) -> ctypes.c_void_p:
    n = (ctypes.c_int64 * 3)(*[int(s) for s in shape])
    p = ctypes.c_void_p()
    _check(load().afft_plan_create_batched(ctypes.byref(p), n, int(batch), int(kind), int(precision)),
           "afft_plan_create_batched")
    return p


def afft_plan_create_axes(shape, batch: int, kind: int, precision: int, axes: int) -> ctypes.c_void_p:
    n = (ctypes.c_int64 * 3)(*[int(s) for s in shape])
    p = ctypes.c_void_p()
    _check(load().afft_plan_create_axes(ctypes.byref(p), n, int(batch), int(kind), int(precision), int(axes)),
           "afft_plan_create_axes")
    return p


def afft_copy_2d(dst_ptr: int, dpitch: int, src_ptr: int, spitch: int, width: int, rows: int, stream: int) -> None:
    """rows x width bytes between pitched buffers (cudaMemcpy2DAsync on the stream)."""
    _check(load().afft_copy_2d(dst_ptr, int(dpitch), src_ptr, int(spitch), int(width), int(rows), stream),
           "afft_copy_2d")


def afft_execute_forward(plan, in_ptr: int, out_ptr: int, stream: int) -> None:
    _check(load().afft_execute_forward(plan, in_ptr, out_ptr, stream), "afft_execute_forward")


def afft_execute_backward(plan, in_ptr: int, out_ptr: int, stream: int) -> None:
    _check(load().afft_execute_backward(plan, in_ptr, out_ptr, stream), "afft_execute_backward")


def afft_execute_forward_host(plan, host_in, host_out, dev_in, dev_out, stream: int) -> None:
    _check(load().afft_execute_forward_host(plan, host_in, host_out, dev_in, dev_out, stream),
           "afft_execute_forward_host")


def afft_execute_backward_host(plan, host_in, host_out, dev_in, dev_out, stream: int) -> None:
    _check(load().afft_execute_backward_host(plan, host_in, host_out, dev_in, dev_out, stream),
           "afft_execute_backward_host")


def afft_plan_destroy(plan) -> None:
    _check(load().afft_plan_destroy(plan), "afft_plan_destroy")


def afft_fill_uniform(ptr: int, count: int, seed: int, precision: int, stream: int) -> None:
    _check(load().afft_fill_uniform(ptr, int(count), int(seed), int(precision), stream),
           "afft_fill_uniform")


def afft_c2r_noalloc(shape, precision: int, in_ptr: int, out_ptr: int, stream: int) -> None:
    """c2r backward without any allocation (fixed 64 MiB device array); see include/afft.h."""
    n = (ctypes.c_int64 * 3)(*[int(s) for s in shape])
    _check(load().afft_c2r_noalloc(n, int(precision), in_ptr, out_ptr, stream), "afft_c2r_noalloc")


# --------------------------------------------------------------- tensor API --

_CDT = {F32: torch.complex64, F64: torch.complex128, F32_SPLIT: torch.complex64}
_RDT = {F32: torch.float32, F64: torch.float64, F32_SPLIT: torch.float32}


class Plan:
    """A resident 3-D FFT plan: ``Plan((n0, n1, n2), "c2c" | "r2c", "f32" | "f64")``.

    ``forward(x)``: unscaled forward transform (c2c: complex -> complex;
    r2c: real [n0, n1, n2] -> complex [n0, n1, n2 // 2 + 1]).
    ``backward(X)``: inverse scaled by 1/N (c2c, or c2r for an r2c plan).
    ``batch``: that many transforms stored back to back.  ``axes``: a bit mask
    (1, 2, 4 for n0, n1, n2) of the axes to transform, for the building blocks
    of the slab and d-dimensional transforms (see afft_plan_create_axes).
    Tensors must be contiguous, on the plan's device, of the plan's dtype.
    Calls are asynchronous on the current (or given) stream.
    """

    def __init__(self, shape, kind="c2c", precision="f32", batch=None, axes=None):
        self.shape = tuple(int(s) for s in shape)
        self.kind = KINDS[kind] if isinstance(kind, str) else int(kind)
        self.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.batch = batch
        self.axes = 7 if axes is None else int(axes)
        if axes is not None:
            self._p = afft_plan_create_axes(self.shape, 1 if batch is None else int(batch), self.kind,
                                            self.precision, self.axes)
        elif batch is None:
            self._p = afft_plan_create(self.shape, self.kind, self.precision)
        else:
            self._p = afft_plan_create_batched(self.shape, int(batch), self.kind, self.precision)
        lib = load()
        self.workspace_bytes = lib.afft_plan_workspace_bytes(self._p)
        self.input_bytes = lib.afft_plan_input_bytes(self._p)
        self.output_bytes = lib.afft_plan_output_bytes(self._p)

    # shapes / dtypes of the forward input and output
    @property
    def spatial_shape(self):
        return self.shape if self.batch is None else (self.batch,) + self.shape

    @property
    def spectral_shape(self):
        n0, n1, n2 = self.shape
        s = (n0, n1, n2 // 2 + 1) if self.kind == R2C else self.shape
        return s if self.batch is None else (self.batch,) + s

    @property
    def spatial_dtype(self):
        return _RDT[self.precision] if self.kind == R2C else _CDT[self.precision]

    @property
    def spectral_dtype(self):
        return _CDT[self.precision]

    def launches(self, backward: bool = False) -> int:
        return load().afft_plan_launches(self._p, int(bool(backward)))

    def _check_tensor(self, t, shape, dtype, what):
        if not isinstance(t, torch.Tensor):
            raise TypeError("%s must be a torch.Tensor" % what)
        if t.device != self.device:
            raise ValueError("%s must be on %s, got %s" % (what, self.device, t.device))
        if t.dtype != dtype:
            raise TypeError("%s must be %s, got %s" % (what, dtype, t.dtype))
        if tuple(t.shape) != tuple(shape):
            raise ValueError("%s must have shape %s, got %s" % (what, shape, tuple(t.shape)))
        if not t.is_contiguous():
            raise ValueError("%s must be contiguous" % what)

    def forward(self, x, out=None, stream=None):
        self._check_tensor(x, self.spatial_shape, self.spatial_dtype, "input")
        if out is None:
            out = torch.empty(self.spectral_shape, dtype=self.spectral_dtype, device=self.device)
        self._check_tensor(out, self.spectral_shape, self.spectral_dtype, "output")
        afft_execute_forward(self._p, x.data_ptr(), out.data_ptr(), _stream_handle(stream))
        return out

    def backward(self, X, out=None, stream=None):
        self._check_tensor(X, self.spectral_shape, self.spectral_dtype, "input")
        if out is None:
            out = torch.empty(self.spatial_shape, dtype=self.spatial_dtype, device=self.device)
        self._check_tensor(out, self.spatial_shape, self.spatial_dtype, "output")
        afft_execute_backward(self._p, X.data_ptr(), out.data_ptr(), _stream_handle(stream))
        return out

    def poisson(self, f, out=None, stream=None):
        """u with -Lap u = f on [0, 2 pi)^3, zero mean (r2c plans; f real, spatial shape)."""
        self._check_tensor(f, self.spatial_shape, self.spatial_dtype, "f")
        if out is None:
            out = torch.empty(self.spatial_shape, dtype=self.spatial_dtype, device=self.device)
        self._check_tensor(out, self.spatial_shape, self.spatial_dtype, "u")
        _check(load().afft_execute_poisson(self._p, f.data_ptr(), out.data_ptr(), _stream_handle(stream)),
               "afft_execute_poisson")
        return out

    def forward_host(self, host_in, host_out, dev_in, dev_out, stream=None):
        """Host -> device copy, forward transform, device -> host copy (one C-ABI call)."""
        self._check_tensor(dev_in, self.spatial_shape, self.spatial_dtype, "dev_in")
        self._check_tensor(dev_out, self.spectral_shape, self.spectral_dtype, "dev_out")
        for t, shape, dt, w in ((host_in, self.spatial_shape, self.spatial_dtype, "host_in"),
                                (host_out, self.spectral_shape, self.spectral_dtype, "host_out")):
            if t.device.type != "cpu" or t.dtype != dt or tuple(t.shape) != shape or not t.is_contiguous():
                raise ValueError("%s must be a contiguous CPU tensor %s %s" % (w, dt, shape))
        afft_execute_forward_host(self._p, host_in.data_ptr(), host_out.data_ptr(), dev_in.data_ptr(),
                                  dev_out.data_ptr(), _stream_handle(stream))

    def backward_host(self, host_in, host_out, dev_in, dev_out, stream=None):
        """Host -> device copy, backward transform, device -> host copy (one C-ABI call)."""
        self._check_tensor(dev_in, self.spectral_shape, self.spectral_dtype, "dev_in")
        self._check_tensor(dev_out, self.spatial_shape, self.spatial_dtype, "dev_out")
        for t, shape, dt, w in ((host_in, self.spectral_shape, self.spectral_dtype, "host_in"),
                                (host_out, self.spatial_shape, self.spatial_dtype, "host_out")):
            if t.device.type != "cpu" or t.dtype != dt or tuple(t.shape) != shape or not t.is_contiguous():
                raise ValueError("%s must be a contiguous CPU tensor %s %s" % (w, dt, shape))
        afft_execute_backward_host(self._p, host_in.data_ptr(), host_out.data_ptr(), dev_in.data_ptr(),
                                   dev_out.data_ptr(), _stream_handle(stream))

    @property
    def backward_scale(self) -> float:
        return float(load().afft_plan_backward_scale(self._p))

    def set_backward_scale(self, scale: float) -> None:
        """The factor of the backward transform (default 1 / product of the transformed n)."""
        _check(load().afft_plan_set_backward_scale(self._p, float(scale)), "afft_plan_set_backward_scale")

    def set_blocked(self, on: bool) -> None:
        """Blocked c2c layout (a workspace of the array's size; see afft_plan_set_blocked)."""
        _check(load().afft_plan_set_blocked(self._p, int(bool(on))), "afft_plan_set_blocked")

    def set_l2_order(self, on: bool) -> None:
        """Alternating tile order of consecutive stages (see afft_plan_set_l2_order)."""
        _check(load().afft_plan_set_l2_order(self._p, int(bool(on))), "afft_plan_set_l2_order")

    @property
    def l2_order(self) -> bool:
        return bool(load().afft_plan_l2_order(self._p))

    def set_l2_chunk(self, nbytes: int) -> None:
        """Slab size for L2-resident fusion of the N2 and N1 stages (0: unfused)."""
        _check(load().afft_plan_set_l2_chunk(self._p, int(nbytes)), "afft_plan_set_l2_chunk")

    @property
    def l2_chunk(self) -> int:
        return int(load().afft_plan_l2_chunk(self._p))

    def tune(self, stream=None, cache: str = None) -> bool:
        """Autotune the launch configuration on temporary buffers (synchronises).  With `cache`
        (a JSON file), a choice stored there for this plan's key (shape, kind, precision, batch,
        GPU name) is applied instead of tuning, and a new one is stored.  Returns True when the
        choice came from the cache."""
        key = tuning_key(self.shape, self.kind, self.precision, self.batch,
                         torch.cuda.get_device_name(self.device)) if cache else None
        if cache:
            cfg = tuning_cache_lookup(cache, key)
            if cfg is not None:
                self.set_tuning(cfg)
                return True
        _check(load().afft_plan_tune(self._p, _stream_handle(stream)), "afft_plan_tune")
        if cache:
            tuning_cache_store(cache, key, self.tuning)
        return False

    @property
    def tuning(self) -> list:
        """[contiguous-stage points per CTA (0: default), N0 pipelined, N1 pipelined, L2 slab bytes,
        N0 row-pair early release, N1 row-pair early release]."""
        cfg = (ctypes.c_int64 * 6)()
        _check(load().afft_plan_get_tuning(self._p, cfg), "afft_plan_get_tuning")
        return [int(v) for v in cfg]

    def set_tuning(self, cfg) -> None:
        """Applies a tuning list (a 4-entry list from an older cache leaves the row-pair choices off)."""
        cfg = [int(v) for v in cfg] + [0] * (6 - len(cfg))
        arr = (ctypes.c_int64 * 6)(*cfg[:6])
        _check(load().afft_plan_set_tuning(self._p, arr), "afft_plan_set_tuning")

    def describe(self) -> dict:
        import json
        buf = ctypes.create_string_buffer(1024)
        _check(load().afft_plan_describe(self._p, buf, len(buf)), "afft_plan_describe")
        return json.loads(buf.value.decode())

    def device_status(self) -> int:
        """Synchronises; returns 0, or 11 (AFFT_ERR_TIMEOUT) if a bounded wait ran out since the last call."""
        return int(load().afft_plan_device_status(self._p))

    def wait_probe(self, limit_us: int, stream=None) -> None:
        """Failure-detection self-test: a kernel whose bounded wait can only run out records a
        timeout in this plan's flag (see afft_plan_wait_probe); device_status() then reports it."""
        _check(load().afft_plan_wait_probe(self._p, int(limit_us), _stream_handle(stream)), "afft_plan_wait_probe")

    def timing_begin(self, capacity: int) -> None:
        """Record per-stage CUDA events for the next ``capacity`` executions."""
        _check(load().afft_plan_timing_begin(self._p, int(capacity)), "afft_plan_timing_begin")
        self._timing_cap = int(capacity)

    def timing_end(self):
        """Per-stage milliseconds, one row of 3 per recorded execution (launch order)."""
        cap = getattr(self, "_timing_cap", 0)
        buf = (ctypes.c_float * (3 * max(cap, 1)))()
        cnt = ctypes.c_int(0)
        _check(load().afft_plan_timing_end(self._p, buf, ctypes.byref(cnt)), "afft_plan_timing_end")
        return [list(buf[3 * r:3 * r + 3]) for r in range(cnt.value)]

    def close(self):
        if getattr(self, "_p", None):
            afft_plan_destroy(self._p)
            self._p = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class Multi:
    """Several plans run as one captured CUDA graph (see afft_multi_* in include/afft.h)."""

    def __init__(self, plans):
        self.plans = list(plans)
        arr = (ctypes.c_void_p * len(self.plans))(*[p._p.value for p in self.plans])
        self._m = ctypes.c_void_p()
        _check(load().afft_multi_create(ctypes.byref(self._m), len(self.plans), arr), "afft_multi_create")

    def _run(self, backward, ins, outs, stream):
        if len(ins) != len(self.plans) or len(outs) != len(self.plans):
            raise ValueError("one input and one output per plan")
        for p, a, b in zip(self.plans, ins, outs):
            if backward:
                p._check_tensor(a, p.spectral_shape, p.spectral_dtype, "input")
                p._check_tensor(b, p.spatial_shape, p.spatial_dtype, "output")
            else:
                p._check_tensor(a, p.spatial_shape, p.spatial_dtype, "input")
                p._check_tensor(b, p.spectral_shape, p.spectral_dtype, "output")
        ia = (ctypes.c_void_p * len(ins))(*[t.data_ptr() for t in ins])
        oa = (ctypes.c_void_p * len(outs))(*[t.data_ptr() for t in outs])
        _check(load().afft_multi_execute(self._m, int(backward), ia, oa, _stream_handle(stream)),
               "afft_multi_execute")

    def forward(self, ins, outs, stream=None):
        self._run(0, ins, outs, stream)

    def backward(self, ins, outs, stream=None):
        self._run(1, ins, outs, stream)

    def close(self):
        if getattr(self, "_m", None) and self._m.value:
            _check(load().afft_multi_destroy(self._m), "afft_multi_destroy")
            self._m = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Queue:
    """Several FP32 r2c plans (one batched plan per size) run as one persistent kernel launch per
    direction (see afft_queue_* in include/afft.h)."""

    def __init__(self, plans):
        self.plans = list(plans)
        arr = (ctypes.c_void_p * len(self.plans))(*[p._p.value for p in self.plans])
        self._q = ctypes.c_void_p()
        _check(load().afft_queue_create(ctypes.byref(self._q), len(self.plans), arr), "afft_queue_create")

    def _run(self, backward, ins, outs, stream):
        n = len(self.plans)
        for p, x, y in zip(self.plans, ins, outs):
            a, b = (p.spectral_shape, p.spatial_shape) if backward else (p.spatial_shape, p.spectral_shape)
            da, db = (p.spectral_dtype, p.spatial_dtype) if backward else (p.spatial_dtype, p.spectral_dtype)
            p._check_tensor(x, a, da, "input")
            p._check_tensor(y, b, db, "output")
        i = (ctypes.c_void_p * n)(*[t.data_ptr() for t in ins])
        o = (ctypes.c_void_p * n)(*[t.data_ptr() for t in outs])
        _check(load().afft_queue_execute(self._q, int(backward), i, o, _stream_handle(stream)), "afft_queue_execute")

    def forward(self, ins, outs, stream=None):
        self._run(False, ins, outs, stream)

    def backward(self, ins, outs, stream=None):
        self._run(True, ins, outs, stream)

    def status(self) -> int:
        """Synchronises; 0, or 11 (AFFT_ERR_TIMEOUT) if a bounded wait ran out since the last call."""
        return int(load().afft_queue_status(self._q))

    def items(self, backward=False) -> int:
        return int(load().afft_queue_items(self._q, int(bool(backward))))

    def close(self):
        if getattr(self, "_q", None):
            _check(load().afft_queue_destroy(self._q), "afft_queue_destroy")
            self._q = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def tuning_key(shape, kind, precision, batch, gpu_name: str) -> str:
    """Cache key of a plan's tuned configuration."""
    kinds = {v: k for k, v in KINDS.items()}
    precs = {v: k for k, v in PRECISIONS.items()}
    return "%s/%s/%s/batch%d/%s" % ("x".join(str(int(n)) for n in shape), kinds.get(kind, kind),
                                    precs.get(precision, precision), int(batch or 1), gpu_name)


def tuning_cache_lookup(path: str, key: str):
    """The stored configuration for `key`, or None (no file, no entry, or a malformed one)."""
    import json
    try:
        with open(path) as fh:
            cfg = json.load(fh).get(key)
    except (OSError, ValueError, AttributeError):
        return None
    if not isinstance(cfg, list) or len(cfg) not in (4, 6) or not all(isinstance(v, int) for v in cfg):
        return None
    return cfg + [0] * (6 - len(cfg))   # entries stored before the row-pair choices existed


def tuning_cache_store(path: str, key: str, cfg) -> None:
    """Adds or replaces `key` in the cache file (written to a temporary file, then renamed)."""
    import json
    try:
        with open(path) as fh:
            data = json.load(fh)
        if not isinstance(data, dict):
            data = {}
    except (OSError, ValueError):
        data = {}
    data[key] = [int(v) for v in cfg]
    tmp = "%s.tmp.%d" % (path, os.getpid())
    with open(tmp, "w") as fh:
        json.dump(data, fh, indent=1, sort_keys=True)
    os.replace(tmp, path)


def fill_uniform(t: torch.Tensor, seed: int, stream=None) -> torch.Tensor:
    """Fill a contiguous complex64/complex128 CUDA tensor with the splitmix64 U[-1, 1) generator."""
    prec = {torch.complex64: F32, torch.complex128: F64}[t.dtype]
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("fill_uniform needs a contiguous CUDA tensor")
    afft_fill_uniform(t.data_ptr(), t.numel(), seed, prec, _stream_handle(stream))
    return t
