"""GB300-native MoA / psi-calculus radix-2 FFT -- Python binding.

A thin ctypes layer over ``libmoafft.so`` (the C ABI declared in
``include/moafft.h``).  Every function here only marshals arguments (torch
tensors or raw device pointers, streams, strings) and checks status codes;
all transform work runs in the library's CUDA kernels.  PyTorch supplies
device memory, streams and autograd plumbing.

The functions keep the C names: :func:`fft_plan`, :func:`fft_plan_ex`,
:func:`fft_plan_many`, :func:`fft_exec`, :func:`fft_exec_adjoint`,
:func:`fft_destroy`, :func:`fft_last_error`, ... .  :class:`Plan` wraps a
plan handle; :class:`FFTFunction` makes a plan differentiable through its
hand-written adjoint.
"""
from __future__ import annotations

import ctypes
import math
import os

PKG_DIR = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG_DIR, "libmoafft.so")

FFT_C64, FFT_C128 = 0, 1
FFT_FORWARD, FFT_INVERSE = -1, 1
FFT_FORM_PLAIN, FFT_FORM_TC_FP16, FFT_FORM_TC_BF16, FFT_FORM_DF64 = 0, 1, 2, 3

FFT_OK = 0
FFT_ERR_ARG = -1
FFT_ERR_NOT_POW2 = -2
FFT_ERR_DTYPE = -3
FFT_ERR_ALIAS = -4
FFT_ERR_ALLOC = -5
FFT_ERR_CUDA = -6
FFT_ERR_TIMEOUT = -7
FFT_ERR_UNSUPPORTED = -8

STATUS_NAMES = {0: "FFT_OK", -1: "FFT_ERR_ARG", -2: "FFT_ERR_NOT_POW2", -3: "FFT_ERR_DTYPE",
                -4: "FFT_ERR_ALIAS", -5: "FFT_ERR_ALLOC", -6: "FFT_ERR_CUDA",
                -7: "FFT_ERR_TIMEOUT", -8: "FFT_ERR_UNSUPPORTED"}

# every symbol include/moafft.h declares
EXPORTS = ["fft_plan", "fft_plan_ex", "fft_plan_many", "fft_plan_nd", "fft_exec", "fft_exec_adjoint",
           "fft_exec_host", "fft_exec_noalloc", "fft_noalloc_check", "fft_plan_check", "fft_plan_set_wait", "fft_plan_profile", "fft_plan_pass_times", "fft_destroy", "fft_last_error", "fft_describe_schedule", "fft_plan_describe",
           "fft_plan_launches", "fft_plan_workspace_bytes", "fft_set_allocator", "fft_tune_candidates", "fft_version",
           "dm_gate", "dm_transpose_vector"]

_LIB = None

ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


class MoaFFTError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile the CUDA library in-tree (nvcc, sm_103a)."""
    from . import _build
    return _build.build(force=force, verbose=verbose)


def lib():
    """The loaded library.  Raises if it has not been built: there is no
    fallback path."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "paper_0803_2386_gb300.build() (nvcc, sm_103a)")
        L = ctypes.CDLL(LIB_PATH)
        vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
        sig = {
            "fft_plan": (i32, [ctypes.POINTER(vp), i64, i64, i32, i32]),
            "fft_plan_ex": (i32, [ctypes.POINTER(vp), i64, i64, i32, i32, i32, ctypes.c_char_p]),
            "fft_plan_many": (i32, [ctypes.POINTER(vp), ctypes.POINTER(i64), i64, i32, i32]),
            "fft_plan_nd": (i32, [ctypes.POINTER(vp), i32, ctypes.POINTER(i64), i64, i32, i32]),
            "fft_exec": (i32, [vp, vp, vp, vp]),
            "fft_exec_adjoint": (i32, [vp, vp, vp, vp]),
            "fft_exec_host": (i32, [vp, vp, vp, vp]),
            "fft_exec_noalloc": (i32, [vp, vp, i64, i64, i32, i32, vp]),
            "fft_noalloc_check": (i32, []),
            "fft_plan_check": (i32, [vp]),
            "fft_plan_set_wait": (i32, [vp, i64, ctypes.c_int32]),
            "fft_plan_profile": (i32, [vp, i32]),
            "fft_plan_pass_times": (i32, [vp, ctypes.POINTER(ctypes.c_double),
                                          ctypes.POINTER(i64), i32]),
            "fft_destroy": (i32, [vp]),
            "fft_last_error": (ctypes.c_char_p, []),
            "fft_describe_schedule": (i32, [i64, i32, i32, ctypes.c_char_p, ctypes.c_char_p, i64]),
            "fft_plan_describe": (i32, [vp, ctypes.c_char_p, i64]),
            "fft_plan_launches": (i64, [vp]),
            "fft_plan_workspace_bytes": (i64, [vp]),
            "fft_set_allocator": (i32, [ALLOC_FN, FREE_FN, vp]),
            "fft_tune_candidates": (i32, [i64, i32, i32, ctypes.c_char_p, i64]),
            "fft_version": (i32, []),
            "dm_gate": (i32, [vp, i32, ctypes.POINTER(i32), i32, vp, i32, vp]),
            "dm_transpose_vector": (i32, [i32, ctypes.POINTER(i32), i32, ctypes.POINTER(i32)]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _LIB = L
    return _LIB


def fft_last_error() -> str:
    return lib().fft_last_error().decode()


def _check(status: int):
    if status != FFT_OK:
        raise MoaFFTError(status, fft_last_error())


def _ptr(x) -> int:
    if x is None:
        return 0
    if isinstance(x, int):
        return x
    return int(x.data_ptr())


def _stream(stream, *tensors) -> int:
    if stream is None:
        try:
            import torch
            for t in tensors:
                if isinstance(t, torch.Tensor) and t.is_cuda:
                    return int(torch.cuda.current_stream(t.device).cuda_stream)
        except ImportError:
            pass
        return 0
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


def _enc(s):
    return None if s is None else s.encode()


# ------------------------------------------------------------- C names ---

def fft_plan(n: int, batch: int = 1, dtype: int = FFT_C128, direction: int = FFT_FORWARD) -> int:
    h = ctypes.c_void_p()
    _check(lib().fft_plan(ctypes.byref(h), n, batch, dtype, direction))
    return h.value


def fft_plan_ex(n: int, batch: int = 1, dtype: int = FFT_C128, direction: int = FFT_FORWARD,
                form: int = FFT_FORM_PLAIN, schedule: str | None = None) -> int:
    h = ctypes.c_void_p()
    _check(lib().fft_plan_ex(ctypes.byref(h), n, batch, dtype, direction, form, _enc(schedule)))
    return h.value


def fft_plan_many(sizes, dtype: int = FFT_C64, direction: int = FFT_FORWARD) -> int:
    sizes = [int(s) for s in sizes]
    arr = (ctypes.c_int64 * max(1, len(sizes)))(*sizes)
    h = ctypes.c_void_p()
    _check(lib().fft_plan_many(ctypes.byref(h), arr, len(sizes), dtype, direction))
    return h.value


def fft_plan_nd(dims, batch: int = 1, dtype: int = FFT_C128, direction: int = FFT_FORWARD) -> int:
    """Plan over arrays of shape dims (row-major, last axis contiguous)."""
    dims = [int(d) for d in dims]
    arr = (ctypes.c_int64 * max(1, len(dims)))(*dims)
    h = ctypes.c_void_p()
    _check(lib().fft_plan_nd(ctypes.byref(h), len(dims), arr, batch, dtype, direction))
    return h.value


def fft_exec(plan: int, inp, out, stream=None):
    _check(lib().fft_exec(plan, _ptr(inp), _ptr(out), _stream(stream, inp, out)))


def fft_exec_adjoint(plan: int, inp, out, stream=None):
    _check(lib().fft_exec_adjoint(plan, _ptr(inp), _ptr(out), _stream(stream, inp, out)))


def fft_exec_host(plan: int, inp, out, stream=None):
    """Host buffers (numpy arrays, pinned torch CPU tensors or raw ints)."""
    def hp(x):
        if isinstance(x, int):
            return x
        if hasattr(x, "ctypes"):
            return x.ctypes.data
        return int(x.data_ptr())
    _check(lib().fft_exec_host(plan, hp(inp), hp(out), _stream(stream)))


def fft_exec_noalloc(inp, out, n: int, batch: int, dtype: int, direction: int = FFT_FORWARD,
                     stream=None):
    """Plan-free transform that allocates no device memory (fixed in-library
    scratch; see include/moafft.h for the limits)."""
    _check(lib().fft_exec_noalloc(_ptr(inp), _ptr(out), n, batch, dtype, direction,
                                  _stream(stream, inp, out)))


def fft_noalloc_check():
    """Synchronise the current device; raise if a bounded wait of an
    fft_exec_noalloc kernel gave up since the last check (then cleared)."""
    _check(lib().fft_noalloc_check())


def _int_array(values):
    arr = (ctypes.c_int * max(1, len(values)))(*[int(v) for v in values])
    return arr


def dm_transpose_vector(n_qubits: int, qubits) -> list:
    """The hyper-cube transpose vector that gathers the gated qubits (host
    logic; Ch. "Density Matrix Operations", Sec. "The Algorithm")."""
    qb = _int_array(qubits)
    out = (ctypes.c_int * (2 * max(1, n_qubits)))()
    _check(lib().dm_transpose_vector(n_qubits, qb, len(qubits), out))
    return list(out)[:2 * n_qubits]


def dm_gate(rho, qubits, u, stream=None):
    """rho <- G rho G^H in place on the GPU, G = u on the gated qubits.
    rho: square complex64/complex128 CUDA tensor of side 2^n; u: 2^q x 2^q
    (numpy or tensor on any device), converted to rho's dtype."""
    import numpy as np
    side = int(rho.shape[-1])
    n = side.bit_length() - 1
    dt = FFT_C128 if str(rho.dtype).endswith("complex128") else FFT_C64
    uu = np.ascontiguousarray(np.asarray(u.cpu() if hasattr(u, "cpu") else u,
                                         dtype=np.complex128 if dt == FFT_C128 else np.complex64))
    qb = _int_array(qubits)
    _check(lib().dm_gate(_ptr(rho), n, qb, len(qubits), uu.ctypes.data, dt, _stream(stream, rho)))


def fft_plan_check(plan: int):
    """Synchronise; raise on a recorded device-side timeout or CUDA error."""
    _check(lib().fft_plan_check(plan))


def fft_plan_set_wait(plan: int, limit_cycles: int = 2000000000, target_offset: int = 0):
    """Bounded waits of a persistent uneven plan: the poll limit in SM
    cycles, and an offset added to every wait's target (nonzero makes every
    wait run out: failure-detection tests)."""
    _check(lib().fft_plan_set_wait(plan, int(limit_cycles), int(target_offset)))


def fft_plan_profile(plan: int, enable: bool = True):
    _check(lib().fft_plan_profile(plan, 1 if enable else 0))


def fft_plan_pass_times(plan: int, max_passes: int = 8):
    """[(total_ms, launches) per pass] since the last read (resets them)."""
    ms = (ctypes.c_double * max_passes)()
    cnt = (ctypes.c_int64 * max_passes)()
    k = lib().fft_plan_pass_times(plan, ms, cnt, max_passes)
    if k < 0:
        _check(k)
    return [(ms[i], cnt[i]) for i in range(k)]


def fft_destroy(plan: int):
    _check(lib().fft_destroy(plan))


def fft_describe_schedule(n: int, dtype: int = FFT_C128, form: int = FFT_FORM_PLAIN,
                          schedule: str | None = None) -> str:
    buf = ctypes.create_string_buffer(8192)
    _check(lib().fft_describe_schedule(n, dtype, form, _enc(schedule), buf, len(buf)))
    return buf.value.decode()


def fft_plan_describe(plan: int) -> str:
    buf = ctypes.create_string_buffer(16384)
    _check(lib().fft_plan_describe(plan, buf, len(buf)))
    return buf.value.decode()


def fft_plan_launches(plan: int) -> int:
    return int(lib().fft_plan_launches(plan))


def fft_plan_workspace_bytes(plan: int) -> int:
    return int(lib().fft_plan_workspace_bytes(plan))


_ALLOC_KEEP = []


def fft_set_allocator(alloc=None, release=None, ctx=None):
    """alloc(bytes) -> device pointer (int) or 0; release(ptr).  None, None
    restores cudaMalloc/cudaFree."""
    if alloc is None and release is None:
        _check(lib().fft_set_allocator(ALLOC_FN(), FREE_FN(), None))
        _ALLOC_KEEP.clear()
        return
    a = ALLOC_FN(lambda nbytes, _c: alloc(nbytes) or None)
    f = FREE_FN(lambda p, _c: release(p))
    _ALLOC_KEEP[:] = [a, f]
    _check(lib().fft_set_allocator(a, f, ctx))


def fft_tune_candidates(n: int, dtype: int = FFT_C64, form: int = FFT_FORM_PLAIN) -> list:
    import json
    buf = ctypes.create_string_buffer(65536)
    _check(lib().fft_tune_candidates(n, dtype, form, buf, len(buf)))
    return json.loads(buf.value.decode())


def fft_version() -> int:
    return int(lib().fft_version())


# ------------------------------------------------------------ wrappers ---

def _dtype_code(t) -> int:
    import torch
    if t.dtype == torch.complex128:
        return FFT_C128
    if t.dtype == torch.complex64:
        return FFT_C64
    raise TypeError(f"unsupported dtype {t.dtype}: complex64 or complex128")


class Plan:
    """Owning wrapper of a plan handle (destroyed on close/garbage collection)."""

    def __init__(self, n: int, batch: int = 1, dtype: int = FFT_C128,
                 direction: int = FFT_FORWARD, form: int = FFT_FORM_PLAIN,
                 schedule: str | None = None):
        self.n, self.batch, self.dtype, self.direction, self.form = n, batch, dtype, direction, form
        self.handle = fft_plan_ex(n, batch, dtype, direction, form, schedule)

    def exec(self, inp, out, stream=None):
        fft_exec(self.handle, inp, out, stream)
        return out

    def exec_adjoint(self, inp, out, stream=None):
        fft_exec_adjoint(self.handle, inp, out, stream)
        return out

    def describe(self) -> str:
        return fft_plan_describe(self.handle)

    @property
    def launches(self) -> int:
        return fft_plan_launches(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            fft_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


_PLAN_CACHE: dict = {}


def _cached_plan(n, batch, dtype, direction, form=FFT_FORM_PLAIN, schedule=None) -> Plan:
    import torch
    key = (n, batch, dtype, direction, form, schedule, torch.cuda.current_device())
    p = _PLAN_CACHE.get(key)
    if p is None:
        p = Plan(n, batch, dtype, direction, form, schedule)
        _PLAN_CACHE[key] = p
    return p


def fft(x, inverse: bool = False, form: int = FFT_FORM_PLAIN, schedule: str | None = None):
    """Transform the last axis of a contiguous complex CUDA tensor."""
    import torch
    x = x.contiguous()
    n = x.shape[-1]
    batch = x.numel() // max(n, 1)
    p = _cached_plan(n, batch, _dtype_code(x), FFT_INVERSE if inverse else FFT_FORWARD, form,
                     schedule)
    out = torch.empty_like(x)
    p.exec(x, out)
    return out


def ifft(x, form: int = FFT_FORM_PLAIN, schedule: str | None = None):
    return fft(x, inverse=True, form=form, schedule=schedule)


class PlanND(Plan):
    """Owning wrapper of a multi-dimensional plan (fft_plan_nd)."""

    def __init__(self, dims, batch: int = 1, dtype: int = FFT_C128, direction: int = FFT_FORWARD):
        self.dims = tuple(int(d) for d in dims)
        self.n = math.prod(self.dims)
        self.batch, self.dtype, self.direction, self.form = batch, dtype, direction, FFT_FORM_PLAIN
        self.handle = fft_plan_nd(self.dims, batch, dtype, direction)


def fftn(x, ndim: int | None = None, inverse: bool = False):
    """Transform the last `ndim` axes (default: all) of a contiguous complex
    CUDA tensor; the leading axes are the batch."""
    import torch
    x = x.contiguous()
    ndim = x.dim() if ndim is None else ndim
    if not 1 <= ndim <= min(x.dim(), 8):
        raise ValueError(f"fftn: ndim = {ndim} for a tensor of {x.dim()} axes (1..8 axes)")
    dims = tuple(x.shape[x.dim() - ndim:])
    batch = x.numel() // max(math.prod(dims), 1)
    key = ("nd", dims, batch, _dtype_code(x), inverse, torch.cuda.current_device())
    p = _PLAN_CACHE.get(key)
    if p is None:
        p = PlanND(dims, batch, _dtype_code(x), FFT_INVERSE if inverse else FFT_FORWARD)
        _PLAN_CACHE[key] = p
    out = torch.empty_like(x)
    p.exec(x, out)
    return out


def ifftn(x, ndim: int | None = None):
    return fftn(x, ndim, inverse=True)


def _make_autograd():
    import torch

    class FFTFunction(torch.autograd.Function):
        """y = F x with the plan's operator; backward applies the adjoint F^H
        through fft_exec_adjoint.  PyTorch's convention for a real loss L of
        complex y: grad_y = dL/dRe(y) + i dL/dIm(y); then grad_x = F^H grad_y."""

        @staticmethod
        def forward(ctx, x, inverse=False, form=FFT_FORM_PLAIN, schedule=None):
            x = x.contiguous()
            n = x.shape[-1]
            p = _cached_plan(n, x.numel() // n, _dtype_code(x),
                             FFT_INVERSE if inverse else FFT_FORWARD, form, schedule)
            ctx.plan = p
            out = torch.empty_like(x)
            p.exec(x, out)
            return out

        @staticmethod
        def backward(ctx, g):
            g = g.contiguous()
            gx = torch.empty_like(g)
            ctx.plan.exec_adjoint(g, gx)
            return gx, None, None, None

    return FFTFunction


_FFTFunction = None


def fft_autograd(x, inverse: bool = False, form: int = FFT_FORM_PLAIN, schedule=None):
    """Differentiable transform of the last axis (hand-written adjoint)."""
    global _FFTFunction
    if _FFTFunction is None:
        _FFTFunction = _make_autograd()
    return _FFTFunction.apply(x, inverse, form, schedule)


def _make_autograd_nd():
    import torch

    class FFTNFunction(torch.autograd.Function):
        """y = F x over the last `ndim` axes (fft_plan_nd); backward applies
        the adjoint F^H through fft_exec_adjoint."""

        @staticmethod
        def forward(ctx, x, ndim, inverse=False):
            x = x.contiguous()
            dims = tuple(x.shape[x.dim() - ndim:])
            batch = x.numel() // max(math.prod(dims), 1)
            key = ("nd", dims, batch, _dtype_code(x), inverse, torch.cuda.current_device())
            p = _PLAN_CACHE.get(key)
            if p is None:
                p = PlanND(dims, batch, _dtype_code(x), FFT_INVERSE if inverse else FFT_FORWARD)
                _PLAN_CACHE[key] = p
            ctx.plan = p
            out = torch.empty_like(x)
            p.exec(x, out)
            return out

        @staticmethod
        def backward(ctx, g):
            g = g.contiguous()
            gx = torch.empty_like(g)
            ctx.plan.exec_adjoint(g, gx)
            return gx, None, None

    return FFTNFunction


_FFTNFunction = None


def fftn_autograd(x, ndim: int | None = None, inverse: bool = False):
    """Differentiable transform of the last `ndim` axes (default: all)."""
    global _FFTNFunction
    if _FFTNFunction is None:
        _FFTNFunction = _make_autograd_nd()
    ndim = x.dim() if ndim is None else ndim
    if not 1 <= ndim <= min(x.dim(), 8):
        raise ValueError(f"fftn_autograd: ndim = {ndim} for a tensor of {x.dim()} axes (1..8 axes)")
    return _FFTNFunction.apply(x, ndim, inverse)
