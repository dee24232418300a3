"""Thin ctypes binding of libdfmnmf.so (include/dfmnmf.h).

Argument marshalling only: every step of the computation runs in the CUDA
library.  Functions keep the C names.  Array arguments may be torch tensors
(CUDA or CPU) or numpy arrays; they must be C-contiguous with the dtype the
header states.  ``stream`` defaults to torch's current CUDA stream.

There is no CPU fallback: if the library cannot be loaded every call raises.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libdfmnmf.so")

DFMNMF_OK, DFMNMF_EINVAL, DFMNMF_ENOMEM, DFMNMF_ECUDA, DFMNMF_ENUMERIC, DFMNMF_ETIMEOUT = range(6)
DFMNMF_FP32, DFMNMF_BF16_TC, DFMNMF_TF32_TC = 0, 1, 2
DFMNMF_IP_F64, DFMNMF_IP_F32X2, DFMNMF_IP_F32 = 0, 1, 2
DFMNMF_STAGE_COV, DFMNMF_STAGE_IP, DFMNMF_STAGE_W, DFMNMF_STAGE_H, DFMNMF_STAGE_G = 1, 2, 3, 4, 5
DFMNMF_BUF_V, DFMNMF_BUF_P, DFMNMF_BUF_LAMBDA = 1, 2, 3
DFMNMF_LOSS_NLL, DFMNMF_LOSS_WIENER_MSE = 1, 2
DFMNMF_OPT_BRANCHES, DFMNMF_OPT_NMF_CTAS, DFMNMF_OPT_VX_GROUPS, DFMNMF_OPT_WUPD_TC, DFMNMF_OPT_WAIT_CYCLES = 1, 2, 3, 4, 5

# Every symbol include/dfmnmf.h declares.
EXPORTED = ("dfmnmf_init", "dfmnmf_set_observation", "dfmnmf_iterate", "dfmnmf_run_stage",
            "dfmnmf_loglik", "dfmnmf_separate", "dfmnmf_get_params", "dfmnmf_set_params",
            "dfmnmf_get_buffer", "dfmnmf_launches_per_iteration", "dfmnmf_kernel_times", "dfmnmf_destroy",
            "dfmnmf_last_error", "dfmnmf_version", "dfmnmf_loglik_noalloc", "dfmnmf_autotune",
            "dfmnmf_cost_gradient", "dfmnmf_init_from_images",
            "dfmnmf_batch_create", "dfmnmf_batch_iterate", "dfmnmf_batch_destroy",
            "dfmnmf_adjoint_create", "dfmnmf_adjoint_run", "dfmnmf_adjoint_destroy",
            "dfmnmf_set_option", "dfmnmf_get_option", "dfmnmf_kernel_times_isolated")


class DfmnmfError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"dfmnmf error {code}: {msg}")
        self.code = code


class dfmnmf_desc(ctypes.Structure):
    _fields_ = [("F", ctypes.c_int), ("T", ctypes.c_int), ("K", ctypes.c_int),
                ("mics", ctypes.POINTER(ctypes.c_int)), ("N", ctypes.c_int), ("B", ctypes.c_int),
                ("precision", ctypes.c_int), ("ip_arith", ctypes.c_int), ("floor_eps", ctypes.c_double)]


_lib = None


def load_library(path: Optional[str] = None):
    """Load libdfmnmf.so (building nothing); raises if it is missing."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise DfmnmfError(DFMNMF_ECUDA, f"{p} not found: run paper_2605_19388_gb300/build.py")
    lib = ctypes.CDLL(p)
    vp, ci, cd = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    sig = {
        "dfmnmf_init": (ci, [ctypes.POINTER(vp), ctypes.POINTER(dfmnmf_desc), vp, vp, vp, vp, vp, vp]),
        "dfmnmf_set_observation": (ci, [vp, vp, vp]),
        "dfmnmf_iterate": (ci, [vp, ci, vp]),
        "dfmnmf_run_stage": (ci, [vp, ci, vp]),
        "dfmnmf_loglik": (ci, [vp, ctypes.POINTER(cd), vp]),
        "dfmnmf_separate": (ci, [vp, vp, vp]),
        "dfmnmf_get_params": (ci, [vp, vp, vp, vp, vp, vp]),
        "dfmnmf_set_params": (ci, [vp, vp, vp, vp, vp, vp]),
        "dfmnmf_get_buffer": (ci, [vp, ci, vp, ctypes.c_size_t, vp]),
        "dfmnmf_launches_per_iteration": (ci, [vp]),
        "dfmnmf_kernel_times": (ci, [vp, ci, ctypes.POINTER(cd), ctypes.POINTER(ctypes.c_char_p), ci,
                                     ctypes.POINTER(ci), vp]),
        "dfmnmf_destroy": (None, [vp]),
        "dfmnmf_last_error": (ctypes.c_char_p, []),
        "dfmnmf_version": (ci, []),
        "dfmnmf_loglik_noalloc": (ci, [ctypes.POINTER(dfmnmf_desc), vp, vp, vp, vp, vp, ctypes.POINTER(cd), vp]),
        "dfmnmf_autotune": (ci, [vp, ci, ctypes.POINTER(ci), ctypes.POINTER(ci), vp]),
        "dfmnmf_cost_gradient": (ci, [vp, vp, vp, vp, vp, ctypes.POINTER(cd), vp]),
        "dfmnmf_init_from_images": (ci, [vp, vp, vp, vp]),
        "dfmnmf_batch_create": (ci, [ctypes.POINTER(vp), ctypes.POINTER(vp), ci]),
        "dfmnmf_batch_iterate": (ci, [vp, ci, vp]),
        "dfmnmf_batch_destroy": (None, [vp]),
        "dfmnmf_adjoint_create": (ci, [ctypes.POINTER(vp), vp, ci, ci]),
        "dfmnmf_adjoint_run": (ci, [vp, ci, vp, ctypes.POINTER(cd), vp, vp, vp, vp, vp]),
        "dfmnmf_adjoint_destroy": (None, [vp]),
        "dfmnmf_set_option": (ci, [vp, ci, ci]),
        "dfmnmf_kernel_times_isolated": (ci, [vp, ci, ctypes.POINTER(cd), ctypes.POINTER(ctypes.c_char_p), ci,
                                             ctypes.POINTER(ci), vp]),
        "dfmnmf_get_option": (ci, [vp, ci]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    if path is None:
        _lib = lib
    return lib


def _check(code: int):
    if code != DFMNMF_OK:
        raise DfmnmfError(code, load_library().dfmnmf_last_error().decode())


def _ptr(a, dtype=None):
    """Raw pointer of a torch tensor / numpy array (None -> NULL)."""
    if a is None:
        return None
    try:
        import torch
        if isinstance(a, torch.Tensor):
            if not a.is_contiguous():
                raise ValueError("tensor must be contiguous")
            if dtype is not None and a.dtype != dtype[0]:
                raise TypeError(f"expected {dtype[0]}, got {a.dtype}")
            return a.data_ptr()
    except ImportError:
        pass
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        if dtype is not None and a.dtype != dtype[1]:
            raise TypeError(f"expected {dtype[1]}, got {a.dtype}")
        return a.ctypes.data
    raise TypeError(f"unsupported array type {type(a)}")


def _dt(name):
    import torch
    return {"c64": (torch.complex64, np.complex64), "c128": (torch.complex128, np.complex128),
            "f32": (torch.float32, np.float32)}[name]


def _stream(stream):
    if stream is not None:
        return int(stream) if not hasattr(stream, "cuda_stream") else stream.cuda_stream
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except ImportError:
        pass
    return 0


class Context:
    """Owns one dfmnmf_ctx*; sizes mirror the descriptor."""

    def __init__(self, handle, F, T, mics, N, B, precision, ip_arith):
        self.handle = handle
        self.F, self.T, self.mics, self.N, self.B = F, T, tuple(mics), N, B
        self.K = len(self.mics)
        self.M = int(sum(self.mics))
        self.precision, self.ip_arith = precision, ip_arith

    def __del__(self):
        try:
            dfmnmf_destroy(self)
        except Exception:
            pass


def dfmnmf_init(F: int, T: int, mics: Sequence[int], N: int, B: int, x, W0, H0, g0, Q0=None,
                precision: int = DFMNMF_FP32, ip_arith: int = DFMNMF_IP_F32X2, floor_eps: float = 1e-6,
                stream=None) -> Context:
    lib = load_library()
    mic_arr = (ctypes.c_int * len(mics))(*[int(m) for m in mics])
    d = dfmnmf_desc(int(F), int(T), len(mics), mic_arr, int(N), int(B), int(precision), int(ip_arith),
                    float(floor_eps))
    h = ctypes.c_void_p()
    _check(lib.dfmnmf_init(ctypes.byref(h), ctypes.byref(d), _ptr(x, _dt("c64")), _ptr(W0, _dt("f32")),
                           _ptr(H0, _dt("f32")), _ptr(g0, _dt("f32")), _ptr(Q0, _dt("c128")),
                           _stream(stream)))
    return Context(h, F, T, mics, N, B, precision, ip_arith)


def dfmnmf_set_observation(ctx: Context, x, stream=None):
    _check(load_library().dfmnmf_set_observation(ctx.handle, _ptr(x, _dt("c64")), _stream(stream)))


def dfmnmf_iterate(ctx: Context, n_iter: int, stream=None):
    _check(load_library().dfmnmf_iterate(ctx.handle, int(n_iter), _stream(stream)))


def dfmnmf_run_stage(ctx: Context, stage: int, stream=None):
    _check(load_library().dfmnmf_run_stage(ctx.handle, int(stage), _stream(stream)))


def dfmnmf_loglik(ctx: Context, stream=None) -> float:
    v = ctypes.c_double()
    _check(load_library().dfmnmf_loglik(ctx.handle, ctypes.byref(v), _stream(stream)))
    return v.value


def dfmnmf_separate(ctx: Context, c_out, stream=None):
    _check(load_library().dfmnmf_separate(ctx.handle, _ptr(c_out, _dt("c64")), _stream(stream)))


def dfmnmf_get_params(ctx: Context, Q=None, W=None, H=None, g=None, stream=None):
    _check(load_library().dfmnmf_get_params(ctx.handle, _ptr(Q, _dt("c128")), _ptr(W, _dt("f32")),
                                            _ptr(H, _dt("f32")), _ptr(g, _dt("f32")), _stream(stream)))


def dfmnmf_set_params(ctx: Context, Q=None, W=None, H=None, g=None, stream=None):
    _check(load_library().dfmnmf_set_params(ctx.handle, _ptr(Q, _dt("c128")), _ptr(W, _dt("f32")),
                                            _ptr(H, _dt("f32")), _ptr(g, _dt("f32")), _stream(stream)))


def dfmnmf_get_buffer(ctx: Context, which: int, dst, stream=None):
    nbytes = dst.numel() * dst.element_size() if hasattr(dst, "numel") else dst.nbytes
    _check(load_library().dfmnmf_get_buffer(ctx.handle, int(which), _ptr(dst), nbytes, _stream(stream)))


def dfmnmf_launches_per_iteration(ctx: Context) -> int:
    return load_library().dfmnmf_launches_per_iteration(ctx.handle)


def dfmnmf_kernel_times(ctx: Context, n_iter: int, stream=None):
    """{kernel name: mean milliseconds} over n_iter event-bracketed iterations."""
    cap = 32
    ms = (ctypes.c_double * cap)()
    names = (ctypes.c_char_p * cap)()
    cnt = ctypes.c_int()
    _check(load_library().dfmnmf_kernel_times(ctx.handle, int(n_iter), ms, names, cap, ctypes.byref(cnt),
                                              _stream(stream)))
    out = []
    for i in range(cnt.value):
        out.append((names[i].decode(), ms[i]))
    return out


def dfmnmf_kernel_times_isolated(ctx: Context, reps: int, stream=None):
    """[(kernel name, mean milliseconds per launch)], each kernel alone, reps launches back to back."""
    cap = 32
    ms = (ctypes.c_double * cap)()
    names = (ctypes.c_char_p * cap)()
    cnt = ctypes.c_int()
    _check(load_library().dfmnmf_kernel_times_isolated(ctx.handle, int(reps), ms, names, cap, ctypes.byref(cnt),
                                                       _stream(stream)))
    return [(names[i].decode(), ms[i]) for i in range(cnt.value)]


def dfmnmf_destroy(ctx: Context):
    if ctx.handle is not None and ctx.handle.value:
        load_library().dfmnmf_destroy(ctx.handle)
        ctx.handle = ctypes.c_void_p()


def dfmnmf_cost_gradient(ctx: Context, dQ=None, dW=None, dH=None, dg=None, stream=None) -> float:
    """Gradient of Eq. (12) at the current state into the given arrays (numpy or torch, host or
    device; None skips one); returns the cost."""
    v = ctypes.c_double()
    _check(load_library().dfmnmf_cost_gradient(ctx.handle, _ptr(dQ, _dt("c128")), _ptr(dW, _dt("f32")),
                                                _ptr(dH, _dt("f32")), _ptr(dg, _dt("f32")), ctypes.byref(v),
                                                _stream(stream)))
    return v.value


def dfmnmf_init_from_images(ctx: Context, c_img, h_out=None, stream=None):
    """Sec. IV-A steps 3, 5, 6 from source images c_img (complex64 [N][F][T][M], device):
    sets the context's Q and g; writes h (float32 [N][F][T], device) when h_out is given."""
    _check(load_library().dfmnmf_init_from_images(ctx.handle, _ptr(c_img, _dt("c64")), _ptr(h_out, _dt("f32")),
                                                  _stream(stream)))


def dfmnmf_autotune(ctx: Context, iters_per_trial: int = 5, stream=None):
    """Time the launch-shape candidates and keep the fastest; returns (branches, nmf_ctas)."""
    br, ct = ctypes.c_int(), ctypes.c_int()
    _check(load_library().dfmnmf_autotune(ctx.handle, int(iters_per_trial), ctypes.byref(br), ctypes.byref(ct),
                                          _stream(stream)))
    return br.value, ct.value


def dfmnmf_set_option(ctx: Context, option: int, value: int):
    _check(load_library().dfmnmf_set_option(ctx.handle, int(option), int(value)))


def dfmnmf_get_option(ctx: Context, option: int) -> int:
    return load_library().dfmnmf_get_option(ctx.handle, int(option))


class Batch:
    """Owns one dfmnmf_batch*; keeps its contexts alive."""

    def __init__(self, handle, ctxs):
        self.handle, self.ctxs = handle, list(ctxs)

    def __del__(self):
        try:
            dfmnmf_batch_destroy(self)
        except Exception:  # pragma: no cover
            pass


def dfmnmf_batch_create(ctxs) -> Batch:
    arr = (ctypes.c_void_p * len(ctxs))(*[c.handle.value for c in ctxs])
    h = ctypes.c_void_p()
    _check(load_library().dfmnmf_batch_create(ctypes.byref(h), arr, len(ctxs)))
    return Batch(h, ctxs)


def dfmnmf_batch_iterate(batch: Batch, n_iter: int, stream=None):
    _check(load_library().dfmnmf_batch_iterate(batch.handle, int(n_iter), _stream(stream)))


def dfmnmf_batch_destroy(batch: Batch):
    if batch.handle is not None and batch.handle.value:
        load_library().dfmnmf_batch_destroy(batch.handle)
        batch.handle = ctypes.c_void_p()


class Adjoint:
    """Owns one dfmnmf_adj* (reverse pass through unrolled iterations); keeps its context alive."""

    def __init__(self, handle, ctx, n_iter, every):
        self.handle, self.ctx, self.n_iter, self.every = handle, ctx, n_iter, every

    def __del__(self):
        try:
            dfmnmf_adjoint_destroy(self)
        except Exception:  # pragma: no cover
            pass


def dfmnmf_adjoint_create(ctx: Context, n_iter: int, every: int = 5) -> Adjoint:
    h = ctypes.c_void_p()
    _check(load_library().dfmnmf_adjoint_create(ctypes.byref(h), ctx.handle, int(n_iter), int(every)))
    return Adjoint(h, ctx, int(n_iter), int(every))


def dfmnmf_adjoint_run(adj: Adjoint, loss: int = DFMNMF_LOSS_NLL, c_true=None, dQ0=None, dW0=None, dH0=None,
                       dg0=None, stream=None) -> float:
    """Runs adj.n_iter iterations from the context's state and writes the gradient of the loss of the
    final state with respect to the initial one (float64 arrays, complex128 for Q); returns the loss."""
    import torch
    f64 = (torch.float64, np.float64)
    v = ctypes.c_double()
    _check(load_library().dfmnmf_adjoint_run(adj.handle, int(loss), _ptr(c_true, _dt("c64")), ctypes.byref(v),
                                             _ptr(dQ0, _dt("c128")), _ptr(dW0, f64), _ptr(dH0, f64),
                                             _ptr(dg0, f64), _stream(stream)))
    return v.value


def dfmnmf_adjoint_destroy(adj: Adjoint):
    if adj.handle is not None and adj.handle.value:
        load_library().dfmnmf_adjoint_destroy(adj.handle)
        adj.handle = ctypes.c_void_p()


def dfmnmf_version() -> int:
    return load_library().dfmnmf_version()


def _device_array(a, dtype, numel: int, name: str):
    """Pointer of a C-contiguous torch CUDA tensor on the current device with `numel` elements of `dtype`
    (raises ValueError or TypeError otherwise, before the library is called)."""
    try:
        import torch
    except ImportError:  # pragma: no cover
        raise ValueError(f"{name} must be a torch CUDA tensor")
    if not isinstance(a, torch.Tensor) or not a.is_cuda:
        raise ValueError(f"{name} must be a torch CUDA tensor (device memory), got {type(a).__name__}"
                         + ("" if not isinstance(a, torch.Tensor) else f" on {a.device}"))
    if a.device.index != torch.cuda.current_device():
        raise ValueError(f"{name} is on {a.device}, the current device is cuda:{torch.cuda.current_device()}")
    if a.numel() != numel:
        raise ValueError(f"{name} has {a.numel()} elements, the sizes need {numel}")
    return _ptr(a, dtype)


def dfmnmf_loglik_noalloc(F: int, T: int, mics: Sequence[int], N: int, B: int, x, Q, W, H, g,
                          floor_eps: float = 1e-6, stream=None) -> float:
    """The cost dfmnmf_loglik returns, from caller-held device arrays, with no device allocation (see the
    header).  x, Q, W, H and g must be CUDA tensors on the current device with exactly the element counts
    F T M, F sum(M_k^2), N F B, N B T and F N M: the library cannot check device pointers itself."""
    lib = load_library()
    mics = [int(m) for m in mics]
    M, q = sum(mics), sum(m * m for m in mics)
    ptrs = [_device_array(a, _dt(dt), n, name) for a, dt, n, name in (
        (x, "c64", F * T * M, "x"), (Q, "c128", F * q, "Q"), (W, "f32", N * F * B, "W"),
        (H, "f32", N * B * T, "H"), (g, "f32", F * N * M, "g"))]
    mic_arr = (ctypes.c_int * len(mics))(*mics)
    d = dfmnmf_desc(int(F), int(T), len(mics), mic_arr, int(N), int(B), 0, 0, float(floor_eps))
    v = ctypes.c_double()
    _check(lib.dfmnmf_loglik_noalloc(ctypes.byref(d), *ptrs, ctypes.byref(v), _stream(stream)))
    return v.value


# --------------------------------------------------------------- convenience
def params_numpy(ctx: Context):
    """(Q complex128 [F][sum M_k^2], W, H, g float32) copied to host numpy arrays."""
    Q = np.empty((ctx.F, sum(m * m for m in ctx.mics)), dtype=np.complex128)
    W = np.empty((ctx.N, ctx.F, ctx.B), dtype=np.float32)
    H = np.empty((ctx.N, ctx.B, ctx.T), dtype=np.float32)
    g = np.empty((ctx.F, ctx.N, ctx.M), dtype=np.float32)
    dfmnmf_get_params(ctx, Q, W, H, g)
    return Q, W, H, g


def buffer_numpy(ctx: Context, which: int):
    mk = ctx.mics[0]
    shapes = {DFMNMF_BUF_V: ((ctx.F, ctx.K, mk, mk, mk), np.complex128),
              DFMNMF_BUF_P: ((ctx.F, ctx.T, ctx.M), np.float32),
              DFMNMF_BUF_LAMBDA: ((ctx.N, ctx.F, ctx.T), np.float32)}
    shape, dt = shapes[which]
    out = np.empty(shape, dtype=dt)
    dfmnmf_get_buffer(ctx, which, out)
    return out
