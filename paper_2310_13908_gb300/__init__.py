"""Python binding of libstokesreg (regularized Stokes layer sums on GB300).

Thin ctypes marshalling over the C ABI declared in include/stokesreg.h; the
functions keep the C names. Every step of an evaluation runs in the CUDA
library: this module only converts arrays to pointers. Host arrays are numpy
float64 (mem = SK_HOST); device arrays are CUDA float64 torch tensors
(mem = SK_DEVICE), whose memory and streams come from PyTorch.

Importing the package does not load the library; the first call does, and
fails loudly (RuntimeError) if libstokesreg.so has not been built: there is
no CPU fallback.
"""

from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libstokesreg.so")

SK_OK, SK_EINVAL, SK_ENOMEM, SK_ECUDA, SK_EBUSY, SK_EAGAIN, SK_ETIMEOUT, SK_ENOTIMPL = range(8)
SK_FP64, SK_FP32C = 0, 1
SK_HOST, SK_DEVICE = 0, 1

_NAMES = {SK_OK: "SK_OK", SK_EINVAL: "SK_EINVAL", SK_ENOMEM: "SK_ENOMEM", SK_ECUDA: "SK_ECUDA",
          SK_EBUSY: "SK_EBUSY", SK_EAGAIN: "SK_EAGAIN", SK_ETIMEOUT: "SK_ETIMEOUT",
          SK_ENOTIMPL: "SK_ENOTIMPL"}

_lib = None
_vp = ctypes.c_void_p
_i64 = ctypes.c_int64
_dbl = ctypes.c_double
_int = ctypes.c_int


class SkError(RuntimeError):
    """A library call returned a status other than SK_OK; .code holds it."""
    def __init__(self, code: int, message: str):
        super().__init__(f"{_NAMES.get(code, code)}: {message}")
        self.code = code


class sk_peaks(ctypes.Structure):
    """sk_peaks of stokesreg.h: measured FFMA2 / DFMA throughput and far-pair rate."""
    _fields_ = [("ffma2_tflops", ctypes.c_double), ("dfma_tflops", ctypes.c_double),
                ("far_pairs_per_s", ctypes.c_double), ("sm_count", ctypes.c_int32)]


class sk_eval_stats(ctypes.Structure):
    """sk_eval_stats of stokesreg.h: counters of the most recent evaluation."""
    _fields_ = [("n_src_active", ctypes.c_int64), ("n_tgt", ctypes.c_int64),
                ("near_pairs", ctypes.c_int64), ("overflow_targets", ctypes.c_int64),
                ("kernel_launches", ctypes.c_int64), ("n_chunks", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("pair_ms", ctypes.c_double),
                ("eval_ms", ctypes.c_double), ("finish_fused", ctypes.c_int32)]


def _declare(lib):
    lib.sk_version.restype = _int
    lib.sk_create.argtypes = [ctypes.POINTER(_vp), _int, ctypes.c_size_t]
    lib.sk_create.restype = _int
    lib.sk_destroy.argtypes = [_vp]
    lib.sk_destroy.restype = None
    lib.sk_last_error.argtypes = [_vp]
    lib.sk_last_error.restype = ctypes.c_char_p
    lib.sk_set_fp32c_thresholds.argtypes = [_vp, _dbl, _dbl]
    lib.sk_set_fp32c_thresholds.restype = _int
    lib.sk_last_eval_stats.argtypes = [_vp, ctypes.POINTER(sk_eval_stats)]
    lib.sk_last_eval_stats.restype = _int
    lib.sk_probe_peaks.argtypes = [_vp, ctypes.POINTER(sk_peaks)]
    lib.sk_probe_peaks.restype = _int
    lib.sk_set_profiling.argtypes = [_vp, _int]
    lib.sk_set_profiling.restype = _int
    lib.stokes_sl_eval.argtypes = [_vp, _int, _int, _i64, _vp, _vp, _vp, _i64, _vp, _vp, _i64,
                                   _dbl, _vp, _vp]
    lib.stokes_sl_eval.restype = _int
    lib.stokes_dl_eval.argtypes = [_vp, _int, _int, _i64, _vp, _vp, _vp, _vp, _i64, _vp, _vp,
                                   _i64, _vp, _vp]
    lib.stokes_dl_eval.restype = _int
    for name, args in _EXTRA_DECLS.items():
        if hasattr(lib, name):
            getattr(lib, name).argtypes = args[0]
            getattr(lib, name).restype = args[1]


_EXTRA_DECLS: dict = {
    "stokes_sl_eval_noalloc": ([_i64, _vp, _vp, _vp, _i64, _vp, _vp, _i64, _dbl, _vp, _vp], _int),
    "serve_create": ([_vp, _vp, ctypes.POINTER(_vp)], _int),
    "serve_submit": ([_vp, _vp, ctypes.POINTER(ctypes.c_uint64)], _int),
    "serve_poll": ([_vp, ctypes.c_uint64, _vp, _vp, ctypes.c_int64], _int),
    "serve_destroy": ([_vp], None),
    "capsule_create": ([_vp, ctypes.POINTER(_vp), _int, _vp, _vp, _vp, _i64, _dbl, _int], _int),
    "capsule_step": ([_vp, _int, _dbl, _vp, _vp], _int),
    "capsule_get": ([_vp, _vp], _int),
    "capsule_set_membrane": ([_vp, _vp, _dbl, _dbl], _int),
    "capsule_set_upsampling": ([_vp, _int], _int),
    "capsule_shape_moments": ([_vp, _vp], _int),
    "capsule_integrate_rkf45": ([_vp, _dbl, ctypes.POINTER(_dbl), _dbl, _vp, _vp, _i64,
                                 ctypes.POINTER(ctypes.c_int64)], _int),
    "capsule_area_volume": ([_vp, ctypes.POINTER(_dbl), ctypes.POINTER(_dbl)], _int),
    "surface_derivatives": ([_vp, _int, _int, _i64, _vp, _vp, _vp, _vp], _int),
    "membrane_force": ([_vp, _int, _int, _vp, _vp, _dbl, _dbl, _vp, _vp, _vp], _int),
    "stokes_sl_eval_upsampled": ([_vp, _int, _int, _int, _vp, _vp, _vp, _dbl, _vp, _vp], _int),
    "stokes_sl_eval_fmm": ([_vp, _int, _int, _i64, _vp, _vp, _vp, _i64, _vp, _vp, _i64, _dbl, _int, _vp,
                            _int, _int, _vp, _vp], _int),
    "capsule_destroy": ([_vp], None),
}


def load():
    """Load libstokesreg.so (RuntimeError if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build the CUDA library first "
                           "(python -c 'import __graft_entry__ as g; g.build()')")
    lib = ctypes.CDLL(LIB_PATH)
    _declare(lib)
    _lib = lib
    return lib


def _check(ctx, code):
    if code != SK_OK:
        raise SkError(code, load().sk_last_error(ctx).decode())


def sk_version() -> int:
    """Library version as an integer (100 for 0.1.0)."""
    return load().sk_version()


def sk_create(device: int = 0, workspace_bytes: int = 0):
    """Create a context on a CUDA device; workspace_bytes = 0 grows it on demand."""
    h = _vp()
    code = load().sk_create(ctypes.byref(h), int(device), int(workspace_bytes))
    if code != SK_OK:
        raise SkError(code, load().sk_last_error(None).decode())
    return h


def sk_destroy(ctx) -> None:
    """Release the context, its stream and workspace (None is ignored)."""
    if ctx:
        load().sk_destroy(ctx)


def sk_last_error(ctx) -> str:
    """Message of the last failure on ctx (or of sk_create when ctx is None)."""
    return load().sk_last_error(ctx).decode()


def sk_set_fp32c_thresholds(ctx, rho_T: float, rho_c: float) -> None:
    """SK_FP32C regime thresholds: FP64 series below rho_T, plain kernel from rho_c."""
    _check(ctx, load().sk_set_fp32c_thresholds(ctx, float(rho_T), float(rho_c)))


def sk_set_profiling(ctx, enable: bool) -> None:
    """Record device times of the pair kernel and of whole evaluations (stats)."""
    _check(ctx, load().sk_set_profiling(ctx, 1 if enable else 0))


def sk_probe_peaks(ctx) -> dict:
    """Measured FFMA2 / DFMA throughput and the far-field pair-loop ceiling."""
    p = sk_peaks()
    _check(ctx, load().sk_probe_peaks(ctx, ctypes.byref(p)))
    return {f[0]: getattr(p, f[0]) for f in p._fields_}


def sk_last_eval_stats(ctx) -> dict:
    """Counters of the most recent evaluation on ctx (waits for it to finish)."""
    st = sk_eval_stats()
    _check(ctx, load().sk_last_eval_stats(ctx, ctypes.byref(st)))
    return {f[0]: getattr(st, f[0]) for f in st._fields_}


# ---- array marshalling ------------------------------------------------------

def _is_torch(a) -> bool:
    return type(a).__module__.startswith("torch")


def _ptr(a, mem: int, shape_tail, name: str):
    """Pointer of a float64 C-contiguous array in the expected memory space."""
    if a is None:
        return None, 0
    if mem == SK_DEVICE:
        if not _is_torch(a) or not a.is_cuda:
            raise TypeError(f"{name}: SK_DEVICE expects a CUDA torch tensor")
        import torch
        if a.dtype != torch.float64 or not a.is_contiguous():
            raise TypeError(f"{name}: expected a contiguous float64 tensor")
        n = a.shape[0] if a.dim() > 0 else 1
        if shape_tail and tuple(a.shape[1:]) != tuple(shape_tail):
            raise ValueError(f"{name}: expected shape (n, {shape_tail})")
        return a.data_ptr(), n
    arr = np.ascontiguousarray(a, dtype=np.float64)
    if shape_tail:
        tail = tuple(shape_tail)
        if (arr.ndim >= 2 and tuple(arr.shape[1:]) != tail) or \
                (arr.ndim <= 1 and arr.size % int(np.prod(tail)) != 0):
            raise ValueError(f"{name}: expected shape (n, {', '.join(map(str, tail))}), "
                             f"got {arr.shape}")
        arr = arr.reshape((-1,) + tail)
    else:
        if arr.ndim > 1:
            raise ValueError(f"{name}: expected a vector, got shape {arr.shape}")
        arr = arr.reshape(-1)
    return arr, arr.shape[0]


def _host_ptr(arr):
    return None if arr is None else arr.ctypes.data_as(_vp)


def _stream_handle(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream  # torch.cuda.Stream


def _alloc_out(like_tensor, mem, M):
    if mem == SK_DEVICE:
        import torch
        return torch.empty((M, 3), dtype=torch.float64, device=like_tensor.device)
    return np.empty((M, 3), dtype=np.float64)


def stokes_sl_eval(ctx, precision: int, mem: int, src_xyz, src_w, f, tgt_xyz, delta,
                   mu: float = 1.0, u_out=None, stream=None):
    """Regularized single layer (Sec. 3.4, Eq. regstokes). Returns u_out (M, 3).

    stream=None makes the call synchronous; a torch.cuda.Stream (or raw
    handle) enqueues it asynchronously on that stream.
    """
    lib = load()
    X, n = _ptr(src_xyz, mem, (3,), "src_xyz")
    W, nw = _ptr(src_w, mem, (), "src_w")
    F, nf = _ptr(f, mem, (3,), "f")
    Y, M = _ptr(tgt_xyz, mem, (3,), "tgt_xyz")
    D, nd = _ptr(delta if mem == SK_DEVICE or not np.isscalar(delta) else [delta], mem, (),
                 "delta")
    if not (n == nw == nf):
        raise ValueError("src_xyz, src_w and f must have the same number of nodes")
    if u_out is None:
        u_out = _alloc_out(tgt_xyz, mem, M)
    U, _ = _ptr(u_out, mem, (3,), "u_out")
    if mem == SK_HOST:
        args = [_host_ptr(X), _host_ptr(W), _host_ptr(F), M, _host_ptr(Y), _host_ptr(D), nd,
                float(mu), _host_ptr(U)]
    else:
        args = [X, W, F, M, Y, D, nd, float(mu), U]
    code = lib.stokes_sl_eval(ctx, int(precision), int(mem), n, *args, _stream_handle(stream))
    _check(ctx, code)
    if mem == SK_HOST and U is not u_out:
        np.copyto(u_out, U.reshape(np.shape(u_out)))
    return u_out


def stokes_dl_eval(ctx, precision: int, mem: int, src_xyz, src_w, src_n, q, tgt_xyz, delta,
                   u_out=None, stream=None):
    """Regularized double layer (stresslet). Returns u_out (M, 3)."""
    lib = load()
    X, n = _ptr(src_xyz, mem, (3,), "src_xyz")
    W, nw = _ptr(src_w, mem, (), "src_w")
    Nn, nn = _ptr(src_n, mem, (3,), "src_n")
    Q, nq = _ptr(q, mem, (3,), "q")
    Y, M = _ptr(tgt_xyz, mem, (3,), "tgt_xyz")
    D, nd = _ptr(delta if mem == SK_DEVICE or not np.isscalar(delta) else [delta], mem, (),
                 "delta")
    if not (n == nw == nn == nq):
        raise ValueError("src_xyz, src_w, src_n and q must have the same number of nodes")
    if u_out is None:
        u_out = _alloc_out(tgt_xyz, mem, M)
    U, _ = _ptr(u_out, mem, (3,), "u_out")
    if mem == SK_HOST:
        args = [_host_ptr(X), _host_ptr(W), _host_ptr(Nn), _host_ptr(Q), M, _host_ptr(Y),
                _host_ptr(D), nd, _host_ptr(U)]
    else:
        args = [X, W, Nn, Q, M, Y, D, nd, U]
    code = lib.stokes_dl_eval(ctx, int(precision), int(mem), n, *args, _stream_handle(stream))
    _check(ctx, code)
    if mem == SK_HOST and U is not u_out:
        np.copyto(u_out, U.reshape(np.shape(u_out)))
    return u_out


def surface_derivatives(ctx, m: int, mem: int, g, stream=None):
    """u- and v-derivatives of node fields g (N, F) by the overset finite
    differences of Sec. 3.5. Returns (g_u, g_v), each (N, F)."""
    lib = load()
    if mem == SK_DEVICE:
        if not _is_torch(g) or not g.is_cuda:
            raise TypeError("g: SK_DEVICE expects a CUDA torch tensor")
        import torch
        G = g.reshape(g.shape[0], -1).contiguous().to(torch.float64)
        gu, gv = torch.empty_like(G), torch.empty_like(G)
        F = G.shape[1]
        _check(ctx, lib.surface_derivatives(ctx, int(m), SK_DEVICE, F, G.data_ptr(),
                                            gu.data_ptr(), gv.data_ptr(), _stream_handle(stream)))
        return gu.reshape(g.shape), gv.reshape(g.shape)
    G = np.ascontiguousarray(g, dtype=np.float64)
    flat = G.reshape(G.shape[0], -1)
    gu, gv = np.empty_like(flat), np.empty_like(flat)
    _check(ctx, lib.surface_derivatives(ctx, int(m), SK_HOST, flat.shape[1], _host_ptr(flat),
                                        _host_ptr(gu), _host_ptr(gv), None))
    return gu.reshape(G.shape), gv.reshape(G.shape)


def membrane_force(ctx, m: int, mem: int, X, X_ref, Es: float, ED: float, weights: bool = False,
                   stream=None):
    """Skalak force f = div_gamma Lambda (Sec. 2.1) at nodes X with reference
    X_ref; returns f (N, 3), or (f, w) with the quadrature weights."""
    lib = load()
    Xa, N = _ptr(X, mem, (3,), "X")
    Xr, Nr = _ptr(X_ref, mem, (3,), "X_ref")
    if N != Nr:
        raise ValueError("X and X_ref must hold the same nodes")
    if mem == SK_DEVICE:
        import torch
        f = torch.empty((N, 3), dtype=torch.float64, device=X.device)
        w = torch.empty((N,), dtype=torch.float64, device=X.device) if weights else None
        args = [Xa, Xr, float(Es), float(ED), f.data_ptr(), w.data_ptr() if weights else None]
    else:
        f = np.empty((N, 3))
        w = np.empty(N) if weights else None
        args = [_host_ptr(Xa), _host_ptr(Xr), float(Es), float(ED), _host_ptr(f), _host_ptr(w)]
    _check(ctx, lib.membrane_force(ctx, int(m), int(mem), *args, _stream_handle(stream)))
    return (f, w) if weights else f


def stokes_sl_eval_upsampled(ctx, precision: int, mem: int, m: int, X, W, f, mu: float = 1.0,
                             stream=None):
    """Single layer at the m-th order nodes from the four-times upsampled grid
    (Sec. 3.4). Returns u (N, 3)."""
    lib = load()
    Xa, N = _ptr(X, mem, (3,), "X")
    Wa, nw = _ptr(W, mem, (), "W")
    Fa, nf = _ptr(f, mem, (3,), "f")
    if not (N == nw == nf):
        raise ValueError("X, W and f must hold the same nodes")
    if mem == SK_DEVICE:
        import torch
        u = torch.empty((N, 3), dtype=torch.float64, device=X.device)
        args = [Xa, Wa, Fa, float(mu), u.data_ptr()]
    else:
        u = np.empty((N, 3))
        args = [_host_ptr(Xa), _host_ptr(Wa), _host_ptr(Fa), float(mu), _host_ptr(u)]
    _check(ctx, lib.stokes_sl_eval_upsampled(ctx, int(precision), int(mem), int(m), *args,
                                             _stream_handle(stream)))
    return u


def stokes_sl_eval_fmm(ctx, mem: int, src_xyz, src_w, f, tgt_xyz, delta, mu: float, centers0,
                       lloyd_iters: int = 10, p: int = 6, stream=None, precision: int = SK_FP64):
    """Single layer by the single-level FMM of Sec. 5 (SK_FP64 or SK_FP32C).
    Returns u (M, 3)."""
    lib = load()
    X, n = _ptr(src_xyz, mem, (3,), "src_xyz")
    W, nw = _ptr(src_w, mem, (), "src_w")
    F, nf = _ptr(f, mem, (3,), "f")
    Y, M = _ptr(tgt_xyz, mem, (3,), "tgt_xyz")
    D, nd = _ptr(delta if mem == SK_DEVICE or not np.isscalar(delta) else [delta], mem, (),
                 "delta")
    C, k = _ptr(centers0, mem, (3,), "centers0")
    if not (n == nw == nf):
        raise ValueError("src_xyz, src_w and f must have the same number of nodes")
    u = _alloc_out(tgt_xyz, mem, M)
    if mem == SK_HOST:
        args = [_host_ptr(X), _host_ptr(W), _host_ptr(F), M, _host_ptr(Y), _host_ptr(D), nd,
                float(mu), k, _host_ptr(C), int(lloyd_iters), int(p), _host_ptr(u)]
    else:
        args = [X, W, F, M, Y, D, nd, float(mu), k, C, int(lloyd_iters), int(p), u.data_ptr()]
    _check(ctx, lib.stokes_sl_eval_fmm(ctx, int(precision), int(mem), n, *args,
                                       _stream_handle(stream)))
    return u


SK_FLOW_NONE, SK_FLOW_SHEAR, SK_FLOW_POISEUILLE = 0, 1, 2


class sk_flow(ctypes.Structure):
    """sk_flow of stokesreg.h: background flow (kind, rate, alpha, R0)."""
    _fields_ = [("kind", ctypes.c_int32), ("rate", ctypes.c_double), ("alpha", ctypes.c_double),
                ("R0", ctypes.c_double)]


class Capsule:
    """Surface nodes advanced by explicit Euler steps (capsule_* of the C ABI)."""

    def __init__(self, ctx, m: int, X, w, delta=None, mu: float = 1.0,
                 precision: int = SK_FP32C):
        Xa, N = _ptr(X, SK_HOST, (3,), "X")
        Wa, _ = _ptr(w, SK_HOST, (), "w")
        if N != 6 * (m - 1) ** 2:
            raise ValueError("X must hold 6 (m-1)^2 nodes")
        D, nd = (None, 0) if delta is None else _ptr(np.atleast_1d(delta), SK_HOST, (), "delta")
        h = _vp()
        _check(ctx, load().capsule_create(ctx, ctypes.byref(h), int(m), _host_ptr(Xa),
                                          _host_ptr(Wa), _host_ptr(D), nd, float(mu),
                                          int(precision)))
        self.ctx, self.handle, self.N = ctx, h, N

    def step(self, n_steps: int, dt: float, f, flow=None):
        """flow: None or (kind, rate, alpha, R0); f None: the membrane force."""
        F, _ = _ptr(f, SK_HOST, (3,), "f") if f is not None else (None, 0)
        fl = ctypes.byref(sk_flow(*flow)) if flow is not None else None
        _check(self.ctx, load().capsule_step(self.handle, int(n_steps), float(dt), fl,
                                             _host_ptr(F)))

    def set_membrane(self, X_ref, Es: float, ED: float):
        """Skalak membrane with stress-free reference X_ref (Sec. 2.1)."""
        Xr, N = _ptr(X_ref, SK_HOST, (3,), "X_ref")
        if N != self.N:
            raise ValueError("X_ref must hold the capsule's nodes")
        _check(self.ctx, load().capsule_set_membrane(self.handle, _host_ptr(Xr), float(Es),
                                                     float(ED)))

    def integrate_rkf45(self, t_end: float, dt: float, tol: float = 1e-6, f=None, flow=None,
                        max_steps: int = 100000):
        """Adaptive RKF45 over t_end (Sec. 3.6); returns (next dt, accepted, rejected)."""
        F, _ = _ptr(f, SK_HOST, (3,), "f") if f is not None else (None, 0)
        fl = ctypes.byref(sk_flow(*flow)) if flow is not None else None
        d = ctypes.c_double(dt)
        stats = (ctypes.c_int64 * 2)()
        _check(self.ctx, load().capsule_integrate_rkf45(self.handle, float(t_end), ctypes.byref(d),
                                                        float(tol), fl, _host_ptr(F),
                                                        int(max_steps), stats))
        return d.value, int(stats[0]), int(stats[1])

    def set_upsampling(self, factor: int):
        """Single layer of every step on the 4x upsampled grid (4) or not (1)."""
        _check(self.ctx, load().capsule_set_upsampling(self.handle, int(factor)))

    def shape_moments(self):
        """(A, V, centroid (3,), inertia tensor about the centroid (3, 3))."""
        out = np.zeros(14)
        _check(self.ctx, load().capsule_shape_moments(self.handle, out.ctypes.data_as(_vp)))
        return out[0], out[1], out[2:5].copy(), out[5:].reshape(3, 3).copy()

    def area_volume(self):
        a, v = ctypes.c_double(), ctypes.c_double()
        _check(self.ctx, load().capsule_area_volume(self.handle, ctypes.byref(a),
                                                    ctypes.byref(v)))
        return a.value, v.value

    def positions(self):
        X = np.empty((self.N, 3))
        _check(self.ctx, load().capsule_get(self.handle, X.ctypes.data_as(_vp)))
        return X

    def close(self):
        if self.handle:
            load().capsule_destroy(self.handle)
            self.handle = None


class sk_serve_cfg(ctypes.Structure):
    """sk_serve_cfg of stokesreg.h: server limits (0 selects the default)."""
    _fields_ = [("max_slots", ctypes.c_int32), ("queue_capacity", ctypes.c_int32),
                ("hbm_budget_bytes", ctypes.c_size_t), ("idle_exit_us", ctypes.c_int64),
                ("host_staging_bytes", ctypes.c_size_t)]


class sk_request(ctypes.Structure):
    """sk_request of stokesreg.h: one single-layer request (host arrays), or
    Euler steps of a resident capsule (capsule != NULL)."""
    _fields_ = [("n_src", ctypes.c_int64), ("src_xyz", _vp), ("src_w", _vp), ("f", _vp),
                ("n_tgt", ctypes.c_int64), ("tgt_xyz", _vp), ("delta", _vp),
                ("n_delta", ctypes.c_int64), ("mu", ctypes.c_double),
                ("capsule", _vp), ("n_steps", ctypes.c_int32), ("dt", ctypes.c_double),
                ("flow", sk_flow)]


class sk_req_stats(ctypes.Structure):
    """sk_req_stats of stokesreg.h: phase timestamps and sizes of a served request."""
    _fields_ = [("submit_us", ctypes.c_double), ("admit_us", ctypes.c_double),
                ("publish_us", ctypes.c_double), ("done_us", ctypes.c_double),
                ("ready_us", ctypes.c_double), ("interactions", ctypes.c_int64),
                ("n_chunks", ctypes.c_int32), ("status", ctypes.c_int32)]


def serve_create(ctx, max_slots: int = 0, queue_capacity: int = 0, hbm_budget_bytes: int = 0,
                 idle_exit_us: int = 0, host_staging_bytes: int = 0):
    """Start a continuous-batching server on ctx (0 = default for every knob)."""
    cfg = sk_serve_cfg(max_slots, queue_capacity, hbm_budget_bytes, idle_exit_us,
                       host_staging_bytes)
    h = _vp()
    _check(ctx, load().serve_create(ctx, ctypes.byref(cfg), ctypes.byref(h)))
    return h


def serve_submit(srv, src_xyz, src_w, f, tgt_xyz, delta, mu: float = 1.0) -> int:
    """Queue one single-layer request (host arrays, copied at once). Returns
    its ticket; raises SkError (SK_EBUSY: retry later, SK_ENOMEM: too large)."""
    X, n = _ptr(src_xyz, SK_HOST, (3,), "src_xyz")
    W, _ = _ptr(src_w, SK_HOST, (), "src_w")
    F, _ = _ptr(f, SK_HOST, (3,), "f")
    Y, M = _ptr(tgt_xyz, SK_HOST, (3,), "tgt_xyz")
    D, nd = _ptr(delta if not np.isscalar(delta) else [delta], SK_HOST, (), "delta")
    req = sk_request(n, _host_ptr(X), _host_ptr(W), _host_ptr(F), M, _host_ptr(Y), _host_ptr(D),
                     nd, float(mu))
    t = ctypes.c_uint64()
    code = load().serve_submit(srv, ctypes.byref(req), ctypes.byref(t))
    if code != SK_OK:
        raise SkError(code, "serve_submit")
    return t.value


def serve_submit_capsule(srv, capsule, n_steps: int, dt: float, flow=None) -> int:
    """Queue n_steps explicit Euler steps of a resident capsule (a Capsule of
    the server's context); serve_poll(srv, ticket, capsule.N) returns its
    nodes after the steps. Raises SkError (SK_EBUSY: the capsule or the queue
    is busy)."""
    req = sk_request()
    req.capsule = capsule.handle
    req.n_steps = int(n_steps)
    req.dt = float(dt)
    if flow is not None:
        req.flow = sk_flow(*flow)
    t = ctypes.c_uint64()
    code = load().serve_submit(srv, ctypes.byref(req), ctypes.byref(t))
    if code != SK_OK:
        raise SkError(code, "serve_submit (capsule)")
    return t.value


def serve_poll(srv, ticket: int, n_tgt: int, timeout_us: int = -1):
    """(status, u (n_tgt, 3) or None, stats dict). SK_EAGAIN: not ready."""
    u = np.empty((n_tgt, 3), dtype=np.float64)
    st = sk_req_stats()
    code = load().serve_poll(srv, ctypes.c_uint64(ticket), u.ctypes.data_as(_vp),
                             ctypes.byref(st), int(timeout_us))
    stats = {f[0]: getattr(st, f[0]) for f in st._fields_}
    return code, (u if code == SK_OK else None), stats


def serve_destroy(srv) -> None:
    """Finish the queued work and free the server."""
    if srv:
        load().serve_destroy(srv)


def stokes_sl_eval_noalloc(src_xyz, src_w, f, tgt_xyz, delta, mu: float = 1.0, u_out=None,
                           stream=None):
    """Single layer (SK_FP32C) that allocates nothing inside the library.

    All arrays are CUDA float64 torch tensors on the current device; the
    library works in its own static 32 MiB device scratch array, so larger
    problems are rejected (SkError SK_EINVAL). Calls that overlap on the GPU
    share that array and must be serialized. Returns u_out (M, 3).
    """
    lib = load()
    X, n = _ptr(src_xyz, SK_DEVICE, (3,), "src_xyz")
    W, nw = _ptr(src_w, SK_DEVICE, (), "src_w")
    F, nf = _ptr(f, SK_DEVICE, (3,), "f")
    Y, M = _ptr(tgt_xyz, SK_DEVICE, (3,), "tgt_xyz")
    D, nd = _ptr(delta, SK_DEVICE, (), "delta")
    if not (n == nw == nf):
        raise ValueError("src_xyz, src_w and f must have the same number of nodes")
    if u_out is None:
        u_out = _alloc_out(tgt_xyz, SK_DEVICE, M)
    U, _ = _ptr(u_out, SK_DEVICE, (3,), "u_out")
    code = lib.stokes_sl_eval_noalloc(n, X, W, F, M, Y, D, nd, float(mu), U,
                                      _stream_handle(stream))
    if code != SK_OK:
        raise SkError(code, "stokes_sl_eval_noalloc failed")
    return u_out


class Context:
    """RAII holder of an sk_ctx*."""

    def __init__(self, device: int = 0, workspace_bytes: int = 0):
        self.handle = sk_create(device, workspace_bytes)

    def close(self):
        if self.handle:
            sk_destroy(self.handle)
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
