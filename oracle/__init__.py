"""FP64 CPU oracle for the regularized Stokes single- and double-layer sums.

TEST INFRASTRUCTURE ONLY: imported by tests/, by the smoke check in
__graft_entry__ and by the CPU-baseline leg of bench.py. The CUDA library and
its Python binding never import it.

The arithmetic lives in stokes_oracle.c (plain C, FP64, libm erf/exp); this
module compiles it with gcc on first use and marshals numpy arrays through
ctypes. See stokes_oracle.c for the formulas and their paper citations
(Sec. 3.4, Eq. regstokes; Sec. 3.3, Eq. smoothint).

Submodules (plain NumPy, same status): membrane.py -- overset finite-difference
surface derivatives and the Skalak membrane force (Sec. 3.5; Sec. 2.1);
timestep.py -- Runge-Kutta-Fehlberg 4(5) adaptive stepping (Sec. 3.6);
upsample.py -- the four-times upsampled single layer (Sec. 3.4);
fmm.py -- the single-level kernel-independent FMM of Sec. 5.
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import tempfile

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
SOURCE = os.path.join(_HERE, "stokes_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")

_dp = ctypes.POINTER(ctypes.c_double)


def compile_library(src: str, out: str) -> str:
    """gcc -O2 -fopenmp -ffp-contract=off: IEEE FP64, same results on x86 and Arm."""
    d = os.path.dirname(os.path.abspath(out))
    fd, tmp = tempfile.mkstemp(suffix=".so", dir=d)
    os.close(fd)
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
           src, "-o", tmp, "-lm"]
    try:
        subprocess.run(cmd, check=True)
        os.replace(tmp, out)
    finally:
        if os.path.exists(tmp):
            os.remove(tmp)
    return out


def build(force: bool = False) -> str:
    """Compile stokes_oracle.c into oracle/liboracle.so if it is missing or stale."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(SOURCE)):
        return _LIB_PATH
    return compile_library(SOURCE, _LIB_PATH)


def _c(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def _ptr(a):
    return a.ctypes.data_as(_dp)


class Oracle:
    """ctypes view of one compiled copy of stokes_oracle.c."""

    def __init__(self, lib_path: str):
        lib = ctypes.CDLL(lib_path)
        i64 = ctypes.c_int64
        lib.oracle_sl.argtypes = [i64, _dp, _dp, _dp, i64, _dp, _dp, i64, ctypes.c_double, _dp,
                                  ctypes.c_int]
        lib.oracle_sl.restype = ctypes.c_int
        lib.oracle_dl.argtypes = [i64, _dp, _dp, _dp, _dp, i64, _dp, _dp, i64, _dp, ctypes.c_int]
        lib.oracle_dl.restype = ctypes.c_int
        lib.oracle_k_batch.argtypes = [ctypes.c_int, ctypes.c_int, i64, _dp, _dp]
        lib.oracle_k_batch.restype = None
        for name in ("oracle_s1", "oracle_s2", "oracle_s3"):
            getattr(lib, name).argtypes = [ctypes.c_double]
            getattr(lib, name).restype = ctypes.c_double
        lib.oracle_plain_stokeslet.argtypes = [i64, _dp, _dp, i64, _dp, _dp, ctypes.c_int]
        lib.oracle_plain_stokeslet.restype = ctypes.c_int
        lib.oracle_max_threads.argtypes = []
        lib.oracle_max_threads.restype = ctypes.c_int
        self.lib = lib
        self.path = lib_path

    def max_threads(self) -> int:
        return int(self.lib.oracle_max_threads())

    def sl(self, src_xyz, w, f, tgt_xyz, delta, mu: float = 1.0, threads: int = 0) -> np.ndarray:
        """Regularized single layer u(x_t), shape (M, 3). delta: scalar, (1,) or (M,)."""
        X = _c(src_xyz, (-1, 3))
        n = X.shape[0]
        w = _c(w, (n,))
        f = _c(f, (n, 3))
        Y = _c(tgt_xyz, (-1, 3))
        M = Y.shape[0]
        d = _c(np.atleast_1d(delta))
        out = np.zeros((M, 3))
        rc = self.lib.oracle_sl(n, _ptr(X), _ptr(w), _ptr(f), M, _ptr(Y), _ptr(d), d.shape[0],
                                float(mu), _ptr(out), int(threads))
        if rc != 0:
            raise ValueError("oracle_sl rejected its arguments")
        return out

    def dl(self, src_xyz, w, nrm, q, tgt_xyz, delta, threads: int = 0) -> np.ndarray:
        """Regularized double layer D(x_t), shape (M, 3). delta: scalar, (1,) or (M,)."""
        X = _c(src_xyz, (-1, 3))
        n = X.shape[0]
        w = _c(w, (n,))
        nr = _c(nrm, (n, 3))
        q = _c(q, (n, 3))
        Y = _c(tgt_xyz, (-1, 3))
        M = Y.shape[0]
        d = _c(np.atleast_1d(delta))
        out = np.zeros((M, 3))
        rc = self.lib.oracle_dl(n, _ptr(X), _ptr(w), _ptr(nr), _ptr(q), M, _ptr(Y), _ptr(d),
                                d.shape[0], _ptr(out), int(threads))
        if rc != 0:
            raise ValueError("oracle_dl rejected its arguments")
        return out

    def plain_stokeslet(self, src_xyz, g, tgt_xyz, threads: int = 0) -> np.ndarray:
        """Plain Stokeslet sum without 1/(8 pi mu): sum g/r + (g . d) d / r^3, (M, 3)."""
        X = _c(src_xyz, (-1, 3))
        n = X.shape[0]
        g = _c(g, (n, 3))
        Y = _c(tgt_xyz, (-1, 3))
        M = Y.shape[0]
        out = np.zeros((M, 3))
        rc = self.lib.oracle_plain_stokeslet(n, _ptr(X), _ptr(g), M, _ptr(Y), _ptr(out),
                                             int(threads))
        if rc != 0:
            raise ValueError("oracle_plain_stokeslet rejected its arguments")
        return out

    def kernel_factor(self, which: int, rho, branch: str = "auto") -> np.ndarray:
        """s1(p)/p (which=1), s2(p)/p^3 (which=2) or s3(p)/p^5 (which=3).

        branch: "auto" (series below p = 1), "series" or "closed".
        """
        b = {"auto": 0, "series": 1, "closed": 2}[branch]
        p = _c(np.atleast_1d(rho))
        out = np.zeros_like(p)
        self.lib.oracle_k_batch(int(which), b, p.shape[0], _ptr(p), _ptr(out))
        return out

    def smoothing(self, which: int, rho) -> np.ndarray:
        """Closed-form s1, s2 or s3 at p."""
        fn = {1: self.lib.oracle_s1, 2: self.lib.oracle_s2, 3: self.lib.oracle_s3}[which]
        return np.array([fn(float(x)) for x in np.atleast_1d(rho)])


_default: Oracle | None = None


def default() -> Oracle:
    global _default
    if _default is None:
        _default = Oracle(build())
    return _default


def max_threads() -> int:
    return default().max_threads()


def sl(*args, **kwargs):
    return default().sl(*args, **kwargs)


def dl(*args, **kwargs):
    return default().dl(*args, **kwargs)


def plain_stokeslet(*args, **kwargs):
    return default().plain_stokeslet(*args, **kwargs)


def kernel_factor(*args, **kwargs):
    return default().kernel_factor(*args, **kwargs)


def smoothing(*args, **kwargs):
    return default().smoothing(*args, **kwargs)
