"""FP64 CPU oracle of the Jacobi-PCA hot path -- TEST INFRASTRUCTURE ONLY.

Only the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA library never loads it and it
never loads the CUDA library: the two share no code.

The arithmetic lives in ``pca_oracle.c`` (plain C, FP64, no BLAS); this module
compiles it with gcc on first use (or through :func:`build`) and wraps it with
ctypes.  Inputs of any dtype are widened to float64 exactly (float32, float16
and bfloat16 all embed in float64) before they reach the C code.

Stage map (Algorithm 1 of the paper):
  band_means      -> stage "BandAverageRemoval", first half (Sec. 4.2 stage 2.1)
  covariance      -> C = X^T X / (N-1)  (Sec. 4.2 stage 3)
  jacobi          -> cyclic Jacobi, Eqs. 2-10 (Sec. 2)
  sort_sign       -> eigen-pair extraction and descending sort (Sec. 4.2 stage 4.3)
  project         -> Q = X V_k (Algorithm 1 stages 5-6)
  backward        -> adjoint of the whole path (not in the paper; written from
                     the standard perturbation theory of symmetric eigenproblems)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pca_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

OK, ERR_ARG, ERR_NOCONV, ERR_NONFINITE = 0, 1, 2, 3
ROW_CYCLIC, ROUND_ROBIN, ODD_EVEN, CLASSICAL, GREEDY = 0, 1, 2, 3, 4


def build(force: bool = False) -> str:
    """Compile pca_oracle.c into _build/liboracle.so (OpenMP on the pixel loops)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c11", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _bind(lib):
    d, i, l = ctypes.c_double, ctypes.c_int, ctypes.c_long
    P = ctypes.c_void_p
    lib.oracle_set_threads.argtypes = [i]
    lib.oracle_band_means.argtypes = [P, l, i, P]
    lib.oracle_covariance.argtypes = [P, l, i, P, P]
    lib.oracle_rotation.argtypes = [d, d, d, P, P]
    lib.oracle_rotation.restype = None
    lib.oracle_jacobi.argtypes = [P, i, d, i, i, P, P, P, P]
    lib.oracle_sort_sign.argtypes = [i, P, P]
    lib.oracle_project.argtypes = [P, l, i, P, P, i, P]
    lib.oracle_pca_fit.argtypes = [P, l, i, i, d, i, i, P, P, P, P, P, P, P]
    lib.oracle_backward.argtypes = [P, l, i, i, P, P, P, P, P, d, P]
    lib.oracle_jacobi_steps.argtypes = [P, i, i, i, d, P]
    lib.oracle_jacobi_steps.restype = l
    return lib


_override = threading.local()


def _load():
    """The oracle library in use: the built one, or a variant set by `using`."""
    global _lib
    lib = getattr(_override, "lib", None)
    if lib is not None:
        return lib
    with _lock:
        if _lib is None:
            _lib = _bind(ctypes.CDLL(build()))
    return _lib


class using:
    """Context manager that routes this module's calls to another build of the
    oracle (tests compile deliberately broken copies to show the pins catch them)."""

    def __init__(self, so_path: str):
        self.lib = _bind(ctypes.CDLL(so_path))

    def __enter__(self):
        self.prev = getattr(_override, "lib", None)
        _override.lib = self.lib
        return self

    def __exit__(self, *exc):
        _override.lib = self.prev
        return False


def compile_variant(src_text: str, out_path: str) -> str:
    """Compile C source text (a modified copy of pca_oracle.c) to a shared library."""
    c_path = out_path + ".c"
    with open(c_path, "w") as f:
        f.write(src_text)
    subprocess.run(["gcc", "-O1", "-shared", "-fPIC", "-std=c11", "-o", out_path, c_path, "-lm"],
                   check=True)
    return out_path


def source() -> str:
    with open(_SRC) as f:
        return f.read()


def set_threads(t: int) -> int:
    """Threads for the pixel loops (covariance, projection); <1 means all cores."""
    return _load().oracle_set_threads(int(t))


def as_f64(a) -> np.ndarray:
    """Exact widening of a numpy array or CPU/GPU torch tensor to C-contiguous float64."""
    try:
        import torch
        if isinstance(a, torch.Tensor):
            a = a.detach().to("cpu", torch.float64).numpy()
    except ImportError:  # pragma: no cover
        pass
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


class OracleError(RuntimeError):
    pass


def _check(st: int, allow=(OK,)):
    if st not in allow:
        raise OracleError(f"oracle status {st}")
    return st


def band_means(Y) -> np.ndarray:
    Y = as_f64(Y)
    N, B = Y.shape
    mu = np.empty(B)
    _check(_load().oracle_band_means(_p(Y), N, B, _p(mu)))
    return mu


def covariance(Y, mu=None) -> np.ndarray:
    Y = as_f64(Y)
    N, B = Y.shape
    mu = band_means(Y) if mu is None else as_f64(mu)
    C = np.empty((B, B))
    _check(_load().oracle_covariance(_p(Y), N, B, _p(mu), _p(C)))
    return C


def rotation(app: float, aqq: float, apq: float):
    c, s = ctypes.c_double(), ctypes.c_double()
    _load().oracle_rotation(app, aqq, apq, ctypes.byref(c), ctypes.byref(s))
    return c.value, s.value


def jacobi(A, tol=1e-14, sweeps_max=60, ordering=ROW_CYCLIC):
    """Returns (A_K, V, info) with info = dict(status, sweeps, off_rel, rotations)."""
    A = as_f64(A).copy()
    B = A.shape[0]
    V = np.empty((B, B))
    sw, off, nrot = ctypes.c_int(), ctypes.c_double(), ctypes.c_long()
    st = _load().oracle_jacobi(_p(A), B, float(tol), int(sweeps_max), int(ordering), _p(V),
                               ctypes.byref(sw), ctypes.byref(off), ctypes.byref(nrot))
    _check(st, (OK, ERR_NOCONV))
    return A, V, dict(status=st, sweeps=sw.value, off_rel=off.value, rotations=nrot.value)


def jacobi_steps(A, ordering, steps, thr=0.0):
    """The first `steps` steps of the classical (one rotation each) or greedy
    (one iteration of disjoint pairs above thr each) ordering, no stop test.
    Returns (A, V, rotations)."""
    A = as_f64(A).copy()
    B = A.shape[0]
    V = np.empty((B, B))
    n = _load().oracle_jacobi_steps(_p(A), B, int(ordering), int(steps), float(thr), _p(V))
    if n < 0:
        raise ValueError("oracle_jacobi_steps rejected its arguments")
    return A, V, int(n)


def sort_sign(lam, V):
    lam = as_f64(lam).copy()
    V = as_f64(V).copy()
    _check(_load().oracle_sort_sign(lam.shape[0], _p(lam), _p(V)))
    return lam, V


def project(Y, mu, V, k) -> np.ndarray:
    Y = as_f64(Y)
    N, B = Y.shape
    mu, V = as_f64(mu), as_f64(V)
    Q = np.empty((N, k))
    _check(_load().oracle_project(_p(Y), N, B, _p(mu), _p(V), int(k), _p(Q)))
    return Q


def pca_fit(Y, k, tol=1e-14, sweeps_max=60, ordering=ROW_CYCLIC, project_q=True):
    """All four stages.  Returns dict(mu, lam, V, Q, status, sweeps, off_rel, rotations)."""
    Y = as_f64(Y)
    N, B = Y.shape
    mu, lam, V = np.empty(B), np.empty(B), np.empty((B, B))
    Q = np.empty((N, k)) if project_q else None
    sw, off, nrot = ctypes.c_int(), ctypes.c_double(), ctypes.c_long()
    st = _load().oracle_pca_fit(_p(Y), N, B, int(k), float(tol), int(sweeps_max), int(ordering),
                                _p(mu), _p(lam), _p(V), _p(Q) if Q is not None else None,
                                ctypes.byref(sw), ctypes.byref(off), ctypes.byref(nrot))
    _check(st, (OK, ERR_NOCONV))
    return dict(mu=mu, lam=lam, V=V, Q=Q, status=st, sweeps=sw.value, off_rel=off.value,
                rotations=nrot.value)


def backward(Y, k, mu, lam, V, dQ, dlam=None, gap_eps=1e-6) -> np.ndarray:
    """dL/dY of the projection layer Q = (Y - 1 mu^T) V_k (and of lam when dlam is
    given) from the forward results; see oracle_backward in pca_oracle.c."""
    Y = as_f64(Y)
    N, B = Y.shape
    mu, lam, V, dQ = as_f64(mu), as_f64(lam), as_f64(V), as_f64(dQ)
    if dQ.shape != (N, k):
        raise ValueError("dQ must be [N, k]")
    dl = as_f64(dlam) if dlam is not None else None
    dY = np.empty((N, B))
    _check(_load().oracle_backward(_p(Y), N, B, int(k), _p(mu), _p(lam), _p(V), _p(dQ),
                                   _p(dl) if dl is not None else None, float(gap_eps), _p(dY)))
    return dY
