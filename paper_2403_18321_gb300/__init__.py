"""GB300 (sm_103a) Jacobi-PCA for hyperspectral cubes -- thin Python binding.

Everything numeric runs in the CUDA library ``_lib/libgbpca.so`` behind the C
ABI of ``include/gbpca.h``; this module only marshals arguments (PyTorch
supplies device memory and the current stream).  There is no CPU path: if
the library is missing or no GPU is present, calls raise.

    mu, eigvals, eigvecs, proj, info = fit(cube, k=10)

Stages (Algorithm 1 of the paper): band means, covariance X^T X/(N-1),
cyclic Jacobi eigen-decomposition sorted in descending order, projection of
the centred cube onto the first k eigenvectors.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

from . import _build

__all__ = ["fit", "fit_host", "fit_batched", "fit_sharded", "Batch", "workspace_size", "load",
           "Info", "PCAError",
           "PREC_P64", "PREC_P32", "PREC_MIX", "STATUS"]

PREC_P64, PREC_P32, PREC_MIX = 0, 1, 2
PRECISIONS = {"p64": PREC_P64, "p32": PREC_P32, "mix": PREC_MIX}
STATUS = {0: "PCA_OK", 1: "PCA_ERR_ARG", 2: "PCA_ERR_NOCONV", 3: "PCA_ERR_NONFINITE",
          4: "PCA_ERR_TIMEOUT", 5: "PCA_ERR_CUDA", 6: "PCA_ERR_WORKSPACE"}
EXPORTS = ("pca_workspace_size", "pca_fit", "pca_covariance", "pca_eigh", "pca_project",
           "pca_read_info", "pca_status_string", "pca_version",
           "pca_kernel_launches", "pca_profile", "pca_profile_collect", "pca_project_noalloc",
           "pca_jacobi_sms", "pca_backward", "pca_backward_workspace_size",
           "pca_batch_workspace_size", "pca_batch_create", "pca_batch_run", "pca_batch_read_info",
           "pca_batch_destroy", "pca_fit_batched", "pca_batch_kernel_launches",
           "pca_combine_moments", "pca_bsq_to_bip", "pca_tuning_defaults", "pca_set_tuning",
           "pca_get_tuning", "pca_batch_jacobi_ctas", "pca_batch_plan_counts",
           "pca_fit_host_workspace_size", "pca_fit_host", "pca_shifted_sums",
           "pca_moments_from_sums")
STAGES = ("covariance", "cov_finalize", "jacobi", "empty", "compact", "refine", "sort_sign",
          "project")


class PCAError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        super().__init__(f"{STATUS.get(status, status)}: {what}")


class Info(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("sweeps", ctypes.c_int),
                ("refine_iters", ctypes.c_int), ("steps", ctypes.c_int),
                ("off_rel", ctypes.c_double), ("tol_used", ctypes.c_double),
                ("refine_res", ctypes.c_double), ("cov_fallback", ctypes.c_int),
                ("proj_fallback", ctypes.c_int)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class Tuning(ctypes.Structure):
    """pca_tuning of include/gbpca.h."""
    _fields_ = [("tc_slot_chunks", ctypes.c_int), ("tc_slot_chunks_f16", ctypes.c_int),
                ("tc_slot_chunks_bf16", ctypes.c_int),
                ("batch_jacobi_ctas", ctypes.c_int * 8),
                ("batch_cov_tc_fixed", ctypes.c_double), ("batch_proj_fixed", ctypes.c_double),
                ("batch_cov_simt_fixed", ctypes.c_double),
                ("batch_simt_items_per_sm", ctypes.c_int), ("proj_tc_stages", ctypes.c_int),
                ("proj_tc_raw_stages", ctypes.c_int), ("tc_slot_chunks_batch", ctypes.c_int),
                ("stream_sms_reserve", ctypes.c_int)]

    def as_dict(self):
        d = {f: getattr(self, f) for f, _ in self._fields_}
        d["batch_jacobi_ctas"] = list(self.batch_jacobi_ctas)
        return d

    @classmethod
    def from_dict(cls, d):
        t = cls()
        load().pca_tuning_defaults(ctypes.byref(t))
        for f, _ in cls._fields_:
            if f not in d:
                continue
            if f == "batch_jacobi_ctas":
                v = list(d[f])
                if len(v) != 8:
                    raise ValueError("batch_jacobi_ctas needs 8 entries")
                for i in range(8):
                    t.batch_jacobi_ctas[i] = int(v[i])
            else:
                setattr(t, f, d[f])
        return t


class Tile(ctypes.Structure):
    """pca_tile of include/gbpca.h."""
    _fields_ = [("cube", ctypes.c_void_p), ("N", ctypes.c_int64), ("B", ctypes.c_int),
                ("k", ctypes.c_int), ("mu", ctypes.c_void_p), ("eigvals", ctypes.c_void_p),
                ("eigvecs", ctypes.c_void_p), ("proj", ctypes.c_void_p)]


_lib = None


def load(build_if_missing: bool = False):
    """The loaded CUDA library (ctypes.CDLL).  Raises if it is not built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_build.LIB):
        if not build_if_missing:
            raise RuntimeError(f"CUDA library not built: {_build.LIB} (run __graft_entry__.build())")
        _build.build()
    lib = ctypes.CDLL(_build.LIB)
    P, i, d, sz, i64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_size_t, ctypes.c_int64
    lib.pca_workspace_size.argtypes = [i64, i, i, i, i]
    lib.pca_workspace_size.restype = sz
    lib.pca_fit.argtypes = [P, i, i64, i, i, d, i, i, P, P, P, P, P, sz, P, ctypes.POINTER(Info)]
    lib.pca_fit.restype = i
    lib.pca_covariance.argtypes = [P, i, i64, i, i, P, P, P, sz, P, ctypes.POINTER(Info)]
    lib.pca_covariance.restype = i
    lib.pca_eigh.argtypes = [P, i, d, i, i, P, P, P, sz, P, ctypes.POINTER(Info)]
    lib.pca_eigh.restype = i
    lib.pca_project.argtypes = [P, i, i64, i, i, P, P, P, P, sz, P]
    lib.pca_project.restype = i
    lib.pca_fit_host_workspace_size.argtypes = [i64, i, i, i, i]
    lib.pca_fit_host_workspace_size.restype = sz
    lib.pca_fit_host.argtypes = [P, i, i64, i, i, d, i, i, P, P, P, P, P, P, P, sz, P,
                                 ctypes.POINTER(Info)]
    lib.pca_fit_host.restype = i
    lib.pca_project_noalloc.argtypes = [P, i, i64, i, i, P, P, P, P]
    lib.pca_project_noalloc.restype = i
    lib.pca_backward_workspace_size.argtypes = [i64, i, i]
    lib.pca_backward_workspace_size.restype = sz
    lib.pca_backward.argtypes = [P, i, i64, i, i, P, P, P, P, P, d, P, P, sz, P,
                                 ctypes.POINTER(Info)]
    lib.pca_backward.restype = i
    lib.pca_read_info.argtypes = [P, P, ctypes.POINTER(Info)]
    lib.pca_read_info.restype = i
    lib.pca_status_string.argtypes = [i]
    lib.pca_status_string.restype = ctypes.c_char_p
    lib.pca_version.restype = i
    lib.pca_kernel_launches.argtypes = [i, i]
    lib.pca_kernel_launches.restype = i
    lib.pca_jacobi_sms.argtypes = [i]
    lib.pca_jacobi_sms.restype = i
    lib.pca_profile.argtypes = [i]
    lib.pca_profile.restype = i
    lib.pca_profile_collect.argtypes = [ctypes.POINTER(ctypes.c_float), i]
    lib.pca_profile_collect.restype = i
    TP = ctypes.POINTER(Tile)
    lib.pca_batch_workspace_size.argtypes = [i, TP, i, i]
    lib.pca_batch_workspace_size.restype = sz
    lib.pca_batch_create.argtypes = [ctypes.POINTER(P), i, TP, i, d, i, i, P, sz,
                                     ctypes.POINTER(i)]
    lib.pca_batch_create.restype = i
    lib.pca_batch_run.argtypes = [P, P]
    lib.pca_batch_run.restype = i
    lib.pca_batch_read_info.argtypes = [P, P, ctypes.POINTER(Info)]
    lib.pca_batch_read_info.restype = i
    lib.pca_batch_destroy.argtypes = [P]
    lib.pca_batch_destroy.restype = None
    lib.pca_batch_kernel_launches.argtypes = [P]
    lib.pca_batch_kernel_launches.restype = i
    lib.pca_fit_batched.argtypes = [i, TP, i, d, i, i, P, sz, P, ctypes.POINTER(Info)]
    lib.pca_fit_batched.restype = i
    lib.pca_combine_moments.argtypes = [i, ctypes.POINTER(i64), P, P, i, P, P, P]
    lib.pca_combine_moments.restype = i
    lib.pca_shifted_sums.argtypes = [i64, P, P, P, i, P, P]
    lib.pca_shifted_sums.restype = i
    lib.pca_moments_from_sums.argtypes = [P, P, i, P, P, P]
    lib.pca_moments_from_sums.restype = i
    lib.pca_bsq_to_bip.argtypes = [P, i, i64, i, P, P]
    lib.pca_bsq_to_bip.restype = i
    TuP = ctypes.POINTER(Tuning)
    lib.pca_tuning_defaults.argtypes = [TuP]
    lib.pca_tuning_defaults.restype = None
    lib.pca_set_tuning.argtypes = [TuP]
    lib.pca_set_tuning.restype = i
    lib.pca_get_tuning.argtypes = [TuP]
    lib.pca_get_tuning.restype = i
    lib.pca_batch_jacobi_ctas.argtypes = [i, i]
    lib.pca_batch_jacobi_ctas.restype = i
    lib.pca_batch_plan_counts.argtypes = [i, TP, i, i, ctypes.POINTER(i)]
    lib.pca_batch_plan_counts.restype = i
    _lib = lib
    return lib


def tuning() -> dict:
    """The library's current tuning parameters (pca_get_tuning)."""
    t = Tuning()
    _check_rc(load().pca_get_tuning(ctypes.byref(t)))
    return t.as_dict()


def tuning_defaults() -> dict:
    t = Tuning()
    load().pca_tuning_defaults(ctypes.byref(t))
    return t.as_dict()


def set_tuning(params: dict | None = None) -> dict:
    """Installs tuning parameters (missing keys take the defaults; None: all
    defaults) and returns the previous ones (pca_set_tuning)."""
    prev = tuning()
    t = Tuning.from_dict(params or {})
    _check_rc(load().pca_set_tuning(ctypes.byref(t)))
    return prev


def _dtype_code(t):
    import torch
    codes = {torch.float32: 0, torch.bfloat16: 1, torch.float16: 2}
    if t.dtype not in codes:
        raise TypeError(f"cube dtype {t.dtype} not supported (float32, bfloat16, float16)")
    return codes[t.dtype]


def _prec_code(precision):
    if isinstance(precision, str):
        return PRECISIONS[precision.lower()]
    return int(precision)


def workspace_size(N: int, B: int, k: int, dtype_code: int = 0, precision="mix") -> int:
    return int(load().pca_workspace_size(int(N), int(B), int(k), int(dtype_code),
                                          _prec_code(precision)))


@dataclass
class Workspace:
    """Reusable device scratch for repeated fits of one problem shape."""
    buf: object
    nbytes: int


def make_workspace(N, B, k, dtype_code=0, precision="mix", device=None):
    import torch
    n = workspace_size(N, B, k, dtype_code, precision)
    if n == 0:
        raise PCAError(1, "pca_workspace_size rejected the shape")
    buf = torch.empty(n + 256, dtype=torch.uint8, device=device or "cuda")
    return Workspace(buf, n)


def _ws_ptr(ws: Workspace) -> int:
    p = ws.buf.data_ptr()
    return (p + 255) & ~255


def bsq_to_bip(cube_bsq, stream=None):
    """A band-sequential device cube [B, N] (each band contiguous, the paper's GPU
    layout) as the pixel-major [N, B] cube the fit reads (pca_bsq_to_bip)."""
    import torch
    if not isinstance(cube_bsq, torch.Tensor) or not cube_bsq.is_cuda:
        raise TypeError("cube must be a CUDA tensor")
    if cube_bsq.dim() != 2 or not cube_bsq.is_contiguous():
        raise ValueError("cube must be a contiguous [B, N] tensor")
    B, N = cube_bsq.shape
    out = torch.empty(N, B, dtype=cube_bsq.dtype, device=cube_bsq.device)
    st = stream if stream is not None else torch.cuda.current_stream(cube_bsq.device)
    _check_rc(load().pca_bsq_to_bip(ctypes.c_void_p(cube_bsq.data_ptr()), _dtype_code(cube_bsq),
                                    N, B, ctypes.c_void_p(out.data_ptr()),
                                    ctypes.c_void_p(st.cuda_stream)))
    return out


def fit(cube, k: int, tol: float = 1e-10, sweeps_max: int = 30, precision="mix",
        out=None, workspace: Workspace | None = None, project: bool = True,
        sync: bool = True, stream=None, layout: str = "bip"):
    """PCA of a device cube (float32/bfloat16/float16): [N, B] pixel-major
    (layout "bip"), or [B, N] band-sequential (layout "bsq", converted first by
    pca_bsq_to_bip).

    Returns (mu [B] f64, eigvals [B] f64, eigvecs [B, B] f64, proj [N, k] f32 or None,
    info dict or None).  With sync=False nothing waits for the GPU and info is None.
    """
    import torch
    if not isinstance(cube, torch.Tensor) or not cube.is_cuda:
        raise TypeError("cube must be a CUDA tensor")
    if cube.dim() != 2 or not cube.is_contiguous():
        raise ValueError("cube must be a contiguous 2-D tensor")
    if layout == "bsq":
        cube = bsq_to_bip(cube, stream)
        if stream is not None:
            cube.record_stream(stream)   # the converted copy stays alive for that stream
    elif layout != "bip":
        raise ValueError("layout must be 'bip' or 'bsq'")
    N, B = cube.shape
    dt = _dtype_code(cube)
    prec = _prec_code(precision)
    dev = cube.device
    if out is None:
        mu = torch.empty(B, dtype=torch.float64, device=dev)
        ev = torch.empty(B, dtype=torch.float64, device=dev)
        V = torch.empty(B, B, dtype=torch.float64, device=dev)
        Q = torch.empty(N, k, dtype=torch.float32, device=dev) if project else None
    else:
        mu, ev, V, Q = out
    if workspace is None:
        workspace = make_workspace(N, B, k, dt, prec, dev)
    st = stream if stream is not None else torch.cuda.current_stream(dev)
    info = Info() if sync else None
    rc = load().pca_fit(ctypes.c_void_p(cube.data_ptr()), dt, N, B, int(k), float(tol),
                        int(sweeps_max), prec, ctypes.c_void_p(mu.data_ptr()),
                        ctypes.c_void_p(ev.data_ptr()), ctypes.c_void_p(V.data_ptr()),
                        ctypes.c_void_p(Q.data_ptr()) if Q is not None else None,
                        ctypes.c_void_p(_ws_ptr(workspace)), workspace.nbytes,
                        ctypes.c_void_p(st.cuda_stream),
                        ctypes.byref(info) if info is not None else None)
    if rc not in (0, 2) and not (rc == 3 and info is not None):
        raise PCAError(rc, load().pca_status_string(rc).decode())
    return mu, ev, V, Q, (info.as_dict() if info is not None else None)


def _check_rc(rc, allow=(0,)):
    if rc not in allow:
        raise PCAError(rc, load().pca_status_string(rc).decode())
    return rc


def covariance(cube, precision="mix", workspace: Workspace | None = None, stream=None):
    """Stages 2-3 only: (mu [B] f64, C [B, B] f64, info)."""
    import torch
    N, B = cube.shape
    dt, prec, dev = _dtype_code(cube), _prec_code(precision), cube.device
    mu = torch.empty(B, dtype=torch.float64, device=dev)
    C = torch.empty(B, B, dtype=torch.float64, device=dev)
    workspace = workspace or make_workspace(N, B, 1, dt, prec, dev)
    st = stream if stream is not None else torch.cuda.current_stream(dev)
    info = Info()
    rc = load().pca_covariance(ctypes.c_void_p(cube.data_ptr()), dt, N, B, prec,
                               ctypes.c_void_p(mu.data_ptr()), ctypes.c_void_p(C.data_ptr()),
                               ctypes.c_void_p(_ws_ptr(workspace)), workspace.nbytes,
                               ctypes.c_void_p(st.cuda_stream), ctypes.byref(info))
    _check_rc(rc, (0, 3))
    return mu, C, info.as_dict()


def eigh(A, tol: float = 1e-10, sweeps_max: int = 30, precision="mix",
         workspace: Workspace | None = None, stream=None):
    """Stage 4 only, on a symmetric device matrix A [B, B] f64: (eigvals, eigvecs, info)."""
    import torch
    B = A.shape[0]
    A = A.contiguous()
    prec, dev = _prec_code(precision), A.device
    ev = torch.empty(B, dtype=torch.float64, device=dev)
    V = torch.empty(B, B, dtype=torch.float64, device=dev)
    workspace = workspace or make_workspace(2, B, 1, 0, prec, dev)
    st = stream if stream is not None else torch.cuda.current_stream(dev)
    info = Info()
    rc = load().pca_eigh(ctypes.c_void_p(A.data_ptr()), B, float(tol), int(sweeps_max), prec,
                         ctypes.c_void_p(ev.data_ptr()), ctypes.c_void_p(V.data_ptr()),
                         ctypes.c_void_p(_ws_ptr(workspace)), workspace.nbytes,
                         ctypes.c_void_p(st.cuda_stream), ctypes.byref(info))
    _check_rc(rc, (0, 2, 3))
    return ev, V, info.as_dict()


def project(cube, mu, eigvecs, k: int, workspace: Workspace | None = None, stream=None):
    """Stages 5-6 only: proj [N, k] f32 = (Y - 1 mu^T) V[:, :k]."""
    import torch
    N, B = cube.shape
    dt, dev = _dtype_code(cube), cube.device
    Q = torch.empty(N, k, dtype=torch.float32, device=dev)
    workspace = workspace or make_workspace(N, B, k, dt, PREC_P32, dev)
    st = stream if stream is not None else torch.cuda.current_stream(dev)
    rc = load().pca_project(ctypes.c_void_p(cube.data_ptr()), dt, N, B, int(k),
                            ctypes.c_void_p(mu.contiguous().data_ptr()),
                            ctypes.c_void_p(eigvecs.contiguous().data_ptr()),
                            ctypes.c_void_p(Q.data_ptr()), ctypes.c_void_p(_ws_ptr(workspace)),
                            workspace.nbytes, ctypes.c_void_p(st.cuda_stream))
    _check_rc(rc)
    return Q


def project_noalloc(cube, mu, eigvecs, k: int, stream=None):
    """Stages 5-6 without any workspace or allocation inside the library call, for
    callers that cannot allocate device memory (e.g. during CUDA-graph capture).
    The library keeps the intermediates in its own fixed device array; calls that
    overlap on the GPU race on it, so serialise them.  Only the output tensor is
    allocated here (by PyTorch, before the call)."""
    import torch
    N, B = cube.shape
    dt, dev = _dtype_code(cube), cube.device
    Q = torch.empty(N, k, dtype=torch.float32, device=dev)
    st = stream if stream is not None else torch.cuda.current_stream(dev)
    rc = load().pca_project_noalloc(ctypes.c_void_p(cube.data_ptr()), dt, N, B, int(k),
                                    ctypes.c_void_p(mu.contiguous().data_ptr()),
                                    ctypes.c_void_p(eigvecs.contiguous().data_ptr()),
                                    ctypes.c_void_p(Q.data_ptr()), ctypes.c_void_p(st.cuda_stream))
    _check_rc(rc)
    return Q


def kernel_launches(precision="mix", k: int = 1) -> int:
    """Kernels one fit enqueues when it projects onto k components (0: none)."""
    return int(load().pca_kernel_launches(_prec_code(precision), int(k)))


def jacobi_sms(B: int) -> int:
    return int(load().pca_jacobi_sms(int(B)))


def batch_plan_counts(shapes, precision="mix", dtype_code: int = 0) -> dict:
    """The plan pca_batch_create would make under the current tuning for tiles of
    shapes [(N, B, k), ...], computed on the host (no device, no workspace)."""
    tiles = (Tile * len(shapes))()
    for t, (N, B, k) in enumerate(shapes):
        tiles[t] = Tile(None, int(N), int(B), int(k), None, None, None, None)
    c = (ctypes.c_int * 4)()
    _check_rc(load().pca_batch_plan_counts(len(shapes), tiles, int(dtype_code),
                                           _prec_code(precision), c))
    return {"cov_items": c[0], "proj_items": c[1], "jacobi_launches": c[2],
            "widest_cluster": c[3]}


def batch_jacobi_ctas(B: int, request: int = 0) -> int:
    """CTAs the batched form gives the Jacobi cluster of a B-band tile when the
    tuning asks for `request` (0: the fewest that hold the matrix)."""
    return int(load().pca_batch_jacobi_ctas(int(B), int(request)))


def profile(enable: bool) -> None:
    load().pca_profile(1 if enable else 0)


def profile_collect(max_records: int = 256):
    """List of dicts {stage: ms} for the fits recorded since profile(True)."""
    buf = (ctypes.c_float * (max_records * len(STAGES)))()
    n = load().pca_profile_collect(buf, max_records)
    return [{s: float(buf[r * len(STAGES) + i]) for i, s in enumerate(STAGES)} for r in range(n)]


class HostFit:
    """Device buffers for repeated pca_fit_host calls of one problem shape: the
    device copy of the cube, the device projection and the workspace."""

    def __init__(self, N: int, B: int, k: int, dtype, precision="mix", device="cuda",
                 project: bool = True):
        import torch
        self.shape, self.k, self.dtype, self.precision = (int(N), int(B)), int(k), dtype, precision
        dt = _dtype_code(torch.empty(0, dtype=dtype))
        n = int(load().pca_fit_host_workspace_size(N, B, k, dt, _prec_code(precision)))
        if n == 0:
            raise PCAError(1, "pca_fit_host_workspace_size rejected the shape")
        self.workspace = Workspace(torch.empty(n + 256, dtype=torch.uint8, device=device), n)
        self.cube_dev = torch.empty(N, B, dtype=dtype, device=device)
        self.proj_dev = torch.empty(N, k, dtype=torch.float32, device=device) if project else None


def fit_host(cube_host, k: int, tol: float = 1e-10, sweeps_max: int = 30, precision="mix",
             buffers: HostFit | None = None, out=None, project: bool = True, sync: bool = True,
             stream=None, device="cuda"):
    """PCA of a host cube [N, B] (float32/bfloat16/float16, pinned memory for
    overlapped copies) through pca_fit_host: the upload overlaps the covariance,
    the download of the projection overlaps the projection.  Returns host
    tensors (mu, eigvals, eigvecs, proj or None, info or None); with
    sync=False nothing waits and info is None (the results are valid once
    `stream` has finished)."""
    import torch
    if not isinstance(cube_host, torch.Tensor) or cube_host.is_cuda:
        raise TypeError("cube_host must be a host tensor")
    if cube_host.dim() != 2 or not cube_host.is_contiguous():
        raise ValueError("cube_host must be a contiguous 2-D tensor")
    N, B = cube_host.shape
    dt = _dtype_code(cube_host)
    if buffers is None:
        buffers = HostFit(N, B, k, cube_host.dtype, precision, device, project)
    if buffers.shape != (N, B) or buffers.k != k or buffers.dtype != cube_host.dtype:
        raise ValueError("buffers were made for another problem shape")
    pin = cube_host.is_pinned()
    if out is None:
        mu = torch.empty(B, dtype=torch.float64, pin_memory=pin)
        ev = torch.empty(B, dtype=torch.float64, pin_memory=pin)
        V = torch.empty(B, B, dtype=torch.float64, pin_memory=pin)
        Q = torch.empty(N, k, dtype=torch.float32, pin_memory=pin) if project else None
    else:
        mu, ev, V, Q = out
    if Q is not None and buffers.proj_dev is None:
        raise ValueError("buffers were made without a projection")
    dev = buffers.cube_dev.device
    st = stream if stream is not None else torch.cuda.current_stream(dev)
    info = Info() if sync else None
    rc = load().pca_fit_host(ctypes.c_void_p(cube_host.data_ptr()), dt, N, B, int(k), float(tol),
                             int(sweeps_max), _prec_code(precision),
                             ctypes.c_void_p(mu.data_ptr()), ctypes.c_void_p(ev.data_ptr()),
                             ctypes.c_void_p(V.data_ptr()),
                             ctypes.c_void_p(Q.data_ptr()) if Q is not None else None,
                             ctypes.c_void_p(buffers.cube_dev.data_ptr()),
                             ctypes.c_void_p(buffers.proj_dev.data_ptr()) if Q is not None else None,
                             ctypes.c_void_p(_ws_ptr(buffers.workspace)), buffers.workspace.nbytes,
                             ctypes.c_void_p(st.cuda_stream),
                             ctypes.byref(info) if info is not None else None)
    if rc not in (0, 2) and not (rc == 3 and info is not None):
        raise PCAError(rc, load().pca_status_string(rc).decode())
    return mu, ev, V, Q, (info.as_dict() if info is not None else None)


def backward(cube, mu, eigvals, eigvecs, dproj, deigvals=None, gap_eps: float = 1e-6,
             sync: bool = True, stream=None):
    """Adjoint of proj = (cube - 1 mu^T) eigvecs[:, :k] (and of eigvals when
    deigvals is given): returns dcube [N, B] float32.  mu, eigvals, eigvecs are
    the forward outputs (float64, device); dproj [N, k] float32."""
    import torch
    N, B = cube.shape
    k = dproj.shape[1]
    dt, dev = _dtype_code(cube), cube.device
    dproj = dproj.to(torch.float32).contiguous()
    dcube = torch.empty(N, B, dtype=torch.float32, device=dev)
    n = load().pca_backward_workspace_size(N, B, k)
    if n == 0:
        raise PCAError(1, "pca_backward_workspace_size rejected the shape")
    ws = Workspace(torch.empty(n + 256, dtype=torch.uint8, device=dev), n)
    dl = deigvals.to(torch.float64).contiguous() if deigvals is not None else None
    st = stream if stream is not None else torch.cuda.current_stream(dev)
    info = Info() if sync else None
    rc = load().pca_backward(ctypes.c_void_p(cube.data_ptr()), dt, N, B, int(k),
                             ctypes.c_void_p(mu.contiguous().data_ptr()),
                             ctypes.c_void_p(eigvals.contiguous().data_ptr()),
                             ctypes.c_void_p(eigvecs.contiguous().data_ptr()),
                             ctypes.c_void_p(dproj.data_ptr()),
                             ctypes.c_void_p(dl.data_ptr()) if dl is not None else None,
                             float(gap_eps), ctypes.c_void_p(dcube.data_ptr()),
                             ctypes.c_void_p(_ws_ptr(ws)), ws.nbytes,
                             ctypes.c_void_p(st.cuda_stream),
                             ctypes.byref(info) if info is not None else None)
    _check_rc(rc)
    return dcube


class Batch:
    """A plan for fitting many device cubes [N_t, B_t] (one dtype) in one go
    (pca_batch_create).  Outputs per tile are allocated here:
    ``results[t] = (mu, eigvals, eigvecs, proj or None)``.  ``run()`` enqueues
    the fits on the current stream (no synchronisation, capturable into a CUDA
    graph); ``info()`` waits and returns (worst status, per-tile info dicts)."""

    def __init__(self, cubes, k, tol: float = 1e-10, sweeps_max: int = 30, precision="mix",
                 project: bool = True, tuning="auto"):
        """tuning: "auto" installs the autotuner's cached parameters for this
        device, dtype and precision while planning (the library defaults when
        nothing is cached); a dict installs those; None plans with whatever the
        library holds."""
        import torch

        from . import tune
        if not cubes:
            raise ValueError("no cubes")
        ks = list(k) if isinstance(k, (list, tuple)) else [int(k)] * len(cubes)
        dt = _dtype_code(cubes[0])
        for c in cubes:
            if not isinstance(c, torch.Tensor) or not c.is_cuda or c.dim() != 2 or not c.is_contiguous():
                raise ValueError("every cube must be a contiguous 2-D CUDA tensor")
            if _dtype_code(c) != dt:
                raise TypeError("all cubes of a batch share one dtype")
        self.cubes = list(cubes)
        self.precision = _prec_code(precision)
        dev = cubes[0].device
        self.results = []
        tiles = (Tile * len(cubes))()
        for t, (c, kt) in enumerate(zip(cubes, ks)):
            N, B = c.shape
            mu = torch.empty(B, dtype=torch.float64, device=dev)
            ev = torch.empty(B, dtype=torch.float64, device=dev)
            V = torch.empty(B, B, dtype=torch.float64, device=dev)
            Q = torch.empty(N, kt, dtype=torch.float32, device=dev) if project else None
            self.results.append((mu, ev, V, Q))
            tiles[t] = Tile(c.data_ptr(), N, B, int(kt), mu.data_ptr(), ev.data_ptr(),
                            V.data_ptr(), Q.data_ptr() if Q is not None else None)
        self._tiles = tiles
        lib = load()
        if tuning == "auto":
            tuning = tune.lookup(tune.device_key(dev, dt, self.precision))
        self.tuning = tuning
        with tune.applied(tuning):
            self._plan_batch(lib, cubes, tiles, dt, tol, sweeps_max, dev)

    def _plan_batch(self, lib, cubes, tiles, dt, tol, sweeps_max, dev):
        import torch
        n = lib.pca_batch_workspace_size(len(cubes), tiles, dt, self.precision)
        if n == 0:
            bad = next(t for t in range(len(cubes))
                       if lib.pca_batch_workspace_size(1, ctypes.byref(tiles[t]), dt,
                                                       self.precision) == 0)
            raise PCAError(1, f"pca_batch_workspace_size rejected tile {bad}")
        self.workspace = Workspace(torch.empty(n + 256, dtype=torch.uint8, device=dev), n)
        self._plan = ctypes.c_void_p()
        bad = ctypes.c_int(-1)
        rc = lib.pca_batch_create(ctypes.byref(self._plan), len(cubes), tiles, dt, float(tol),
                                  int(sweeps_max), self.precision,
                                  ctypes.c_void_p(_ws_ptr(self.workspace)), n, ctypes.byref(bad))
        if rc != 0:
            raise PCAError(rc, f"pca_batch_create (tile {bad.value})")

    def run(self, stream=None):
        import torch
        st = stream if stream is not None else torch.cuda.current_stream(self.cubes[0].device)
        _check_rc(load().pca_batch_run(self._plan, ctypes.c_void_p(st.cuda_stream)))

    def info(self, stream=None):
        import torch
        st = stream if stream is not None else torch.cuda.current_stream(self.cubes[0].device)
        infos = (Info * len(self.cubes))()
        rc = load().pca_batch_read_info(self._plan, ctypes.c_void_p(st.cuda_stream), infos)
        if rc in (1, 5, 6):
            raise PCAError(rc, "pca_batch_read_info")
        return rc, [i.as_dict() for i in infos]

    def kernel_launches(self) -> int:
        return int(load().pca_batch_kernel_launches(self._plan))

    def close(self):
        if self._plan:
            load().pca_batch_destroy(self._plan)
            self._plan = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def fit_batched(cubes, k, tol: float = 1e-10, sweeps_max: int = 30, precision="mix",
                project: bool = True):
    """Fits every cube of the list (pca_batch_*): returns (results, status, infos) with
    results[t] = (mu, eigvals, eigvecs, proj or None)."""
    b = Batch(cubes, k, tol, sweeps_max, precision, project)
    b.run()
    status, infos = b.info()
    b.close()
    return b.results, status, infos


def combine_moments(counts, mus, Cs, stream=None):
    """Pooled (mu [B], C [B, B]) of shards with pixel counts `counts` (ints),
    means mus [G, B] and covariances Cs [G, B, B] (float64, device)."""
    import torch
    mus = mus.to(torch.float64).contiguous()
    Cs = Cs.to(torch.float64).contiguous()
    G, B = mus.shape
    mu = torch.empty(B, dtype=torch.float64, device=mus.device)
    C = torch.empty(B, B, dtype=torch.float64, device=mus.device)
    n = (ctypes.c_int64 * G)(*[int(c) for c in counts])
    st = stream if stream is not None else torch.cuda.current_stream(mus.device)
    _check_rc(load().pca_combine_moments(G, n, ctypes.c_void_p(mus.data_ptr()),
                                         ctypes.c_void_p(Cs.data_ptr()), B,
                                         ctypes.c_void_p(mu.data_ptr()),
                                         ctypes.c_void_p(C.data_ptr()),
                                         ctypes.c_void_p(st.cuda_stream)))
    return mu, C


def sums_length(B: int) -> int:
    """Length of the vector pca_shifted_sums writes: 1 + B + B(B+1)/2."""
    return 1 + B + B * (B + 1) // 2


def shifted_sums(n, mu, C, s, stream=None):
    """(n, S1, S2 upper) of one shard about the common shift s, as one FP64
    vector of sums_length(B) values on the device (pca_shifted_sums)."""
    import torch
    mu, C, s = (t.to(torch.float64).contiguous() for t in (mu, C, s))
    B = mu.shape[0]
    sums = torch.empty(sums_length(B), dtype=torch.float64, device=mu.device)
    st = stream if stream is not None else torch.cuda.current_stream(mu.device)
    _check_rc(load().pca_shifted_sums(int(n), ctypes.c_void_p(mu.data_ptr()),
                                      ctypes.c_void_p(C.data_ptr()), ctypes.c_void_p(s.data_ptr()),
                                      B, ctypes.c_void_p(sums.data_ptr()),
                                      ctypes.c_void_p(st.cuda_stream)))
    return sums


def moments_from_sums(sums, s, stream=None):
    """(mu [B], C [B, B]) of the cube from the shards' summed shifted sums
    (pca_moments_from_sums)."""
    import torch
    sums, s = sums.to(torch.float64).contiguous(), s.to(torch.float64).contiguous()
    B = s.shape[0]
    if sums.numel() != sums_length(B):
        raise ValueError("sums has the wrong length for B")
    mu = torch.empty(B, dtype=torch.float64, device=s.device)
    C = torch.empty(B, B, dtype=torch.float64, device=s.device)
    st = stream if stream is not None else torch.cuda.current_stream(s.device)
    _check_rc(load().pca_moments_from_sums(ctypes.c_void_p(sums.data_ptr()),
                                           ctypes.c_void_p(s.data_ptr()), B,
                                           ctypes.c_void_p(mu.data_ptr()),
                                           ctypes.c_void_p(C.data_ptr()),
                                           ctypes.c_void_p(st.cuda_stream)))
    return mu, C


class _LibraryOps:
    """The stages of a pixel-sharded fit, on this rank's GPU."""

    def __init__(self, precision, tol, sweeps_max):
        self.precision, self.tol, self.sweeps_max = precision, tol, sweeps_max

    def moments(self, cube):
        mu, C, _ = covariance(cube, self.precision)
        return mu, C

    def shifted_sums(self, n, mu, C, s):
        return shifted_sums(n, mu, C, s)

    def from_sums(self, sums, s):
        return moments_from_sums(sums, s)

    def eigh(self, C):
        ev, V, info = eigh(C, self.tol, self.sweeps_max, self.precision)
        return ev, V, info

    def project(self, cube, mu, V, k):
        return project(cube, mu, V, k)


def fit_sharded(cube, k: int, tol: float = 1e-10, sweeps_max: int = 30, precision="mix",
                group=None, ops=None):
    """PCA of a cube whose pixels are split over the ranks of a torch.distributed
    group: `cube` is this rank's [N_r, B] slice (contiguous and 16-byte aligned,
    N_r >= 2; clone a slice of a larger cube whose first row does not start on a
    16-byte boundary).  Each rank computes its band means and covariance; rank 0
    of the group sends its mean as the common shift s; every rank turns its
    moments into (n, S1, S2) about s (pca_shifted_sums) and ONE all-reduce sums
    them -- 1 + B + B(B+1)/2 FP64 values whatever the number of ranks; every rank
    recovers the pooled mean and covariance (pca_moments_from_sums).  Rank 0
    solves the pooled covariance and broadcasts eigenvalues and eigenvectors, so
    that every rank holds the same bits; each rank projects its own pixels.
    Returns (mu, eigvals, eigvecs, proj of this rank's pixels, info of the
    eigen-solve on rank 0 or None).  `ops` replaces the stages (used to test the
    exchange on CPU ranks)."""
    import torch
    import torch.distributed as dist
    ops = ops if ops is not None else _LibraryOps(precision, tol, sweeps_max)
    rank = dist.get_rank(group)
    N, B = cube.shape
    mu_r, C_r = ops.moments(cube)
    dev = mu_r.device
    root = dist.get_global_rank(group, 0) if group is not None else 0
    s = mu_r.clone() if rank == 0 else torch.empty(B, dtype=torch.float64, device=dev)
    dist.broadcast(s, root, group=group)
    sums = ops.shifted_sums(N, mu_r, C_r, s)
    dist.all_reduce(sums, op=dist.ReduceOp.SUM, group=group)
    mu, C = ops.from_sums(sums, s)
    info = None
    if rank == 0:
        ev, V, info = ops.eigh(C)
        ev, V = ev.contiguous(), V.contiguous()
    else:
        ev = torch.empty(B, dtype=torch.float64, device=dev)
        V = torch.empty(B, B, dtype=torch.float64, device=dev)
    dist.broadcast(ev, root, group=group)
    dist.broadcast(V, root, group=group)
    Q = ops.project(cube, mu, V, k)
    return mu, ev, V, Q, info


def _autograd_function():
    import torch

    class PCAProjection(torch.autograd.Function):
        """proj = PCAProjection.apply(cube, k, precision, tol, sweeps_max, gap_eps):
        the forward pass is pca_fit, the backward pass pca_backward (gradient
        with respect to the cube; the centred cube is recomputed, not stored)."""

        @staticmethod
        def forward(ctx, cube, k, precision="p64", tol=1e-10, sweeps_max=30, gap_eps=1e-6):
            mu, ev, V, Q, _ = fit(cube.detach().contiguous(), int(k), tol=tol,
                                  sweeps_max=sweeps_max, precision=precision)
            ctx.save_for_backward(cube, mu, ev, V)
            ctx.gap_eps = gap_eps
            return Q

        @staticmethod
        def backward(ctx, dQ):
            cube, mu, ev, V = ctx.saved_tensors
            dY = backward(cube.detach().contiguous(), mu, ev, V, dQ.contiguous(),
                          gap_eps=ctx.gap_eps)
            return dY.to(cube.dtype), None, None, None, None, None

    return PCAProjection


_pca_projection = None


def __getattr__(name):
    global _pca_projection
    if name == "PCAProjection":
        if _pca_projection is None:
            _pca_projection = _autograd_function()
        return _pca_projection
    raise AttributeError(name)
