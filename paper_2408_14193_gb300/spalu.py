"""ctypes binding of the spaLU C ABI (include/spalu.h): argument marshalling only.

Every numerical step runs in the CUDA library; device arrays are passed as torch CUDA
tensors (their data pointers) together with the current torch CUDA stream.  There is no
CPU fallback: when the library is missing, loading fails with an error that says so.
"""
from __future__ import annotations

import ctypes
import json
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = None

SPALU_OK = 0
_STATUS = {
    0: "ok", -1: "invalid argument", -2: "allocation failed", -3: "zero pivot in an LU",
    -4: "refinement did not converge", -5: "bounded device wait expired", -6: "CUDA runtime error",
    -7: "unsupported request", -8: "non-finite value in the factor", -9: "handle in the wrong state",
}


class SpaluError(RuntimeError):
    def __init__(self, status: int, where: str):
        super().__init__(f"{where}: {status_string(status)} (status {status})")
        self.status = status


def status_string(s: int) -> str:
    return _STATUS.get(int(s), "unknown status")


def library_path() -> str:
    return os.path.join(_HERE, "_build", "libspalu.so")


class Options(ctypes.Structure):
    """Mirror of spalu_opts."""
    _fields_ = [
        ("eps_id", ctypes.c_double),
        ("precision", ctypes.c_int),
        ("symmetric", ctypes.c_int),
        ("p_oversample", ctypes.c_int),
        ("near_radius", ctypes.c_int),
        ("h0", ctypes.c_int),
        ("seed", ctypes.c_ulonglong),
        ("gmres_m", ctypes.c_int),
        ("gmres_maxit", ctypes.c_int),
        ("gmres_tol", ctypes.c_double),
        ("spars_ctas", ctypes.c_int),
        ("schur_tc", ctypes.c_int),
        ("sketch_tc", ctypes.c_int),
        ("leaf_bwd", ctypes.c_int),
    ]

    @classmethod
    def default(cls, **kw) -> "Options":
        o = cls()
        load_library().spalu_default_opts(ctypes.byref(o))
        for k, v in kw.items():
            if not hasattr(o, k):
                raise AttributeError(k)
            setattr(o, k, v)
        return o


_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double

# (name, restype, argtypes) of every entry point declared in include/spalu.h
SIGNATURES = [
    ("spalu_default_opts", None, [_P]),
    ("spalu_status_string", ctypes.c_char_p, [_I]),
    ("spalu_nd_build_grid", _I, [_I, _I, _I, _P, _P]),
    ("spalu_nd_export", _I, [_P, _P, _P, _P, _I]),
    ("spalu_nd_export_segments", _I, [_P, _P, _I]),
    ("spalu_nd_destroy", None, [_P]),
    ("spalu_nd_order_csr", _I, [_I, _P, _P, _P, _P, _I, _P, _P]),
    ("spalu_factor_create", _I, [_P, _P, _P]),
    ("spalu_factor_numeric", _I, [_P, _P, _P, _P, _I, _P]),
    ("spalu_factor_numeric_batch", _I, [_I, _P, _P, _P, _P, _P, _P]),
    ("spalu_solve_batch", _I, [_I, _P, _P, _P, _P, _P, _P]),
    ("spalu_tune_solve", _I, [_P, _I, _P]),
    ("spalu_tune_factor", _I, [_P, _P]),
    ("spalu_factor_numeric_host", _I, [_P, _P, _P, _P, _I, _P]),
    ("spalu_solve", _I, [_P, _P, _P, _I, _I, _P]),
    ("spalu_refine", _I, [_P, _P, _P, _I, _I, _P, _P, _P]),
    ("spalu_solve_host", _I, [_P, _P, _P, _I, _I, _I, _P, _P, _P]),
    ("spalu_factor_solve_host", _I, [_P, _P, _P, _P, _I, _P, _P, _I, _I, _I, _P, _P, _P]),
    ("spalu_factor_solve_graph", _I, [_P, _P, _P, _P, _I, _P, _P, _I, _I, _P, _P, _P]),
    ("spalu_batch_graph_create", _I, [_I, _P, _P, _P, _P, _P, _P, _P, _P, _P, _I, _I, _P, _P]),
    ("spalu_batch_graph_run", _I, [_P, _P, _P, _P]),
    ("spalu_batch_graph_destroy", None, [_P]),
    ("spalu_stats", _I, [_P, ctypes.c_char_p, ctypes.c_size_t]),
    ("spalu_factor_export_level", _I, [_P, _I, _P, _P, _P, _P, _P, _P, _P]),
    ("spalu_residual_noalloc", _I, [_P, _P, _P, _I, _I, _P, _P]),
    ("spalu_set_timing", _I, [_P, _I]),
    ("spalu_kernel_launches", ctypes.c_ulonglong, []),
    ("spalu_measure_fma_peak", _I, [_I, _P, _P]),
    ("spalu_factor_destroy", None, [_P]),
    ("spalu_predictor_create", _I, [_P, _P]),
    ("spalu_predictor_get_params", _I, [_P, _P, _P]),
    ("spalu_predictor_set_norm", _I, [_P, _P, _P, _P]),
    ("spalu_predictor_get_norm", _I, [_P, _P, _P, _P]),
    ("spalu_predictor_fit_norm", _I, [_P, _P, _I, _P]),
    ("spalu_predictor_loss_grad", _I, [_P, _P, _P, _I, _P, _P, _P]),
    ("spalu_predictor_train", _I, [_P, _P, _P, _I, _I, _I, ctypes.c_float, _P, _P]),
    ("spalu_predictor_infer", _I, [_P, _P, _I, _P, _P]),
    ("spalu_predictor_destroy", None, [_P]),
    ("spalu_factor_set_predictor", _I, [_P, _P, _I, ctypes.c_double]),
    ("spalu_factor_export_training", _I, [_P, _P, _P, _I, _P, _P]),
]

PRED_NFEAT = 16
PRED_NPARAM = 1218
PRED_MODES = {"off": 0, "record": 1, "predict": 2}


def load_library(path: str | None = None):
    """Load the CUDA library (building is done by __graft_entry__.build or build.py)."""
    global _LIB
    if _LIB is not None and path is None:
        return _LIB
    p = path or library_path()
    if not os.path.exists(p):
        raise RuntimeError(
            f"spaLU CUDA library not found at {p}: build it first "
            "(python -c 'import __graft_entry__ as g; g.build()')")
    lib = ctypes.CDLL(p)
    for name, res, args in SIGNATURES:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    if path is None:
        _LIB = lib
    return lib


def kernel_launches() -> int:
    return int(load_library().spalu_kernel_launches())


def measure_fma_peak(precision: int, stream=None) -> float:
    """spalu_measure_fma_peak: FP64 (0) or FP32 (1) FMA throughput of the device in FLOP/s."""
    v = ctypes.c_double(0.0)
    _check(load_library().spalu_measure_fma_peak(precision, ctypes.byref(v), _stream_ptr(stream)),
           "spalu_measure_fma_peak")
    return v.value


def _stream_ptr(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _check(status: int, where: str):
    if status != SPALU_OK:
        raise SpaluError(status, where)


def _dev_ptr(t, dtype):
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == dtype and t.is_contiguous()):
        raise TypeError(f"expected a contiguous CUDA tensor of {dtype}")
    return ctypes.c_void_p(t.data_ptr())


def nd_order_csr(rowptr, colind, xy, leaf_size: int, boundary=None):
    """spalu_nd_order_csr: nested dissection of a general graph with coordinates (host
    computation); returns (perm, level) as int32 arrays."""
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int32)
    colind = np.ascontiguousarray(colind, dtype=np.int32)
    xy = np.ascontiguousarray(xy, dtype=np.float64)
    n = rowptr.size - 1
    if xy.shape != (n, 2):
        raise ValueError("xy must have shape (n, 2)")
    bd = None if boundary is None else np.ascontiguousarray(boundary, dtype=np.uint8)
    if bd is not None and bd.size != n:
        raise ValueError("boundary must have n entries")
    perm = np.empty(n, dtype=np.int32)
    level = np.empty(n, dtype=np.int32)
    _check(load_library().spalu_nd_order_csr(n, rowptr.ctypes.data, colind.ctypes.data, xy.ctypes.data,
                                             None if bd is None else bd.ctypes.data, int(leaf_size),
                                             perm.ctypes.data, level.ctypes.data), "spalu_nd_order_csr")
    return perm, level


class NestedDissection:
    """spalu_nd_build_grid: nested dissection of an nx x ny grid (leaf pitch 16)."""

    def __init__(self, nx: int, ny: int | None = None, leaf_pitch: int = 16, stream=None):
        self.lib = load_library()
        self.nx = nx
        self.ny = nx if ny is None else ny
        h = ctypes.c_void_p()
        _check(self.lib.spalu_nd_build_grid(nx, self.ny, leaf_pitch, _stream_ptr(stream), ctypes.byref(h)),
               "spalu_nd_build_grid")
        self.handle = h

    def export(self):
        n = self.nx * self.ny
        perm = np.empty(n, dtype=np.int32)
        iperm = np.empty(n, dtype=np.int32)
        levels = np.zeros(8 * 64, dtype=np.int32)
        _check(self.lib.spalu_nd_export(self.handle, perm.ctypes.data, iperm.ctypes.data,
                                        levels.ctypes.data, levels.size), "spalu_nd_export")
        L = int(levels[0])
        table = levels[8: 8 * (L + 1)].reshape(L, 8) if L else np.zeros((0, 8), np.int32)
        return perm, iperm, L, table

    def finest_segments(self, nseg: int) -> np.ndarray:
        out = np.empty(15 * nseg, dtype=np.int32)
        _check(self.lib.spalu_nd_export_segments(self.handle, out.ctypes.data, out.size),
               "spalu_nd_export_segments")
        return out.reshape(nseg, 15)

    def __del__(self):
        h = getattr(self, "handle", None)
        if h:
            self.lib.spalu_nd_destroy(h)
            self.handle = None


class Factor:
    """spalu_factor_create / _numeric / spalu_solve / spalu_refine on one grid."""

    def __init__(self, nd: NestedDissection, opts: Options | None = None, **kw):
        self.lib = load_library()
        self.nd = nd
        self.opts = opts if opts is not None else Options.default(**kw)
        h = ctypes.c_void_p()
        _check(self.lib.spalu_factor_create(nd.handle, ctypes.byref(self.opts), ctypes.byref(h)),
               "spalu_factor_create")
        self.handle = h
        self.N = nd.nx * nd.ny

    def factor(self, rowptr, colind, val, stream=None):
        """Numeric factorization of a device CSR matrix (torch int32/int32/float64)."""
        import torch
        self._csr_shape(rowptr, colind, val)
        _check(self.lib.spalu_factor_numeric(self.handle, _dev_ptr(rowptr, torch.int32),
                                             _dev_ptr(colind, torch.int32), _dev_ptr(val, torch.float64),
                                             int(val.numel()), _stream_ptr(stream)),
               "spalu_factor_numeric")

    def _csr_shape(self, rowptr, colind, val):
        if len(rowptr) != self.N + 1 or len(colind) != len(val):
            raise ValueError(f"CSR arrays must have N + 1 = {self.N + 1} row pointers and as many column "
                             f"indices as values, got {len(rowptr)}, {len(colind)}, {len(val)}")

    def factor_host(self, rowptr: np.ndarray, colind: np.ndarray, val: np.ndarray, stream=None):
        rowptr = np.ascontiguousarray(rowptr, dtype=np.int32)
        colind = np.ascontiguousarray(colind, dtype=np.int32)
        val = np.ascontiguousarray(val, dtype=np.float64)
        self._csr_shape(rowptr, colind, val)
        _check(self.lib.spalu_factor_numeric_host(self.handle, rowptr.ctypes.data, colind.ctypes.data,
                                                  val.ctypes.data, int(val.size), _stream_ptr(stream)),
               "spalu_factor_numeric_host")

    def _nrhs(self, B, X):
        """Right-hand-side count of B, shaped (N,) or (nrhs, N), with X shaped like B; the
        kernels index both with leading dimension N, so a short tensor is refused here."""
        if B.dim() not in (1, 2) or B.shape[-1] != self.N:
            raise ValueError(f"B must have shape (N,) or (nrhs, N) with N = {self.N}, got {tuple(B.shape)}")
        if X is not None and tuple(X.shape) != tuple(B.shape):
            raise ValueError(f"X must have the shape of B {tuple(B.shape)}, got {tuple(X.shape)}")
        return 1 if B.dim() == 1 else B.shape[0]

    def solve(self, B, X=None, stream=None):
        """X = spaLU^{-1} B for a device float64 tensor B of shape (N,) or (nrhs, N) laid
        out column by column (row k of the tensor is right-hand side k)."""
        import torch
        if X is None:
            X = torch.empty_like(B)
        nrhs = self._nrhs(B, X)
        _check(self.lib.spalu_solve(self.handle, _dev_ptr(B, torch.float64), _dev_ptr(X, torch.float64),
                                    nrhs, self.N, _stream_ptr(stream)), "spalu_solve")
        return X

    def factor_solve_graph(self, rowptr, colind, val, B, X, stream=None, check=True):
        """spalu_factor_solve_graph: factor (device CSR), solve B into X and refine X, as one
        CUDA graph after the first call; returns (iterations, relative residuals)."""
        import torch
        self._csr_shape(rowptr, colind, val)
        nrhs = self._nrhs(B, X)
        it = ctypes.c_int(0)
        rel = np.zeros(nrhs)
        st = self.lib.spalu_factor_solve_graph(
            self.handle, _dev_ptr(rowptr, torch.int32), _dev_ptr(colind, torch.int32), _dev_ptr(val, torch.float64),
            int(val.numel()), _dev_ptr(B, torch.float64), _dev_ptr(X, torch.float64), nrhs, self.N,
            ctypes.byref(it), rel.ctypes.data, _stream_ptr(stream))
        if check:
            _check(st, "spalu_factor_solve_graph")
        return it.value, rel

    def tune_solve(self, nrhs: int = 16, stream=None):
        """Time the level-solve kernels with 2- and 8-warp CTAs per level and keep the fastest."""
        _check(self.lib.spalu_tune_solve(self.handle, nrhs, _stream_ptr(stream)), "spalu_tune_solve")

    def tune_factor(self, stream=None):
        """Re-factor the last matrix under each candidate shared-memory budget of the sparsify
        kernel and keep the fastest per level (the handle is factored on return)."""
        _check(self.lib.spalu_tune_factor(self.handle, _stream_ptr(stream)), "spalu_tune_factor")

    def refine(self, B, X, stream=None, check=True):
        """GMRES refinement of X in place; returns (iterations, relative residuals)."""
        import torch
        nrhs = self._nrhs(B, X)
        it = ctypes.c_int(0)
        rel = np.zeros(nrhs)
        st = self.lib.spalu_refine(self.handle, _dev_ptr(B, torch.float64), _dev_ptr(X, torch.float64),
                                   nrhs, self.N, ctypes.byref(it), rel.ctypes.data, _stream_ptr(stream))
        if check:
            _check(st, "spalu_refine")
        return it.value, rel

    def solve_host(self, B: np.ndarray, refine: bool = False, stream=None, out: np.ndarray | None = None):
        """Host arrays in and out (copies inside the call); B has shape (nrhs, N).  ``out``
        (same shape, float64, C-contiguous; page-locked for full copy bandwidth) receives the
        solution; a new array otherwise."""
        B = np.ascontiguousarray(B, dtype=np.float64)
        if B.ndim not in (1, 2) or B.shape[-1] != self.N:
            raise ValueError(f"B must have shape (N,) or (nrhs, N) with N = {self.N}, got {B.shape}")
        nrhs = 1 if B.ndim == 1 else B.shape[0]
        if out is not None:
            if out.shape != B.shape or out.dtype != np.float64 or not out.flags.c_contiguous:
                raise ValueError("out must be a C-contiguous float64 array shaped like B")
            X = out
        else:
            X = np.empty_like(B)
        it = ctypes.c_int(0)
        rel = np.zeros(nrhs)
        _check(self.lib.spalu_solve_host(self.handle, B.ctypes.data, X.ctypes.data, nrhs, self.N,
                                         1 if refine else 0, ctypes.byref(it), rel.ctypes.data,
                                         _stream_ptr(stream)), "spalu_solve_host")
        return X, it.value, rel

    def factor_solve_host(self, rowptr: np.ndarray, colind: np.ndarray, val: np.ndarray, B: np.ndarray,
                          refine: bool = False, stream=None, out: np.ndarray | None = None):
        """spalu_factor_solve_host: factor the host CSR matrix and solve for the host B (shape
        (nrhs, N)) in one call, the upload of B overlapping the factorization.  Returns
        (X, iterations, relative residuals); ``out`` as in solve_host."""
        rowptr = np.ascontiguousarray(rowptr, dtype=np.int32)
        colind = np.ascontiguousarray(colind, dtype=np.int32)
        val = np.ascontiguousarray(val, dtype=np.float64)
        self._csr_shape(rowptr, colind, val)
        B = np.ascontiguousarray(B, dtype=np.float64)
        if B.ndim not in (1, 2) or B.shape[-1] != self.N:
            raise ValueError(f"B must have shape (N,) or (nrhs, N) with N = {self.N}, got {B.shape}")
        nrhs = 1 if B.ndim == 1 else B.shape[0]
        if out is not None:
            if out.shape != B.shape or out.dtype != np.float64 or not out.flags.c_contiguous:
                raise ValueError("out must be a C-contiguous float64 array shaped like B")
            X = out
        else:
            X = np.empty_like(B)
        it = ctypes.c_int(0)
        rel = np.zeros(nrhs)
        _check(self.lib.spalu_factor_solve_host(self.handle, rowptr.ctypes.data, colind.ctypes.data,
                                                val.ctypes.data, int(val.size), B.ctypes.data, X.ctypes.data,
                                                nrhs, self.N, 1 if refine else 0, ctypes.byref(it),
                                                rel.ctypes.data, _stream_ptr(stream)),
               "spalu_factor_solve_host")
        return X, it.value, rel

    def residual_noalloc(self, B, X, stream=None):
        """||B - A X|| / ||B|| per column without any device allocation (nrhs <= 64)."""
        import torch
        nrhs = self._nrhs(B, X)
        rel = np.zeros(nrhs)
        _check(self.lib.spalu_residual_noalloc(self.handle, _dev_ptr(B, torch.float64),
                                               _dev_ptr(X, torch.float64), nrhs, self.N,
                                               rel.ctypes.data, _stream_ptr(stream)),
               "spalu_residual_noalloc")
        return rel

    def export_level(self, l: int) -> dict:
        """spalu_factor_export_level: the index tables of level l as numpy arrays: cnt, kk,
        nodes and skel (nseg x capS), pcnt (nparent x 2) and pmap (nparent x ldFp x 2)."""
        info = np.zeros(4, dtype=np.int32)
        _check(self.lib.spalu_factor_export_level(self.handle, l, info.ctypes.data, None, None, None, None,
                                                  None, None), "spalu_factor_export_level")
        nseg, cap, npar, ldp = (int(v) for v in info)
        out = {"cnt": np.zeros(nseg, np.int32), "kk": np.zeros(nseg, np.int32),
               "nodes": np.zeros((nseg, cap), np.int32), "skel": np.zeros((nseg, cap), np.int32),
               "pcnt": np.zeros((npar, 2), np.int32), "pmap": np.full((npar, ldp, 2), -1, np.int32)}
        _check(self.lib.spalu_factor_export_level(self.handle, l, info.ctypes.data,
                                                  *[out[k].ctypes.data for k in
                                                    ("cnt", "kk", "nodes", "skel", "pcnt", "pmap")]),
               "spalu_factor_export_level")
        out["info"] = info
        return out

    def set_timing(self, on: bool = True):
        _check(self.lib.spalu_set_timing(self.handle, 1 if on else 0), "spalu_set_timing")

    def set_predictor(self, predictor: "Predictor | None", mode: str = "predict", margin: float = 0.35):
        """spalu_factor_set_predictor: mode "off", "record" or "predict" for the next factor."""
        self._pred = predictor             # keep it alive while the factor may use it
        _check(self.lib.spalu_factor_set_predictor(self.handle, predictor.handle if predictor else None,
                                                   PRED_MODES[mode], float(margin)),
               "spalu_factor_set_predictor")

    def export_training(self, cap: int | None = None, stream=None):
        """spalu_factor_export_training: (X, Y) device float32 tensors of the recorded rows."""
        import torch
        if cap is None:
            cap = sum(lv["nseg"] for lv in self.stats()["levels"])
        X = torch.empty((max(cap, 1), PRED_NFEAT), dtype=torch.float32, device="cuda")
        Y = torch.empty((max(cap, 1), 2), dtype=torch.float32, device="cuda")
        n = ctypes.c_int(0)
        _check(self.lib.spalu_factor_export_training(self.handle, _dev_ptr(X, torch.float32),
                                                     _dev_ptr(Y, torch.float32), int(cap), ctypes.byref(n),
                                                     _stream_ptr(stream)), "spalu_factor_export_training")
        m = min(n.value, cap)
        return X[:m], Y[:m]

    def stats(self) -> dict:
        buf = ctypes.create_string_buffer(1 << 16)
        _check(self.lib.spalu_stats(self.handle, buf, len(buf)), "spalu_stats")
        return json.loads(buf.value.decode())

    def __del__(self):
        h = getattr(self, "handle", None)
        if h:
            self.lib.spalu_factor_destroy(h)
            self.handle = None


def factor_batch(factors, csrs, streams):
    """Numeric factorization of independent problems: factors[i] from csrs[i] = (rowptr, colind,
    val) device tensors on streams[i]; all problems are enqueued before any is waited for."""
    import torch
    n = len(factors)
    if not (len(csrs) == n and len(streams) == n):
        raise ValueError("factors, csrs and streams must have the same length")
    P = ctypes.c_void_p * n
    hs = P(*[f.handle for f in factors])
    rp = P(*[_dev_ptr(c[0], torch.int32).value for c in csrs])
    ci = P(*[_dev_ptr(c[1], torch.int32).value for c in csrs])
    va = P(*[_dev_ptr(c[2], torch.float64).value for c in csrs])
    nz = (ctypes.c_int * n)(*[int(c[2].numel()) for c in csrs])
    st = P(*[_stream_ptr(s).value for s in streams])
    _check(load_library().spalu_factor_numeric_batch(n, hs, rp, ci, va, nz, st), "spalu_factor_numeric_batch")


def solve_batch(factors, Bs, Xs, streams):
    """X_i = spaLU_i^{-1} B_i on streams[i] for every problem (device float64 tensors shaped
    (nrhs, N) or (N,)); enqueued only, not synchronised."""
    import torch
    n = len(factors)
    if not (len(Bs) == n and len(Xs) == n and len(streams) == n):
        raise ValueError("factors, Bs, Xs and streams must have the same length")
    P = ctypes.c_void_p * n
    hs = P(*[f.handle for f in factors])
    bp = P(*[_dev_ptr(B, torch.float64).value for B in Bs])
    xp = P(*[_dev_ptr(X, torch.float64).value for X in Xs])
    nr = (ctypes.c_int * n)(*[f._nrhs(B, X) for f, B, X in zip(factors, Bs, Xs)])
    ld = (ctypes.c_int * n)(*[f.N for f in factors])
    st = P(*[_stream_ptr(s).value for s in streams])
    _check(load_library().spalu_solve_batch(n, hs, bp, xp, nr, ld, st), "spalu_solve_batch")


class Predictor:
    """spalu_predictor_*: the learned rank predictor (16 -> 64 ReLU -> 2; BF16 inference,
    FP32 training with Adam, all on the device)."""

    def __init__(self, params: np.ndarray):
        self.lib = load_library()
        p = np.ascontiguousarray(params, dtype=np.float32)
        if p.size != PRED_NPARAM:
            raise ValueError(f"expected {PRED_NPARAM} parameters")
        h = ctypes.c_void_p()
        _check(self.lib.spalu_predictor_create(p.ctypes.data, ctypes.byref(h)), "spalu_predictor_create")
        self.handle = h

    def params(self, stream=None) -> np.ndarray:
        out = np.empty(PRED_NPARAM, dtype=np.float32)
        _check(self.lib.spalu_predictor_get_params(self.handle, out.ctypes.data, _stream_ptr(stream)),
               "spalu_predictor_get_params")
        return out

    def set_norm(self, mu, isd, stream=None):
        mu = np.ascontiguousarray(mu, dtype=np.float32)
        isd = np.ascontiguousarray(isd, dtype=np.float32)
        _check(self.lib.spalu_predictor_set_norm(self.handle, mu.ctypes.data, isd.ctypes.data,
                                                 _stream_ptr(stream)), "spalu_predictor_set_norm")

    def norm(self, stream=None):
        mu = np.empty(PRED_NFEAT, dtype=np.float32)
        isd = np.empty(PRED_NFEAT, dtype=np.float32)
        _check(self.lib.spalu_predictor_get_norm(self.handle, mu.ctypes.data, isd.ctypes.data,
                                                 _stream_ptr(stream)), "spalu_predictor_get_norm")
        return mu, isd

    def fit_norm(self, X, stream=None):
        import torch
        _check(self.lib.spalu_predictor_fit_norm(self.handle, _dev_ptr(X, torch.float32), int(X.shape[0]),
                                                 _stream_ptr(stream)), "spalu_predictor_fit_norm")

    def loss_grad(self, X, Y, stream=None):
        import torch
        loss = ctypes.c_float(0.0)
        g = np.empty(PRED_NPARAM, dtype=np.float32)
        _check(self.lib.spalu_predictor_loss_grad(self.handle, _dev_ptr(X, torch.float32),
                                                  _dev_ptr(Y, torch.float32), int(X.shape[0]),
                                                  ctypes.byref(loss), g.ctypes.data, _stream_ptr(stream)),
               "spalu_predictor_loss_grad")
        return loss.value, g

    def train(self, X, Y, epochs: int, batch: int = 256, lr: float = 1e-3, stream=None) -> float:
        import torch
        loss = ctypes.c_float(0.0)
        _check(self.lib.spalu_predictor_train(self.handle, _dev_ptr(X, torch.float32),
                                              _dev_ptr(Y, torch.float32), int(X.shape[0]), int(epochs),
                                              int(batch), float(lr), ctypes.byref(loss), _stream_ptr(stream)),
               "spalu_predictor_train")
        return loss.value

    def infer(self, X, stream=None):
        import torch
        out = torch.empty((X.shape[0], 2), dtype=torch.float32, device=X.device)
        _check(self.lib.spalu_predictor_infer(self.handle, _dev_ptr(X, torch.float32), int(X.shape[0]),
                                              _dev_ptr(out, torch.float32), _stream_ptr(stream)),
               "spalu_predictor_infer")
        return out

    def __del__(self):
        h = getattr(self, "handle", None)
        if h:
            self.lib.spalu_predictor_destroy(h)
            self.handle = None


class BatchGraph:
    """spalu_batch_graph_*: the steps (factor, solve, optionally one GMRES cycle) of many
    independent problems captured as one CUDA graph; run() replays it."""

    def __init__(self, factors, csrs, Bs, Xs, nstreams: int = 16, refine: bool = True, stream=None):
        import torch
        n = len(factors)
        if not (len(csrs) == n and len(Bs) == n and len(Xs) == n):
            raise ValueError("factors, csrs, Bs and Xs must have the same length")
        self.lib = load_library()
        self.factors = list(factors)
        self._keep = (list(csrs), list(Bs), list(Xs))
        P = ctypes.c_void_p * n
        for f, (rp, ci, va) in zip(factors, csrs):
            f._csr_shape(rp, ci, va)
        self.nrhs = [f._nrhs(B, X) for f, B, X in zip(factors, Bs, Xs)]
        args = [P(*[f.handle for f in factors]),
                P(*[_dev_ptr(c[0], torch.int32).value for c in csrs]),
                P(*[_dev_ptr(c[1], torch.int32).value for c in csrs]),
                P(*[_dev_ptr(c[2], torch.float64).value for c in csrs]),
                (ctypes.c_int * n)(*[int(c[2].numel()) for c in csrs]),
                P(*[_dev_ptr(B, torch.float64).value for B in Bs]),
                P(*[_dev_ptr(X, torch.float64).value for X in Xs]),
                (ctypes.c_int * n)(*self.nrhs),
                (ctypes.c_int * n)(*[f.N for f in factors])]
        h = ctypes.c_void_p()
        _check(self.lib.spalu_batch_graph_create(n, *args, int(nstreams), 1 if refine else 0, _stream_ptr(stream),
                                                 ctypes.byref(h)), "spalu_batch_graph_create")
        self.handle = h
        self.n = n

    def run(self, stream=None, check=True):
        """Replay the graph; returns (iterations per problem, largest relative residual per problem)."""
        it = np.zeros(self.n, dtype=np.int32)
        rel = np.zeros(self.n)
        st = self.lib.spalu_batch_graph_run(self.handle, it.ctypes.data, rel.ctypes.data, _stream_ptr(stream))
        if check:
            _check(st, "spalu_batch_graph_run")
        return it, rel

    def __del__(self):
        h = getattr(self, "handle", None)
        if h:
            self.lib.spalu_batch_graph_destroy(h)
            self.handle = None
