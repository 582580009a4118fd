"""Python binding of ``libhsolve.so`` (ctypes; argument marshalling only).

Every step of the factorization, the substitution sweeps and the Krylov
solve runs in the library's CUDA kernels.  Device buffers are torch CUDA
tensors (float64, column-major n x nrhs, i.e. a C-contiguous (nrhs, n)
tensor); the library never falls back to any host computation: if the
library cannot be loaded, every call raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libhsolve.so")

OK = 0
STATUS = {0: "OK", -1: "ERR_ARG", -2: "ERR_CUDA", -3: "ERR_OOM", -4: "ERR_SINGULAR",
          -5: "ERR_NOT_SPD", -6: "ERR_NO_CONVERGENCE", -7: "ERR_BUDGET", -8: "ERR_TIMEOUT",
          -9: "ERR_STATE"}
PRECISION = {"fp64": 0, "mixed_fp32": 1, "mixed_tf32": 2, "mixed_bf16": 3, "mixed_3xtf32": 4}
KRYLOV = {"pcg": 0, "gmres": 1}


class HsolveError(RuntimeError):
    def __init__(self, code, msg=""):
        self.code = code
        super().__init__(f"hsolve {STATUS.get(code, code)}: {msg}")


class Csr(C.Structure):
    _fields_ = [("n", C.c_int64), ("nnz", C.c_int64), ("rowptr", C.c_void_p),
                ("col", C.c_void_p), ("val", C.c_void_p)]


class Opts(C.Structure):
    _fields_ = [("leaf_size", C.c_int32), ("symmetric", C.c_int32), ("top_size", C.c_int64),
                ("max_rank", C.c_int32), ("gmres_restart", C.c_int32), ("compress", C.c_int32),
                ("cluster_qr", C.c_int32), ("equilibrate", C.c_int32)]


class SolveInfo(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("rel_residual", C.c_double),
                ("factor_ms", C.c_double), ("solve_ms", C.c_double)]


class Stats(C.Structure):
    _fields_ = [("levels", C.c_int32), ("clusters0", C.c_int32), ("colours_total", C.c_int32),
                ("top_size", C.c_int32), ("coarse_total", C.c_int64),
                ("factor_bytes", C.c_int64), ("block_bytes", C.c_int64),
                ("apply_bytes", C.c_int64), ("factor_flops", C.c_double),
                ("schur_flops", C.c_double), ("prep_flops", C.c_double),
                ("gemm_flops", C.c_double), ("kernel_launches", C.c_int32),
                ("precision", C.c_int32), ("launches_total", C.c_int64),
                ("qr_flops", C.c_double)]


class ClusterExport(C.Structure):
    _fields_ = [("m", C.c_int32), ("k", C.c_int32), ("nw", C.c_int32), ("nnb", C.c_int32),
                ("colour", C.c_int32), ("npiv", C.c_int32), ("T", C.c_int64), ("TR", C.c_int64),
                ("Y", C.c_int64), ("XT", C.c_int64), ("piv", C.c_int64), ("nb", C.c_int64)]


class LevelExport(C.Structure):
    _fields_ = [("nclu", C.c_int32), ("dense_top", C.c_int32), ("symmetric", C.c_int32),
                ("precision", C.c_int32), ("fac_elems", C.c_int64), ("piv_total", C.c_int64),
                ("nbr_total", C.c_int64)]


class PhaseTime(C.Structure):
    _fields_ = [("name", C.c_char * 24), ("ms", C.c_double), ("launches", C.c_int32)]


EXPORTS = {
    "hsolve_default_opts": (None, [C.POINTER(Opts)]),
    "hsolve_analyze": (C.c_int, [C.POINTER(Csr), C.c_void_p, C.c_int, C.POINTER(Opts), C.c_void_p,
                                 C.POINTER(C.c_void_p)]),
    "hsolve_factor": (C.c_int, [C.c_void_p, C.c_double, C.c_int]),
    "hsolve_factor_forced": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_int32,
                                       C.c_void_p]),
    "hsolve_apply": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_int64]),
    "hsolve_apply_noalloc": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_int64]),
    "hsolve_solve": (C.c_int, [C.c_void_p, C.c_int, C.c_double, C.c_int, C.c_void_p, C.c_void_p,
                               C.c_int, C.c_int64, C.POINTER(SolveInfo)]),
    "hsolve_solve_host": (C.c_int, [C.c_void_p, C.c_int, C.c_double, C.c_int, C.c_void_p,
                                    C.c_void_p, C.c_int, C.c_int64, C.POINTER(SolveInfo)]),
    "hsolve_spmv": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_int64]),
    "hsolve_get_stats": (C.c_int, [C.c_void_p, C.POINTER(Stats)]),
    "hsolve_get_level": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_int32), C.c_void_p,
                                   C.c_void_p, C.c_void_p, C.c_int32]),
    "hsolve_get_perm": (C.c_int, [C.c_void_p, C.c_void_p]),
    "hsolve_export_level": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(LevelExport), C.c_void_p,
                                      C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "hsolve_export_cluster": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.POINTER(ClusterExport),
                                        C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                        C.c_void_p, C.c_void_p, C.c_void_p]),
    "hsolve_get_phase_times": (C.c_int, [C.c_void_p, C.POINTER(PhaseTime), C.c_int32,
                                         C.POINTER(C.c_int32)]),
    "hsolve_set_profiling": (C.c_int, [C.c_void_p, C.c_int]),
    "hsolve_last_error": (C.c_char_p, [C.c_void_p]),
    "hsolve_destroy": (None, [C.c_void_p]),
    "hsolve_wait_selftest": (C.c_int, [C.c_int, C.c_int64, C.c_void_p]),
    "hsolve_tc_gemm": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_int64,
                                 C.c_int64, C.c_void_p, C.c_int64, C.c_int64, C.c_void_p,
                                 C.c_int64, C.c_float, C.c_float, C.c_int, C.c_void_p]),
}

TC_MODES = {"tf32": 0, "3xtf32": 1, "bf16": 2}


class ServerOpts(C.Structure):
    _fields_ = [("memory_budget", C.c_int64), ("max_batch_rhs", C.c_int32),
                ("workers", C.c_int32)]


class ServerResult(C.Structure):
    _fields_ = [("status", C.c_int32), ("iterations", C.c_int32), ("rel_residual", C.c_double),
                ("queue_ms", C.c_double), ("service_ms", C.c_double),
                ("latency_ms", C.c_double), ("batch_rhs", C.c_int32), ("factored", C.c_int32),
                ("message", C.c_char * 128)]


class ServerStats(C.Structure):
    _fields_ = [(n, C.c_int64) for n in (
        "requests_submitted", "requests_done", "rhs_done", "batches", "factorizations",
        "evictions", "resident", "resident_bytes", "peak_resident_bytes", "queued")]


EXPORTS.update({
    "hsolve_server_default_opts": (None, [C.POINTER(ServerOpts)]),
    "hsolve_server_create": (C.c_int, [C.POINTER(ServerOpts), C.POINTER(C.c_void_p)]),
    "hsolve_server_add_matrix": (C.c_int, [C.c_void_p, C.POINTER(Csr), C.c_void_p, C.c_int,
                                           C.POINTER(Opts), C.c_double, C.c_int, C.c_int,
                                           C.c_double, C.c_int, C.POINTER(C.c_int32)]),
    "hsolve_server_submit": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_int32, C.c_int64,
                                       C.POINTER(C.c_int64)]),
    "hsolve_server_wait": (C.c_int, [C.c_void_p, C.c_int64, C.c_void_p, C.c_int64,
                                     C.POINTER(ServerResult), C.c_double]),
    "hsolve_server_get_stats": (C.c_int, [C.c_void_p, C.POINTER(ServerStats)]),
    "hsolve_server_destroy": (None, [C.c_void_p]),
})

_lib = None


def load(path: str = LIB_PATH):
    """Load libhsolve.so (raises if it is missing: there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise HsolveError(-2, f"{path} not built; run paper_1712_07297_gb300.build.build()")
    lib = C.CDLL(path)
    for name, (res, args) in EXPORTS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def default_opts() -> Opts:
    o = Opts()
    load().hsolve_default_opts(C.byref(o))
    return o


def _check(code, handle=None):
    if code != OK:
        msg = ""
        if handle:
            m = load().hsolve_last_error(handle)
            msg = m.decode() if m else ""
        raise HsolveError(code, msg)


def _dev_ptr(t, n):
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64):
        raise TypeError("expected a float64 CUDA tensor")
    if t.dim() == 1:
        if t.shape[0] != n or not t.is_contiguous():
            raise ValueError("vector of length n expected")
        return t.data_ptr(), 1, n
    if t.dim() != 2 or t.shape[1] != n or t.stride(1) != 1:
        raise ValueError("(nrhs, n) tensor with unit stride along n expected")
    return t.data_ptr(), t.shape[0], t.stride(0)


class Solver:
    """One analysed matrix: analyze -> factor -> apply / solve."""

    def __init__(self, rowptr, col, val, coords=None, *, leaf_size=128, symmetric=-1, top_size=0,
                 max_rank=0, gmres_restart=50, compress=0, cluster_qr=1, equilibrate=0,
                 stream=None):
        lib = load()
        self.rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
        self.col = np.ascontiguousarray(col, dtype=np.int32)
        self.val = np.ascontiguousarray(val, dtype=np.float64)
        self.n = len(self.rowptr) - 1
        csr = Csr(self.n, len(self.col), self.rowptr.ctypes.data, self.col.ctypes.data,
                  self.val.ctypes.data)
        o = default_opts()
        o.leaf_size, o.symmetric, o.top_size = leaf_size, symmetric, top_size
        o.max_rank, o.gmres_restart, o.compress = max_rank, gmres_restart, compress
        o.cluster_qr = cluster_qr
        o.equilibrate = equilibrate
        h = C.c_void_p()
        cptr, dim = None, 0
        if coords is not None:
            self._coords = np.ascontiguousarray(coords, dtype=np.float64)
            cptr, dim = self._coords.ctypes.data, self._coords.shape[1]
        st = None
        if stream is not None:
            st = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
        _check(lib.hsolve_analyze(C.byref(csr), cptr, dim, C.byref(o), st, C.byref(h)))
        self.h = h

    @classmethod
    def from_problem(cls, prob, **kw):
        return cls(prob.rowptr, prob.col, prob.val, prob.coords, **kw)

    def close(self):
        if getattr(self, "h", None):
            load().hsolve_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def factor(self, eps: float, precision="fp64"):
        p = PRECISION[precision] if isinstance(precision, str) else int(precision)
        _check(load().hsolve_factor(self.h, float(eps), p), self.h)

    def factor_forced(self, precision, ranks_per_level, pivots_per_level=None):
        """Factor with every cluster's rank fixed (hsolve_factor_forced):
        ranks_per_level[l] = the ranks of level l's clusters; optionally
        pivots_per_level[l][s] = cluster s's pivot order (ranks_per_level[l][s]
        column indices)."""
        p = PRECISION[precision] if isinstance(precision, str) else int(precision)
        counts = np.array([len(r) for r in ranks_per_level], dtype=np.int32)
        flat = np.ascontiguousarray(np.concatenate([np.asarray(r, dtype=np.int32)
                                                    for r in ranks_per_level]))
        pv = None
        if pivots_per_level is not None:
            parts = [np.asarray(q, dtype=np.int32).ravel()
                     for lv in pivots_per_level for q in lv]
            for lv, rk in zip(pivots_per_level, ranks_per_level):
                if [len(q) for q in lv] != [int(k) for k in rk]:
                    raise ValueError("pivot lists must have ranks[s] entries")
            pv = np.ascontiguousarray(np.concatenate(parts) if parts else
                                      np.zeros(1, dtype=np.int32))
        _check(load().hsolve_factor_forced(self.h, p, flat.ctypes.data, counts.ctypes.data,
                                           len(counts), None if pv is None else pv.ctypes.data),
               self.h)

    def apply(self, rhs, out=None):
        """out = M^{-1} rhs on the device (torch float64 CUDA tensors)."""
        import torch
        ptr, nrhs, ld = _dev_ptr(rhs, self.n)
        if out is None:
            out = torch.empty_like(rhs)
        optr, onrhs, old = _dev_ptr(out, self.n)
        if onrhs != nrhs or old != ld:
            raise ValueError("rhs/out layouts differ")
        _check(load().hsolve_apply(self.h, ptr, optr, nrhs, ld), self.h)
        return out

    def apply_noalloc(self, rhs, out):
        """out = M^{-1} rhs through hsolve_apply_noalloc: the library
        allocates no device memory (temporaries come from its fixed scratch
        array); `out` must be given."""
        ptr, nrhs, ld = _dev_ptr(rhs, self.n)
        optr, onrhs, old = _dev_ptr(out, self.n)
        if onrhs != nrhs or old != ld:
            raise ValueError("rhs/out layouts differ")
        _check(load().hsolve_apply_noalloc(self.h, ptr, optr, nrhs, ld), self.h)
        return out

    def spmv(self, x, y=None):
        import torch
        ptr, nrhs, ld = _dev_ptr(x, self.n)
        if y is None:
            y = torch.empty_like(x)
        yptr, _, _ = _dev_ptr(y, self.n)
        _check(load().hsolve_spmv(self.h, ptr, yptr, nrhs, ld), self.h)
        return y

    def solve(self, b, x=None, *, krylov="pcg", tol=1e-10, maxit=1000, check=True):
        import torch
        ptr, nrhs, ld = _dev_ptr(b, self.n)
        if x is None:
            x = torch.empty_like(b)
        xptr, _, _ = _dev_ptr(x, self.n)
        info = SolveInfo()
        code = load().hsolve_solve(self.h, KRYLOV[krylov], tol, maxit, ptr, xptr, nrhs, ld,
                                   C.byref(info))
        if check:
            _check(code, self.h)
        return x, info

    def solve_host(self, b: np.ndarray, *, krylov="pcg", tol=1e-10, maxit=1000, check=True):
        """Host arrays in and out (copies are part of the call)."""
        b = np.ascontiguousarray(b, dtype=np.float64)
        bb = b[None, :] if b.ndim == 1 else b
        x = np.empty_like(bb)
        info = SolveInfo()
        code = load().hsolve_solve_host(self.h, KRYLOV[krylov], tol, maxit, bb.ctypes.data,
                                        x.ctypes.data, bb.shape[0], self.n, C.byref(info))
        if check:
            _check(code, self.h)
        return (x[0] if b.ndim == 1 else x), info

    def stats(self) -> dict:
        s = Stats()
        _check(load().hsolve_get_stats(self.h, C.byref(s)), self.h)
        return {k: getattr(s, k) for k, _ in Stats._fields_}

    def level(self, level: int):
        lib = load()
        nc = C.c_int32()
        _check(lib.hsolve_get_level(self.h, level, C.byref(nc), None, None, None, 0), self.h)
        sizes = np.zeros(nc.value, dtype=np.int32)
        ranks = np.zeros(nc.value, dtype=np.int32)
        colour = np.zeros(nc.value, dtype=np.int32)
        _check(lib.hsolve_get_level(self.h, level, C.byref(nc), sizes.ctypes.data,
                                    ranks.ctypes.data, colour.ctypes.data, nc.value), self.h)
        return sizes, ranks, colour

    def export_level(self, level: int, blocks: bool = True) -> dict:
        """The stored operators of one level (hsolve_export_level): a dict with
        the level's flags and, per cluster, m, k, nw, colour, pivots,
        neighbours (id, width) and (blocks=True) the blocks T', T'_R^T, Y, X^T
        as float64 arrays (None where the factorization keeps none)."""
        lib = load()
        info = LevelExport()
        _check(lib.hsolve_export_level(self.h, level, C.byref(info), None, None, None, None,
                                       None), self.h)
        nc = info.nclu
        recs = (ClusterExport * max(nc, 1))()
        fac = np.zeros(max(info.fac_elems, 1) if blocks else 1, dtype=np.float64)
        piv = np.zeros(max(info.piv_total, 1), dtype=np.int32)
        nid = np.zeros(max(info.nbr_total, 1), dtype=np.int32)
        nw = np.zeros(max(info.nbr_total, 1), dtype=np.int32)
        _check(lib.hsolve_export_level(self.h, level, C.byref(info), recs,
                                       fac.ctypes.data if blocks else None, piv.ctypes.data,
                                       nid.ctypes.data, nw.ctypes.data), self.h)

        def blk(off, rows, cols):
            if not blocks or off < 0 or rows == 0 or cols == 0:
                return None
            return fac[off:off + rows * cols].reshape(cols, rows).T.copy()

        out = []
        for s in range(nc):
            r = recs[s]
            m, k = r.m, r.k
            out.append(dict(
                m=m, k=k, nw=r.nw, colour=r.colour, piv=piv[r.piv:r.piv + r.npiv].copy(),
                nbrs=list(zip(nid[r.nb:r.nb + r.nnb].tolist(), nw[r.nb:r.nb + r.nnb].tolist())),
                T=blk(r.T, m, m), TRt=blk(r.TR, m, m), Y=blk(r.Y, m, r.nw),
                XT=blk(r.XT, m, r.nw)))
        return dict(nclu=nc, dense_top=bool(info.dense_top), symmetric=bool(info.symmetric),
                    precision=info.precision, clusters=out)

    def export_cluster(self, level: int, cluster: int) -> dict:
        """One cluster's record and blocks (hsolve_export_cluster): the same
        keys as a cluster of export_level."""
        lib = load()
        r = ClusterExport()
        _check(lib.hsolve_export_cluster(self.h, level, cluster, C.byref(r), None, None, None,
                                         None, None, None, None), self.h)
        m, k, nw, nnb = r.m, r.k, r.nw, r.nnb
        T = np.zeros(max(m * m, 1)) if r.T >= 0 else None
        TRt = np.zeros(max(m * m, 1)) if r.TR >= 0 else None
        Y = np.zeros(max(m * nw, 1)) if r.Y >= 0 else None
        XT = np.zeros(max(m * nw, 1)) if r.XT >= 0 else None
        piv = np.zeros(max(k, 1), dtype=np.int32)
        nid = np.zeros(max(nnb, 1), dtype=np.int32)
        nwd = np.zeros(max(nnb, 1), dtype=np.int32)
        ptr = lambda a: None if a is None else a.ctypes.data  # noqa: E731
        _check(lib.hsolve_export_cluster(self.h, level, cluster, C.byref(r), ptr(T), ptr(TRt),
                                         ptr(Y), ptr(XT), piv.ctypes.data, nid.ctypes.data,
                                         nwd.ctypes.data), self.h)

        def mat(a, cols):
            return None if a is None else a[:m * cols].reshape(cols, m).T.copy()

        return dict(m=m, k=k, nw=nw, colour=r.colour, piv=piv[:k].copy(),
                    nbrs=list(zip(nid[:nnb].tolist(), nwd[:nnb].tolist())),
                    T=mat(T, m), TRt=mat(TRt, m), Y=mat(Y, nw), XT=mat(XT, nw))

    def perm(self) -> np.ndarray:
        p = np.zeros(self.n, dtype=np.int64)
        _check(load().hsolve_get_perm(self.h, p.ctypes.data), self.h)
        return p

    def set_profiling(self, on, per_level=False, deferred=False):
        v = 0 if not on else (2 if per_level else (3 if deferred else 1))
        _check(load().hsolve_set_profiling(self.h, v), self.h)

    def phase_times(self) -> dict:
        lib = load()
        cnt = C.c_int32()
        _check(lib.hsolve_get_phase_times(self.h, None, 0, C.byref(cnt)), self.h)
        arr = (PhaseTime * max(cnt.value, 1))()
        _check(lib.hsolve_get_phase_times(self.h, arr, cnt.value, C.byref(cnt)), self.h)
        return {arr[i].name.decode(): (arr[i].ms, arr[i].launches) for i in range(cnt.value)}


def wait_selftest(kind: str, limit_cycles: int) -> int:
    """Run one bounded device wait that nothing signals (hsolve_wait_selftest):
    kind "mbarrier" (the tensor-core kernels' wait); returns the status code
    (HSOLVE_ERR_TIMEOUT = -8 when it gave up)."""
    return load().hsolve_wait_selftest({"mbarrier": 0}[kind], int(limit_cycles), None)


def tc_gemm(mode, A, B, C_, alpha=1.0, beta=0.0, lower=False, stream=None):
    """C_ = beta C_ + alpha A B^T on the tensor cores (hsolve_tc_gemm).

    A (M x K), B (N x K): float32 CUDA tensors of any strides; C_: float32
    CUDA tensor (M x N) stored column-major (C_.stride() == (1, ldc)).
    mode: "tf32", "3xtf32" or "bf16"."""
    M, K = A.shape
    N, K2 = B.shape
    if K2 != K or tuple(C_.shape) != (M, N) or C_.stride(0) != 1:
        raise ValueError("tc_gemm: shapes or C layout")
    for t in (A, B, C_):
        if t.dtype.__str__() != "torch.float32" or not t.is_cuda:
            raise ValueError("tc_gemm: float32 CUDA tensors")
    st = None if stream is None else C.c_void_p(stream.cuda_stream)
    _check(load().hsolve_tc_gemm(TC_MODES[mode], M, N, K, A.data_ptr(), A.stride(0), A.stride(1),
                                 B.data_ptr(), B.stride(0), B.stride(1), C_.data_ptr(),
                                 max(C_.stride(1), M), float(alpha), float(beta), int(lower), st))
    return C_


class Server:
    """The serving runtime (hsolve_server_*): register matrices, submit
    host right-hand sides (numpy (nrhs, n)), wait for solutions."""

    def __init__(self, memory_budget=60 << 30, max_batch_rhs=256, workers=4):
        o = ServerOpts(int(memory_budget), int(max_batch_rhs), int(workers))
        self.h = C.c_void_p()
        _check(load().hsolve_server_create(C.byref(o), C.byref(self.h)))
        self.n = {}

    def add_matrix(self, prob, eps, precision="mixed_fp32", krylov="pcg", tol=1e-10, maxit=500,
                   leaf_size=128, symmetric=-1, top_size=0, equilibrate=0):
        import numpy as np
        rp = np.ascontiguousarray(prob.rowptr, dtype=np.int64)
        col = np.ascontiguousarray(prob.col, dtype=np.int32)
        val = np.ascontiguousarray(prob.val, dtype=np.float64)
        xyz = np.ascontiguousarray(prob.coords, dtype=np.float64)
        csr = Csr(prob.n, len(col), rp.ctypes.data, col.ctypes.data, val.ctypes.data)
        o = default_opts()
        o.leaf_size, o.symmetric, o.top_size, o.equilibrate = leaf_size, symmetric, top_size, \
            equilibrate
        mid = C.c_int32()
        p = PRECISION[precision] if isinstance(precision, str) else int(precision)
        _check(load().hsolve_server_add_matrix(self.h, C.byref(csr), xyz.ctypes.data,
                                               xyz.shape[1], C.byref(o), float(eps), p,
                                               KRYLOV[krylov], float(tol), int(maxit),
                                               C.byref(mid)))
        self.n[mid.value] = prob.n
        return mid.value

    def submit(self, matrix_id, b):
        import numpy as np
        b = np.ascontiguousarray(b, dtype=np.float64)
        if b.ndim == 1:
            b = b[None, :]
        rid = C.c_int64()
        _check(load().hsolve_server_submit(self.h, int(matrix_id), b.ctypes.data, b.shape[0],
                                           b.shape[1], C.byref(rid)))
        return rid.value, b.shape

    def wait(self, ticket, timeout=600.0, want_x=True):
        """Block until the request is served; returns (x (nrhs, n) or None,
        result record)."""
        import numpy as np
        rid, shape = ticket
        x = np.empty(shape, dtype=np.float64) if want_x else None
        res = ServerResult()
        code = load().hsolve_server_wait(self.h, rid, x.ctypes.data if want_x else None,
                                         shape[1], C.byref(res), float(timeout))
        if code != OK:
            raise HsolveError(code, res.message.decode(errors="replace"))
        return x, {k: getattr(res, k) for k, _ in ServerResult._fields_}

    def stats(self):
        st = ServerStats()
        _check(load().hsolve_server_get_stats(self.h, C.byref(st)))
        return {k: getattr(st, k) for k, _ in ServerStats._fields_}

    def close(self):
        if getattr(self, "h", None):
            load().hsolve_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
