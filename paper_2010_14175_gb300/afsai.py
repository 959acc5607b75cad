"""Python binding of libafsai.so: argument marshalling only.

Every step of the set-up, the preconditioner application and PCG runs in
the CUDA library (``csrc/``) behind the C ABI declared in
``include/afsai.h``.  PyTorch is used for device memory and streams:
tensors are passed by ``data_ptr()`` and the current stream by handle.
There is no CPU fallback: if the library is missing or no GPU is present,
the calls raise.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

_lock = threading.Lock()
_lib = None

STATUS = {
    0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ENOTSPD", 4: "ENOCONV", 5: "ECUDA", 6: "ETIMEOUT", 7: "EAGAIN",
    8: "EBUSY", 9: "ENOTSUP",
}
OK, EINVAL, ENOMEM, ENOTSPD, ENOCONV, ECUDA, ETIMEOUT, EAGAIN, EBUSY, ENOTSUP = range(10)

# names exported by include/afsai.h (checked by the ABI test)
EXPORTS = (
    "afsai_setup", "afsai_apply", "afsai_spmv", "pcg_solve", "afsai_solve_host", "afsai_get_info",
    "afsai_export_G", "afsai_export_Gt", "afsai_export_rows", "afsai_destroy", "afsai_last_error", "afsai_version",
    "afsai_kernel_launches", "afsai_apply_static", "afsai_batch_solve", "serve_create", "serve_register",
    "serve_submit", "serve_poll", "serve_get_stats", "serve_destroy", "afsai_spmv_engine", "afsai_check_arith",
    "afsai_trim_pool", "afsai_pool_stats",
)


class AfsaiError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Csr(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("nnz", ctypes.c_int64), ("rowptr", ctypes.c_void_p),
                ("col", ctypes.c_void_p), ("val", ctypes.c_void_p)]


class Params(ctypes.Structure):
    _fields_ = [("kiter", ctypes.c_int32), ("s", ctypes.c_int32), ("eps", ctypes.c_double),
                ("exit_mode", ctypes.c_int32), ("g_prec", ctypes.c_int32), ("chol_prec", ctypes.c_int32),
                ("block_rows", ctypes.c_int32), ("block_power", ctypes.c_int32)]


class Info(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("nnz_G", ctypes.c_int64), ("max_row", ctypes.c_int32),
                ("g_prec", ctypes.c_int32), ("n_retry", ctypes.c_int32), ("setup_ms", ctypes.c_double),
                ("kernel_ms", ctypes.c_double)]


class BatchInfo(ctypes.Structure):
    _fields_ = [("nsys", ctypes.c_int32), ("converged", ctypes.c_int32), ("max_iters", ctypes.c_int32),
                ("graph_launches", ctypes.c_int32), ("total_rows", ctypes.c_int64), ("nnz_G", ctypes.c_int64),
                ("setup_ms", ctypes.c_double), ("solve_ms", ctypes.c_double)]


class ServeResult(ctypes.Structure):
    _fields_ = [("nrhs", ctypes.c_int32), ("max_iters", ctypes.c_int32), ("converged", ctypes.c_int32),
                ("pad", ctypes.c_int32), ("max_relres_true", ctypes.c_double), ("queue_ms", ctypes.c_double),
                ("setup_ms", ctypes.c_double), ("latency_ms", ctypes.c_double)]


class ServeStats(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int64) for k in ("requests_submitted", "requests_done", "solves", "steps",
                                              "peak_mem_bytes", "mem_used_bytes", "queued", "running")]


class PcgInfo(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("converged", ctypes.c_int32), ("relres_rec", ctypes.c_double),
                ("relres_true", ctypes.c_double), ("solve_ms", ctypes.c_double), ("kernel_ms", ctypes.c_double * 5)]


def _as_dict(s):
    out = {}
    for k, _ in s._fields_:
        v = getattr(s, k)
        out[k] = list(v) if isinstance(v, ctypes.Array) else v
    return out


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libafsai.so (building it first if needed)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if build_if_missing and not _build.up_to_date():
            _build.build()
        if not os.path.exists(path):
            raise RuntimeError(f"libafsai.so not built ({path}); run paper_2010_14175_gb300.build.build()")
        lib = ctypes.CDLL(path)
        P = ctypes.c_void_p
        st = ctypes.c_int
        lib.afsai_setup.argtypes = [ctypes.POINTER(Csr), ctypes.POINTER(Params), P, ctypes.POINTER(P)]
        lib.afsai_setup.restype = st
        lib.afsai_apply.argtypes = [P, P, P, P]
        lib.afsai_apply.restype = st
        lib.afsai_apply_static.argtypes = [P, P, P, P]
        lib.afsai_apply_static.restype = st
        lib.afsai_spmv.argtypes = [ctypes.POINTER(Csr), P, P, P]
        lib.afsai_spmv.restype = st
        lib.pcg_solve.argtypes = [ctypes.POINTER(Csr), P, P, P, ctypes.c_double, ctypes.c_int32, P,
                                  ctypes.POINTER(PcgInfo)]
        lib.pcg_solve.restype = st
        lib.afsai_solve_host.argtypes = [ctypes.POINTER(Csr), ctypes.POINTER(Params), P, P, ctypes.c_double,
                                         ctypes.c_int32, P, ctypes.POINTER(Info), ctypes.POINTER(PcgInfo)]
        lib.afsai_solve_host.restype = st
        lib.afsai_get_info.argtypes = [P, ctypes.POINTER(Info)]
        lib.afsai_get_info.restype = st
        for fn in (lib.afsai_export_G, lib.afsai_export_Gt):
            fn.argtypes = [P, P, P, P]
            fn.restype = st
        lib.afsai_export_rows.argtypes = [P, P, P]
        lib.afsai_export_rows.restype = st
        lib.afsai_destroy.argtypes = [P]
        lib.afsai_destroy.restype = None
        lib.afsai_last_error.argtypes = []
        lib.afsai_last_error.restype = ctypes.c_char_p
        lib.afsai_version.argtypes = []
        lib.afsai_version.restype = ctypes.c_char_p
        lib.afsai_batch_solve.argtypes = [ctypes.c_int32, P, ctypes.POINTER(Params), P, P, ctypes.c_double,
                                          ctypes.c_int32, P, P, ctypes.POINTER(BatchInfo)]
        lib.afsai_batch_solve.restype = st
        lib.serve_create.argtypes = [ctypes.c_size_t, ctypes.c_int32, ctypes.POINTER(Params), ctypes.c_int32,
                                     ctypes.c_int32, ctypes.POINTER(P)]
        lib.serve_create.restype = st
        lib.serve_register.argtypes = [P, ctypes.POINTER(Csr), ctypes.POINTER(ctypes.c_int32)]
        lib.serve_register.restype = st
        lib.serve_submit.argtypes = [P, ctypes.c_int32, P, ctypes.c_int32, ctypes.c_double,
                                     ctypes.POINTER(ctypes.c_int64)]
        lib.serve_submit.restype = st
        lib.serve_poll.argtypes = [P, ctypes.c_int64, P, P, ctypes.POINTER(ServeResult)]
        lib.serve_poll.restype = st
        lib.serve_get_stats.argtypes = [P, ctypes.POINTER(ServeStats)]
        lib.serve_get_stats.restype = st
        lib.serve_destroy.argtypes = [P]
        lib.serve_destroy.restype = None
        lib.afsai_spmv_engine.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int64, ctypes.c_int32]
        lib.afsai_spmv_engine.restype = ctypes.c_int32
        lib.afsai_check_arith.argtypes = [ctypes.c_int64, ctypes.c_uint64, P, P]
        lib.afsai_check_arith.restype = ctypes.c_int
        lib.afsai_kernel_launches.argtypes = []
        lib.afsai_kernel_launches.restype = ctypes.c_int64
        lib.afsai_trim_pool.argtypes = []
        lib.afsai_trim_pool.restype = ctypes.c_int
        lib.afsai_pool_stats.argtypes = [P, P]
        lib.afsai_pool_stats.restype = ctypes.c_int
        _lib = lib
        return lib


def spmv_engine(role: int, n: int, nnz: int, vtype: int = 0) -> int:
    """Engine chosen for role 0 (A), 1 (G), 2 (G^T) of a matrix shape (0: none)."""
    return int(load().afsai_spmv_engine(int(role), int(n), int(nnz), int(vtype)))


def check_arith(n: int, seed: int = 1, stream=None):
    """Mismatch counts (divisions, square roots) of the library's integer-
    pipe FP64 arithmetic against the hardware IEEE operations on n operand
    sets drawn on the device."""
    out = (ctypes.c_int64 * 2)()
    _check(load().afsai_check_arith(int(n), int(seed) & 0xFFFFFFFFFFFFFFFF, ctypes.cast(out, ctypes.c_void_p),
                                    _stream(stream)))
    return int(out[0]), int(out[1])


def kernel_launches() -> int:
    """Kernels launched by the library so far in this process."""
    return int(load().afsai_kernel_launches())


def pool_stats():
    """(bytes in use, bytes reserved) of the library's memory pool on the
    current device."""
    used, reserved = ctypes.c_int64(), ctypes.c_int64()
    _check(load().afsai_pool_stats(ctypes.cast(ctypes.byref(used), ctypes.c_void_p),
                                   ctypes.cast(ctypes.byref(reserved), ctypes.c_void_p)))
    return int(used.value), int(reserved.value)


def trim_pool():
    """Returns the unused memory of the library's pool on the current device."""
    _check(load().afsai_trim_pool())


def _check(status):
    if status != OK:
        raise AfsaiError(status, load().afsai_last_error().decode())


def _stream(stream):
    import torch

    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _device_array(t, dtype_name, n, what):
    """Device address of a contiguous CUDA tensor of n entries of the given
    dtype.  The library reads and writes these addresses from its kernels,
    so a host tensor, another dtype or a shorter tensor is refused here,
    before the call (there is no CPU path)."""
    if not getattr(t, "is_cuda", False):
        raise ValueError(f"{what}: a CUDA tensor is required (the library has no CPU path)")
    if str(t.dtype) != "torch." + dtype_name:
        raise ValueError(f"{what}: dtype {dtype_name} expected, got {t.dtype}")
    if not t.is_contiguous() or t.numel() != n:
        raise ValueError(f"{what}: a contiguous tensor of {n} entries expected (got {t.numel()})")
    return ctypes.c_void_p(t.data_ptr())


def _vec(t, n, what):
    return _device_array(t, "float64", n, what)


class DeviceCSR:
    """A CSR matrix in device memory (torch tensors int32/int32/float64)."""

    def __init__(self, n, rowptr, col, val):
        self.n = int(n)
        self.rowptr, self.col, self.val = rowptr, col, val
        self.nnz = int(col.numel())

    @classmethod
    def from_host(cls, A, device="cuda"):
        import torch

        return cls(A.n, torch.from_numpy(np.ascontiguousarray(A.rowptr, dtype=np.int32)).to(device),
                   torch.from_numpy(np.ascontiguousarray(A.col, dtype=np.int32)).to(device),
                   torch.from_numpy(np.ascontiguousarray(A.val, dtype=np.float64)).to(device))

    def c(self) -> Csr:
        rp = _device_array(self.rowptr, "int32", self.n + 1, "rowptr")
        ci = _device_array(self.col, "int32", self.nnz, "col")
        va = _device_array(self.val, "float64", self.nnz, "val")
        return Csr(self.n, self.nnz, rp.value, ci.value, va.value)


def params(kiter, s, eps, exit_mode=0, g_prec=0, chol_prec=0, block_rows=0, block_power=1) -> Params:
    return Params(int(kiter), int(s), float(eps), int(exit_mode), int(g_prec), int(chol_prec), int(block_rows),
                  int(block_power))


class Precond:
    """Owns an afsai_precond* (G, G^T, per-row results in device memory)."""

    def __init__(self, handle):
        self._h = handle
        self._n = None

    @property
    def handle(self):
        return self._h

    @property
    def n(self) -> int:
        if self._n is None:
            self._n = self.info()["n"]
        return self._n

    def info(self) -> dict:
        inf = Info()
        _check(load().afsai_get_info(self._h, ctypes.byref(inf)))
        return _as_dict(inf)

    def export(self, transpose=False):
        """(rowptr, col, val) of G (or G^T) as numpy arrays (val as float64)."""
        inf = self.info()
        n, nnz = inf["n"], inf["nnz_G"]
        rp = np.zeros(n + 1, dtype=np.int32)
        ci = np.zeros(max(nnz, 1), dtype=np.int32)
        va = np.zeros(max(nnz, 1), dtype=np.float64)
        fn = load().afsai_export_Gt if transpose else load().afsai_export_G
        _check(fn(self._h, rp.ctypes.data_as(ctypes.c_void_p), ci.ctypes.data_as(ctypes.c_void_p),
                  va.ctypes.data_as(ctypes.c_void_p)))
        return rp, ci[:nnz], va[:nnz]

    def rows(self):
        """(psi, steps) per row as numpy arrays."""
        n = self.info()["n"]
        psi = np.zeros(n, dtype=np.float64)
        steps = np.zeros(n, dtype=np.int32)
        _check(load().afsai_export_rows(self._h, psi.ctypes.data_as(ctypes.c_void_p),
                                        steps.ctypes.data_as(ctypes.c_void_p)))
        return psi, steps

    def close(self):
        if self._h:
            load().afsai_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def afsai_setup(A: DeviceCSR, prm: Params, stream=None) -> Precond:
    lib = load()
    h = ctypes.c_void_p()
    csr = A.c()
    _check(lib.afsai_setup(ctypes.byref(csr), ctypes.byref(prm), _stream(stream), ctypes.byref(h)))
    return Precond(h)


def afsai_apply(M: Precond, r, z, stream=None):
    n = M.n
    _check(load().afsai_apply(M.handle, _vec(r, n, "r"), _vec(z, n, "z"), _stream(stream)))


def afsai_apply_static(M: Precond, r, z, stream=None):
    """z = G^T (G r) without any device allocation (n <= 2^20)."""
    n = M.n
    _check(load().afsai_apply_static(M.handle, _vec(r, n, "r"), _vec(z, n, "z"), _stream(stream)))


def afsai_spmv(A: DeviceCSR, x, y, stream=None):
    csr = A.c()
    _check(load().afsai_spmv(ctypes.byref(csr), _vec(x, A.n, "x"), _vec(y, A.n, "y"), _stream(stream)))


def pcg_solve(A: DeviceCSR, M, b, x, rtol=1e-8, maxit=10000, stream=None, raise_on_noconv=True) -> dict:
    inf = PcgInfo()
    csr = A.c()
    st = load().pcg_solve(ctypes.byref(csr), M.handle if M is not None else None, _vec(b, A.n, "b"),
                          _vec(x, A.n, "x"), float(rtol), int(maxit), _stream(stream), ctypes.byref(inf))
    if st != OK and not (st == ENOCONV and not raise_on_noconv):
        _check(st)
    out = _as_dict(inf)
    out["status"] = st
    return out


def afsai_batch_solve(As, prm: Params, bs, xs, rtol=1e-8, maxit=10000, stream=None, raise_on_noconv=True):
    """Batched aFSAI-PCG over independent systems (lists of DeviceCSR and
    device vectors; xs hold the initial guesses and receive the solutions).
    Returns (list of per-system info dicts, batch info dict)."""
    n = len(As)
    csrs = (Csr * n)(*[A.c() for A in As])
    bp = (ctypes.c_void_p * n)(*[_vec(b, A.n, f"b[{k}]").value for k, (A, b) in enumerate(zip(As, bs))])
    xp = (ctypes.c_void_p * n)(*[_vec(x, A.n, f"x[{k}]").value for k, (A, x) in enumerate(zip(As, xs))])
    infos = (PcgInfo * n)()
    binfo = BatchInfo()
    st = load().afsai_batch_solve(n, ctypes.cast(csrs, ctypes.c_void_p), ctypes.byref(prm),
                                  ctypes.cast(bp, ctypes.c_void_p), ctypes.cast(xp, ctypes.c_void_p), float(rtol),
                                  int(maxit), _stream(stream), ctypes.cast(infos, ctypes.c_void_p), ctypes.byref(binfo))
    if st != OK and not (st == ENOCONV and not raise_on_noconv):
        _check(st)
    return [_as_dict(i) for i in infos], dict(_as_dict(binfo), status=st)


class Server:
    """Solve server (continuous batching) on the current device."""

    def __init__(self, mem_budget_bytes, max_slots, prm: Params, maxit=10000, iters_per_step=4):
        h = ctypes.c_void_p()
        _check(load().serve_create(int(mem_budget_bytes), int(max_slots), ctypes.byref(prm), int(maxit),
                                   int(iters_per_step), ctypes.byref(h)))
        self._h = h
        self._n = {}

    def register(self, A) -> int:
        """A: host CSR (n, rowptr, col, val numpy arrays) or DeviceCSR."""
        if isinstance(A, DeviceCSR):
            csr = A.c()
        else:
            self._keep = getattr(self, "_keep", [])
            arrs = (np.ascontiguousarray(A.rowptr, dtype=np.int32), np.ascontiguousarray(A.col, dtype=np.int32),
                    np.ascontiguousarray(A.val, dtype=np.float64))
            self._keep.append(arrs)
            csr = Csr(A.n, int(arrs[1].size), arrs[0].ctypes.data, arrs[1].ctypes.data, arrs[2].ctypes.data)
        mid = ctypes.c_int32()
        _check(load().serve_register(self._h, ctypes.byref(csr), ctypes.byref(mid)))
        self._n[mid.value] = A.n
        return mid.value

    def submit(self, matrix_id, b: np.ndarray, rtol=1e-8) -> int:
        """b: (n,) or (nrhs, n) float64 host array."""
        b = np.ascontiguousarray(b, dtype=np.float64)
        nrhs = 1 if b.ndim == 1 else b.shape[0]
        t = ctypes.c_int64()
        _check(load().serve_submit(self._h, int(matrix_id), b.ctypes.data_as(ctypes.c_void_p), nrhs, float(rtol),
                                   ctypes.byref(t)))
        return t.value, matrix_id, nrhs

    def poll(self, ticket):
        """None while running, else (x (nrhs, n), [info dicts], result dict)."""
        t, mid, nrhs = ticket
        n = self._n[mid]
        x = np.zeros((nrhs, n))
        infos = (PcgInfo * nrhs)()
        res = ServeResult()
        st = load().serve_poll(self._h, t, x.ctypes.data_as(ctypes.c_void_p), ctypes.cast(infos, ctypes.c_void_p),
                               ctypes.byref(res))
        if st == EAGAIN:
            return None
        if st not in (OK, ENOCONV):
            _check(st)
        return x, [_as_dict(i) for i in infos], _as_dict(res)

    def wait(self, ticket, timeout_s=120.0, sleep_s=0.0005):
        import time

        t0 = time.time()
        while True:
            r = self.poll(ticket)
            if r is not None:
                return r
            if time.time() - t0 > timeout_s:
                raise TimeoutError("request did not finish")
            time.sleep(sleep_s)

    def stats(self):
        s = ServeStats()
        _check(load().serve_get_stats(self._h, ctypes.byref(s)))
        return _as_dict(s)

    def close(self):
        if self._h:
            load().serve_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def afsai_solve_host(A, prm: Params, b: np.ndarray, x: np.ndarray, rtol=1e-8, maxit=10000, stream=None):
    """End-to-end solve from host arrays (A: object with n, rowptr, col, val
    numpy arrays; b, x: float64 numpy arrays, x receives the solution)."""
    rp = np.ascontiguousarray(A.rowptr, dtype=np.int32)
    ci = np.ascontiguousarray(A.col, dtype=np.int32)
    va = np.ascontiguousarray(A.val, dtype=np.float64)
    assert b.dtype == np.float64 and x.dtype == np.float64 and b.flags.c_contiguous and x.flags.c_contiguous
    csr = Csr(A.n, int(ci.size), rp.ctypes.data, ci.ctypes.data, va.ctypes.data)
    sinf, pinf = Info(), PcgInfo()
    st = load().afsai_solve_host(ctypes.byref(csr), ctypes.byref(prm), b.ctypes.data_as(ctypes.c_void_p),
                                 x.ctypes.data_as(ctypes.c_void_p), float(rtol), int(maxit), _stream(stream),
                                 ctypes.byref(sinf), ctypes.byref(pinf))
    if st not in (OK, ENOCONV):
        _check(st)
    return _as_dict(sinf), _as_dict(pinf)
