"""Plain FP64 CPU oracle for aFSAI set-up and aFSAI-PCG (test infrastructure).

Only the tests, the package smoke check and the benchmark's CPU-baseline leg
import this package.  The CUDA library neither imports nor links it; the two
share no code.  The arithmetic lives in ``afsai_oracle.c`` (compiled here
with gcc, ``-ffp-contract=off``, OpenMP over independent rows); this module
only builds it and marshals numpy arrays.

Every function cites the part of the paper it follows:
  * ``afsai_setup``   - Section 2 (Eqs. "DensSys", "blocksys", "diagScal",
    "kap2", "grapsi", "exit_crit"); optional locality bound of Section 4
    (stripe graph of G inside the lower part of Ahat^k).
  * ``row_trace``     - the same iteration for one row, step by step.
  * ``spmv``/``apply``- Eq. "prec": M^{-1} r = G^T (G r).
  * ``pcg``           - PCG with M^{-1} = G^T G, stopping at an 8-order
    reduction of the residual (Section 5.2).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "afsai_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libafsai_oracle.so")
_lock = threading.Lock()
_lib = None

OK, EINVAL, ENOMEM, ENOTSPD = 0, 1, 2, 3


def _compile(src: str, out: str) -> None:
    base = ["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-std=c11", "-o", out, src, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)


def build(force: bool = False) -> str:
    """Compile the oracle shared library with gcc (OpenMP if available)."""
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    _compile(_SRC, _LIB + ".tmp")
    os.replace(_LIB + ".tmp", _LIB)
    return _LIB


def build_variant(source_text: str, out_dir: str) -> str:
    """Compile a modified copy of the oracle's C source into out_dir (same
    flags) and return the library path.  For the tests that plant a mistake
    in the oracle and check that its pins catch it; such a library is used
    by a process that sets AFSAI_ORACLE_LIB to its path."""
    src = os.path.join(out_dir, "afsai_oracle_variant.c")
    with open(src, "w") as f:
        f.write(source_text)
    lib = os.path.join(out_dir, "libafsai_oracle_variant.so")
    _compile(src, lib)
    return lib


def source_text() -> str:
    with open(_SRC) as f:
        return f.read()


def _load():
    global _lib
    with _lock:
        if _lib is None:
            path = os.environ.get("AFSAI_ORACLE_LIB") or build()
            lib = ctypes.CDLL(path)
            P = ctypes.c_void_p
            i32, f64 = ctypes.c_int32, ctypes.c_double
            lib.oracle_afsai_rows.argtypes = [i32, P, P, P, i32, i32, f64, i32, i32, i32, i32, i32, i32, P, P, P, P,
                                              P]
            lib.oracle_afsai_rows.restype = ctypes.c_int
            lib.oracle_afsai_row_trace.argtypes = [i32, P, P, P, i32, i32, f64, i32, i32, P, P, P, P, P]
            lib.oracle_afsai_row_trace.restype = ctypes.c_int
            lib.oracle_spmv.argtypes = [i32, P, P, P, P, P]
            lib.oracle_spmv.restype = None
            lib.oracle_apply.argtypes = [i32, P, P, P, P, P, P]
            lib.oracle_apply.restype = None
            lib.oracle_pcg.argtypes = [i32, P, P, P, P, P, P, P, P, f64, i32, P, P, P, P]
            lib.oracle_pcg.restype = ctypes.c_int
            lib.oracle_num_threads.argtypes = []
            lib.oracle_num_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _csr_args(A):
    rp = np.ascontiguousarray(A.rowptr, dtype=np.int32)
    ci = np.ascontiguousarray(A.col, dtype=np.int32)
    va = np.ascontiguousarray(A.val, dtype=np.float64)
    return rp, ci, va


def num_threads() -> int:
    return int(_load().oracle_num_threads())


def set_threads(k: int) -> int:
    """Sets the OpenMP thread count of the oracle's parallel loops (the SpMV
    of PCG, the set-up without an explicit ``nthreads``); returns the count
    that was in effect.  For timing the oracle at one thread and at all
    cores; no effect on any result (rows and SpMV rows are independent)."""
    before = num_threads()
    import ctypes.util

    name = ctypes.util.find_library("gomp") or "libgomp.so.1"
    try:
        ctypes.CDLL(name).omp_set_num_threads(int(k))
    except OSError:
        pass
    return before


class OracleG:
    """Result of the oracle set-up: G in CSR (sorted columns) plus per-row
    psi (final Kaporin row measure) and number of enlargement steps."""

    def __init__(self, n, rowptr, col, val, psi, steps):
        self.n = n
        self.rowptr = rowptr
        self.col = col
        self.val = val
        self.psi = psi
        self.steps = steps

    @property
    def nnz(self):
        return int(self.rowptr[-1])

    def to_scipy(self):
        import scipy.sparse as sp

        return sp.csr_matrix((self.val, self.col, self.rowptr), shape=(self.n, self.n))


def afsai_setup(A, kiter: int, s: int, eps: float, exit_mode: int = 0, rows=None, nthreads: int = 0,
                block_rows: int = 0, block_power: int = 1) -> OracleG:
    """aFSAI set-up (Section 2) for all rows, or for rows [r0, r1) when
    ``rows=(r0, r1)`` (the returned G then holds only those rows, with
    row pointers relative to r0).  ``block_rows > 0`` applies the locality
    bound of the distributed set-up (Section 4): stripes of ``block_rows``
    rows, candidates only from stripes allowed by the stripe adjacency raised
    to ``block_power``."""
    lib = _load()
    rp, ci, va = _csr_args(A)
    r0, r1 = (0, A.n) if rows is None else rows
    nr = r1 - r0
    mcap = 1 + kiter * s
    Gc = np.zeros(max(nr, 1) * mcap, dtype=np.int32)
    Gv = np.zeros(max(nr, 1) * mcap, dtype=np.float64)
    m = np.zeros(max(nr, 1), dtype=np.int32)
    psi = np.zeros(max(nr, 1), dtype=np.float64)
    steps = np.zeros(max(nr, 1), dtype=np.int32)
    st = lib.oracle_afsai_rows(A.n, _p(rp), _p(ci), _p(va), kiter, s, float(eps), exit_mode, int(block_rows),
                               int(block_power), r0, r1, nthreads, _p(Gc), _p(Gv), _p(m), _p(psi), _p(steps))
    if st != OK:
        raise RuntimeError(f"oracle_afsai_rows failed with status {st}")
    m = m[:nr]
    rowptr = np.zeros(nr + 1, dtype=np.int64)
    np.cumsum(m, out=rowptr[1:])
    sel = (np.arange(mcap)[None, :] < m[:, None]).reshape(-1)
    col = Gc[: nr * mcap][sel]
    val = Gv[: nr * mcap][sel]
    return OracleG(nr, rowptr.astype(np.int32), col, val, psi[:nr], steps[:nr])


def row_trace(A, i: int, kiter: int, s: int, eps: float, exit_mode: int = 0):
    """Per-step history of row i: list of (P_k, g_k, psi_k), k = 0..nsteps."""
    lib = _load()
    rp, ci, va = _csr_args(A)
    mcap = 1 + kiter * s
    mk = np.zeros(kiter + 1, dtype=np.int32)
    Pk = np.zeros((kiter + 1) * mcap, dtype=np.int32)
    gk = np.zeros((kiter + 1) * mcap, dtype=np.float64)
    pk = np.zeros(kiter + 1, dtype=np.float64)
    ns = np.zeros(1, dtype=np.int32)
    st = lib.oracle_afsai_row_trace(A.n, _p(rp), _p(ci), _p(va), kiter, s, float(eps), exit_mode, i, _p(mk), _p(Pk),
                                    _p(gk), _p(pk), _p(ns))
    if st != OK:
        raise RuntimeError(f"oracle_afsai_row_trace failed with status {st}")
    out = []
    for k in range(int(ns[0]) + 1):
        m = int(mk[k])
        out.append((Pk[k * mcap:k * mcap + m].copy(), gk[k * mcap:k * mcap + m].copy(), float(pk[k])))
    return out


def spmv(A, x: np.ndarray) -> np.ndarray:
    lib = _load()
    rp, ci, va = _csr_args(A)
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.zeros(A.n, dtype=np.float64)
    lib.oracle_spmv(A.n, _p(rp), _p(ci), _p(va), _p(x), _p(y))
    return y


def apply(G: OracleG, r: np.ndarray) -> np.ndarray:
    """z = G^T (G r) (Eq. "prec")."""
    lib = _load()
    rp, ci, va = _csr_args(G)
    r = np.ascontiguousarray(r, dtype=np.float64)
    t = np.zeros(G.n, dtype=np.float64)
    z = np.zeros(G.n, dtype=np.float64)
    lib.oracle_apply(G.n, _p(rp), _p(ci), _p(va), _p(r), _p(t), _p(z))
    return z


def pcg(A, G: OracleG, b: np.ndarray, rtol: float = 1e-8, maxit: int = 10000, history: bool = False):
    """PCG with M^{-1} = G^T G; returns (x, iters, relres_rec, relres_true),
    plus the recursive relative residual after each iteration (entry 0: the
    initial one) when ``history`` is set."""
    lib = _load()
    rp, ci, va = _csr_args(A)
    grp, gci, gva = _csr_args(G)
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.zeros(A.n, dtype=np.float64)
    it = np.zeros(1, dtype=np.int32)
    rr = np.zeros(1, dtype=np.float64)
    rt = np.zeros(1, dtype=np.float64)
    hist = np.zeros(int(maxit) + 1, dtype=np.float64) if history else None
    st = lib.oracle_pcg(A.n, _p(rp), _p(ci), _p(va), _p(grp), _p(gci), _p(gva), _p(b), _p(x), float(rtol), int(maxit),
                        _p(it), _p(rr), _p(rt), _p(hist) if history else None)
    if st != OK:
        raise RuntimeError(f"oracle_pcg failed with status {st}")
    if history:
        return x, int(it[0]), float(rr[0]), float(rt[0]), hist[: min(int(it[0]), int(maxit)) + 1]
    return x, int(it[0]), float(rr[0]), float(rt[0])
