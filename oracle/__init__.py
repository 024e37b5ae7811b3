"""CPU oracle for the 3-way hash joins -- TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library
and its Python binding) never imports, links or calls it, and it shares no
code with that path.

``linear`` and ``cyclic`` evaluate the plain relational definitions of
Section 3 (linear R(A,B) S(B,C) T(C,D); cyclic R(A,B) S(B,C) T(C,A)) under
bag semantics with a single-threaded C hash join (``oracle.c``);
``linear4`` the chain one relation longer, R(A,B) S(B,C) T(C,D) U(D,E)
(Section 7's additional hash levels), for COUNT and GROUP BY A.  Counts are
unsigned 64-bit with wraparound and are returned as ``int64`` views of the
same bits, the width the CUDA path reports.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIBDIR = os.path.join(_HERE, "_lib")
_LIB = os.path.join(_LIBDIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

COUNT, GROUP_BY_A, MATERIALIZE = 0, 1, 2


class OracleError(RuntimeError):
    pass


def build(force: bool = False) -> str:
    """Compile oracle.c into _lib/liboracle.so with the host C compiler."""
    src = os.path.join(_HERE, "oracle.c")
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(src)):
        return _LIB
    os.makedirs(_LIBDIR, exist_ok=True)
    tmp = _LIB + f".{os.getpid()}.tmp"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", src, "-o", tmp])
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            P = ctypes.c_void_p
            I64 = ctypes.c_int64
            sig = [P, P, I64, P, P, I64, P, P, I64, ctypes.c_int, ctypes.c_int32,
                   P, P, P, I64, P]
            for name in ("oracle_linear", "oracle_cyclic"):
                f = getattr(lib, name)
                f.argtypes = sig
                f.restype = ctypes.c_int
            lib.oracle_linear4.argtypes = [P, P, I64, P, P, I64, P, P, I64, P, P, I64, ctypes.c_int,
                                           ctypes.c_int32, P, P]
            lib.oracle_linear4.restype = ctypes.c_int
            lib.oracle_binary_count.argtypes = [P, I64, P, I64, P]
            lib.oracle_binary_count.restype = ctypes.c_int
            _lib = lib
    return _lib


def _col(v):
    a = np.ascontiguousarray(np.asarray(v, dtype=np.int32))
    return a, a.ctypes.data


def _run(fn, R, S, T, mode, a_domain, capacity, arity):
    Rx, pRx = _col(R[0]); Ry, pRy = _col(R[1])
    Sx, pSx = _col(S[0]); Sy, pSy = _col(S[1])
    Tx, pTx = _col(T[0]); Ty, pTy = _col(T[1])
    if not (len(Rx) == len(Ry) and len(Sx) == len(Sy) and len(Tx) == len(Ty)):
        raise ValueError("column lengths differ")
    total = np.zeros(1, dtype=np.uint64)
    cnt = None
    p_cnt = None
    if mode == GROUP_BY_A:
        cnt = np.zeros(int(a_domain), dtype=np.uint64)
        p_cnt = cnt.ctypes.data
    rows = None
    p_rows = None
    n_rows = np.zeros(1, dtype=np.int64)
    cap = 0
    if mode == MATERIALIZE:
        cap = int(capacity)
        rows = np.zeros((max(cap, 1), arity), dtype=np.int32)
        p_rows = rows.ctypes.data
    rc = fn(pRx, pRy, len(Rx), pSx, pSy, len(Sx), pTx, pTy, len(Tx), int(mode),
            int(a_domain or 0), total.ctypes.data, p_cnt, p_rows, cap, n_rows.ctypes.data)
    out = {"rc": rc, "total": int(total.view(np.int64)[0])}
    if cnt is not None:
        out["counts"] = cnt.view(np.int64)
    if mode == MATERIALIZE:
        out["n_rows"] = int(n_rows[0])
        out["rows"] = rows[: min(int(n_rows[0]), cap)]
    return out


def linear(R, S, T, mode=COUNT, a_domain=None, capacity=None, check=True):
    """R(A,B) S(B,C) T(C,D); R, S, T are (x, y) column pairs."""
    if mode == MATERIALIZE and capacity is None:
        capacity = count_linear_rows(R, S, T)
    out = _run(_load().oracle_linear, R, S, T, mode, a_domain, capacity, 4)
    if check and out["rc"] != 0:
        raise OracleError(f"oracle_linear returned {out['rc']}")
    return out


def cyclic(R, S, T, mode=COUNT, a_domain=None, capacity=None, check=True):
    """R(A,B) S(B,C) T(C,A); T's columns are (c, a)."""
    if mode == MATERIALIZE and capacity is None:
        capacity = cyclic(R, S, T, COUNT)["total"]
    out = _run(_load().oracle_cyclic, R, S, T, mode, a_domain, capacity, 3)
    if check and out["rc"] != 0:
        raise OracleError(f"oracle_cyclic returned {out['rc']}")
    return out


def linear4(R, S, T, U, mode=COUNT, a_domain=None, check=True):
    """R(A,B) S(B,C) T(C,D) U(D,E): COUNT or COUNT GROUP BY A."""
    cols = [_col(c) for rel in (R, S, T, U) for c in rel]
    for k in range(0, 8, 2):
        if len(cols[k][0]) != len(cols[k + 1][0]):
            raise ValueError("column lengths differ")
    total = np.zeros(1, dtype=np.uint64)
    cnt = np.zeros(int(a_domain), dtype=np.uint64) if mode == GROUP_BY_A else None
    args = []
    for k in range(0, 8, 2):
        args += [cols[k][1], cols[k + 1][1], len(cols[k][0])]
    rc = _load().oracle_linear4(*args, int(mode), int(a_domain or 0), total.ctypes.data,
                                cnt.ctypes.data if cnt is not None else None)
    if check and rc != 0:
        raise OracleError(f"oracle_linear4 returned {rc}")
    out = {"rc": rc, "total": int(total.view(np.int64)[0])}
    if cnt is not None:
        out["counts"] = cnt.view(np.int64)
    return out


def count_linear_rows(R, S, T) -> int:
    return linear(R, S, T, COUNT)["total"]


def binary_count(R, S) -> int:
    """|R(A,B) join S(B,C)|, the cascade's intermediate size."""
    Rb, pRb = _col(R[1])
    Sb, pSb = _col(S[0])
    c = np.zeros(1, dtype=np.uint64)
    rc = _load().oracle_binary_count(pRb, len(Rb), pSb, len(Sb), c.ctypes.data)
    if rc:
        raise OracleError(f"oracle_binary_count returned {rc}")
    return int(c[0])
