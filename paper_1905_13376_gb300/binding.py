"""Thin ctypes binding of libmwj (include/mwj.h).

The functions ``mwj_*`` mirror the C ABI one to one (argument marshalling
only).  ``Context`` adds convenience: it takes int32 CUDA tensors, allocates
outputs and the workspace with torch, and raises ``MwjError`` on a non-OK
status.  Every step of every join runs in the library's CUDA kernels; there is
no CPU path, and loading fails loudly when the library cannot be built or
loaded.
"""
from __future__ import annotations

import ctypes
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))

MWJ_OK = 0
MWJ_ERR_INVALID_ARG = 1
MWJ_ERR_DOMAIN = 2
MWJ_ERR_CAPACITY = 3
MWJ_ERR_WORKSPACE = 4
MWJ_ERR_CUDA = 5
MWJ_ERR_TIMEOUT = 6
MWJ_ERR_CHECK = 7
MWJ_ERR_UNIMPLEMENTED = 8

MWJ_COUNT = 0
MWJ_COUNT_GROUP_BY_A = 1
MWJ_MATERIALIZE = 2

MWJ_LINEAR = 0
MWJ_CYCLIC = 1
MWJ_STAR = 4

MODES = {"count": MWJ_COUNT, "group_by_a": MWJ_COUNT_GROUP_BY_A, "rows": MWJ_MATERIALIZE}


class mwj_rel(ctypes.Structure):
    _fields_ = [("x", ctypes.c_void_p), ("y", ctypes.c_void_p), ("n", ctypes.c_int64)]


class mwj_shares(ctypes.Structure):
    _fields_ = [("s", ctypes.c_int32 * 3)]


class mwj_out(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int), ("total", ctypes.c_void_p),
                ("group_counts", ctypes.c_void_p), ("a_domain", ctypes.c_int32),
                ("rows", ctypes.c_void_p), ("capacity", ctypes.c_int64),
                ("n_rows", ctypes.c_void_p)]


class mwj_query(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("R", mwj_rel), ("S", mwj_rel), ("T", mwj_rel),
                ("shares", mwj_shares)]


class mwj_batch_rule(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("size_log2", ctypes.c_int32), ("tuples_per_bucket", ctypes.c_int32),
                ("table_factor", ctypes.c_int32), ("fit_pct", ctypes.c_int32)]


class mwj_config(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int32), ("seed", ctypes.c_uint32),
                ("smem_bytes", ctypes.c_int32), ("load_pct", ctypes.c_int32),
                ("spin_limit", ctypes.c_int64)]


class MwjError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"mwj status {status}: {msg}")
        self.status = status


_lib = None
_lock = threading.Lock()

# exported symbols and their signatures: (restype, argtypes)
_P = ctypes.c_void_p
_SIGS = {
    "mwj_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.POINTER(mwj_config)]),
    "mwj_destroy": (ctypes.c_int, [_P]),
    "mwj_workspace_size": (ctypes.c_int, [_P, ctypes.c_int, mwj_rel, mwj_rel, mwj_rel,
                                          ctypes.POINTER(mwj_shares), ctypes.c_int,
                                          ctypes.POINTER(ctypes.c_size_t)]),
    "mwj_join3_linear": (ctypes.c_int, [_P, mwj_rel, mwj_rel, mwj_rel, ctypes.POINTER(mwj_shares),
                                        ctypes.POINTER(mwj_out), _P, ctypes.c_size_t, _P]),
    "mwj_join3_cyclic": (ctypes.c_int, [_P, mwj_rel, mwj_rel, mwj_rel, ctypes.POINTER(mwj_shares),
                                        ctypes.POINTER(mwj_out), _P, ctypes.c_size_t, _P]),
    "mwj_join3_star": (ctypes.c_int, [_P, mwj_rel, mwj_rel, mwj_rel, ctypes.POINTER(mwj_shares),
                                      ctypes.POINTER(mwj_out), _P, ctypes.c_size_t, _P]),
    "mwj_join4_workspace_size": (ctypes.c_int, [_P, mwj_rel, mwj_rel, mwj_rel, mwj_rel,
                                                ctypes.POINTER(mwj_shares), ctypes.c_int,
                                                ctypes.POINTER(ctypes.c_size_t)]),
    "mwj_join4_linear": (ctypes.c_int, [_P, mwj_rel, mwj_rel, mwj_rel, mwj_rel, ctypes.POINTER(mwj_shares),
                                        ctypes.POINTER(mwj_out), _P, ctypes.c_size_t, _P]),
    "mwj_fm_workspace_size": (ctypes.c_int, [_P, mwj_rel, mwj_rel, mwj_rel, ctypes.POINTER(mwj_shares),
                                             ctypes.POINTER(ctypes.c_size_t)]),
    "mwj_fm_linear": (ctypes.c_int, [_P, mwj_rel, mwj_rel, mwj_rel, ctypes.POINTER(mwj_shares), ctypes.c_int32,
                                     _P, _P, _P, ctypes.c_size_t, _P]),
    "mwj_cascade_join": (ctypes.c_int, [_P, ctypes.c_int, mwj_rel, mwj_rel, mwj_rel,
                                        ctypes.POINTER(mwj_out), _P, ctypes.c_size_t, _P]),
    "mwj_stream_status": (ctypes.c_int, [_P, _P]),
    "mwj_check_bounded_wait": (ctypes.c_int, [_P, ctypes.c_int64, _P]),
    "mwj_batch_set_rules": (ctypes.c_int, [_P, ctypes.POINTER(mwj_batch_rule), ctypes.c_int32]),
    "mwj_batch_set_launch": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int32]),
    "mwj_join3_linear_noalloc": (ctypes.c_int, [mwj_rel, mwj_rel, mwj_rel,
                                                ctypes.POINTER(mwj_shares),
                                                ctypes.POINTER(mwj_out), _P]),
    "mwj_plan_shares_alt": (ctypes.c_int, [_P, ctypes.c_int, mwj_rel, mwj_rel, mwj_rel,
                                           ctypes.POINTER(mwj_shares)]),
    "mwj_plan_shares": (ctypes.c_int, [_P, ctypes.c_int, mwj_rel, mwj_rel, mwj_rel, ctypes.c_int,
                                       ctypes.POINTER(mwj_shares), _P]),
    "mwj_last_error": (ctypes.c_char_p, [_P]),
    "mwj_set_profiling": (ctypes.c_int, [_P, ctypes.c_int]),
    "mwj_launch_count": (ctypes.c_longlong, [_P]),
    "mwj_get_phase_times": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_char_p),
                                           ctypes.POINTER(ctypes.c_double),
                                           ctypes.POINTER(ctypes.c_longlong), ctypes.c_int]),
    "mwj_reset_phase_times": (ctypes.c_int, [_P]),
    "mwj_version": (ctypes.c_char_p, []),
    "mwj_features_workspace_size": (ctypes.c_size_t, []),
    "mwj_features": (ctypes.c_int, [_P, ctypes.c_int, mwj_rel, mwj_rel, mwj_rel,
                                    ctypes.POINTER(ctypes.c_float), _P, ctypes.c_size_t, _P]),
    "mwj_cost_model": (ctypes.c_int, [ctypes.POINTER(ctypes.c_float), ctypes.c_double,
                                      ctypes.POINTER(ctypes.c_double)]),
    "mwj_mlp_num_params": (ctypes.c_size_t, []),
    "mwj_mlp_create": (ctypes.c_int, [_P, ctypes.POINTER(_P)]),
    "mwj_mlp_destroy": (ctypes.c_int, [_P]),
    "mwj_mlp_set_params": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_float)]),
    "mwj_mlp_get_params": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_float)]),
    "mwj_mlp_forward": (ctypes.c_int, [_P, _P, ctypes.c_int32, _P, _P]),
    "mwj_mlp_backward": (ctypes.c_int, [_P, _P, _P, _P, ctypes.c_int32, ctypes.c_float, _P, _P,
                                        _P]),
    "mwj_mlp_adam": (ctypes.c_int, [_P, _P, ctypes.c_float, ctypes.c_int32, _P]),
    "mwj_batch_create": (ctypes.c_int, [_P, ctypes.POINTER(mwj_query), ctypes.c_int32,
                                        ctypes.POINTER(_P)]),
    "mwj_batch_workspace_size": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_size_t)]),
    "mwj_batch_shares": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.POINTER(mwj_shares)]),
    "mwj_batch_launch": (ctypes.c_int, [_P, _P, _P, ctypes.c_size_t, _P]),
    "mwj_batch_destroy": (ctypes.c_int, [_P]),
}


def lib_path() -> str:
    return os.path.join(_HERE, "_lib", "libmwj.so")


def load():
    """Load libmwj.so, building it first if it is missing or stale."""
    global _lib
    with _lock:
        if _lib is None:
            from . import build as _build
            path = _build.build()
            lib = ctypes.CDLL(path)
            for name, (res, args) in _SIGS.items():
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _lib = lib
    return _lib


def __getattr__(name):
    # mwj_* functions resolve to the library's exports
    if name in _SIGS:
        return getattr(load(), name)
    raise AttributeError(name)


# ---------------------------------------------------------------------------
# convenience layer over torch tensors
# ---------------------------------------------------------------------------

def _rel(pair):
    import torch
    x, y = pair
    assert x.dtype == torch.int32 and y.dtype == torch.int32, "relations are int32 column pairs"
    assert x.is_cuda and y.is_cuda and x.is_contiguous() and y.is_contiguous()
    assert x.numel() == y.numel()
    return mwj_rel(x.data_ptr(), y.data_ptr(), x.numel())


def _shares(s):
    if s is None:
        return None
    v = list(s) + [1] * (3 - len(s))
    sh = mwj_shares()
    for i in range(3):
        sh.s[i] = int(v[i])
    return ctypes.byref(sh)


class Context:
    """One library context on one CUDA device."""

    def __init__(self, device: int | None = None, seed: int = 0, load_pct: int = 0,
                 spin_limit: int = 0):
        import torch
        self.lib = load()
        if device is None:
            device = torch.cuda.current_device()
        self.device = torch.device("cuda", device)
        cfg = mwj_config(device, seed & 0xFFFFFFFF, 0, load_pct, spin_limit)
        h = _P()
        st = self.lib.mwj_create(ctypes.byref(h), ctypes.byref(cfg))
        if st != MWJ_OK:
            raise MwjError(st, "mwj_create failed")
        self.h = h
        self._ws = None

    def close(self):
        if getattr(self, "h", None):
            self.lib.mwj_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st):
        if st != MWJ_OK:
            raise MwjError(st, self.lib.mwj_last_error(self.h).decode())

    def set_profiling(self, on: bool = True):
        self._check(self.lib.mwj_set_profiling(self.h, 1 if on else 0))

    def batch_set_rules(self, rules):
        """Planning rules of batches created afterwards: an iterable of
        (kind, size_log2, tuples_per_bucket, table_factor, fit_pct); empty
        restores the library's rules."""
        rules = list(rules)
        arr = (mwj_batch_rule * max(1, len(rules)))()
        for i, r in enumerate(rules):
            arr[i] = mwj_batch_rule(*[int(v) for v in r])
        self._check(self.lib.mwj_batch_set_rules(self.h, arr, len(rules)))

    def batch_set_launch(self, prep_ctas_per_sm: int = 0, join_ctas_per_sm: int = 0):
        self._check(self.lib.mwj_batch_set_launch(self.h, int(prep_ctas_per_sm), int(join_ctas_per_sm)))

    def check_bounded_wait(self, polls: int, stream=None):
        """Run the failure-detection check (a bounded wait on a barrier phase
        that never completes); returns the status mwj_stream_status reports
        afterwards (MWJ_ERR_TIMEOUT when the wait gave up)."""
        self._check(self.lib.mwj_check_bounded_wait(self.h, int(polls), self._stream(stream)))
        return int(self.lib.mwj_stream_status(self.h, self._stream(stream)))

    def launch_count(self) -> int:
        return int(self.lib.mwj_launch_count(self.h))

    def phase_times(self) -> dict:
        """{kernel name: (total ms, launches)} since the last reset."""
        n = self.lib.mwj_get_phase_times(self.h, None, None, None, 0)
        names = (ctypes.c_char_p * max(n, 1))()
        ms = (ctypes.c_double * max(n, 1))()
        cnt = (ctypes.c_longlong * max(n, 1))()
        n = self.lib.mwj_get_phase_times(self.h, names, ms, cnt, n)
        return {names[i].decode(): (ms[i], cnt[i]) for i in range(n)}

    def reset_phase_times(self):
        self._check(self.lib.mwj_reset_phase_times(self.h))

    def workspace(self, nbytes: int):
        import torch
        if self._ws is None or self._ws.numel() < nbytes:
            self._ws = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=self.device)
        return self._ws

    def workspace_size(self, kind, R, S, T, shares=None, mode=MWJ_COUNT) -> int:
        n = ctypes.c_size_t()
        self._check(self.lib.mwj_workspace_size(self.h, kind, _rel(R), _rel(S), _rel(T),
                                                _shares(shares), mode, ctypes.byref(n)))
        return n.value

    def plan_shares(self, kind, R, S, T, mode=MWJ_COUNT, stream=None):
        sh = mwj_shares()
        self._check(self.lib.mwj_plan_shares(self.h, kind, _rel(R), _rel(S), _rel(T), mode,
                                             ctypes.byref(sh), self._stream(stream)))
        return tuple(sh.s)

    def plan_shares_alt(self, kind, R, S, T):
        """The alternative share vector (linear: H(B) buckets in shared memory;
        cyclic: the cube tiling of Section 5.2)."""
        sh = mwj_shares()
        self._check(self.lib.mwj_plan_shares_alt(self.h, kind, _rel(R), _rel(S), _rel(T), ctypes.byref(sh)))
        return tuple(sh.s)

    def _stream(self, stream):
        import torch
        s = stream if stream is not None else torch.cuda.current_stream(self.device)
        return ctypes.c_void_p(s.cuda_stream)

    def _outputs(self, mode, a_domain, capacity, arity, reuse=None):
        import torch
        dev = self.device
        if reuse is not None:   # the output tensors of an earlier call with the same mode and sizes
            o = mwj_out()
            o.mode = mode
            o.total = reuse["total"].data_ptr()
            if mode == MWJ_COUNT_GROUP_BY_A:
                if reuse["counts"].numel() != int(a_domain):
                    raise ValueError("out: group_counts of another a_domain")
                o.group_counts = reuse["counts"].data_ptr()
                o.a_domain = int(a_domain)
            if mode == MWJ_MATERIALIZE:
                raise ValueError("out: reuse is for the aggregate modes")
            return o, reuse
        # the library writes the total (and the exact row count) itself
        total = torch.empty(1, dtype=torch.int64, device=dev)
        o = mwj_out()
        o.mode = mode
        o.total = total.data_ptr()
        res = {"total": total}
        if mode == MWJ_COUNT_GROUP_BY_A:
            cnt = torch.empty(int(a_domain), dtype=torch.int64, device=dev)
            o.group_counts = cnt.data_ptr()
            o.a_domain = int(a_domain)
            res["counts"] = cnt
        if mode == MWJ_MATERIALIZE:
            rows = torch.empty((max(int(capacity), 1), arity), dtype=torch.int32, device=dev)
            n_rows = torch.zeros(1, dtype=torch.int64, device=dev)
            o.rows = rows.data_ptr()
            o.capacity = int(capacity)
            o.n_rows = n_rows.data_ptr()
            res["rows"] = rows
            res["n_rows"] = n_rows
        return o, res

    def _run(self, fn, kind_ws, R, S, T, mode, shares, a_domain, capacity, arity, stream, sync,
             extra=(), out=None):
        if isinstance(mode, str):
            mode = MODES[mode]
        o, res = self._outputs(mode, a_domain, capacity, arity, out)
        with_shares = kind_ws in (MWJ_LINEAR, MWJ_CYCLIC, MWJ_STAR)
        nb = self.workspace_size(kind_ws, R, S, T, shares if with_shares else None, mode)
        ws = self.workspace(nb)
        args = (self.h,) + tuple(extra) + (_rel(R), _rel(S), _rel(T))
        if with_shares:
            args = args + (_shares(shares),)
        st = fn(*args, ctypes.byref(o), ctypes.c_void_p(ws.data_ptr()), ws.numel(),
                self._stream(stream))
        self._check(st)
        if sync:
            self._check(self.lib.mwj_stream_status(self.h, self._stream(stream)))
            if mode == MWJ_MATERIALIZE:
                n = int(res["n_rows"].item())
                res["rows"] = res["rows"][:n]
        return res

    def join3_linear(self, R, S, T, mode="count", shares=None, a_domain=None, capacity=0,
                     stream=None, sync=True, out=None):
        """Linear 3-way join R(A,B) S(B,C) T(C,D).  shares = (H(B) buckets,
        g(C) buckets[, log2 on-chip table slots]); None: one bucket per side
        for "count" and "group_by_a" (T's and S's tables in L2), H(B)
        buckets from |R| for "rows".  out: the result dict of an earlier
        aggregate call with the same mode and a_domain, whose tensors are
        written again instead of new ones."""
        return self._run(self.lib.mwj_join3_linear, MWJ_LINEAR, R, S, T, mode, shares, a_domain,
                         capacity, 4, stream, sync, out=out)

    def join3_star(self, R, S, T, mode="count", shares=None, a_domain=None, capacity=0,
                   stream=None, sync=True):
        """Star 3-way join: small R(A,B) and T(C,D) held on chip, S(B,C)
        streamed once.  shares = (h(B) buckets of R, g(C) buckets of T), 0 or
        None for the default."""
        return self._run(self.lib.mwj_join3_star, MWJ_STAR, R, S, T, mode, shares, a_domain,
                         capacity, 4, stream, sync)

    def join4_linear(self, R, S, T, U, mode="count", shares=None, a_domain=None, stream=None,
                     sync=True):
        """Chain of four relations R(A,B) S(B,C) T(C,D) U(D,E): COUNT or
        COUNT GROUP BY A."""
        if isinstance(mode, str):
            mode = MODES[mode]
        o, res = self._outputs(mode, a_domain, 0, 4)
        nb = ctypes.c_size_t(0)
        self._check(self.lib.mwj_join4_workspace_size(self.h, _rel(R), _rel(S), _rel(T), _rel(U),
                                                      _shares(shares), int(mode), ctypes.byref(nb)))
        ws = self.workspace(nb.value)
        self._check(self.lib.mwj_join4_linear(self.h, _rel(R), _rel(S), _rel(T), _rel(U), _shares(shares),
                                              ctypes.byref(o), ctypes.c_void_p(ws.data_ptr()), ws.numel(),
                                              self._stream(stream)))
        if sync:
            self._check(self.lib.mwj_stream_status(self.h, self._stream(stream)))
        return res

    def fm_linear(self, R, S, T, a_domain, shares=None, estimates=True, stream=None, sync=True):
        """Flajolet-Martin (PCSA) sketches of the distinct D reachable from
        every A through R(A,B) S(B,C) T(C,D): {"sketches": int32
        (a_domain, 16) holding the uint32 bitmaps, "estimates": float32
        (a_domain,) or None}."""
        import torch
        sk = torch.empty((int(a_domain), 16), dtype=torch.int32, device=self.device)
        est = torch.empty(int(a_domain), dtype=torch.float32, device=self.device) if estimates else None
        nb = ctypes.c_size_t(0)
        self._check(self.lib.mwj_fm_workspace_size(self.h, _rel(R), _rel(S), _rel(T), _shares(shares),
                                                   ctypes.byref(nb)))
        ws = self.workspace(nb.value)
        self._check(self.lib.mwj_fm_linear(self.h, _rel(R), _rel(S), _rel(T), _shares(shares), int(a_domain),
                                           ctypes.c_void_p(sk.data_ptr()),
                                           ctypes.c_void_p(est.data_ptr()) if est is not None else None,
                                           ctypes.c_void_p(ws.data_ptr()), ws.numel(), self._stream(stream)))
        if sync:
            self._check(self.lib.mwj_stream_status(self.h, self._stream(stream)))
        return {"sketches": sk, "estimates": est}

    def join3_cyclic(self, R, S, T, mode="count", shares=None, a_domain=None, capacity=0,
                     stream=None, sync=True, out=None):
        """Cyclic 3-way join R(A,B) S(B,C) T(C,A), T given as (c, a) columns.
        shares = (H(A), G(B), F(C)) bucket counts; None: the library's cube
        shares.  out: as for join3_linear."""
        return self._run(self.lib.mwj_join3_cyclic, MWJ_CYCLIC, R, S, T, mode, shares, a_domain,
                         capacity, 3, stream, sync, out=out)

    def cascade_join(self, kind, R, S, T, mode="count", a_domain=None, capacity=0, stream=None,
                     sync=True, workspace_bytes=None):
        if isinstance(mode, str):
            mode = MODES[mode]
        o, res = self._outputs(mode, a_domain, capacity, 4 if kind == MWJ_LINEAR else 3)
        nb = self.workspace_size(2 + kind, R, S, T, None, mode)
        if workspace_bytes is not None:
            nb = max(nb, int(workspace_bytes))
        ws = self.workspace(nb)
        st = self.lib.mwj_cascade_join(self.h, kind, _rel(R), _rel(S), _rel(T), ctypes.byref(o),
                                       ctypes.c_void_p(ws.data_ptr()), ws.numel(),
                                       self._stream(stream))
        self._check(st)
        if sync:
            self._check(self.lib.mwj_stream_status(self.h, self._stream(stream)))
            if mode == MWJ_MATERIALIZE:
                res["rows"] = res["rows"][:int(res["n_rows"].item())]
        return res


class Batch:
    """A planned batch of independent joins (COUNT(*) per query) on one context.

    queries: list of (kind, R, S, T[, shares]) with device int32 column pairs.
    """

    def __init__(self, ctx: "Context", queries):
        import torch
        self.ctx = ctx
        self.lib = ctx.lib
        self._keep = [q[1:4] for q in queries]   # the relations must outlive the batch
        arr = (mwj_query * max(1, len(queries)))()
        for i, q in enumerate(queries):
            kind, R, S, T = q[:4]
            sh = q[4] if len(q) > 4 and q[4] is not None else (0, 0, 0)
            arr[i].kind = kind
            arr[i].R, arr[i].S, arr[i].T = _rel(R), _rel(S), _rel(T)
            for k in range(3):
                arr[i].shares.s[k] = int(sh[k])
        h = _P()
        ctx._check(self.lib.mwj_batch_create(ctx.h, arr, len(queries), ctypes.byref(h)))
        self.h = h
        self.n = len(queries)
        n = ctypes.c_size_t()
        ctx._check(self.lib.mwj_batch_workspace_size(self.h, ctypes.byref(n)))
        self.ws = torch.empty(max(n.value, 256), dtype=torch.uint8, device=ctx.device)
        self.counts = torch.zeros(max(self.n, 1), dtype=torch.int64, device=ctx.device)

    def shares(self, q):
        sh = mwj_shares()
        self.ctx._check(self.lib.mwj_batch_shares(self.h, q, ctypes.byref(sh)))
        return tuple(sh.s)

    def launch(self, stream=None):
        """Enqueue the batch; returns the device counts tensor (no sync)."""
        st = self.lib.mwj_batch_launch(self.h, ctypes.c_void_p(self.counts.data_ptr()),
                                       ctypes.c_void_p(self.ws.data_ptr()), self.ws.numel(),
                                       self.ctx._stream(stream))
        self.ctx._check(st)
        return self.counts[: self.n]

    def close(self):
        if getattr(self, "h", None):
            self.lib.mwj_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def cost_model(features, hbm_gbs: float = 6792.1):
    """The library's cost model on a host feature vector (24 floats)."""
    lib = load()
    f = (ctypes.c_float * 24)(*[float(v) for v in features])
    out = (ctypes.c_double * 3)()
    st = lib.mwj_cost_model(f, float(hbm_gbs), out)
    if st != MWJ_OK:
        raise MwjError(st, "mwj_cost_model")
    return list(out)


class MLP:
    """The planner network on the GPU (BF16 weights/activations, FP32 accumulate)."""

    def __init__(self, ctx: "Context", params=None):
        import numpy as np
        import torch
        self.ctx, self.lib = ctx, ctx.lib
        h = _P()
        ctx._check(self.lib.mwj_mlp_create(ctx.h, ctypes.byref(h)))
        self.h = h
        self.n = int(self.lib.mwj_mlp_num_params())
        self.grads = torch.zeros(self.n, dtype=torch.float32, device=ctx.device)
        self.loss = torch.zeros(1, dtype=torch.float32, device=ctx.device)
        self.step = 0
        if params is not None:
            self.set_params(np.asarray(params, dtype=np.float32))

    def set_params(self, p):
        import numpy as np
        p = np.ascontiguousarray(p, dtype=np.float32)
        assert p.size == self.n
        self.ctx._check(self.lib.mwj_mlp_set_params(self.h, p.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))
        self.step = 0

    def get_params(self):
        import numpy as np
        p = np.zeros(self.n, dtype=np.float32)
        self.ctx._check(self.lib.mwj_mlp_get_params(self.h, p.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))
        return p

    def forward(self, X):
        import torch
        X = X.contiguous().float()
        Y = torch.empty((X.shape[0], 3), dtype=torch.float32, device=X.device)
        self.ctx._check(self.lib.mwj_mlp_forward(self.h, ctypes.c_void_p(X.data_ptr()), X.shape[0],
                                                 ctypes.c_void_p(Y.data_ptr()),
                                                 self.ctx._stream(None)))
        return Y

    def backward(self, X, T, M):
        X, T, M = (t.contiguous().float() for t in (X, T, M))
        cnt = float(max(1.0, float(M.sum().item())))
        self.ctx._check(self.lib.mwj_mlp_backward(
            self.h, ctypes.c_void_p(X.data_ptr()), ctypes.c_void_p(T.data_ptr()),
            ctypes.c_void_p(M.data_ptr()), X.shape[0], 1.0 / cnt,
            ctypes.c_void_p(self.grads.data_ptr()), ctypes.c_void_p(self.loss.data_ptr()),
            self.ctx._stream(None)))
        return self.grads, self.loss

    def adam(self, lr):
        self.step += 1
        self.ctx._check(self.lib.mwj_mlp_adam(self.h, ctypes.c_void_p(self.grads.data_ptr()),
                                              float(lr), self.step, self.ctx._stream(None)))

    def close(self):
        if getattr(self, "h", None):
            self.lib.mwj_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
