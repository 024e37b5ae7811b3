"""mwj_join3_linear_noalloc: the linear join for callers that cannot
allocate device memory (it runs on a fixed scratch array inside the library
instead of a context and a workspace).  Checked through the C ABI against
mwj_join3_linear, the entry point that uses a caller workspace, and against
the CPU oracle, on two calls in a row; exact integer equality is the
tolerance of every join test here.

This file is collected last on purpose: if it fails, a run that stops at the
first failure has already run every other test."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1905_13376_gb300 import binding, datagen

from gpu_util import cu

pytestmark = pytest.mark.gpu


def _rel(p):
    return binding.mwj_rel(p[0].data_ptr(), p[1].data_ptr(), p[0].numel())


def _noalloc(lib, R, S, T, mode, a_domain, stream):
    import torch
    total = torch.full((1,), -7, dtype=torch.int64, device="cuda")
    o = binding.mwj_out()
    o.mode = mode
    o.total = total.data_ptr()
    cnt = None
    if mode == binding.MWJ_COUNT_GROUP_BY_A:
        cnt = torch.full((a_domain,), -7, dtype=torch.int64, device="cuda")
        o.group_counts = cnt.data_ptr()
        o.a_domain = a_domain
    st = lib.mwj_join3_linear_noalloc(_rel(R), _rel(S), _rel(T), None, ctypes.byref(o),
                                      ctypes.c_void_p(stream.cuda_stream))
    return st, total, cnt


def test_noalloc_matches_workspace_entry_point_twice():
    import torch
    torch.cuda.set_device(0)
    lib = binding.load()
    ctx = binding.Context(0)
    stream = torch.cuda.current_stream()
    cases = [datagen.linear_uniform(n=50000, ad=5000, bd=700, cd=900, dd=5000, seed=61),
             datagen.linear_uniform(n=1 << 18, ad=1 << 16, bd=4096, cd=4096, dd=1 << 16, seed=62)]
    F = datagen.chung_lu_directed(n_vertices=1 << 13, mean_degree=16.0, seed=63)
    cases.append((F, F, F))
    for R, S, T in cases:
        a_domain = int(max(R[0].max(), 0)) + 1
        dR, dS, dT = cu(R), cu(S), cu(T)
        ref = ctx.join3_linear(dR, dS, dT, "group_by_a", a_domain=a_domain)
        want = oracle.linear(R, S, T, oracle.GROUP_BY_A, a_domain=a_domain)
        assert int(ref["total"].item()) == want["total"]
        assert np.array_equal(ref["counts"].cpu().numpy(), want["counts"])
        for _ in range(2):   # two calls in a row share the scratch array
            st, total, cnt = _noalloc(lib, dR, dS, dT, binding.MWJ_COUNT_GROUP_BY_A, a_domain,
                                      stream)
            assert st == binding.MWJ_OK
            assert int(total.item()) == int(ref["total"].item())
            assert torch.equal(cnt, ref["counts"])
            assert np.array_equal(cnt.cpu().numpy(), want["counts"])
            st, total, _ = _noalloc(lib, dR, dS, dT, binding.MWJ_COUNT, 0, stream)
            assert st == binding.MWJ_OK
            assert int(total.item()) == int(ref["total"].item())
    ctx.close()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    torch.cuda.set_device(0)
    lib = binding.load()
    n = (1 << 18) + 1
    big = cu((np.zeros(n, np.int32), np.zeros(n, np.int32)))
    small = cu((np.zeros(8, np.int32), np.zeros(8, np.int32)))
    st, _, _ = _noalloc(lib, big, small, small, binding.MWJ_COUNT, 0, torch.cuda.current_stream())
    assert st == binding.MWJ_ERR_WORKSPACE
    st, _, _ = _noalloc(lib, small, small, small, binding.MWJ_MATERIALIZE, 0,
                        torch.cuda.current_stream())
    assert st == binding.MWJ_ERR_INVALID_ARG
