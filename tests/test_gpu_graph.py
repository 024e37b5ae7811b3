"""A linear-join call captured into a CUDA graph: the work the call forks onto
the context's side streams (T's table, and with partitions R's partition) is
captured through the event fork/join and replays to the oracle's result, with
the default plan (one bucket per side) and a partitioned one."""
import numpy as np
import pytest

import oracle
from paper_1905_13376_gb300 import binding, datagen

from gpu_util import cu

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("shares", [(64, 1), None])
def test_linear_group_by_in_a_cuda_graph(shares):
    import torch
    torch.cuda.set_device(0)
    ctx = binding.Context(0)
    R, S, T = datagen.linear_uniform(n=1 << 15, ad=1 << 12, bd=1 << 10, cd=1 << 10, dd=1 << 12,
                                     seed=datagen.SEED_BASE + 110)
    dR, dS, dT = cu(R), cu(S), cu(T)
    want = oracle.linear(R, S, T, oracle.GROUP_BY_A, a_domain=1 << 12)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        # warm-up outside the capture: sizes the context's workspace
        ctx.join3_linear(dR, dS, dT, "group_by_a", shares=shares, a_domain=1 << 12, stream=s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        out = ctx.join3_linear(dR, dS, dT, "group_by_a", shares=shares, a_domain=1 << 12, stream=s,
                               sync=False)
    for _ in range(2):
        g.replay()
        torch.cuda.synchronize()
        assert int(out["total"].item()) == want["total"]
        assert np.array_equal(out["counts"].cpu().numpy(), want["counts"])
    ctx.close()
