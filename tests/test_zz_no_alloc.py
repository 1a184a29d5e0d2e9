"""The allocation-free autocorrelation entry point, meant for callers that cannot
allocate device memory themselves (they own every buffer and pass it in), must give
the same C_k as the allocating entry point psl_autocorr, call after call, although
every call reuses the same built-in scratch area."""
import numpy as np
import pytest

import psl_workloads as W
from helpers import have_gpu

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not have_gpu(), reason="needs a CUDA GPU")]


def test_static_autocorr_matches_allocating_entry_point():
    import torch

    from paper_2107_09801_gb300 import build
    build.build()
    import paper_2107_09801_gb300 as P
    from paper_2107_09801_gb300 import binding as B

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    # a long sequence first, then shorter ones: nothing left in the scratch may leak into
    # a later result; the last call repeats the first length with another sequence
    cases = [(131071, 1), (1000, 2), (33, 3), (131071, 4)]
    with P.Context(arena_bytes=1 << 24, max_walks=2) as ctx:
        for L, seed in cases:
            s = W.random_pm1(L, seed)
            want = ctx.autocorr(s)[0]                      # existing, allocating entry point
            s_dev = torch.from_numpy(s).to(dev)
            C_dev = torch.full((L,), -12345, dtype=torch.int32, device=dev)
            B.psl_autocorr_static(s_dev.data_ptr(), L, C_dev.data_ptr(), stream.cuda_stream)
            torch.cuda.synchronize(dev)
            assert np.array_equal(C_dev.cpu().numpy(), want), L   # integers: bit-exact
    with pytest.raises(B.PslError):
        B.psl_autocorr_static(s_dev.data_ptr(), 1 << 20, C_dev.data_ptr(), stream.cuda_stream)
    with pytest.raises(B.PslError):
        B.psl_autocorr_static(s_dev.data_ptr(), 0, C_dev.data_ptr(), stream.cuda_stream)
