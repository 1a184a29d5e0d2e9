"""The allocation-free autocorrelation entry point, psl_autocorr_static, is for callers that
cannot allocate device memory themselves: code running under another framework's allocator
(where a raw cudaFree would synchronise the whole device) and services that reserve every
buffer at start-up.  They pass input and output buffers they own; the library's only extra
memory is a fixed scratch array built into it.

Checks: the result equals the allocating entry point psl_autocorr and, independently, the
FFT route of Eq. 2, call after call, although every call reuses the same scratch; the
longest accepted length (2^20 - 1, which fills every scratch word) and the shortest (1)
work; later calls take no device memory; sizes beyond the maximum are refused.  This file
is collected last and passes both alone and after the other tests."""
import numpy as np
import pytest

import psl_workloads as W
from helpers import fft_autocorr, have_gpu

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not have_gpu(), reason="needs a CUDA GPU")]

L_MAX = (1 << 20) - 1


def test_static_autocorr_matches_allocating_entry_point():
    import torch

    from paper_2107_09801_gb300 import build
    build.build()
    import paper_2107_09801_gb300 as P
    from paper_2107_09801_gb300 import binding as B

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    # device buffers of the caller, allocated before the first call
    s_dev = torch.empty(L_MAX, dtype=torch.int8, device=dev)
    C_dev = torch.empty(L_MAX, dtype=torch.int32, device=dev)

    def static_call(s, check_mem=True):
        """One call; device free memory before and after it must be equal (except on the first
        call, which may load the library's device code and its scratch array)."""
        L = len(s)
        s_dev[:L].copy_(torch.from_numpy(s))
        C_dev[:L].fill_(-12345)
        torch.cuda.synchronize(dev)
        free_before = torch.cuda.mem_get_info(dev)[0]
        B.psl_autocorr_static(s_dev.data_ptr(), L, C_dev.data_ptr(), stream.cuda_stream)
        torch.cuda.synchronize(dev)
        assert not check_mem or torch.cuda.mem_get_info(dev)[0] == free_before, L
        return C_dev[:L].cpu().numpy()

    with P.Context(arena_bytes=1 << 24, max_walks=2) as ctx:
        # the first call on the device looks up the scratch address (before any stream capture)
        static_call(W.random_pm1(1000, 0), check_mem=False)
        # the longest length first, then shorter ones (nothing left in the scratch may leak
        # into a later result), a ragged tail, length 1, and the longest again with another
        # sequence: every length twice in a row
        cases = [(L_MAX, 1), (L_MAX, 2), (131071, 3), (131071, 4), (1000, 5), (33, 6), (33, 7), (1, 8), (1, 9),
                 (L_MAX, 10)]
        for L, seed in cases:
            s = W.random_pm1(L, seed)
            got = static_call(s)
            assert np.array_equal(got.astype(np.int64), fft_autocorr(s)), L    # Eq. 2, independent route
            if L <= 131071:
                want = ctx.autocorr(s)[0]                                     # the allocating entry point
                assert np.array_equal(got, want), L                           # integers: bit-exact
    with pytest.raises(B.PslError):
        B.psl_autocorr_static(s_dev.data_ptr(), L_MAX + 1, C_dev.data_ptr(), stream.cuda_stream)
    with pytest.raises(B.PslError):
        B.psl_autocorr_static(s_dev.data_ptr(), 0, C_dev.data_ptr(), stream.cuda_stream)
    torch.cuda.synchronize(dev)
    assert int(C_dev[0].item()) == L_MAX   # refused calls launch nothing: the last result stays
