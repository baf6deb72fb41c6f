"""bm_threshold_noalloc: the threshold query for callers that cannot call
cudaMalloc (for example a plugin whose host program owns all device memory,
or a service that must not allocate once running).  It keeps its ids in a
fixed device array inside the library instead of pool-allocated buffers.

Checked through the C ABI against bm_threshold (the pool entry point) on two
calls in a row, the second with fewer ids so that stale ids left in the shared
array by the first call would show.  Integer outputs: bit-exact."""
from __future__ import annotations

import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def test_noalloc_matches_pool_entry_point(dg):
    assert torch.cuda.is_available(), "GPU test needs a CUDA device"
    import paper_1402_4073_gb300 as bm

    r_bits = 64 * 20000 + 29
    nbm = 48
    words = dg.bernoulli(dg.STREAM_TESTS + 9500, r_bits, np.linspace(0.02, 0.7, nbm))
    calls = [
        (dg.floyd(dg.STREAM_TESTS + 9501, nbm, 40).astype(np.uint32), 9),
        (np.array([3, 3, 17, 5, 40], dtype=np.uint32), 2),  # fewer ids, a repeat
    ]
    with bm.Pool(r_bits, nbm) as pool:
        pool.put_dense(words)
        info = pool.info()
        base, stride = info["dense_base"], info["stride_words"]
        stream = torch.cuda.current_stream().cuda_stream
        for ids, theta in calls:
            want = pool.empty_words()
            want_card = torch.zeros(1, dtype=torch.int64, device="cuda")
            bm.threshold(pool, ids, theta, want, want_card)

            got = pool.empty_words()
            got.fill_(-1)
            got_card = torch.full((1,), -1, dtype=torch.int64, device="cuda")
            rc = bm.lib.bm_threshold_noalloc(
                ctypes.c_void_p(base), stride, nbm, r_bits, ids.ctypes.data, len(ids), theta,
                got.data_ptr(), got_card.data_ptr(), stream)
            assert rc == 0, bm.lib.bm_strerror(rc)
            torch.cuda.synchronize()
            assert torch.equal(got, want)
            assert int(got_card.item()) == int(want_card.item()) > 0

        # sizes beyond the fixed scratch array are refused
        too_many = np.zeros(16385, dtype=np.uint32)
        out = pool.empty_words()
        rc = bm.lib.bm_threshold_noalloc(ctypes.c_void_p(base), stride, nbm, r_bits,
                                         too_many.ctypes.data, len(too_many), 1, out.data_ptr(),
                                         None, stream)
        assert rc == bm.BM_EINVAL
