"""The allocation-free resampling entry point, spa_resample_systematic_noalloc.

It serves callers that cannot call cudaMalloc: a process whose device memory belongs
to another allocator's pool, a latency-critical path where an allocation would
synchronise the device, or a service that must keep its device footprint fixed. They pass
device buffers, and the kernel's scratch is a fixed device array inside the library.
These checks go through the C ABI. The ancestors must equal those of the allocating
spa_resample_systematic (bit for bit, as in the other resampling tests) on several
calls in a row, because every call reuses the previous call's scratch contents. Sizes
beyond the fixed scratch must be rejected. This file sorts last, so a run that stops at
the first failure has already run every other test.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_noalloc_resampling_matches_allocating_entry_point():
    import __graft_entry__

    __graft_entry__.build()
    import torch

    import paper_1106_0322_gb300 as spa

    rng = np.random.default_rng(2024)
    stream = torch.cuda.Stream()
    for call, N in enumerate([8192, 3001, 8192]):
        W = rng.gamma(0.4 + call, size=N)
        W /= W.sum()
        u = float(rng.random())
        ref = spa.resample_systematic(W, u)
        W_dev = torch.tensor(W, dtype=torch.float64, device="cuda")
        idx_dev = torch.full((N,), -1, dtype=torch.int32, device="cuda")
        # the buffers were filled on torch's current stream; order the side stream after it
        stream.wait_stream(torch.cuda.current_stream())
        spa.resample_systematic_noalloc(W_dev, u, idx_dev, stream.cuda_stream)
        stream.synchronize()
        assert np.array_equal(idx_dev.cpu().numpy(), ref), f"call {call}"
    # equal weights on the largest size the fixed scratch holds: the identity map
    N = spa.NOALLOC_RESAMPLE_MAX_N
    W_dev = torch.full((N,), 1.0 / N, dtype=torch.float64, device="cuda")
    idx_dev = torch.empty(N, dtype=torch.int32, device="cuda")
    stream.wait_stream(torch.cuda.current_stream())
    spa.resample_systematic_noalloc(W_dev, 0.5, idx_dev, stream.cuda_stream)
    stream.synchronize()
    assert np.array_equal(idx_dev.cpu().numpy(), np.arange(N, dtype=np.int32))
    # one more than the fixed scratch holds: rejected with a clear error
    big = torch.zeros(N + 1, dtype=torch.float64, device="cuda")
    idx = torch.zeros(N + 1, dtype=torch.int32, device="cuda")
    stream.wait_stream(torch.cuda.current_stream())
    with pytest.raises(spa.SpaError) as err:
        spa.resample_systematic_noalloc(big, 0.5, idx, stream.cuda_stream)
    assert err.value.code == spa.SPA_EINVAL
    assert "SPA_NOALLOC_RESAMPLE_MAX_N" in str(err.value)
