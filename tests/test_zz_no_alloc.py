"""The exclusive scan that allocates nothing, for callers that cannot obtain
device memory (a program whose GPU memory is all held by its own pool
allocator, or a plug-in whose host framework forbids cudaMalloc/cudaFree
during its step).  Its scratch is a fixed device array inside the library;
the result must equal the scan that takes caller scratch, call after call.

Collected last on purpose, and written to pass both on its own in a fresh
process and after the rest of the suite."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    from paper_2312_16981_gb300 import binding
    binding.load()
    return binding


def _noalloc(B, counts_dev, n):
    out = torch.full((n + 1,), -1, dtype=torch.int32, device="cuda")
    code = B.load().ugkwp_exclusive_scan_noalloc(
        ctypes.c_void_p(counts_dev.data_ptr() if n else 0), n, ctypes.c_void_p(out.data_ptr()),
        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert code == 0, B.load().ugkwp_last_error(None)
    return out.to(torch.int64) & 0xFFFFFFFF


def test_noalloc_scan_matches_scan_with_caller_scratch_two_calls(B):
    rng = np.random.Generator(np.random.Philox(2024))
    # two calls in a row with different sizes: the shared static scratch keeps
    # the first call's partials, and the second must not depend on them
    for n in (1_000_003, 70_001):
        counts = rng.integers(0, 3000, size=n, dtype=np.int64)
        counts[rng.random(n) < 0.3] = 0
        dev = torch.from_numpy(counts).to(torch.int32).cuda()
        got = _noalloc(B, dev, n)
        ref = B.exclusive_scan(dev)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(got.cpu().numpy(), ref.cpu().numpy())
        assert int(got[-1]) == int(counts.sum())


def test_noalloc_scan_edge_sizes_and_limit(B):
    for n in (0, 1, 4096, 4097):
        counts = torch.arange(n, dtype=torch.int32, device="cuda") % 7
        got = _noalloc(B, counts, n)
        np.testing.assert_array_equal(got.cpu().numpy(), B.exclusive_scan(counts).cpu().numpy())
    # beyond the static scratch: rejected with a clear error, nothing launched
    big = (1 << 24) + 1
    code = B.load().ugkwp_exclusive_scan_noalloc(ctypes.c_void_p(1), big, ctypes.c_void_p(1), None)
    assert code == -1
    assert b"static scratch" in B.load().ugkwp_last_error(None)
