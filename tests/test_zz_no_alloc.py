"""csc_sample_noalloc, the sampling entry point that allocates no device memory,
against csc_sample through the C ABI.

It exists for callers that cannot allocate device memory (all device memory owned
by their own allocator, a fixed memory budget, or a latency-critical path where
cudaMalloc / cudaFree may synchronize the device).  Its scratch is a fixed array
inside the library shared by all calls, so the test makes two calls in a row (the
second on a smaller problem than the first) and checks each against the allocating
entry point: sampling results are bit-exact, so the comparison is exact equality.
This file is collected last on purpose."""
import ctypes

import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    from paper_1602_02018_gb300 import _native, build

    build.build()
    return _native


def _run(fn, N, n, seed):
    out = torch.full((n,), -1, dtype=torch.int64, device="cuda")
    st = fn(N, n, seed, ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st, out


def test_noalloc_matches_allocating_sampler_on_two_calls_in_a_row(L):
    lib = L.lib()
    cases = [(100_000, 2_120, 0), (1_000, 120, 5)]
    got = []
    for N, n, seed in cases:  # two calls of the no-alloc entry point back to back
        st, out = _run(lib.csc_sample_noalloc, N, n, seed)
        assert st == L.CSC_OK, lib.csc_last_error()
        got.append(out)
    torch.cuda.synchronize()
    for (N, n, seed), out in zip(cases, got):
        st, ref = _run(lib.csc_sample, N, n, seed)
        assert st == L.CSC_OK, lib.csc_last_error()
        torch.cuda.synchronize()
        assert torch.equal(out, ref)


def test_noalloc_rejects_sizes_beyond_its_scratch(L):
    lib = L.lib()
    out = torch.full((10,), -1, dtype=torch.int64, device="cuda")
    st = lib.csc_sample_noalloc(2**26 + 1, 10, 0, ctypes.c_void_p(out.data_ptr()), None)
    assert st == L.CSC_E_UNSUPPORTED
    torch.cuda.synchronize()
    assert torch.all(out == -1)  # rejected before any work
    assert b"scratch" in lib.csc_last_error()
