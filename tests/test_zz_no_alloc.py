"""pip_shuffle_noalloc: the shuffle for callers that cannot allocate device memory.

Such callers (an application that has reserved the whole GPU for its own
memory pool, a latency-critical path that must not enter the CUDA allocator)
get the same result as pip_shuffle, with the scratch taken from a fixed 16 MiB
area built into the library.  The test calls the entry point through the C
ABI twice in a row and compares each result with pip_shuffle's on the same
input, bit for bit (the tolerance of every parity test here).  This file is
collected last so that a failure here does not hide any other test.
"""
import ctypes

import numpy as np
import pytest

import workloads
from tests.gpu_util import from_dev, load_pip, to_dev, torch_cuda

pytestmark = pytest.mark.gpu

CASES = [((1 << 22) + 3, "u64", 0.5, 11), (1_000_003, "u32", 0.5, 12), (300_007, "rec128", 0.6, 13),
         (1 << 20, "u64", 0.8, 14)]


@pytest.fixture(scope="module")
def pip():
    torch_cuda()
    return load_pip()


def noalloc(pip, A, n, dtype, seed, eps):
    torch = torch_cuda()
    stream = torch.cuda.current_stream().cuda_stream
    return pip.lib().pip_shuffle_noalloc(ctypes.c_void_p(A.data_ptr()), n, pip.DTYPES[dtype], seed, eps,
                                         ctypes.c_void_p(stream))


@pytest.mark.parametrize("n,dtype,eps,seed", CASES)
def test_noalloc_matches_pip_shuffle_twice_in_a_row(pip, n, dtype, eps, seed):
    host = workloads.make(n, dtype)
    a = to_dev(host)  # through the no-allocation entry point
    b = to_dev(host)  # through pip_shuffle
    for _ in range(2):  # second call reuses the area the first one left behind
        assert noalloc(pip, a, n, dtype, seed, eps) == pip.PIP_OK
        pip.shuffle(b, seed=seed, eps=eps)
        pip.check()
        assert np.array_equal(from_dev(a, host), from_dev(b, host))
    assert not np.array_equal(from_dev(a, host), host)


def test_noalloc_refuses_requests_beyond_the_area(pip):
    n = 1 << 26
    plan = pip.plan(n, "u64", 0.1, flags=pip.FLAG_FORCE_GRID)
    assert plan["aux_bytes"] > (16 << 20)
    host = workloads.iota(n, "u64")
    a = to_dev(host)
    assert noalloc(pip, a, n, "u64", 1, 0.1) == pip.PIP_ETOOLARGE
    pip.check()
    assert np.array_equal(from_dev(a, host), host)
    # and invalid arguments are still refused
    assert noalloc(pip, a, n, "u64", 1, 1.5) == pip.PIP_EINVAL
