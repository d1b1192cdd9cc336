"""pip_shuffle_noalloc: the shuffle for callers that cannot allocate device memory.

Such callers (an application that has reserved the whole GPU for its own
memory pool, a latency-critical path that must not enter the CUDA allocator)
get the same result as pip_shuffle, with the scratch taken from a fixed 16 MiB
area built into the library.  The tests call the entry point through the C ABI
and check:

* two calls in a row (the second reuses the area the first left behind), each
  against the sequential oracle and against pip_shuffle on the same input, bit
  for bit (the tolerance of every parity test here);
* that a call allocates nothing: after the set-up call, the device's free
  memory, torch's reserved bytes and the default memory pool's reserved and
  used bytes do not move across calls;
* the refusals: plans larger than the area, invalid arguments and host memory.

This file is collected last so that a failure here does not hide any other test.
"""
import ctypes
import ctypes.util
import glob
import os

import numpy as np
import pytest

import oracle
import workloads
from tests.gpu_util import from_dev, load_pip, to_dev, torch_cuda

pytestmark = pytest.mark.gpu

CASES = [((1 << 22) + 3, "u64", 0.5, 11), (1_000_003, "u32", 0.5, 12), (300_007, "rec128", 0.6, 13),
         (1 << 20, "u64", 0.8, 14)]


@pytest.fixture(scope="module")
def pip():
    torch_cuda()
    p = load_pip()
    # set-up call (n = 0): reserves and looks up the area on this device
    assert p.lib().pip_shuffle_noalloc(None, 0, p.DTYPES["u64"], 0, 0.5, None) == p.PIP_OK
    return p


def noalloc(pip, A, n, dtype, seed, eps):
    torch = torch_cuda()
    stream = torch.cuda.current_stream().cuda_stream
    return pip.lib().pip_shuffle_noalloc(ctypes.c_void_p(A.data_ptr()), n, pip.DTYPES[dtype], seed, eps,
                                         ctypes.c_void_p(stream))


def oracle_shuffle(host, seed):
    want = host.copy()
    oracle.knuth_hash(want, seed)
    return want


@pytest.mark.parametrize("n,dtype,eps,seed", CASES)
def test_noalloc_equals_the_oracle_and_pip_shuffle_twice_in_a_row(pip, n, dtype, eps, seed):
    host = workloads.make(n, dtype)
    for call in range(2):  # the second call reuses the area the first one left behind
        s = seed + 1000 * call
        want = oracle_shuffle(host, s)
        a = to_dev(host)  # through the no-allocation entry point
        b = to_dev(host)  # through pip_shuffle
        assert noalloc(pip, a, n, dtype, s, eps) == pip.PIP_OK
        pip.check()
        got = from_dev(a, host)
        assert np.array_equal(got, want)
        pip.shuffle(b, seed=s, eps=eps)
        pip.check()
        assert np.array_equal(got, from_dev(b, host))
        assert not np.array_equal(got, host)


def _default_pool_bytes(torch):
    """(reserved, used) bytes of the device's default memory pool, read
    through the CUDA runtime, or None when no runtime library is found."""
    cands = [ctypes.util.find_library("cudart")]
    for root in [os.path.dirname(torch.__file__), "/usr/local/cuda/lib64"]:
        cands += sorted(glob.glob(os.path.join(root, "**", "libcudart.so*"), recursive=True))
    for c in [c for c in cands if c]:
        try:
            rt = ctypes.CDLL(c)
        except OSError:
            continue
        pool = ctypes.c_void_p()
        if rt.cudaDeviceGetDefaultMemPool(ctypes.byref(pool), torch.cuda.current_device()) != 0:
            continue
        out = []
        for attr in (5, 7):  # cudaMemPoolAttrReservedMemCurrent, cudaMemPoolAttrUsedMemCurrent
            v = ctypes.c_uint64()
            if rt.cudaMemPoolGetAttribute(pool, attr, ctypes.byref(v)) != 0:
                return None
            out.append(v.value)
        return tuple(out)
    return None


def _memory_state(torch):
    """Free device memory, torch's reserved bytes and the default pool's
    (reserved, used) bytes: each grows when anything allocates.  (torch's
    allocated bytes are left out: tensors of earlier tests freed by the
    garbage collector can lower them at any time.)"""
    torch.cuda.synchronize()
    return (torch.cuda.mem_get_info()[0], torch.cuda.memory_reserved(), _default_pool_bytes(torch))


def test_noalloc_allocates_nothing(pip):
    import gc

    torch = torch_cuda()
    gc.collect()
    n, dtype = (1 << 22) + 3, "u64"
    host = workloads.make(n, dtype)
    a = to_dev(host)
    assert noalloc(pip, a, n, dtype, 21, 0.5) == pip.PIP_OK  # warm-up: kernels loaded
    pip.check()
    _memory_state(torch)  # loads the runtime library the pool query uses
    before = _memory_state(torch)
    for s in (22, 23):
        assert noalloc(pip, a, n, dtype, s, 0.5) == pip.PIP_OK
        free_during = torch.cuda.mem_get_info()[0]  # while the kernel may still run
        pip.check()
        assert free_during == before[0]
        assert _memory_state(torch) == before


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


def test_noalloc_refuses_host_memory(pip):
    torch = torch_cuda()
    for pinned in (False, True):
        h = torch.arange(4096, dtype=torch.int64)
        if pinned:
            h = h.pin_memory()
        assert noalloc(pip, h, 4096, "u64", 1, 0.5) == pip.PIP_EINVAL
        pip.check()
        assert torch.equal(h, torch.arange(4096, dtype=torch.int64))
