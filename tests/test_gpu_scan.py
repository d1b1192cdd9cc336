"""GPU parity of the in-place exclusive scan (Section 5.1) against the CPU
oracle (Algorithm 3's up-sweep / down-sweep), bit for bit: integer addition
modulo 2^w is associative, so the output is unique."""
import numpy as np
import pytest

import oracle
from tests.gpu_util import from_dev, load_pip, to_dev, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pip():
    torch_cuda()
    return load_pip()


def gpu_scan(pip, a: np.ndarray, **kw):
    torch = torch_cuda()
    A = to_dev(a)
    tot = torch.zeros(1, dtype=A.dtype, device="cuda")
    pip.scan(A, total=tot, **kw)
    pip.check()
    return from_dev(A, a), int(tot.cpu().numpy().view(a.dtype)[0])


def expected(a: np.ndarray):
    b = a.copy()
    t = oracle.scan_exclusive(b)
    return b, t


TILE = {np.uint32: 12288, np.uint64: 5120}  # elements per tile (48 KB for u32, 40 KB for u64)


@pytest.mark.parametrize("dtype", [np.uint32, np.uint64])
@pytest.mark.parametrize("k", [0, 1, 2, 3, 31, 32, 33, 1000])
def test_small_and_ragged(pip, dtype, k):
    for n in sorted({k, TILE[dtype] - 1 + k % 3, TILE[dtype] + k, 3 * TILE[dtype] + 7 + k}):
        rng = np.random.default_rng(n)
        a = rng.integers(0, np.iinfo(dtype).max, size=n, dtype=dtype, endpoint=True)
        got, tot = gpu_scan(pip, a)
        want, wt = expected(a)
        assert np.array_equal(got, want), n
        assert tot == wt, n


@pytest.mark.parametrize("dtype", [np.uint32, np.uint64])
@pytest.mark.parametrize("n", [(1 << 20) + 3, 10**7 + 11, 1 << 26])
def test_large(pip, dtype, n):
    rng = np.random.default_rng(n + 1)
    a = rng.integers(0, 1 << 20, size=n, dtype=dtype)
    got, tot = gpu_scan(pip, a)
    want, wt = expected(a)
    assert np.array_equal(got, want)
    assert tot == wt


def test_closed_forms_and_wraparound(pip):
    n = 5 * 8192 + 3
    ones = np.ones(n, dtype=np.uint64)
    got, tot = gpu_scan(pip, ones)
    assert tot == n and np.array_equal(got, np.arange(n, dtype=np.uint64))
    big = np.full(n, 0xFFFFFFFF, dtype=np.uint32)
    got, tot = gpu_scan(pip, big)
    assert tot == (n * 0xFFFFFFFF) % (1 << 32)
    assert np.array_equal(got, ((np.arange(n, dtype=np.uint64) * 0xFFFFFFFF) % (1 << 32)).astype(np.uint32))


def test_caller_scratch_and_repeat(pip):
    torch = torch_cuda()
    n = 3 * 10**6 + 5
    a = np.random.default_rng(7).integers(0, 1000, size=n, dtype=np.uint64)
    want, wt = expected(a)
    aux = torch.empty(pip.scan_aux_bytes(), dtype=torch.uint8, device="cuda")
    for _ in range(3):  # the scratch is reused; every call starts from a clean state
        got, tot = gpu_scan(pip, a, aux=aux)
        assert np.array_equal(got, want) and tot == wt


def test_argument_errors(pip):
    torch = torch_cuda()
    A = torch.zeros(100, dtype=torch.int64, device="cuda")
    assert pip.lib().pip_scan(A.data_ptr() + 8, 10, pip.U64, None, None) == pip.PIP_EINVAL  # not 16-byte aligned
    assert pip.lib().pip_scan(A.data_ptr(), 10, pip.REC128, None, None) == pip.PIP_EINVAL
    assert pip.lib().pip_scan(None, 0, pip.U64, None, None) == pip.PIP_OK
