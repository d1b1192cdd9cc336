"""GPU parity of the host-memory path (pip_shuffle_host_stream): every array
copied in, shuffled and copied back must equal the oracle's sequential Knuth
shuffle of that array with its seed, bit for bit, whatever the overlap of the
copies with the neighbouring shuffles."""
import numpy as np
import pytest

import oracle
import workloads
from tests.gpu_util import load_pip, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pip():
    torch_cuda()
    return load_pip()


def host_tensor(torch, arr: np.ndarray, pinned: bool):
    view = {4: np.int32, 8: np.int64}[arr.dtype.itemsize] if arr.ndim == 1 else np.int64
    t = torch.from_numpy(np.ascontiguousarray(arr).view(view).copy())
    return t.pin_memory() if pinned else t


def to_np(t, like: np.ndarray) -> np.ndarray:
    return t.numpy().view(like.dtype).reshape(like.shape)


def expected(arr: np.ndarray, seed: int) -> np.ndarray:
    return oracle.knuth_hash(arr.copy(), seed)


@pytest.mark.parametrize("dtype,pinned,in_place", [("u64", True, False), ("u32", False, True), ("u64", True, True),
                                                   ("rec128", True, False)])
def test_sequence_of_host_arrays(pip, dtype, pinned, in_place):
    torch = torch_cuda()
    n, count = (1 << 20) + 3, 5
    base = workloads.make(n, dtype)
    arrays = [base.copy() for _ in range(count)]
    for j, a in enumerate(arrays):  # different contents per array
        if a.ndim == 1:
            a ^= np.array(j, dtype=a.dtype)
    ins = [host_tensor(torch, a, pinned) for a in arrays]
    outs = ins if in_place else [host_tensor(torch, np.zeros_like(a), pinned) for a in arrays]
    seeds = [11 * j + 3 for j in range(count)]
    pip.shuffle_host_stream(ins, outs, seeds, eps=0.5)
    pip.check()
    for j in range(count):
        assert np.array_equal(to_np(outs[j], arrays[j]), expected(arrays[j], seeds[j])), j


def test_single_array_and_caller_buffer(pip):
    torch = torch_cuda()
    n = 300007
    a = workloads.make(n, "u64")
    t = host_tensor(torch, a, True)
    buf = torch.empty(((n * 8 + 255) // 256) * 256, dtype=torch.uint8, device="cuda")
    pip.shuffle_host_stream([t], [t], [5], eps=0.25, dev_buf=buf)
    pip.check()
    assert np.array_equal(to_np(t, a), expected(a, 5))
    # two arrays need two buffers: one is too small
    t2 = host_tensor(torch, a, True)
    with pytest.raises(pip.PipError) as e:
        pip.shuffle_host_stream([t, t2], [t, t2], [1, 2], eps=0.25, dev_buf=buf)
    assert e.value.code == pip.PIP_EINVAL
    # five arrays go round three caller buffers
    slot = ((n * 8 + 255) // 256) * 256
    buf3 = torch.empty(3 * slot, dtype=torch.uint8, device="cuda")
    ts = [host_tensor(torch, a, True) for _ in range(5)]
    pip.shuffle_host_stream(ts, ts, [20, 21, 22, 23, 24], eps=0.25, dev_buf=buf3)
    pip.check()
    for j, tj in enumerate(ts):
        assert np.array_equal(to_np(tj, a), expected(a, 20 + j)), j
    # seven arrays go round four caller buffers (room for a fourth is used),
    # and round three when the area holds three and a half
    for nslots in (4.0, 3.5):
        bufx = torch.empty(int(nslots * slot), dtype=torch.uint8, device="cuda")
        ts = [host_tensor(torch, a, True) for _ in range(7)]
        pip.shuffle_host_stream(ts, ts, [30 + j for j in range(7)], eps=0.25, dev_buf=bufx)
        pip.check()
        for j, tj in enumerate(ts):
            assert np.array_equal(to_np(tj, a), expected(a, 30 + j)), (nslots, j)


def test_larger_arrays_many_steps(pip):
    torch = torch_cuda()
    n, count = (1 << 24) + 1, 4
    a = workloads.make(n, "u64")
    ins = [host_tensor(torch, a, True) for _ in range(count)]
    outs = [host_tensor(torch, np.zeros_like(a), True) for _ in range(count)]
    seeds = [2, 2, 9, 2]
    pip.shuffle_host_stream(ins, outs, seeds, eps=0.25)
    pip.check()
    want2, want9 = expected(a, 2), expected(a, 9)
    for j in range(count):
        assert np.array_equal(to_np(outs[j], a), want9 if seeds[j] == 9 else want2), j
    # the inputs were not modified
    for t in ins:
        assert np.array_equal(to_np(t, a), a)


def test_tiny_and_empty(pip):
    torch = torch_cuda()
    for n in (1, 2, 3):
        a = workloads.make(n, "u64")
        t0, t1 = host_tensor(torch, a, True), host_tensor(torch, a, True)
        pip.shuffle_host_stream([t0, t1], [t0, t1], [4, 5], eps=0.5)
        pip.check()
        assert np.array_equal(to_np(t0, a), expected(a, 4)) and np.array_equal(to_np(t1, a), expected(a, 5))
    pip.shuffle_host_stream([], [], [], eps=0.5)
    pip.check()
