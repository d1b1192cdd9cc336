"""Parity at the full sizes of the benchmark configurations, in the launch
configuration ``bench.py`` times (default plans).

* n = 10^9 uint64, seed 2: the whole output for eps = 0.25, 0.5 and 0.75 is
  compared with one run of the sequential oracle (the permutation does not
  depend on eps).
* n = 2^30 16-byte records, seed 3, eps = 0.5: the keys form a permutation and
  every record keeps its payload (properties that hold at any size).
* the 8192-array batch (sizes log-uniform in [2^8, 2^22], stream seed 7): every
  array against the oracle, computed by a process pool started with ``spawn``.
* scratch: with caller-provided scratch of exactly the planned size the
  device's free memory does not move, and the plan obeys the aux bound.
"""
import multiprocessing as mp
import os

import numpy as np
import pytest

import oracle
import workloads
from tests.gpu_util import load_pip, torch_cuda

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def pip():
    torch_cuda()
    return load_pip()


def test_headline_1e9_every_eps_equals_the_oracle(pip):
    torch = torch_cuda()
    n, seed = 10**9, 2
    expected = workloads.iota(n, "u64")
    oracle.knuth_hash(expected, seed)
    exp_t = torch.from_numpy(expected.view(np.int64))
    for eps in (0.25, 0.5, 0.75):
        A = torch.arange(n, dtype=torch.int64, device="cuda")
        st = torch.zeros(pip.STATS_BYTES, dtype=torch.uint8, device="cuda")
        pip.shuffle(A, seed=seed, eps=eps, stats=st)
        pip.check()
        s = pip.read_stats(st)
        assert s.status == 0 and s.attempts == (n - 1) + s.losers
        got = A.cpu()
        del A
        assert torch.equal(got, exp_t), eps
        del got
        torch.cuda.empty_cache()


def test_records_2pow30_keep_keys_and_payloads(pip):
    torch = torch_cuda()
    n, seed = 1 << 30, 3
    A = torch.empty((n, 2), dtype=torch.int64, device="cuda")
    A[:, 0] = torch.arange(n, dtype=torch.int64, device="cuda")
    # payloads from the workload generator, built on the host in chunks
    chunk = 1 << 26
    for c0 in range(0, n, chunk):
        keys = np.arange(c0, min(n, c0 + chunk), dtype=np.uint64)
        A[c0:c0 + keys.size, 1] = torch.from_numpy(workloads.record_payload(keys).view(np.int64)).cuda()
    pip.shuffle(A, seed=seed, eps=0.5)
    pip.check()
    keys = A[:, 0]
    seen = torch.zeros(n, dtype=torch.bool, device="cuda")
    seen[keys] = True
    assert bool(seen.all())
    del seen
    assert not torch.equal(keys[:1000], torch.arange(1000, dtype=torch.int64, device="cuda"))
    for c0 in range(0, n, chunk):
        blk = A[c0:c0 + chunk].cpu().numpy().view(np.uint64)
        assert np.array_equal(blk[:, 1], workloads.record_payload(blk[:, 0]))


def _oracle_slice(args):
    """Worker: oracle outputs of arrays [j0, j1) written into the shared buffer."""
    shm_name, total, offsets, sizes, seeds, j0, j1 = args
    from multiprocessing import shared_memory

    import oracle as orc

    shm = shared_memory.SharedMemory(name=shm_name)
    try:
        buf = np.ndarray((total,), dtype=np.uint32, buffer=shm.buf)
        for j in range(j0, j1):
            a = buf[offsets[j]:offsets[j] + sizes[j]]
            a[:] = np.arange(sizes[j], dtype=np.uint32)
            orc.knuth_hash(a, int(seeds[j]))
    finally:
        shm.close()
    return j1 - j0


def test_batch_8192_arrays_all_equal_the_oracle(pip):
    from multiprocessing import shared_memory

    torch = torch_cuda()
    sizes, seeds = workloads.batch_workload()
    offs = np.zeros(len(sizes) + 1, dtype=np.int64)
    offs[1:] = np.cumsum(sizes)
    total = int(offs[-1])
    shm = shared_memory.SharedMemory(create=True, size=total * 4)
    try:
        ctx = mp.get_context("spawn")
        nproc = max(1, min(16, os.cpu_count() or 1))
        chunks = np.array_split(np.arange(len(sizes)), nproc * 4)
        jobs = [(shm.name, total, offs[:-1].tolist(), sizes.tolist(), seeds.tolist(), int(c[0]), int(c[-1]) + 1)
                for c in chunks if len(c)]
        with ctx.Pool(nproc) as pool:
            async_res = pool.map_async(_oracle_slice, jobs)
            buf = torch.empty(total, dtype=torch.int32, device="cuda")
            arrays = [buf[int(offs[j]):int(offs[j + 1])] for j in range(len(sizes))]
            for a in arrays:
                a.copy_(torch.arange(a.shape[0], dtype=torch.int32, device="cuda"))
            pip.Batch(arrays, [int(s) for s in seeds], eps=0.5).run()
            pip.check()
            got = buf.cpu().numpy().view(np.uint32)
            assert sum(async_res.get()) == len(sizes)
        want = np.ndarray((total,), dtype=np.uint32, buffer=shm.buf)
        bad = [j for j in range(len(sizes)) if not np.array_equal(got[offs[j]:offs[j + 1]], want[offs[j]:offs[j + 1]])]
        del want
        assert not bad, bad[:10]
    finally:
        shm.close()
        shm.unlink()


@pytest.mark.parametrize("eps", [0.25, 0.5, 0.75])
def test_scratch_is_exactly_the_plan(pip, eps):
    torch = torch_cuda()
    n = 10**8
    p = pip.plan(n, "u64", eps)
    assert p["aux_bytes"] + p["smem_bytes"] <= p["aux_bound_bytes"]
    A = torch.arange(n, dtype=torch.int64, device="cuda")
    aux = torch.empty(p["aux_bytes"], dtype=torch.uint8, device="cuda")
    small = torch.arange(1 << 16, dtype=torch.int64, device="cuda")
    flag = {pip.DRIVER_GRID: 32, pip.DRIVER_CTA: 64, pip.DRIVER_CLUSTER: 128}[p["driver"]]
    pip.shuffle(small, seed=4, eps=eps, aux=aux, flags=flag)  # loads the kernel
    pip.check()
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    pip.shuffle(A, seed=4, eps=eps, aux=aux)
    free1, _ = torch.cuda.mem_get_info()  # while the kernel may still run
    pip.check()
    free2, _ = torch.cuda.mem_get_info()
    assert free1 == free0 and free2 == free0
    seen = torch.zeros(n, dtype=torch.bool, device="cuda")
    seen[A] = True
    assert bool(seen.all())
