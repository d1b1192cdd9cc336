"""Parity at the full sizes of the benchmark configurations, in the launch
configuration ``bench.py`` times (default plans).

* n = 10^9 uint64, seed 2: the whole output for eps = 0.25, 0.5 and 0.75 is
  compared with one run of the sequential oracle (the permutation does not
  depend on eps).
* n = 2^30 16-byte records, seed 3, eps = 0.5: the whole output against one
  run of the sequential oracle.
* the 8192-array batch (sizes log-uniform in [2^8, 2^22], stream seed 7): every
  array against the oracle, computed by a process pool started with ``spawn``.
* serving: the served workload's four largest requests (near 2^28 elements,
  uint32 and uint64) with its first 16 requests, under the 120 GB budget,
  each against the oracle.
* scratch: with caller-provided scratch of exactly the planned size the
  device's free memory does not move, and the plan obeys the aux bound.
* tree contraction of 2^25 leaves and list contraction of 2^26 nodes at
  their default plans (the tree's has the bench launch's shape), and the scan
  of 10^9 uint32 values (the bench's size): whole outputs against the oracle.
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


def test_records_2pow30_equal_the_oracle(pip):
    # the record configuration at its stated size (2^30 16-byte records,
    # 16 GiB, seed 3, eps = 0.5, default plan): the whole output against one
    # run of the sequential oracle on the same input, record by record
    torch = torch_cuda()
    n, seed = 1 << 30, 3
    host = np.empty((n, 2), dtype=np.uint64)
    chunk = 1 << 26
    for c0 in range(0, n, chunk):
        keys = np.arange(c0, min(n, c0 + chunk), dtype=np.uint64)
        host[c0:c0 + keys.size, 0] = keys
        host[c0:c0 + keys.size, 1] = workloads.record_payload(keys)
    A = torch.from_numpy(host.view(np.int64)).cuda()
    plan = pip.plan(n, "rec128", 0.5)
    st = torch.zeros(pip.STATS_BYTES, dtype=torch.uint8, device="cuda")
    pip.shuffle(A, seed=seed, eps=0.5, stats=st)
    pip.check()
    s = pip.read_stats(st)
    assert s.status == 0 and s.attempts == (n - 1) + s.losers
    assert plan["driver"] == pip.DRIVER_GRID
    got = A.cpu().numpy().view(np.uint64)
    del A
    torch.cuda.empty_cache()
    assert not np.array_equal(got[:1000, 0], np.arange(1000, dtype=np.uint64))
    oracle.knuth_hash(host, seed)  # in place: host becomes the expected output
    for c0 in range(0, n, chunk):
        assert np.array_equal(got[c0:c0 + chunk], host[c0:c0 + chunk]), c0


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


def _oracle_request(args):
    """Worker: the oracle's output of one served request (A[i] = i, seed =
    request id) written into its slice of the shared buffer."""
    shm_name, off, n, itemsize, seed = args
    from multiprocessing import shared_memory

    import oracle as orc

    shm = shared_memory.SharedMemory(name=shm_name)
    try:
        dt = np.uint32 if itemsize == 4 else np.uint64
        a = np.ndarray((n,), dtype=dt, buffer=shm.buf, offset=off)
        a[:] = np.arange(n, dtype=dt)
        orc.knuth_hash(a, seed)
    finally:
        shm.close()
    return n


def test_served_largest_requests_equal_the_oracle(pip):
    # the serving workload's largest requests (sizes near 2^28, both element
    # types) served together with the stream's first 16 requests, under the
    # 120 GB budget: every result against the oracle
    from multiprocessing import shared_memory

    sizes, dtypes, seeds, _ = workloads.serve_workload()
    top = [int(j) for j in np.argsort(-sizes)[:4]]
    ids = top + [j for j in range(16) if j not in top]
    assert {dtypes[j] for j in top} == {"u32", "u64"}
    item = {j: 4 if dtypes[j] == "u32" else 8 for j in ids}
    offs, total = {}, 0
    for j in ids:
        offs[j] = total
        total += (int(sizes[j]) * item[j] + 255) // 256 * 256
    shm = shared_memory.SharedMemory(create=True, size=total)
    try:
        ctx = mp.get_context("spawn")
        with ctx.Pool(max(1, min(16, os.cpu_count() or 1))) as pool:
            jobs = [(shm.name, offs[j], int(sizes[j]), item[j], int(seeds[j])) for j in ids]
            async_res = pool.map_async(_oracle_request, jobs)
            got = {}
            with pip.Server(120 * 10**9) as srv:
                tickets = {j: srv.submit(int(sizes[j]), str(dtypes[j]), seed=int(seeds[j]), eps=0.5) for j in ids}
                for j, t in tickets.items():
                    ptr, st = srv.wait(t)
                    assert st.status == 0, j
                    n = int(sizes[j])
                    got[j] = pip.device_view(ptr, n, str(dtypes[j])).cpu().numpy().copy()
                    assert st.attempts == (n - 1) + st.losers
                    srv.release(t)
                assert srv.info().status == 0
            assert sum(async_res.get()) == int(sum(sizes[j] for j in ids))
        for j in ids:
            dt = np.uint32 if item[j] == 4 else np.uint64
            want = np.ndarray((int(sizes[j]),), dtype=dt, buffer=shm.buf, offset=offs[j])
            assert np.array_equal(got[j].view(dt), want), (j, int(sizes[j]), dtypes[j])
            del want
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


def test_tree_contraction_in_the_bench_launch_shape(pip):
    # 2^25 leaves (6.7e7 nodes, 2 GB): the default plan at eps = 0.25 has
    # the bench launch's shape (L2-sized prefix, 304 blocks, phase-B cache);
    # the whole output against the oracle's schedule, and every rake undone
    torch = torch_cuda()
    rec = workloads.random_tree(1 << 25, rng_seed=25)
    n = rec.shape[0]
    plan = pip.tree_plan(n, 0.25)
    F = plan["fresh_per_round"]
    assert plan["max_active"] == F * 5 // 2 + 2
    t = torch.from_numpy(rec.view(np.int64)).cuda()
    pip.tree_contract(t, eps=0.25)
    pip.check()
    out = t.cpu().numpy().view(np.uint64).reshape(rec.shape)
    del t
    torch.cuda.empty_cache()
    # schedule-free check first: every rake undone back to the input
    rc, back = oracle.tree_uncontract(out, rec)
    assert rc == 0 and np.array_equal(back, rec)
    del back
    # then the records under the schedule reading (F, kmax = 2.5 F + 2)
    want = rec.copy()
    oracle.tree_contract(want, F, F * 5 // 2 + 2)
    assert np.array_equal(out, want)


def test_list_contraction_one_long_list(pip):
    # one random list of 2^26 nodes at the default plan (eps = 0.25)
    torch = torch_cuda()
    rec = workloads.random_lists(1 << 26, rng_seed=26)
    t = torch.from_numpy(rec.view(np.int64)).cuda()
    pip.list_contract(t, eps=0.25)
    pip.check()
    out = t.cpu().numpy().view(np.uint64).reshape(rec.shape)
    del t
    torch.cuda.empty_cache()
    assert np.array_equal(out, oracle.list_contract(rec.copy()))


def test_scan_1e9_u32(pip):
    # the bench's scan size: 10^9 uint32 values below 2^20, whole output and
    # total against the oracle's up-sweep / down-sweep
    torch = torch_cuda()
    n = 10**9
    a = np.random.default_rng(9).integers(0, 1 << 20, size=n, dtype=np.uint32)
    t = torch.from_numpy(a.view(np.int32)).cuda()
    tot = torch.zeros(1, dtype=torch.int32, device="cuda")
    pip.scan(t, total=tot)
    pip.check()
    got = t.cpu().numpy().view(np.uint32)
    got_tot = int(tot.cpu().numpy().view(np.uint32)[0])
    del t
    torch.cuda.empty_cache()
    want_tot = oracle.scan_exclusive(a)  # in place on the host copy
    assert got_tot == want_tot
    assert np.array_equal(got, a)
