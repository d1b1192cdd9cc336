"""GPU tests of the request server: admission by memory, continuous batching,
and results identical to the single-array call whether a request runs alone
or in a mix (tolerance zero: a shuffle has one correct output)."""
import time

import numpy as np
import pytest

import oracle
import workloads
from tests.gpu_util import from_dev, load_pip, to_dev, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pip():
    torch_cuda()
    return load_pip()


def expected(n, dtype, seed):
    a = workloads.make(n, dtype)
    oracle.knuth_hash(a, seed)
    return a


def result(pip, ptr, n, dtype):
    like = workloads.make(0, dtype)
    return pip.device_view(ptr, n, dtype).cpu().numpy().view(like.dtype).reshape((n, 2) if dtype == "rec128" else (n,))


def test_mixed_requests_equal_the_oracle(pip):
    rng = np.random.default_rng(3)
    reqs = []
    with pip.Server(8 << 30, rounds_per_tick=16) as srv:
        for j in range(80):
            n = int(2 ** rng.uniform(0, 21))
            dtype = ["u32", "u64", "rec128"][j % 3]
            eps = [0.3, 0.5, 0.7][j % 3]
            reqs.append((srv.submit(n, dtype, seed=j, eps=eps), n, dtype, j))
        for t, n, dtype, seed in reqs:
            ptr, st = srv.wait(t)
            assert st.status == 0
            assert np.array_equal(result(pip, ptr, n, dtype), expected(n, dtype, seed)), (n, dtype)
            if n >= 2:
                assert st.attempts == (n - 1) + st.losers and st.rounds >= 1
            srv.release(t)
        info = srv.info()
        assert info.completed == 80 and info.used_bytes == 0 and info.status == 0


def test_alone_equals_in_the_mix(pip):
    n, seed, eps = 300_007, 42, 0.5
    with pip.Server(4 << 30) as srv:
        t = srv.submit(n, "u64", seed, eps)
        alone = result(pip, *srv.wait(t)[:1], n, "u64").copy()
        srv.release(t)
    with pip.Server(4 << 30, rounds_per_tick=8) as srv:
        others = [srv.submit(int(s), "u32", seed=k, eps=0.6) for k, s in enumerate([10**5, 7, 2**18, 999, 2**20])]
        t = srv.submit(n, "u64", seed, eps)
        more = [srv.submit(2**16 + k, "u64", seed=k, eps=0.4) for k in range(5)]
        mixed = result(pip, srv.wait(t)[0], n, "u64").copy()
        for o in others + more:
            srv.wait(o)
    A = to_dev(workloads.iota(n, "u64"))
    pip.shuffle(A, seed=seed, eps=eps)
    pip.check()
    single = from_dev(A, workloads.iota(n, "u64"))
    assert np.array_equal(alone, mixed)
    assert np.array_equal(alone, single)
    assert np.array_equal(alone, expected(n, "u64", seed))


def test_client_arrays_and_budget_admission(pip):
    torch = torch_cuda()
    sizes = [1 << 20] * 12
    budget = 3 * ((1 << 20) * 8) + (1 << 20)  # room for three arrays at a time
    host = [workloads.iota(n, "u64") for n in sizes]
    dev = [to_dev(a) for a in host]
    with pip.Server(budget, rounds_per_tick=4) as srv:
        tickets = [srv.submit(n, "u64", seed=k, eps=0.5, A=d) for k, (n, d) in enumerate(zip(sizes, dev))]
        stats = []
        for k, t in enumerate(tickets):
            ptr, st = srv.wait(t)
            assert ptr == dev[k].data_ptr()
            stats.append(st)
            srv.release(t)
        info = srv.info()
        assert info.peak_used_bytes <= budget
        assert info.completed == 12
    torch.cuda.synchronize()
    for k, (a, d) in enumerate(zip(host, dev)):
        out = from_dev(d, a)
        want = a.copy()
        oracle.knuth_hash(want, k)
        assert np.array_equal(out, want)
    # at most three requests were ever resident together: admissions wait for releases
    admits = sorted(s.admit_ns for s in stats)
    dones = sorted(s.done_ns for s in stats)
    assert admits[3] >= dones[0]


def test_oversize_request_is_refused(pip):
    with pip.Server(1 << 20) as srv:
        with pytest.raises(pip.PipError) as e:
            srv.submit(1 << 20, "u64", 1, 0.5)
        assert e.value.code == pip.PIP_EINVAL


def test_late_arrivals_overlap_running_requests(pip):
    """Continuous batching: a request submitted while a long one runs is
    admitted and finishes before the long one does."""
    with pip.Server(8 << 30, rounds_per_tick=32, lanes=pip.SERVE_NO_LANES) as srv:
        long_t = srv.submit(1 << 26, "u64", seed=1, eps=0.5)
        time.sleep(0.05)
        short_t = srv.submit(1 << 12, "u32", seed=2, eps=0.5)
        _, s_short = srv.wait(short_t)
        _, s_long = srv.wait(long_t)
        assert s_short.admit_ns < s_long.done_ns
        assert s_short.done_ns < s_long.done_ns
        assert s_long.ticks > 1
        assert np.array_equal(result(pip, srv.poll(short_t)[0], 1 << 12, "u32"), expected(1 << 12, "u32", 2))


def test_next_done_returns_completion_order(pip):
    with pip.Server(8 << 30, lanes=pip.SERVE_NO_LANES) as srv:
        big = srv.submit(1 << 24, "u64", seed=1, eps=0.5)
        smalls = [srv.submit(1000 + k, "u32", seed=k, eps=0.5) for k in range(20)]
        got = [srv.next_done() for _ in range(21)]
        assert sorted(got) == sorted([big] + smalls)
        assert got[-1] == big  # the long request finishes last
        for t in got:
            srv.release(t)
        assert srv.next_done(timeout_ms=10) is None


# ------------------------------------------------------------------ lanes
def test_lane_requests_equal_the_oracle_alone_and_in_the_mix(pip):
    """Large requests run on lanes (the grid driver on a slice of the GPU,
    next to the ticks); each result equals the oracle, the same request
    served without lanes, and pip_shuffle."""
    big = [((1 << 22) + 17, "u64", 5), ((1 << 23) + 3, "u32", 6), ((1 << 22) + 1, "rec128", 7)]
    small = [(int(2 ** (8 + k % 12)), ["u32", "u64"][k % 2], 100 + k) for k in range(40)]
    results = {}
    for lanes in (0, pip.SERVE_NO_LANES):  # 0 = default lanes
        with pip.Server(16 << 30, lanes=lanes) as srv:
            tickets = {}
            for j, (n, d, sd) in enumerate(big + small):
                tickets[j] = srv.submit(n, d, seed=sd, eps=0.5)
            for j, (n, d, sd) in enumerate(big + small):
                ptr, st = srv.wait(tickets[j])
                assert st.status == 0
                results.setdefault(j, []).append(result(pip, ptr, n, d).copy())
                srv.release(tickets[j])
            info = srv.info()
            assert info.status == 0 and info.used_bytes == 0
            assert (info.lane_requests == len(big)) if lanes == 0 else (info.lane_requests == 0)
    for j, (n, d, sd) in enumerate(big + small):
        a, b = results[j]
        assert np.array_equal(a, b), (n, d)
        assert np.array_equal(a, expected(n, d, sd)), (n, d)
    # alone: one lane request on an idle server
    n, d, sd = big[0]
    with pip.Server(16 << 30) as srv:
        t = srv.submit(n, d, seed=sd, eps=0.5)
        ptr, st = srv.wait(t)
        assert np.array_equal(result(pip, ptr, n, d), results[0][0])
        assert st.attempts == (n - 1) + st.losers


def test_lane_request_is_much_faster_than_one_block(pip):
    n = 1 << 26
    times = {}
    for lanes in (0, pip.SERVE_NO_LANES):
        with pip.Server(8 << 30, lanes=lanes) as srv:
            t = srv.submit(n, "u64", seed=3, eps=0.5)
            ptr, st = srv.wait(t)
            assert st.status == 0
            times[lanes] = (st.done_ns - st.admit_ns) / 1e6
            out = result(pip, ptr, n, "u64")
            srv.release(t)
    assert times[0] * 4 < times[pip.SERVE_NO_LANES], times
    assert np.array_equal(out, expected(n, "u64", 3))


def test_small_requests_pass_a_large_one_waiting_for_a_lane(pip):
    """With one lane, a second large request waits for it while small
    requests behind it are admitted to tick blocks and finish first."""
    with pip.Server(16 << 30, lanes=1) as srv:
        a = srv.submit(1 << 26, "u64", seed=1, eps=0.5)
        b = srv.submit(1 << 26, "u64", seed=2, eps=0.5)
        smalls = [srv.submit(4096 + k, "u32", seed=k, eps=0.5) for k in range(8)]
        _, sb = srv.wait(b)
        for k, t in enumerate(smalls):
            ptr, st = srv.wait(t)
            assert st.done_ns < sb.done_ns
            assert np.array_equal(result(pip, ptr, 4096 + k, "u32"), expected(4096 + k, "u32", k))
        _, sa = srv.wait(a)
        assert sa.done_ns <= sb.admit_ns + 1_000_000  # b took the lane once a had left it
        for t, sd in ((a, 1), (b, 2)):
            assert np.array_equal(result(pip, srv.poll(t)[0], 1 << 26, "u64"), expected(1 << 26, "u64", sd))
