"""GPU parity of the batched path: many independent arrays in one launch.

Every array of a batch must come out exactly as the sequential Knuth shuffle
of the oracle with its own targets, and exactly as the single-array call.
"""
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


def expected(arr, seed=None, H=None):
    out = arr.copy()
    if H is not None:
        oracle.knuth_explicit(out, H)
    else:
        oracle.knuth_hash(out, seed)
    return out


SIZES = [0, 1, 2, 3, 31, 256, 257, 1000, 4096, 65536 + 3, 300001, 1 << 20]


@pytest.mark.parametrize("dtype", ["u32", "u64", "rec128"])
def test_batch_matches_oracle(pip, dtype):
    host = [workloads.make(n, dtype) for n in SIZES]
    seeds = [17 * j + 1 for j in range(len(SIZES))]
    dev = [to_dev(a) if a.size else to_dev(np.zeros(0, dtype=a.dtype)).reshape(a.shape) for a in host]
    pip.shuffle_batch(dev, seeds, eps=0.5)
    pip.check()
    for a, d, s in zip(host, dev, seeds):
        assert np.array_equal(from_dev(d, a), expected(a, s)), a.shape


@pytest.mark.parametrize("eps", [0.25, 0.5, 0.75])
def test_batch_equals_single_calls(pip, eps):
    torch = torch_cuda()
    rng = np.random.default_rng(5)
    sizes = [int(x) for x in rng.integers(2, 200000, size=40)]
    host = [workloads.iota(n, "u32") for n in sizes]
    seeds = list(range(100, 140))
    batch = [to_dev(a) for a in host]
    single = [to_dev(a) for a in host]
    b = pip.Batch(batch, seeds, eps=eps)
    stats = torch.zeros(pip.JOB_STATS_BYTES * len(sizes), dtype=torch.uint8, device="cuda")
    b.run(stats=stats)
    for t, s in zip(single, seeds):
        pip.shuffle(t, seed=s, eps=eps)
    pip.check()
    js = pip.read_job_stats(stats, len(sizes))
    for a, x, y, s, st, n in zip(host, batch, single, seeds, js, sizes):
        got = from_dev(x, a)
        assert np.array_equal(got, from_dev(y, a))
        assert np.array_equal(got, expected(a, s))
        assert st.status == 0 and st.attempts == (n - 1) + st.losers and st.rounds >= 1


def test_batch_explicit_targets_and_closed_forms(pip):
    n = 5000
    Hs = [np.zeros(n, dtype=np.uint32),
          np.maximum(np.arange(n, dtype=np.int64) - 1, 0).astype(np.uint32),
          workloads.random_targets(n, 1), None]
    host = [workloads.iota(n, "u64") for _ in Hs]
    dev = [to_dev(a) for a in host]
    Hd = [to_dev(h) if h is not None else None for h in Hs]
    b = pip.Batch(dev, [0, 0, 0, 9], eps=0.5, H=Hd, fresh_per_round=64)
    b.run()
    pip.check()
    assert from_dev(dev[0], host[0]).tolist() == [(i + 1) % n for i in range(n)]
    assert from_dev(dev[1], host[1]).tolist() == [n - 1] + list(range(n - 1))
    assert np.array_equal(from_dev(dev[2], host[2]), expected(host[2], H=Hs[2]))
    assert np.array_equal(from_dev(dev[3], host[3]), expected(host[3], 9))


def test_batch_invalid_targets_reported_and_arrays_untouched(pip):
    n = 1000
    H = workloads.random_targets(n, 4)
    H[500] = 900
    host = [workloads.iota(n, "u32") for _ in range(3)]
    dev = [to_dev(a) for a in host]
    b = pip.Batch(dev, [1, 2, 3], eps=0.5, H=[None, to_dev(H), None])
    b.run()
    with pytest.raises(pip.PipError) as e:
        pip.check()
    assert e.value.code == pip.PIP_EINVAL
    for a, d in zip(host, dev):
        assert np.array_equal(from_dev(d, a), a)


def test_graph_replay_repeats_the_shuffle(pip):
    torch = torch_cuda()
    sizes = [3000, 70000, 256, 1 << 18]
    host = [workloads.iota(n, "u32") for n in sizes]
    dev = [to_dev(a) for a in host]
    seeds = [1, 2, 3, 4]
    b = pip.Batch(dev, seeds, eps=0.5)
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        b.run(stream=s)  # warm-up outside capture (sets kernel attributes)
    s.synchronize()
    for a, d in zip(host, dev):  # reset inputs
        d.copy_(to_dev(a))
    torch.cuda.synchronize()
    with torch.cuda.graph(g, stream=s):
        b.run(stream=s)
    g.replay()
    g.replay()
    torch.cuda.synchronize()
    pip.check()
    for a, d, sd in zip(host, dev, seeds):
        twice = expected(expected(a, sd), sd)
        assert np.array_equal(from_dev(d, a), twice)


def test_batch_workload_sample(pip):
    """A slice of the 8192-array workload (sizes log-uniform in [2^8, 2^22], seed 7)."""
    sizes, seeds = workloads.batch_workload()
    idx = list(range(0, 8192, 64))  # 128 arrays spread over the size mix
    host = [workloads.iota(int(sizes[j]), "u32") for j in idx]
    dev = [to_dev(a) for a in host]
    pip.shuffle_batch(dev, [int(seeds[j]) for j in idx], eps=0.5)
    pip.check()
    for a, d, j in zip(host, dev, idx):
        assert np.array_equal(from_dev(d, a), expected(a, int(seeds[j])))


def test_autotuned_options_keep_the_output(pip, tmp_path, monkeypatch):
    from paper_2103_01216_gb300 import autotune

    monkeypatch.setenv("PIP_TUNE_CACHE", str(tmp_path / "tune.json"))
    n = (1 << 16) + 3
    entry = autotune.tune_single(n, "u64", 0.5, reps=1)
    assert entry["options"] and entry["ms"] > 0
    host = workloads.iota(n, "u64")
    A = to_dev(host)
    pip.shuffle(A, seed=5, eps=0.5, tuned=True)
    pip.check()
    assert np.array_equal(from_dev(A, host), expected(host, 5))
    sizes = [300, 5000, 70000]
    arrays = [to_dev(workloads.iota(s, "u32")) for s in sizes]
    b = autotune.tune_batch(arrays, [1, 2, 3], eps=0.5, reps=1)
    assert b["options"]
