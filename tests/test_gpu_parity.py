"""GPU parity: the CUDA round driver against the CPU oracle, bit for bit.

Every case runs the C ABI (through the Python binding) on a GB300 and compares
the whole output array with the sequential Knuth shuffle of ``oracle/`` on the
same input and the same targets.  The tolerance is zero: a shuffle has exactly
one correct output for given targets.
"""
import itertools

import numpy as np
import pytest

import oracle
import workloads
from tests.gpu_util import gpu_shuffle, load_pip, torch_cuda
from tests.conftest import read_golden

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pip():
    torch_cuda()
    return load_pip()


# the three round drivers: persistent grid, one block, one cluster (DSMEM tables),
# and the first two under the two-reservation rule of Algorithm 1 as printed
# and the grid driver under each commit mode (the exchange at L2, and plain
# loads and stores) whatever the prefix size
DRIVERS = {"grid": 32, "cta": 64, "cluster": 128, "grid_tworeserve": 32 | 512, "cta_tworeserve": 64 | 512,
           "grid_exchange": 32 | 8, "grid_loadstore": 32 | 4, "grid_tworeserve_exchange": 32 | 512 | 8,
           "grid_exchange_early": 32 | 8 | 4096}


def expect_hashed(arr, seed):
    out = arr.copy()
    oracle.knuth_hash(out, seed)
    return out


def expect_explicit(arr, H):
    out = arr.copy()
    oracle.knuth_explicit(out, H)
    return out


# ------------------------------------------------------------------ explicit targets
@pytest.mark.parametrize("driver", sorted(DRIVERS))
@pytest.mark.parametrize("F", [1, 2, 3, 8])
def test_figure3_worked_example(pip, F, driver):
    g = read_golden("fig3_worked_example.txt")
    H = np.array([int(x) for x in g["h_zero_based"].split()], dtype=np.uint32)
    expected = [int(x) for x in g["expected_output_zero_based"].split()]
    for dt in ("u32", "u64"):
        out, stats = gpu_shuffle(pip, workloads.iota(8, dt), H=H, fresh_per_round=F, with_stats=True,
                                 flags=DRIVERS[driver])
        assert out.tolist() == expected
        assert stats.status == 0
        assert stats.attempts == 7 + stats.losers


@pytest.mark.parametrize("driver", sorted(DRIVERS))
@pytest.mark.parametrize("n", [2, 3, 4, 5, 6])
def test_every_target_sequence_small_n(pip, n, driver):
    for F in sorted({1, 2, n - 1}):
        for Ht in itertools.product(*[range(i + 1) for i in range(n)]):
            H = np.array(Ht, dtype=np.uint32)
            arr = workloads.iota(n, "u64")
            out, _ = gpu_shuffle(pip, arr, H=H, fresh_per_round=F, flags=DRIVERS[driver])
            assert np.array_equal(out, expect_explicit(arr, H)), (F, Ht)


@pytest.mark.slow
def test_every_target_sequence_n7(pip):
    n = 7
    seen = set()
    for Ht in itertools.product(*[range(i + 1) for i in range(n)]):
        H = np.array(Ht, dtype=np.uint32)
        arr = workloads.iota(n, "u32")
        out, _ = gpu_shuffle(pip, arr, H=H, fresh_per_round=3)
        assert np.array_equal(out, expect_explicit(arr, H)), Ht
        seen.add(tuple(out.tolist()))
    assert len(seen) == 5040  # the bijection, seen through the GPU path


def closed_form_targets(n):
    return {
        "zero": np.zeros(n, dtype=np.uint32),
        "prev": np.maximum(np.arange(n, dtype=np.int64) - 1, 0).astype(np.uint32),
        "self": np.arange(n, dtype=np.uint32),
    }


@pytest.mark.parametrize("driver", sorted(DRIVERS))
@pytest.mark.parametrize("n", [2, 3, 1000, 20011])
@pytest.mark.parametrize("F", [1, 7, 3000])
def test_closed_form_worst_cases(pip, n, F, driver):
    for name, H in closed_form_targets(n).items():
        arr = workloads.iota(n, "u64")
        out, stats = gpu_shuffle(pip, arr, H=H, fresh_per_round=F, with_stats=True, flags=DRIVERS[driver])
        if name == "zero":
            assert out.tolist() == [(i + 1) % n for i in range(n)]
            assert stats.rounds == n - 1  # depth n-1 chain: exactly one commit per round
        elif name == "prev":
            assert out.tolist() == [n - 1] + list(range(n - 1))
            assert stats.rounds == n - 1
        else:
            assert out.tolist() == list(range(n))
        assert stats.attempts == (n - 1) + stats.losers


@pytest.mark.parametrize("n", [5, 1001, 65539])
def test_sattolo_targets(pip, n):
    rng = np.random.default_rng(n)
    H = np.zeros(n, dtype=np.uint32)
    H[1:] = np.floor(rng.random(n - 1) * np.arange(1, n)).astype(np.uint32)  # strictly below i
    arr = workloads.iota(n, "u32")
    out, _ = gpu_shuffle(pip, arr, H=H, fresh_per_round=max(1, n // 50))
    assert np.array_equal(out, expect_explicit(arr, H))


@pytest.mark.parametrize("driver", sorted(DRIVERS))
@pytest.mark.parametrize("n,F", [(1000, 1), (1000, 64), (65537, 256), (300007, 3000), (1 << 20, 100000)])
def test_random_explicit_targets(pip, n, F, driver):
    if driver.startswith("cta") and F > 3000:
        pytest.skip("prefix larger than one block's shared memory")
    H = workloads.random_targets(n, rng_seed=n + F)
    arr = workloads.iota(n, "u64")
    out, stats = gpu_shuffle(pip, arr, H=H, fresh_per_round=F, with_stats=True, flags=DRIVERS[driver])
    assert np.array_equal(out, expect_explicit(arr, H))
    assert stats.rounds >= -(-(n - 1) // F)
    assert stats.attempts == (n - 1) + stats.losers


# ------------------------------------------------------------------ losers under conflicts
@pytest.mark.parametrize("name", ["zero", "prev"])
@pytest.mark.parametrize("commit", [8, 4])
def test_grid_losers_under_conflicts(pip, name, commit):
    """Every fresh swap but one loses in every round, so the losers overflow
    the blocks' on-chip lists into the queue in device memory: with all
    targets at 0 nothing targets a loser's own location; with H[i] = i-1
    every own location is taken."""
    n = 50021
    H = closed_form_targets(n)[name]
    for F in (7, 3000):
        arr = workloads.iota(n, "u64")
        out, st = gpu_shuffle(pip, arr, eps=0.25, H=H, fresh_per_round=F, flags=pip.FLAG_FORCE_GRID | commit,
                              with_stats=True)
        assert np.array_equal(out, expect_explicit(arr, H)), F
        assert st.rounds == n - 1 and st.attempts == (n - 1) + st.losers


# ------------------------------------------------------------------ phase order
@pytest.mark.parametrize("dtype", ["u32", "u64", "rec128"])
def test_phase_order_equal_the_oracle(pip, dtype):
    """A prefix above the planner's 128K threshold runs with the reservations
    and the cleaning after the commit; forced early it gives the same result."""
    n = (1 << 21) + 5
    F = 150000
    fl = pip.FLAG_FORCE_GRID
    assert not pip.plan(n, dtype, 0.2, fresh_per_round=F, flags=fl)["flags"] & pip.FLAG_EARLY_RESERVE
    assert pip.plan(n, dtype, 0.2, fresh_per_round=4096, flags=fl)["flags"] & pip.FLAG_EARLY_RESERVE
    arr = workloads.records(n) if dtype == "rec128" else workloads.iota(n, dtype)
    want = expect_hashed(arr, 9)
    for extra in (0, pip.FLAG_EARLY_RESERVE):
        out, st = gpu_shuffle(pip, arr, seed=9, eps=0.2, fresh_per_round=F, flags=fl | extra, with_stats=True)
        assert np.array_equal(out, want), extra
        assert st.status == 0 and st.attempts == (n - 1) + st.losers


# ------------------------------------------------------------------ hashed targets
@pytest.mark.parametrize("driver", sorted(DRIVERS))
def test_config_2pow20_u64_seed1_eps_half(pip, driver):
    n = 1 << 20
    arr = workloads.iota(n, "u64")
    out, stats = gpu_shuffle(pip, arr, seed=1, eps=0.5, with_stats=True, flags=DRIVERS[driver])
    assert np.array_equal(out, expect_hashed(arr, 1))
    assert stats.status == 0 and stats.attempts == (n - 1) + stats.losers
    p = pip.plan(n, "u64", 0.5, flags=DRIVERS[driver])
    assert stats.rounds >= p["min_rounds"]
    assert stats.max_active <= p["max_active"]


@pytest.mark.parametrize("driver", sorted(DRIVERS))
@pytest.mark.parametrize("n", [2, 3, 31, 32, 33, 1023, 1025, 4097, 100003])
@pytest.mark.parametrize("dtype", ["u32", "u64", "rec128"])
def test_ragged_sizes_all_dtypes(pip, n, dtype, driver):
    arr = workloads.make(n, dtype)
    seed = 1000 + n
    out, _ = gpu_shuffle(pip, arr, seed=seed, eps=0.5, flags=DRIVERS[driver])
    assert np.array_equal(out, expect_hashed(arr, seed))


@pytest.mark.parametrize("eps", [0.1, 0.25, 0.5, 0.75, 0.9])
def test_eps_sweep(pip, eps):
    n = (1 << 18) + 13
    arr = workloads.iota(n, "u64")
    out, stats = gpu_shuffle(pip, arr, seed=7, eps=eps, with_stats=True)
    assert np.array_equal(out, expect_hashed(arr, 7))
    p = pip.plan(n, "u64", eps)
    assert p["aux_bytes"] <= p["aux_bound_bytes"]
    assert stats.max_active <= p["max_active"]


def test_output_does_not_depend_on_launch_shape(pip):
    n, seed = 300007, 11
    arr = workloads.iota(n, "u32")
    ref = expect_hashed(arr, seed)
    configs = [
        dict(fresh_per_round=13),
        dict(fresh_per_round=1000, slot_factor=2),
        dict(fresh_per_round=1000, slot_factor=16),
        dict(fresh_per_round=50000, grid_blocks=1),
        dict(fresh_per_round=50000, grid_blocks=2, block_threads=128),
        dict(fresh_per_round=50000, block_threads=256),
        dict(fresh_per_round=n - 1),
        dict(prefix_c=0.01),
        dict(fresh_per_round=4096, flags=2),
        dict(flags=2),
        dict(flags=DRIVERS["cta"]),
        dict(flags=DRIVERS["cta"], fresh_per_round=17, slot_factor=2),
        dict(flags=DRIVERS["cta"], fresh_per_round=3000, slot_factor=8, block_threads=256),
        dict(flags=DRIVERS["grid"], fresh_per_round=3000),
        dict(flags=DRIVERS["cluster"]),
        dict(flags=DRIVERS["cluster"], fresh_per_round=50000, slot_factor=3),
        dict(flags=DRIVERS["cluster"], fresh_per_round=7, block_threads=256),
        dict(flags=DRIVERS["grid"] | 256, fresh_per_round=3000),
        dict(flags=DRIVERS["grid"] | 256, fresh_per_round=50000),
        dict(flags=512),
        dict(flags=DRIVERS["grid_tworeserve"], fresh_per_round=50000, slot_factor=2),
        dict(flags=DRIVERS["cta_tworeserve"], fresh_per_round=700),
        dict(flags=DRIVERS["cta_tworeserve"] | 2, fresh_per_round=2000, block_threads=1024),
    ]
    for c in configs:
        out, _ = gpu_shuffle(pip, arr, seed=seed, eps=0.5, **c)
        assert np.array_equal(out, ref), c


@pytest.mark.parametrize("dtype", ["u32", "u64", "rec128"])
@pytest.mark.parametrize("mode", ["exchange", "loadstore", "speculate"])
@pytest.mark.parametrize("n,F", [(100003, 977), ((1 << 20) + 5, 150000), (3 << 16, 4096)])
def test_commit_modes_equal_the_oracle(pip, dtype, mode, n, F):
    # every commit mode of the grid driver on every element size, at prefixes
    # on both sides of the planner's switch between them
    flags = DRIVERS["grid"] | {"exchange": 8, "loadstore": 4, "speculate": 256}[mode]
    arr = workloads.make(n, dtype)
    out, stats = gpu_shuffle(pip, arr, seed=n % 97, eps=0.5, fresh_per_round=F, with_stats=True, flags=flags)
    assert np.array_equal(out, expect_hashed(arr, n % 97))
    assert stats.status == 0 and stats.attempts == (n - 1) + stats.losers


def test_planner_picks_the_commit_mode_by_prefix(pip):
    small = pip.plan(10**9, "u64", 0.5)
    large = pip.plan(10**9, "u64", 0.25)
    assert small["driver"] == large["driver"] == pip.DRIVER_GRID
    assert small["flags"] & 256 and not small["flags"] & 8
    assert large["flags"] & 8 and not large["flags"] & 256
    forced = pip.plan(10**9, "u64", 0.25, flags=4)
    assert not forced["flags"] & 8


def test_records_keep_their_payload(pip):
    n, seed = (1 << 19) + 7, 3
    arr = workloads.records(n)
    out, _ = gpu_shuffle(pip, arr, seed=seed, eps=0.5)
    assert np.array_equal(out, expect_hashed(arr, seed))
    assert np.array_equal(out[:, 1], workloads.record_payload(out[:, 0]))


def test_deterministic_repeat(pip):
    n = 200003
    arr = workloads.iota(n, "u64")
    a, _ = gpu_shuffle(pip, arr, seed=5, eps=0.4)
    b, _ = gpu_shuffle(pip, arr, seed=5, eps=0.4)
    assert np.array_equal(a, b)


@pytest.mark.parametrize("eps", [0.25, 0.5, 0.75])
def test_2pow24_against_oracle(pip, eps):
    n = 1 << 24
    arr = workloads.iota(n, "u64")
    out, stats = gpu_shuffle(pip, arr, seed=2, eps=eps, with_stats=True)
    assert np.array_equal(out, expect_hashed(arr, 2))
    assert stats.attempts == (n - 1) + stats.losers


# ------------------------------------------------------------------ errors
def test_invalid_explicit_targets_leave_array_untouched(pip):
    torch = torch_cuda()
    from tests.gpu_util import to_dev, from_dev

    n = 4096
    arr = workloads.iota(n, "u64")
    H = workloads.random_targets(n, 3)
    H[1234] = 1300  # > i
    A = to_dev(arr)
    pip.shuffle(A, H=to_dev(H), eps=0.5)
    with pytest.raises(pip.PipError) as e:
        pip.check()
    assert e.value.code == pip.PIP_EINVAL
    assert np.array_equal(from_dev(A, arr), arr)
    # the latch was cleared and the library keeps working
    out, _ = gpu_shuffle(pip, arr, seed=1, eps=0.5)
    assert np.array_equal(out, expect_hashed(arr, 1))
    del torch


def test_barrier_wait_runs_out_and_reports_timeout(pip):
    """A block that never arrives makes every bounded wait give up (no hang)."""
    from tests.gpu_util import to_dev, from_dev

    n = 1 << 16
    arr = workloads.iota(n, "u64")
    A = to_dev(arr)
    pip.shuffle(A, seed=1, eps=0.5, grid_blocks=4, flags=pip.FLAG_TEST_SKIP_BARRIER | pip.FLAG_FORCE_GRID,
                wait_timeout_ns=50_000_000)
    with pytest.raises(pip.PipError) as e:
        pip.check()
    assert e.value.code == pip.PIP_ETIMEOUT
    assert np.array_equal(from_dev(A, arr), arr)
    out, _ = gpu_shuffle(pip, arr, seed=1, eps=0.5)
    assert np.array_equal(out, expect_hashed(arr, 1))


@pytest.mark.parametrize("dtype", ["u32", "u64", "rec128"])
def test_gated_launch_equals_the_oracle(pip, dtype):
    # the grid driver as a serving lane runs it: no cooperative attribute,
    # the blocks meet at a start gate first; alone on the GPU they all
    # check in, and the result is the oracle's
    n = (1 << 20) + 3
    arr = workloads.make(n, dtype)
    for F in (4096, 200000):  # both commit modes
        out, stats = gpu_shuffle(pip, arr, seed=6, eps=0.5, fresh_per_round=F, with_stats=True,
                                 flags=pip.FLAG_TEST_GATED | pip.FLAG_FORCE_GRID)
        assert stats.status == 0
        assert np.array_equal(out, expect_hashed(arr, 6))


def test_start_gate_gives_up_before_touching_anything(pip):
    """A block that never checks in makes the start gate give up: every block
    leaves before touching the array or the tables, the run reports
    PIP_EBUSY in its own stats, and the per-device latch stays clear."""
    torch = torch_cuda()
    from tests.gpu_util import to_dev, from_dev

    n = 1 << 18
    arr = workloads.iota(n, "u64")
    A = to_dev(arr)
    st = torch.zeros(pip.STATS_BYTES, dtype=torch.uint8, device="cuda")
    pip.shuffle(A, seed=1, eps=0.5, grid_blocks=8, stats=st,
                flags=pip.FLAG_TEST_GATED | pip.FLAG_TEST_SKIP_BARRIER | pip.FLAG_FORCE_GRID,
                wait_timeout_ns=50_000_000)
    pip.check()  # the gate's decision is the run's own, not the device's
    assert pip.read_stats(st).status == pip.PIP_EBUSY
    assert np.array_equal(from_dev(A, arr), arr)
    out, _ = gpu_shuffle(pip, arr, seed=1, eps=0.5)
    assert np.array_equal(out, expect_hashed(arr, 1))


def test_caller_provided_scratch(pip):
    torch = torch_cuda()
    from tests.gpu_util import to_dev, from_dev

    n = 1 << 18
    arr = workloads.iota(n, "u32")
    for flags in (DRIVERS["grid"], DRIVERS["cta"]):
        p = pip.plan(n, "u32", 0.5, flags=flags)
        aux = torch.empty(p["aux_bytes"], dtype=torch.uint8, device="cuda")
        A = to_dev(arr)
        pip.shuffle(A, seed=9, eps=0.5, aux=aux, flags=flags)
        pip.check()
        assert np.array_equal(from_dev(A, arr), expect_hashed(arr, 9))
    p = pip.plan(n, "u32", 0.5, flags=DRIVERS["grid"])
    small = torch.empty(p["aux_bytes"] - 256, dtype=torch.uint8, device="cuda")
    with pytest.raises(pip.PipError):
        pip.shuffle(A, seed=9, eps=0.5, aux=small, flags=DRIVERS["grid"])
